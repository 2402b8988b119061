"""Memory-bounded evaluation of the FP64 oracle on large meshes, for a few bin pairs.

TEST INFRASTRUCTURE ONLY (like the rest of oracle/).  Only tests/ and the scripts under
tests/golden/ call it.

A 512^3 survey with window (5e7 randoms, local line of sight) needs 12 complex FP64 spectra
per catalogue and per pass: about 100 GB if held in memory as catalogue_spectra holds them.
Here the same spectra are built one (L, M) channel at a time, with the same expressions in the
same order as catalogue_spectra (so the arrays are identical bit for bit), and kept in .npy
files opened as read-only memory maps.  The estimator and its shot noise are then the oracle's
own bispectrum_raw_fft and shot_noise_fft (Eq. bi_estimator_FFTs, Eq. ShotNoise), called for one
multipole and one bin pair at a time, so that at most one pair's filtered fields are held.
"""
from __future__ import annotations

import dataclasses
import os

import numpy as np

from . import estimator as E


def _store(workdir, name, arr):
    path = os.path.join(workdir, name + ".npy")
    mm = np.lib.format.open_memmap(path, mode="w+", dtype=arr.dtype, shape=arr.shape)
    mm[...] = arr
    mm.flush()
    del mm
    return np.load(path, mmap_mode="r")


def catalogue_spectra_on_disk(params, gal, ran, workdir):
    """The dict catalogue_spectra returns ('data' and, with params.window, 'window'), with every
    spectrum kept in a file under workdir.  Same arithmetic as catalogue_spectra (Sec. 4.1,
    Eq. dn, Eq. nlm; N_L^M and Sbar_L^M of Eq. ShotNoise; I of Eq. normalization)."""
    os.makedirs(workdir, exist_ok=True)
    Ls = params.needed_L()
    wg = E.object_weights(gal, params.P0)
    wr = E.object_weights(ran, params.P0) if ran is not None else None
    if params.los == "local" and ran is None:
        raise ValueError("local line of sight needs a random catalogue")
    if params.window and ran is None:
        raise ValueError("window needs randoms")
    alpha = float(wg.sum() / wr.sum()) if ran is not None else None
    glob = params.los == "global"

    def per_cat(cat, w, L, M):
        yc = E.los_yconj(params, cat["xyz"], L, M)
        d = E.spectrum(params, cat["xyz"], w * yc)
        n = E.spectrum(params, cat["xyz"], w * w * np.conj(yc))
        return d, n, complex(np.sum(w ** 3 * yc))

    D, Nk, S, WD, WN, WS = {}, {}, {}, {}, {}, {}
    for L in Ls:
        for M in range(-L, L + 1):
            if glob and M != 0:
                continue
            key = (L, M)
            if glob and L > 0:  # the global line of sight aliases every L to the monopole
                D[key], Nk[key], S[key] = D[(0, 0)], Nk[(0, 0)], S[(0, 0)]
                if params.window:
                    WD[key], WN[key], WS[key] = WD[(0, 0)], WN[(0, 0)], WS[(0, 0)]
                continue
            tag = f"L{L}_M{M}".replace("-", "m")
            dg, ng, sg = per_cat(gal, wg, L, M)
            if ran is not None:
                dr, nr, sr = per_cat(ran, wr, L, M)
                d = dg - alpha * dr
                n = ng + alpha ** 2 * nr
                s = sg - alpha ** 3 * sr
            else:
                d, n, s = dg, ng, sg
            del dg, ng
            d = d.copy()
            d[0, 0, 0] = 0.0
            D[key] = _store(workdir, "data_D_" + tag, d)
            del d
            Nk[key] = _store(workdir, "data_N_" + tag, n)
            del n
            S[key] = s
            if params.window:
                WD[key] = _store(workdir, "window_D_" + tag, alpha * dr)
                WN[key] = _store(workdir, "window_N_" + tag, alpha ** 2 * nr)
                WS[key] = alpha ** 3 * sr
            if ran is not None:
                del dr, nr
    if ran is not None:
        R = E.assign(ran["xyz"], wr, params.N, params.L, params.mas, 0.0)
        I = alpha ** 3 * float(np.sum(R ** 3)) / params.H ** 6
        del R
    else:
        I = float(wg.sum()) ** 3 / params.V ** 2
    out = {"data": E.Spectra(D, Nk, S, I, alpha, "data")}
    if params.window:
        out["window"] = E.Spectra(WD, WN, WS, I, alpha, "window")
    return out


def measure_pairs(params, specs, pairs_by_mult):
    """Oracle values at the requested bins: pairs_by_mult maps a multipole (l1, l2, L) of
    params.ells to a list of (b1, b2).  Returns {(l1, l2, L, b1, b2): {'raw', 'shot', 'B'}
    and, with a window pass, 'window_raw', 'window_shot', 'window'}."""
    out = {}
    for mult, pairs in pairs_by_mult.items():
        if tuple(mult) not in [tuple(e) for e in params.ells]:
            raise ValueError(f"{mult} is not a multipole of the plan")
        q = dataclasses.replace(params, ells=[tuple(mult)])
        for (b1, b2) in pairs:
            rec = {}
            for pas, pre in (("data", ""), ("window", "window_")):
                if pas not in specs:
                    continue
                raw = float(E.bispectrum_raw_fft(q, specs[pas], [(b1, b2)])[0, b1, b2])
                shot = float(E.shot_noise_fft(q, specs[pas], [(b1, b2)])[0, b1, b2])
                rec[pre + "raw"] = raw
                rec[pre + "shot"] = shot
                rec["window" if pre else "B"] = raw - shot
            out[tuple(mult) + (b1, b2)] = rec
    return out
