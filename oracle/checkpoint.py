"""Checkpointed runs of the FP64 oracle for large meshes, where one measurement takes hours.

TEST INFRASTRUCTURE ONLY (like the rest of oracle/).

The oracle is evaluated one k1 row at a time (every k2 of one k1 bin); after each row the
results so far are written to a .npz file (written to a temporary name, then renamed, so an
interrupted run never leaves a half-written file), and a later call resumes after the last
completed row.  A fingerprint of the parameters and the catalogues guards against resuming with
different inputs.
"""
from __future__ import annotations

import hashlib
import os

import numpy as np

from . import estimator as E

KEYS = ("raw", "shot", "window_raw", "window_shot")


def fingerprint(params, gal, ran):
    h = hashlib.sha256()
    h.update(repr((params.N, params.L, list(map(float, params.edges)), list(map(tuple, params.ells)), params.los,
                   tuple(params.observer), params.mas, params.interlace, params.P0, params.window)).encode())
    for cat in (gal, ran):
        if cat is None:
            h.update(b"none")
            continue
        for k in sorted(cat):
            h.update(k.encode())
            h.update(np.ascontiguousarray(cat[k]).tobytes())
    return h.hexdigest()


def measure_rows(params, gal, ran, path, max_rows=None):
    """Measure with a checkpoint file at `path`; returns the oracle's result dict (as
    estimator.measure) once every row is done, or None when max_rows rows were computed in this
    call and rows remain."""
    nb = len(params.edges) - 1
    nm = len(params.ells)
    fp = fingerprint(params, gal, ran)
    arrays = {}
    done = np.zeros(nb, dtype=bool)
    if os.path.exists(path):
        st = np.load(path, allow_pickle=False)
        if str(st["fingerprint"]) != fp:
            raise ValueError(f"{path}: checkpoint of a different measurement")
        done = st["done"].copy()
        arrays = {k: st[k].copy() for k in KEYS if k in st.files}
    specs = E.catalogue_spectra(params, gal, ran)
    passes = [("raw", "shot", specs["data"])]
    if "window" in specs:
        passes.append(("window_raw", "window_shot", specs["window"]))
    for kr, ks, _ in passes:
        for k in (kr, ks):
            arrays.setdefault(k, np.full((nm, nb, nb), np.nan))
    rows = 0
    for b1 in range(nb):
        if done[b1]:
            continue
        if max_rows is not None and rows >= max_rows:
            return None
        pairs = [(b1, b2) for b2 in range(nb)]
        for kr, ks, sp in passes:
            arrays[kr][:, b1, :] = E.bispectrum_raw_fft(params, sp, pairs)[:, b1, :]
            arrays[ks][:, b1, :] = E.shot_noise_fft(params, sp, pairs)[:, b1, :]
        done[b1] = True
        rows += 1
        tmp = path + ".tmp.npz"
        np.savez(tmp, fingerprint=np.array(fp), done=done, **arrays)
        os.replace(tmp, path)
    if not done.all():
        return None
    sd = specs["data"]
    res = {"raw": arrays["raw"], "shot": arrays["shot"], "B": arrays["raw"] - arrays["shot"], "I": sd.I,
           "alpha": sd.alpha, "nmodes": E.FieldCache(params, None).nmodes.astype(np.float64)}
    if "window_raw" in arrays:
        res.update(window_raw=arrays["window_raw"], window_shot=arrays["window_shot"],
                   window=arrays["window_raw"] - arrays["window_shot"])
    return res
