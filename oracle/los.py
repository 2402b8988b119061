"""FP64 oracle of the bispectrum multipoles with the line of sight on x1 or x2 instead of x3
(App. B; the estimator of Eq. bi_estimator_FFTs with the y_L^{M*} weight moved to another
object of the triplet).

TEST INFRASTRUCTURE ONLY.  Plain sums over the definitions; shares no code with the library.
Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may import it.

With the line of sight on object p (p = 3 is the main text's choice), the three slots of the
mesh sum (k1 shell, k2 shell, G) take the spectra
    X_s = delta n_L^M  if s = p,  else delta n_0^0,
and the shot-noise terms of Eq. shotnoise follow the object that carries the weight (reading):
* i = j = k:  Sbar_L^M Y1 Y2, for every p;
* a distinct object in slot s and a coincident pair in the other two:
  the shell (or, for s = 3, the unit-shell mesh sum) of  X_s conj(N_pair) - Sbar_L^M C/W^2,
  with N_pair = N_L^M if the pair holds p, else N_0^0, and X_s = delta n_L^M if s = p.
For p = 3 this is the main text's estimator (oracle/estimator.py).
"""
from __future__ import annotations

import numpy as np

from . import estimator as E
from .sph import h_lll, n_lll


def _key(p, slot, L, M):
    return (L, M) if slot == p else (0, 0)


def bispectrum_raw_fft(params, spec, p):
    """hat B with the line of sight on object p, [n_mult, nb, nb]."""
    nb = len(params.edges) - 1
    out = np.zeros((len(params.ells), nb, nb))
    fcs, G = {}, {}

    def fc(key):
        if key not in fcs:
            fcs[key] = E.FieldCache(params, spec.D[key])
        return fcs[key]

    glob = params.los == "global"
    for im, (l1, l2, L) in enumerate(params.ells):
        pref = n_lll(l1, l2, L) * h_lll(l1, l2, L) / spec.I
        terms = E._m_terms(l1, l2, L, glob)
        for b1 in range(nb):
            for b2 in range(nb):
                acc = 0.0 + 0.0j
                for m1, m2, M, c3 in terms:
                    k3 = _key(p, 3, L, M)
                    if k3 not in G:
                        G[k3] = E.g_field(params, spec.D[k3])
                    F1 = fc(_key(p, 1, L, M)).get(l1, m1, b1)
                    F2 = fc(_key(p, 2, L, M)).get(l2, m2, b2)
                    acc += c3 * params.V / params.Ng * np.sum(F1 * F2 * G[k3])
                out[im, b1, b2] = pref * acc.real
    return out


def _pair_spectrum(params, spec, p, s, L, M, cw):
    """X_s conj(N_pair) - Sbar_L^M C/W^2 for a distinct object in slot s."""
    X = spec.D[(L, M)] if s == p else spec.D[(0, 0)]
    Npair = spec.Nk[(L, M)] if s != p else spec.Nk[(0, 0)]
    q = X * np.conj(Npair) - spec.Sbar[(L, M)] * cw
    q[E.nyquist_mask(params.N)] = 0.0
    return q


def shot_noise_fft(params, spec, p):
    """The four shot-noise terms with the line of sight on object p, summed, [n_mult, nb, nb]."""
    nb = len(params.edges) - 1
    out = np.zeros((len(params.ells), nb, nb))
    uc = E.FieldCache(params, None)
    cw = E.cw2(params)
    glob = params.los == "global"
    qs, qx = {}, {}

    def shell_avg(l, m, b, q):
        nm = uc.nmodes[b]
        return complex(np.sum((uc.harmonic(l, m) * q)[uc.bins == b]) / nm) if nm else 0.0

    for im, (l1, l2, L) in enumerate(params.ells):
        pref = n_lll(l1, l2, L) * h_lll(l1, l2, L) / spec.I
        terms = E._m_terms(l1, l2, L, glob)
        for b1 in range(nb):
            for b2 in range(nb):
                t = 0.0 + 0.0j
                for m1, m2, M, c3 in terms:
                    for s in (1, 2, 3):
                        if (s, L, M) not in qs:
                            qs[(s, L, M)] = _pair_spectrum(params, spec, p, s, L, M, cw)
                    Y1 = E.shell_average_y(params, uc, l1, m1, b1)
                    Y2 = E.shell_average_y(params, uc, l2, m2, b2)
                    t += c3 * spec.Sbar[(L, M)] * Y1 * Y2
                    t += c3 * shell_avg(l1, m1, b1, qs[(1, L, M)]) * Y2
                    t += c3 * Y1 * shell_avg(l2, m2, b2, qs[(2, L, M)])
                    if (L, M) not in qx:
                        qx[(L, M)] = params.Ng * np.fft.ifftn(qs[(3, L, M)])
                    t += c3 / params.Ng * np.sum(uc.get(l1, m1, b1) * uc.get(l2, m2, b2) * qx[(L, M)])
                out[im, b1, b2] = pref * t.real
    return out


def measure(params, gal, ran, p):
    """{'B', 'shot', 'raw', and 'window', 'window_shot' if requested} with the line of sight on p."""
    specs = E.catalogue_spectra(params, gal, ran)
    sd = specs["data"]
    raw = bispectrum_raw_fft(params, sd, p)
    shot = shot_noise_fft(params, sd, p)
    res = {"raw": raw, "shot": shot, "B": raw - shot}
    if "window" in specs:
        sw = specs["window"]
        wraw = bispectrum_raw_fft(params, sw, p)
        wshot = shot_noise_fft(params, sw, p)
        res.update(window_raw=wraw, window_shot=wshot, window=wraw - wshot)
    return res


def raw_direct(params, acc, I, p, l1, l2, L, modes1, modes2):
    """The triangle sum (N H / I) sum 3j (1/(Nm1 Nm2)) sum_{k1 k2} y1* y2* X1(k1) X2(k2) X3(-k1-k2)."""
    glob = params.los == "global"
    n1 = np.asarray(modes1)
    n2 = np.asarray(modes2)
    tot = 0.0 + 0.0j
    for m1, m2, M, c3 in E._m_terms(l1, l2, L, glob):
        a1 = E._yk(params, l1, m1, n1) * acc.D(*_key(p, 1, L, M), n1)
        a2 = E._yk(params, l2, m2, n2) * acc.D(*_key(p, 2, L, M), n2)
        s = 0.0 + 0.0j
        for i in range(len(n1)):
            n3 = -(n1[i][None, :] + n2)
            s += a1[i] * np.sum(a2 * acc.D(*_key(p, 3, L, M), n3))
        tot += c3 * s / (len(n1) * len(n2))
    return n_lll(l1, l2, L) * h_lll(l1, l2, L) / I * tot.real


def shot_direct(params, acc, I, p, l1, l2, L, modes1, modes2):
    """The four shot-noise terms from shell and triangle sums over the modes, with any spectrum
    accessor (the exact one has C/W^2 = 1)."""
    glob = params.los == "global"
    n1 = np.asarray(modes1)
    n2 = np.asarray(modes2)

    def q(s, M, n):
        X = acc.D(L, M, n) if s == p else acc.D(0, 0, n)
        Np = acc.N(L, M, n) if s != p else acc.N(0, 0, n)
        return X * np.conj(Np) - acc.Sbar(L, M) * acc.cw2(n)

    tot = 0.0 + 0.0j
    for m1, m2, M, c3 in E._m_terms(l1, l2, L, glob):
        y1 = E._yk(params, l1, m1, n1)
        y2 = E._yk(params, l2, m2, n2)
        Y1, Y2 = y1.mean(), y2.mean()
        tot += c3 * acc.Sbar(L, M) * Y1 * Y2
        tot += c3 * np.mean(y1 * q(1, M, n1)) * Y2
        tot += c3 * Y1 * np.mean(y2 * q(2, M, n2))
        s = 0.0 + 0.0j
        for i in range(len(n1)):
            s += y1[i] * np.sum(y2 * q(3, M, -(n1[i][None, :] + n2)))
        tot += c3 * s / (len(n1) * len(n2))
    return n_lll(l1, l2, L) * h_lll(l1, l2, L) / I * tot.real


def distinct_triplet_sum(params, acc, I, p, l1, l2, L, modes1, modes2):
    """Brute force over distinct objects i != j != k: s w s w s w y_L^{M*}(x of the object in
    slot p) A1(x_i - x_k) A2(x_j - x_k)."""
    glob = params.los == "global"
    n1 = np.asarray(modes1, dtype=np.float64)
    n2 = np.asarray(modes2, dtype=np.float64)
    x, sw = acc.x, acc.s * acc.w
    dx = x[:, None, :] - x[None, :, :]
    npart = len(x)
    mask = np.ones((npart, npart, npart), dtype=bool)
    ii = np.arange(npart)
    mask[ii, ii, :] = False
    mask[ii, :, ii] = False
    mask[:, ii, ii] = False
    tot = 0j
    for m1, m2, M, c3 in E._m_terms(l1, l2, L, glob):
        y1 = E._yk(params, l1, m1, n1)
        y2 = E._yk(params, l2, m2, n2)
        A1 = np.exp(-1j * acc.kF * np.einsum("ikd,nd->ikn", dx, n1)) @ y1 / len(n1)
        A2 = np.exp(-1j * acc.kF * np.einsum("ikd,nd->ikn", dx, n2)) @ y2 / len(n2)
        yc = acc.yc(L, M)
        wi = sw * (yc if p == 1 else 1.0)
        wj = sw * (yc if p == 2 else 1.0)
        wk = sw * (yc if p == 3 else 1.0)
        T = (wi[:, None, None] * A1[:, None, :]) * (wj[None, :, None] * A2[None, :, :]) * wk[None, None, :]
        tot += c3 * np.sum(T[mask])
    return n_lll(l1, l2, L) * h_lll(l1, l2, L) / I * tot.real
