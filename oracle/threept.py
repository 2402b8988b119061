"""FP64 CPU oracle of the FFT-based three-point-function multipoles (Sec. 4.3) and the
three-point window multipoles Q (Sec. 6.1, Eq. Q).

TEST INFRASTRUCTURE ONLY.  Plain, slow and obviously correct; it shares no code with the
CUDA path.  Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may
import it.

What it computes (Eq. three_point_es, Eq. reduced_xi_estimator):

    zeta_{l1 l2 L}(r_a, r_b) = (N H / I) sum_{m1 m2 M} 3j
        int d^3x F_{l1}^{m1}(x; a) F_{l2}^{m2}(x; b) G_L^M(x),

with F_l^m(x; a) the average over the separations s of r-bin a of y_l^{m*}(s_hat)
delta n(x + s) and G_L^M(x) = delta n_L^M(x).  In Fourier space the average is the filter
K_a(k) = (1/N_r(a)) sum_{s in a} y_l^{m*}(s_hat) e^{i k.s}; for a thin continuous shell it is
i^l j_l(k r) y_l^{m*}(k_hat), the filter the paper writes.

Readings where the paper is silent (the CUDA path takes the same ones):
* r-bins are sets of mesh separations: s integer with |s_i| <= N/2 - 1, in bin a when
  e_a <= H |s| < e_{a+1} (FP64, the same comparison as the k-bins); N_r(a) counts them.  A bin
  that starts at 0 holds s = 0, where y_l^m(0) is taken as delta_{l0} (the r = 0 bin of the
  window multipoles, Sec. 6.1);
* the continuous integrals become sums over cells and separations: int d^3x -> (V/N_g)
  sum_x, densities are mesh weights / H^3, deconvolved by W_mass like the bispectrum's;
* shot noise: of the bispectrum's four terms only i = j != k reaches r_1, r_2 > 0 (Sec. 4.3);
  it lives on r_a = r_b and is the Q_L^M = delta n_L^M N_0^{0*} - Sbar_L^M C/W^2 correlation
  (the bispectrum's Q field) at the separations of the bin, weighted by y_{l1}^{m1*} y_{l2}^{m2*}.
  The terms at r = 0 (i != j = k, i = k != j, i = j = k) are not subtracted;
* the window multipoles Q_{l1 l2 L}: the same estimator on the randoms-only pass
  (nbar = alpha sum_ran w delta_D), its i = j != k term subtracted like the data's.
"""
from __future__ import annotations

import numpy as np

from . import estimator as E
from .sph import h_lll, n_lll


# --------------------------------------------------------------------------------------
# r-bins of mesh separations
# --------------------------------------------------------------------------------------


def r_bin_of_q(params, q):
    """Bin of separations with |s|^2 = q: e_a <= H sqrt(q) < e_{a+1}."""
    r = params.H * np.sqrt(np.asarray(q, dtype=np.float64))
    e = np.asarray(params.edges, dtype=np.float64)
    a = np.searchsorted(e, r, side="right") - 1
    return np.where((a >= 0) & (a < len(e) - 1), a, -1)


def offset_bins(params):
    """r-bin of every separation s, indexed by s mod N on the N^3 grid (-1: in no bin)."""
    sx, sy, sz = E.mode_grids(params.N)
    q = sx * sx + sy * sy + sz * sz
    a = r_bin_of_q(params, q)
    return np.where(E.nyquist_mask(params.N), -1, a)


def shell_offsets(params, a, bins=None):
    """Signed separations (n, 3) of r-bin a."""
    if bins is None:
        bins = offset_bins(params)
    return E.signed_modes(params.N)[np.argwhere(bins == a)]


def _ys(params, l, m, s):
    """y_l^{m*}(s_hat) of integer separations s (n, 3); y(0) = delta_{l0}."""
    s = np.asarray(s, dtype=np.float64)
    r = np.sqrt(np.sum(s * s, axis=-1))
    out = np.zeros(len(s), dtype=np.complex128)
    nz = r > 0
    if nz.any():
        out[nz] = np.conj(E._y(params, l, m, s[nz, 0], s[nz, 1], s[nz, 2]))
    if l == 0:
        out[~nz] = 1.0
    return out


def shell_filter(params, l, m, a, bins=None):
    """K_a(k) = (1/N_r(a)) sum_{s in a} y_l^{m*}(s_hat) e^{i k.s} on the full k grid."""
    if bins is None:
        bins = offset_bins(params)
    idx = np.argwhere(bins == a)
    c = np.zeros((params.N,) * 3, dtype=np.complex128)
    if len(idx) == 0:
        return c
    s = E.signed_modes(params.N)[idx]
    c[idx[:, 0], idx[:, 1], idx[:, 2]] = _ys(params, l, m, s) / len(idx)
    return params.Ng * np.fft.ifftn(c)  # sum_s c(s) e^{+i k.s}


# --------------------------------------------------------------------------------------
# estimator, FFT mode (Eq. reduced_xi_estimator)
# --------------------------------------------------------------------------------------


class FilterFields:
    """F_l^m(x; a) = (Ng/V) ifft(D(k) K_a(k)) (densities), computed on demand."""

    def __init__(self, params, D00):
        self.p, self.D = params, D00
        self.bins = offset_bins(params)
        self.nr = np.bincount(self.bins[self.bins >= 0].ravel(), minlength=len(params.edges) - 1)
        self.cache = {}

    def get(self, l, m, a):
        key = (l, m, a)
        if key not in self.cache:
            K = shell_filter(self.p, l, m, a, self.bins)
            self.cache[key] = self.p.Ng / self.p.V * np.fft.ifftn(self.D * K)
        return self.cache[key]


def threept_raw_fft(params, spec):
    """hat zeta_{l1 l2 L}(r_a, r_b) before shot-noise subtraction, [n_mult, nb, nb]."""
    nb = len(params.edges) - 1
    out = np.zeros((len(params.ells), nb, nb))
    ff = FilterFields(params, spec.D[(0, 0)])
    G = {}
    glob = params.los == "global"
    for im, (l1, l2, L) in enumerate(params.ells):
        pref = n_lll(l1, l2, L) * h_lll(l1, l2, L) / spec.I
        terms = E._m_terms(l1, l2, L, glob)
        for a in range(nb):
            for b in range(nb):
                acc = 0.0 + 0.0j
                for m1, m2, M, c3 in terms:
                    if (L, M) not in G:
                        G[(L, M)] = E.g_field(params, spec.D[(L, M)])
                    acc += c3 * params.V / params.Ng * np.sum(ff.get(l1, m1, a) * ff.get(l2, m2, b) * G[(L, M)])
                out[im, a, b] = pref * acc.real
    return out


def threept_shot_fft(params, spec, cw=None):
    """The i = j != k term: on r_a = r_b,
    (N H / I) sum 3j (1/N_r^2) sum_{s in a} y_{l1}^{m1*} y_{l2}^{m2*}(s_hat) (Ng/V^2) q(-s),
    q(x) = sum_k Q_L^M(k) e^{ikx}; zero off the diagonal."""
    nb = len(params.edges) - 1
    out = np.zeros((len(params.ells), nb, nb))
    if cw is None:
        cw = E.cw2(params)
    bins = offset_bins(params)
    glob = params.los == "global"
    qx = {}
    for im, (l1, l2, L) in enumerate(params.ells):
        pref = n_lll(l1, l2, L) * h_lll(l1, l2, L) / spec.I
        for a in range(nb):
            s = shell_offsets(params, a, bins)
            if len(s) == 0:
                continue
            neg = (-s) % params.N
            acc = 0.0 + 0.0j
            for m1, m2, M, c3 in E._m_terms(l1, l2, L, glob):
                if (L, M) not in qx:
                    # Q_L^M = delta n_L^M N_0^{0*} - Sbar_L^M C/W^2 (zero on the Nyquist planes
                    # with the estimator's spectra and C/W^2)
                    q = spec.D[(L, M)] * np.conj(spec.Nk[(0, 0)]) - spec.Sbar[(L, M)] * cw
                    qx[(L, M)] = params.Ng * np.fft.ifftn(q)
                w = _ys(params, l1, m1, s) * _ys(params, l2, m2, s)
                acc += c3 * np.sum(w * qx[(L, M)][neg[:, 0], neg[:, 1], neg[:, 2]])
            out[im, a, a] = pref * acc.real * params.Ng / params.V ** 2 / len(s) ** 2
    return out


def measure(params, gal, ran=None):
    """Full oracle: {'zeta', 'shot', 'raw', 'nr', and 'window' (= Q), 'window_shot' if requested}."""
    specs = E.catalogue_spectra(params, gal, ran)
    sd = specs["data"]
    raw = threept_raw_fft(params, sd)
    shot = threept_shot_fft(params, sd)
    res = {"raw": raw, "shot": shot, "zeta": raw - shot, "I": sd.I, "alpha": sd.alpha}
    if "window" in specs:
        sw = specs["window"]
        wraw = threept_raw_fft(params, sw)
        wshot = threept_shot_fft(params, sw)
        res.update(window_raw=wraw, window_shot=wshot, window=wraw - wshot)
    bins = offset_bins(params)
    res["nr"] = np.bincount(bins[bins >= 0].ravel(), minlength=len(params.edges) - 1).astype(np.float64)
    return res


# --------------------------------------------------------------------------------------
# direct mode: the separation sums of Eq. three_point_es written out on the mesh
# --------------------------------------------------------------------------------------


def threept_raw_direct(params, spec, l1, l2, L, a, b):
    """hat zeta for one multipole and bin pair with F formed by explicit sums over the
    separations of each bin (np.roll of the density mesh), no filter in k space."""
    bins = offset_bins(params)
    s1, s2 = shell_offsets(params, a, bins), shell_offsets(params, b, bins)
    if len(s1) == 0 or len(s2) == 0:
        return 0.0
    dens = {}

    def field(L_, M_):
        if (L_, M_) not in dens:
            dens[(L_, M_)] = E.g_field(params, spec.D[(L_, M_)])
        return dens[(L_, M_)]

    def F(l, m, s):
        ys = _ys(params, l, m, s)
        out = np.zeros((params.N,) * 3, dtype=np.complex128)
        d = field(0, 0)
        for i in range(len(s)):
            out += ys[i] * np.roll(d, shift=tuple(-s[i]), axis=(0, 1, 2))  # delta n(x + s)
        return out / len(s)

    acc = 0.0 + 0.0j
    for m1, m2, M, c3 in E._m_terms(l1, l2, L, params.los == "global"):
        acc += c3 * params.V / params.Ng * np.sum(F(l1, m1, s1) * F(l2, m2, s2) * field(L, M))
    return n_lll(l1, l2, L) * h_lll(l1, l2, L) / spec.I * acc.real


def node_spectra(params, xyz, w, ran_xyz=None, ran_w=None):
    """Spectra of objects that sit on mesh nodes, without deconvolution (W = C = 1): the
    exact DFTs, for the separation-space brute force.  xyz are node indices (n, 3)."""
    N = params.N

    def mesh(ix, v):
        m = np.zeros((N,) * 3, dtype=np.complex128)
        np.add.at(m, (ix[:, 0] % N, ix[:, 1] % N, ix[:, 2] % N), v)
        return np.fft.fftn(m)

    def yconj(ix, L, M):
        pos = (np.asarray(ix, dtype=np.float64) + 0.0) * params.H
        return E.los_yconj(params, pos, L, M)

    alpha = float(np.sum(w) / np.sum(ran_w)) if ran_xyz is not None else None
    D, Nk, S = {}, {}, {}
    for L in params.needed_L():
        for M in range(-L, L + 1):
            if params.los == "global" and M != 0:
                continue
            yg = yconj(xyz, L, M) if params.los == "local" else np.ones(len(xyz))
            D[(L, M)] = mesh(xyz, w * yg)
            Nk[(L, M)] = mesh(xyz, w * w * np.conj(yg))
            S[(L, M)] = complex(np.sum(w ** 3 * yg))
            if ran_xyz is not None:
                yr = yconj(ran_xyz, L, M) if params.los == "local" else np.ones(len(ran_xyz))
                D[(L, M)] = D[(L, M)] - alpha * mesh(ran_xyz, ran_w * yr)
                Nk[(L, M)] = Nk[(L, M)] + alpha ** 2 * mesh(ran_xyz, ran_w ** 2 * np.conj(yr))
                S[(L, M)] -= alpha ** 3 * complex(np.sum(ran_w ** 3 * yr))
    return E.Spectra(D, Nk, S, 1.0, alpha, "data")


def distinct_triplet_sum(params, xyz, w, l1, l2, L, a, b, ran_xyz=None, ran_w=None):
    """(N H / I) sum 3j (1/(N_r(a) N_r(b) H^6)) sum over distinct objects i != j != k with
    x_i - x_k in r-bin a and x_j - x_k in r-bin b of w_i w_j w_k y_{l1}^{m1*} y_{l2}^{m2*}
    y_L^{M*}(x_k hat), I = 1 (objects: the data with weight w, the randoms with -alpha w)."""
    N = params.N
    bins = offset_bins(params)
    nr = np.bincount(bins[bins >= 0].ravel(), minlength=len(params.edges) - 1)
    pos = np.asarray(xyz, dtype=np.int64)
    wt = np.asarray(w, dtype=np.float64)
    if ran_xyz is not None:
        alpha = float(np.sum(w) / np.sum(ran_w))
        pos = np.concatenate([pos, np.asarray(ran_xyz, dtype=np.int64)])
        wt = np.concatenate([wt, -alpha * np.asarray(ran_w, dtype=np.float64)])
    sgn = E.signed_modes(N)
    n = len(pos)
    tot = 0.0 + 0.0j
    for m1, m2, M, c3 in E._m_terms(l1, l2, L, params.los == "global"):
        if params.los == "local":
            yk = E.los_yconj(params, pos.astype(np.float64) * params.H, L, M)
        else:
            yk = np.ones(n)
        for k in range(n):
            d = (pos - pos[k]) % N
            ab = bins[d[:, 0], d[:, 1], d[:, 2]]
            s = sgn[d]
            y1 = _ys(params, l1, m1, s)
            y2 = _ys(params, l2, m2, s)
            i1 = np.flatnonzero(ab == a)
            i2 = np.flatnonzero(ab == b)
            for i in i1:
                if i == k:
                    continue
                j = i2[(i2 != i) & (i2 != k)]
                tot += c3 * wt[i] * y1[i] * np.sum(wt[j] * y2[j]) * wt[k] * yk[k]
    return n_lll(l1, l2, L) * h_lll(l1, l2, L) * tot.real / (nr[a] * nr[b] * params.H ** 6)
