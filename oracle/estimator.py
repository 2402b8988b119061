"""FP64 CPU oracle of the FFT-based TripoSH bispectrum-multipole estimator.

TEST INFRASTRUCTURE ONLY.  This is the plain, slow, obviously-correct reference the
CUDA path is checked against; it shares no code with it.  Only tests/,
__graft_entry__.smoke() and bench.py's CPU-baseline leg may import it.

It follows Sec. 4 of the paper step by step, in FP64 with numpy (numpy's FFT is the
only library primitive used as a step):

1. weights, FKP weight w = 1/(1 + nbar P0) (Sec. 5.2, Eq. weight), alpha (Sec. 4.1);
2. mass assignment NGP/CIC/TSC in particle order (Sec. 4.2, App. C), optional
   interlacing (a reading, see below);
3. FFT and division by W_mass(k) (Sec. 4.2);
4. y_L^{M*}(x)-weighted density delta n_L^M (Eq. nlm) -> G_L^M(x) (Eq. nlm_bi);
5. shell-filtered fields F_l^m(x; k) (Eq. nlm_bi, Eq. angular_integral);
6. the mesh sum of F F G contracted with 3j symbols (Eq. bi_estimator_FFTs; global
   line of sight: Eq. simulation_estimator);
7. shot noise, four terms (Eq. shotnoise, Eq. ShotNoise);
8. normalisation I (Eq. normalization; periodic box I = Np^3/V^2, Sec. 4.4).

It also evaluates the same estimator as the mode sum over triangles (Eq. bi_estimator,
"direct mode") and, for a handful of particles, with exact DFTs ("particle-exact mode").

Readings where the paper is silent or garbled (the CUDA path takes the same ones):
* bins are [e_b, e_{b+1}) in k = kF sqrt(|n|^2), decided in FP64; modes on a Nyquist
  plane (any |n_i| = N/2) and k = 0 are in no bin; N_mode counts the full cube;
* every spectrum is zero on the Nyquist planes (the interlaced combination is not
  Hermitian there and no shell reaches them);
* mesh node c sits at x = c H; CIC uses floor(u), NGP and TSC round(u), u = x/H;
* interlacing: a second mesh filled at u - 1/2, combined as
  (D1 + exp(-i pi (nx+ny+nz)/N) D2)/2 with signed integer n;
* shot noise is taken in its discrete form (shell averages of y instead of Kronecker
  deltas, and the i=j!=k term as the same mesh sum with unit shells and
  Q = D_L^M conj(N_0^0) - Sbar_L^M C/W^2), C(k) the alias sum of W^2 (even images only
  when interlaced), no C on the i=j=k term (Sec. 4.2);
* D(k=0) is set to zero for the data pass (delta n has no mean), kept for the window;
* window bispectrum: the same estimator on nbar = alpha sum_ran w delta_D, with
  Sbar = alpha^3 sum w^3 y*, N = alpha^2 sum w^2 y, same I.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Sequence

import numpy as np

from .sph import allowed_multipole, h_lll, n_lll, wigner3j, ylm

# --------------------------------------------------------------------------------------
# plan
# --------------------------------------------------------------------------------------


@dataclass
class Params:
    N: int
    L: float
    edges: Sequence[float]
    ells: Sequence[tuple]
    los: str = "global"          # 'global' (z axis) or 'local'
    observer: tuple = (0.0, 0.0, 0.0)
    mas: int = 2                 # p = 1, 2, 3 for NGP, CIC, TSC
    interlace: bool = False
    P0: float = 0.0
    window: bool = False
    polar_axis: str = "z"        # axis of the spherical harmonics ('z' or 'x'), a test knob
    condon_shortley: bool = True  # phase convention of y_l^m (the result does not depend on it)
    ells_all_orders: bool = False  # allow l1 < l2 (test knob)
    extra: dict = field(default_factory=dict)

    @property
    def V(self):
        return float(self.L) ** 3

    @property
    def Ng(self):
        return self.N ** 3

    @property
    def H(self):
        return self.L / self.N

    @property
    def kF(self):
        return 2.0 * np.pi / self.L

    def needed_L(self):
        return sorted({int(c[2]) for c in self.ells} | {0})

    def needed_l(self):
        s = set()
        for l1, l2, _ in self.ells:
            s.add(int(l1))
            s.add(int(l2))
        return sorted(s)


def _axes(params, x, y, z):
    """Spherical-harmonic polar axis: 'z' (default) or 'x' (cyclic relabelling)."""
    if params.polar_axis == "z":
        return x, y, z
    if params.polar_axis == "x":
        return y, z, x
    raise ValueError(params.polar_axis)


def _y(params, l, m, x, y, z):
    a, b, c = _axes(params, x, y, z)
    return ylm(l, m, a, b, c, condon_shortley=params.condon_shortley)


# --------------------------------------------------------------------------------------
# k-space geometry
# --------------------------------------------------------------------------------------


def signed_modes(N):
    """Signed integer frequencies of the FFT grid (index j -> j or j - N)."""
    j = np.arange(N)
    return np.where(j < N // 2, j, j - N).astype(np.int64)


def mode_grids(N):
    n = signed_modes(N)
    return n[:, None, None], n[None, :, None], n[None, None, :]


def nyquist_mask(N):
    nx, ny, nz = mode_grids(N)
    h = N // 2
    return (np.abs(nx) == h) | (np.abs(ny) == h) | (np.abs(nz) == h)


def bin_of_q(params, q):
    """Bin of modes with |n|^2 = q: e_b <= kF sqrt(q) < e_{b+1} (Eq. angular_integral, reading)."""
    kF = 2.0 * np.pi / params.L
    k = kF * np.sqrt(np.asarray(q, dtype=np.float64))
    e = np.asarray(params.edges, dtype=np.float64)
    b = np.searchsorted(e, k, side="right") - 1
    return np.where((b >= 0) & (b < len(e) - 1), b, -1)


def bin_grid(params):
    """Bin index of every mode of the full N^3 grid (-1: in no bin)."""
    nx, ny, nz = mode_grids(params.N)
    q = nx * nx + ny * ny + nz * nz
    b = bin_of_q(params, q)
    b = np.where(nyquist_mask(params.N) | (q == 0), -1, b)
    return b


def shell_modes(params, b, bins=None):
    """Integer vectors (n, 3) of the modes in bin b."""
    if bins is None:
        bins = bin_grid(params)
    idx = np.argwhere(bins == b)
    n = signed_modes(params.N)
    return n[idx]


def mas_window(N, p):
    """W_mass(k) = prod_i sinc(pi n_i / N)^p (Sec. 4.2)."""
    nx, ny, nz = mode_grids(N)
    return (np.sinc(nx / N) * np.sinc(ny / N) * np.sinc(nz / N)) ** p


def c_shot(N, p, interlace, mmax=None):
    """Alias sum C(k) = sum_m W^2(k + 2 kN m) (Jing 2005, cited in Sec. 4.2); with
    interlacing only images with even m_x+m_y+m_z survive.  Truncated direct sum."""
    if mmax is None:
        mmax = 4000 if p == 1 else 600
    n = signed_modes(N).astype(np.float64)
    m = np.arange(-mmax, mmax + 1, dtype=np.float64)
    t = np.sinc((n[:, None] + N * m[None, :]) / N) ** (2 * p)
    E = t.sum(axis=1)
    O = (t * np.where(m % 2 == 0, 1.0, -1.0)[None, :]).sum(axis=1)
    EE = E[:, None, None] * E[None, :, None] * E[None, None, :]
    if not interlace:
        return EE
    OO = O[:, None, None] * O[None, :, None] * O[None, None, :]
    return 0.5 * (EE + OO)


# --------------------------------------------------------------------------------------
# mass assignment (Sec. 4.2, App. C)
# --------------------------------------------------------------------------------------


def grid_coords(xyz, N, L, shift=0.0):
    """u = x / H - shift in FP64, H = L / N."""
    H = L / N
    return np.asarray(xyz, dtype=np.float32).astype(np.float64) / H - shift


def home_cells(u, p):
    """Home node of each coordinate: floor(u) for CIC, floor(u + 1/2) for NGP and TSC."""
    if p == 2:
        return np.floor(u)
    return np.floor(u + 0.5)


def cell_keys(xyz, N, L, p, shift=0.0):
    """Linear index (hx N + hy) N + hz of each particle's home node (periodic)."""
    u = grid_coords(xyz, N, L, shift)
    h = home_cells(u, p).astype(np.int64) % N
    return (h[:, 0] * N + h[:, 1]) * N + h[:, 2]


def stable_cell_order(xyz, N, L, p):
    """Particle permutation sorted by home cell, ties kept in input order."""
    return np.argsort(cell_keys(xyz, N, L, p), kind="stable")


def _kernel_1d(d, s, p):
    """1D assignment weight of a particle at offset d from its home node onto node home+s."""
    if p == 1:
        return np.ones_like(d) if s == 0 else np.zeros_like(d)
    if p == 2:
        return {0: 1.0 - d, 1: d}.get(s, np.zeros_like(d))
    if p == 3:
        if s == -1:
            return 0.5 * (0.5 - d) ** 2
        if s == 0:
            return 0.75 - d * d
        if s == 1:
            return 0.5 * (0.5 + d) ** 2
        return np.zeros_like(d)
    raise ValueError(p)


def _offsets(p):
    return {1: (0,), 2: (0, 1), 3: (-1, 0, 1)}[p]


def assign(xyz, vals, N, L, p, shift=0.0):
    """Mesh m(c) = sum_i vals_i W_p(c - u_i), FP64, in particle order (complex vals allowed)."""
    vals = np.asarray(vals)
    u = grid_coords(xyz, N, L, shift)
    hf = home_cells(u, p)
    d = u - hf
    h = hf.astype(np.int64)
    cplx = np.iscomplexobj(vals)
    mesh_r = np.zeros(N ** 3, dtype=np.float64)
    mesh_i = np.zeros(N ** 3, dtype=np.float64) if cplx else None
    for sx in _offsets(p):
        wx = _kernel_1d(d[:, 0], sx, p)
        ix = (h[:, 0] + sx) % N
        for sy in _offsets(p):
            wy = _kernel_1d(d[:, 1], sy, p)
            iy = (h[:, 1] + sy) % N
            for sz in _offsets(p):
                wz = _kernel_1d(d[:, 2], sz, p)
                iz = (h[:, 2] + sz) % N
                idx = (ix * N + iy) * N + iz
                wt = wx * wy * wz
                mesh_r += np.bincount(idx, weights=wt * np.real(vals), minlength=N ** 3)
                if cplx:
                    mesh_i += np.bincount(idx, weights=wt * np.imag(vals), minlength=N ** 3)
    m = mesh_r.reshape(N, N, N)
    if cplx:
        m = m + 1j * mesh_i.reshape(N, N, N)
    return m


def spectrum(params, xyz, vals):
    """delta n|_FFT(k) / W_mass(k), interlaced if requested, zero on Nyquist planes."""
    N, L, p = params.N, params.L, params.mas
    D = np.fft.fftn(assign(xyz, vals, N, L, p, 0.0))
    if params.interlace:
        D2 = np.fft.fftn(assign(xyz, vals, N, L, p, 0.5))
        nx, ny, nz = mode_grids(N)
        D = 0.5 * (D + np.exp(-1j * np.pi * (nx + ny + nz) / N) * D2)
    D = D / mas_window(N, p)
    D[nyquist_mask(N)] = 0.0
    return D


# --------------------------------------------------------------------------------------
# catalogues -> spectra (Sec. 4.1, Eq. mean_n, dn, nlm, ShotNoise definitions)
# --------------------------------------------------------------------------------------


def object_weights(cat, P0):
    n = len(cat["xyz"])
    w = np.ones(n) if cat.get("w") is None else np.asarray(cat["w"], dtype=np.float32).astype(np.float64)
    if P0 and P0 > 0 and cat.get("nbar") is not None:
        nb = np.asarray(cat["nbar"], dtype=np.float32).astype(np.float64)
        w = w / (1.0 + nb * P0)
    return w


def los_yconj(params, xyz, L, M):
    """y_L^{M*}(x_hat) per object: the local line of sight from the observer, or the z axis."""
    n = len(xyz)
    if params.los == "global":
        if params.polar_axis != "z":
            raise ValueError("global LOS is the z axis")
        return np.full(n, 1.0 + 0j) if M == 0 else np.zeros(n, dtype=np.complex128)
    d = np.asarray(xyz, dtype=np.float32).astype(np.float64) - np.asarray(params.observer, dtype=np.float64)[None, :]
    return np.conj(_y(params, L, M, d[:, 0], d[:, 1], d[:, 2]))


@dataclass
class Spectra:
    """Fourier-space inputs of one estimator pass (data or window)."""
    D: dict          # (L, M) -> delta n_L^M(k)/W   (full grid)
    Nk: dict         # (L, M) -> N_L^M(k)/W
    Sbar: dict       # (L, M) -> Sbar_L^M
    I: float
    alpha: float | None
    kind: str        # 'data' or 'window'


def catalogue_spectra(params, gal, ran=None):
    """Spectra of the data pass and, if params.window, of the randoms-only window pass."""
    Ls = params.needed_L()
    wg = object_weights(gal, params.P0)
    wr = object_weights(ran, params.P0) if ran is not None else None
    if params.los == "local" and ran is None:
        raise ValueError("local line of sight needs a random catalogue")
    alpha = float(wg.sum() / wr.sum()) if ran is not None else None

    def per_cat(cat, w):
        D, Nk, S = {}, {}, {}
        for L in Ls:
            for M in range(-L, L + 1):
                if params.los == "global" and M != 0:
                    continue
                yc = los_yconj(params, cat["xyz"], L, M)
                if params.los == "global" and L > 0:
                    D[(L, M)], Nk[(L, M)], S[(L, M)] = D[(0, 0)], Nk[(0, 0)], S[(0, 0)]
                    continue
                D[(L, M)] = spectrum(params, cat["xyz"], w * yc)
                Nk[(L, M)] = spectrum(params, cat["xyz"], w * w * np.conj(yc))
                S[(L, M)] = complex(np.sum(w ** 3 * yc))
        return D, Nk, S

    Dg, Ng_, Sg = per_cat(gal, wg)
    if ran is not None:
        Dr, Nr, Sr = per_cat(ran, wr)
        D = {k: Dg[k] - alpha * Dr[k] for k in Dg}
        Nk = {k: Ng_[k] + alpha ** 2 * Nr[k] for k in Ng_}
        S = {k: Sg[k] - alpha ** 3 * Sr[k] for k in Sg}
        R = assign(ran["xyz"], wr, params.N, params.L, params.mas, 0.0)
        I = alpha ** 3 * float(np.sum(R ** 3)) / params.H ** 6
    else:
        D, Nk, S = dict(Dg), dict(Ng_), dict(Sg)
        I = float(wg.sum()) ** 3 / params.V ** 2
    for k in D:
        D[k] = D[k].copy()
        D[k][0, 0, 0] = 0.0
    out = {"data": Spectra(D, Nk, S, I, alpha, "data")}
    if params.window:
        if ran is None:
            raise ValueError("window needs randoms")
        out["window"] = Spectra({k: alpha * v for k, v in Dr.items()},
                                {k: alpha ** 2 * v for k, v in Nr.items()},
                                {k: alpha ** 3 * v for k, v in Sr.items()}, I, alpha, "window")
    return out


# --------------------------------------------------------------------------------------
# estimator, FFT mode (Eq. bi_estimator_FFTs, Eq. nlm_bi)
# --------------------------------------------------------------------------------------


def _k_harmonic(params, l, m):
    """conj(y_l^m(k_hat)) on the full grid."""
    nx, ny, nz = mode_grids(params.N)
    shape = (params.N,) * 3
    return np.conj(_y(params, l, m, np.broadcast_to(nx, shape), np.broadcast_to(ny, shape),
                      np.broadcast_to(nz, shape)))


def _m_terms(l1, l2, L, global_los):
    """(m1, m2, M, 3j) with m1 + m2 + M = 0 and a non-zero 3j symbol."""
    out = []
    for m1 in range(-l1, l1 + 1):
        for m2 in range(-l2, l2 + 1):
            M = -m1 - m2
            if abs(M) > L or (global_los and M != 0):
                continue
            c = wigner3j(l1, l2, L, m1, m2, M)
            if c != 0.0:
                out.append((m1, m2, M, c))
    return out


class FieldCache:
    """F_l^m(x; b) (or unit-shell U fields when D is None) computed on demand."""

    def __init__(self, params, D00):
        self.p = params
        self.D = D00
        self.bins = bin_grid(params)
        self.nmodes = np.bincount(self.bins[self.bins >= 0].ravel(), minlength=len(params.edges) - 1)
        self.cache = {}
        self.harm = {}

    def harmonic(self, l, m):
        if (l, m) not in self.harm:
            self.harm[(l, m)] = _k_harmonic(self.p, l, m)
        return self.harm[(l, m)]

    def get(self, l, m, b):
        key = (l, m, b)
        if key not in self.cache:
            mask = self.bins == b
            spec = self.harmonic(l, m) * mask
            if self.D is not None:
                spec = spec * self.D
            nm = self.nmodes[b]
            self.cache[key] = self.p.Ng * np.fft.ifftn(spec) / nm if nm > 0 else np.zeros_like(spec)
        return self.cache[key]


def g_field(params, spec_LM):
    """G_L^M(x) = int d^3k/(2pi)^3 e^{ikx} delta n_L^M(k)/W  ->  (Ng/V) ifft."""
    return params.Ng / params.V * np.fft.ifftn(spec_LM)


def _pairs(nb, pairs):
    return [(b1, b2) for b1 in range(nb) for b2 in range(nb)] if pairs is None else list(pairs)


def bispectrum_raw_fft(params, spec, pairs=None):
    """hat B_{l1 l2 L}(k1, k2) before shot-noise subtraction (Eq. bi_estimator_FFTs).

    Returns array [n_mult, nb, nb] (NaN where a pair was not requested)."""
    nb = len(params.edges) - 1
    out = np.full((len(params.ells), nb, nb), np.nan)
    fc = FieldCache(params, spec.D[(0, 0)])
    G = {}
    glob = params.los == "global"
    for im, (l1, l2, L) in enumerate(params.ells):
        pref = n_lll(l1, l2, L) * h_lll(l1, l2, L) / spec.I
        terms = _m_terms(l1, l2, L, glob)
        for (b1, b2) in _pairs(nb, pairs):
            acc = 0.0 + 0.0j
            for m1, m2, M, c3 in terms:
                key = (L, M)
                if key not in G:
                    G[key] = g_field(params, spec.D[key])
                acc += c3 * params.V / params.Ng * np.sum(fc.get(l1, m1, b1) * fc.get(l2, m2, b2) * G[key])
            out[im, b1, b2] = pref * acc.real
    return out


# --------------------------------------------------------------------------------------
# shot noise (Eq. shotnoise, Eq. ShotNoise; discrete reading)
# --------------------------------------------------------------------------------------


def shell_average_y(params, fc, l, m, b):
    """Y = (1/N_mode) sum_{k in shell} y_l^{m*}(k_hat)."""
    nm = fc.nmodes[b]
    return complex(np.sum(fc.harmonic(l, m)[fc.bins == b]) / nm) if nm else 0.0


def cw2(params):
    """C_shot(k) / W_mass(k)^2 on the full grid, zero on Nyquist planes."""
    v = c_shot(params.N, params.mas, params.interlace) / mas_window(params.N, params.mas) ** 2
    v[nyquist_mask(params.N)] = 0.0
    return v


def shell_average_z(params, spec, fc, l, m, L, M, b, cw=None):
    """Z = (1/N_mode) sum_{k in shell} y_l^{m*}(k_hat) [D(k) N_L^{M*}(k) - Sbar_L^M C/W^2]."""
    nm = fc.nmodes[b]
    if not nm:
        return 0.0
    if cw is None:
        cw = cw2(params)
    mask = fc.bins == b
    val = spec.D[(0, 0)] * np.conj(spec.Nk[(L, M)]) - spec.Sbar[(L, M)] * cw
    return complex(np.sum((fc.harmonic(l, m) * val)[mask]) / nm)


def q_spectrum(params, spec, L, M, cw=None):
    """Q_L^M(k) = delta n_L^M(k) N_0^{0*}(k) - Sbar_L^M C(k)/W^2(k), zero on Nyquist planes."""
    if cw is None:
        cw = cw2(params)
    q = spec.D[(L, M)] * np.conj(spec.Nk[(0, 0)]) - spec.Sbar[(L, M)] * cw
    q[nyquist_mask(params.N)] = 0.0
    return q


def shot_noise_fft(params, spec, pairs=None, parts=False):
    """Sum of the four shot-noise terms for every multipole and requested pair."""
    nb = len(params.edges) - 1
    out = np.full((len(params.ells), nb, nb), np.nan)
    comp = {k: np.full((len(params.ells), nb, nb), np.nan) for k in ("iii", "ijj", "iji", "iij")}
    uc = FieldCache(params, None)
    cw = cw2(params)
    qf = {}
    glob = params.los == "global"
    for im, (l1, l2, L) in enumerate(params.ells):
        pref = n_lll(l1, l2, L) * h_lll(l1, l2, L) / spec.I
        terms = _m_terms(l1, l2, L, glob)
        for (b1, b2) in _pairs(nb, pairs):
            t = {k: 0.0 + 0.0j for k in comp}
            for m1, m2, M, c3 in terms:
                Y1 = shell_average_y(params, uc, l1, m1, b1)
                Y2 = shell_average_y(params, uc, l2, m2, b2)
                t["iii"] += c3 * spec.Sbar[(L, M)] * Y1 * Y2
                t["ijj"] += c3 * shell_average_z(params, spec, uc, l1, m1, L, M, b1, cw) * Y2
                t["iji"] += c3 * Y1 * shell_average_z(params, spec, uc, l2, m2, L, M, b2, cw)
                if (L, M) not in qf:
                    qf[(L, M)] = params.Ng * np.fft.ifftn(q_spectrum(params, spec, L, M, cw))
                t["iij"] += c3 / params.Ng * np.sum(uc.get(l1, m1, b1) * uc.get(l2, m2, b2) * qf[(L, M)])
            tot = 0.0
            for k in comp:
                comp[k][im, b1, b2] = pref * t[k].real
                tot += pref * t[k].real
            out[im, b1, b2] = tot
    return (out, comp) if parts else out


def measure(params, gal, ran=None, pairs=None):
    """Full oracle: {'B', 'shot', 'raw', 'nmodes', and 'window', 'window_shot' if requested}."""
    for (l1, l2, L) in params.ells:
        if not (allowed_multipole(l1, l2, L) or (params.ells_all_orders and allowed_multipole(l2, l1, L))):
            raise ValueError(f"multipole {(l1, l2, L)} violates the selection rules")
    specs = catalogue_spectra(params, gal, ran)
    res = {}
    sd = specs["data"]
    raw = bispectrum_raw_fft(params, sd, pairs)
    shot = shot_noise_fft(params, sd, pairs)
    res.update(raw=raw, shot=shot, B=raw - shot, I=sd.I, alpha=sd.alpha)
    if "window" in specs:
        sw = specs["window"]
        wraw = bispectrum_raw_fft(params, sw, pairs)
        wshot = shot_noise_fft(params, sw, pairs)
        res.update(window_raw=wraw, window_shot=wshot, window=wraw - wshot)
    fc = FieldCache(params, None)
    res["nmodes"] = fc.nmodes.astype(np.float64)
    return res


# --------------------------------------------------------------------------------------
# direct mode: the triangle sum of Eq. bi_estimator with k3 = -k1-k2 (mod N)
# --------------------------------------------------------------------------------------


class MeshSpectrumAccess:
    """Spectra looked up on the FFT grid, k3 wrapped mod N (the discrete identity of the FFT form)."""

    def __init__(self, params, spec):
        self.p, self.s = params, spec
        self.cw = cw2(params)

    def _idx(self, n):
        N = self.p.N
        n = np.asarray(n) % N
        return n[..., 0], n[..., 1], n[..., 2]

    def D(self, L, M, n):
        return self.s.D[(L, M)][self._idx(n)]

    def N(self, L, M, n):
        return self.s.Nk[(L, M)][self._idx(n)]

    def cw2(self, n):
        return self.cw[self._idx(n)]

    def Sbar(self, L, M):
        return self.s.Sbar[(L, M)]

    def q(self, L, M, n):
        return self.D(L, M, n) * np.conj(self.N(0, 0, n)) - self.Sbar(L, M) * self.cw2(n)


def _yk(params, l, m, n):
    n = np.asarray(n, dtype=np.float64)
    return np.conj(_y(params, l, m, n[..., 0], n[..., 1], n[..., 2]))


def bispectrum_raw_direct(params, acc, I, l1, l2, L, b1, b2, modes1, modes2, kernel="D"):
    """(N H / I) sum_m 3j (1/(Nm1 Nm2)) sum_{k1,k2} y1* y2* X(k1) X(k2) D_L^M(-k1-k2).

    kernel='D' gives hat B; kernel='Q' gives the i=j!=k shot term (X = 1, Q instead of D)."""
    glob = params.los == "global"
    tot = 0.0 + 0.0j
    n1 = np.asarray(modes1)
    n2 = np.asarray(modes2)
    for m1, m2, M, c3 in _m_terms(l1, l2, L, glob):
        y1 = _yk(params, l1, m1, n1)
        y2 = _yk(params, l2, m2, n2)
        if kernel == "D":
            a1 = y1 * acc.D(0, 0, n1)
            a2 = y2 * acc.D(0, 0, n2)
        else:
            a1, a2 = y1, y2
        s = 0.0 + 0.0j
        for i in range(len(n1)):
            n3 = -(n1[i][None, :] + n2)
            g = acc.D(L, M, n3) if kernel == "D" else acc.q(L, M, n3)
            s += a1[i] * np.sum(a2 * g)
        tot += c3 * s / (len(n1) * len(n2))
    return n_lll(l1, l2, L) * h_lll(l1, l2, L) / I * tot.real


def shot_noise_direct(params, acc, I, l1, l2, L, modes1, modes2):
    """The four shot-noise terms from shell sums (i=j=k, i!=j=k, i=k!=j) and the triangle
    sum (i=j!=k), written with an arbitrary spectrum accessor."""
    glob = params.los == "global"
    n1 = np.asarray(modes1)
    n2 = np.asarray(modes2)
    t = {"iii": 0j, "ijj": 0j, "iji": 0j}
    for m1, m2, M, c3 in _m_terms(l1, l2, L, glob):
        y1 = _yk(params, l1, m1, n1)
        y2 = _yk(params, l2, m2, n2)
        Y1, Y2 = y1.mean(), y2.mean()
        S = acc.Sbar(L, M)
        Z1 = np.mean(y1 * (acc.D(0, 0, n1) * np.conj(acc.N(L, M, n1)) - S * acc.cw2(n1)))
        Z2 = np.mean(y2 * (acc.D(0, 0, n2) * np.conj(acc.N(L, M, n2)) - S * acc.cw2(n2)))
        t["iii"] += c3 * S * Y1 * Y2
        t["ijj"] += c3 * Z1 * Y2
        t["iji"] += c3 * Y1 * Z2
    pref = n_lll(l1, l2, L) * h_lll(l1, l2, L) / I
    out = {k: pref * v.real for k, v in t.items()}
    out["iij"] = bispectrum_raw_direct(params, acc, I, l1, l2, L, None, None, n1, n2, kernel="Q")
    return out


# --------------------------------------------------------------------------------------
# particle-exact mode: exact DFTs of a few particles, W = C = 1
# --------------------------------------------------------------------------------------


class ExactSpectrumAccess:
    """delta n_L^M(k), N_L^M(k) as exact sums over particles at unwrapped integer k."""

    def __init__(self, params, gal, ran, alpha):
        self.p = params
        self.kF = 2.0 * np.pi / params.L
        pos, s, w = [np.asarray(gal["xyz"], np.float64)], [np.ones(len(gal["xyz"]))], [object_weights(gal, params.P0)]
        if ran is not None:
            pos.append(np.asarray(ran["xyz"], np.float64))
            s.append(np.full(len(ran["xyz"]), -alpha))
            w.append(object_weights(ran, params.P0))
        self.x = np.concatenate(pos)
        self.s = np.concatenate(s)
        self.w = np.concatenate(w)
        self.cache = {}

    def yc(self, L, M):
        if (L, M) not in self.cache:
            self.cache[(L, M)] = los_yconj(self.p, self.x, L, M)
        return self.cache[(L, M)]

    def _phase(self, n):
        n = np.asarray(n, dtype=np.float64)
        return np.exp(-1j * self.kF * (n @ self.x.T))  # (..., Np)

    def D(self, L, M, n):
        return self._phase(n) @ (self.s * self.w * self.yc(L, M))

    def N(self, L, M, n):
        return self._phase(n) @ (self.s ** 2 * self.w ** 2 * np.conj(self.yc(L, M)))

    def Sbar(self, L, M):
        return complex(np.sum(self.s ** 3 * self.w ** 3 * self.yc(L, M)))

    def cw2(self, n):
        return np.ones(np.asarray(n).shape[:-1])

    def q(self, L, M, n):
        return self.D(L, M, n) * np.conj(self.N(0, 0, n)) - self.Sbar(L, M)


def distinct_triplet_sum(params, acc, I, l1, l2, L, modes1, modes2):
    """Brute force over distinct particle triplets i != j != k of the particle-form
    estimator (Sec. 4.2): sum s w s w s w y_L^{M*}(x_k) A1(x_i - x_k) A2(x_j - x_k)."""
    glob = params.los == "global"
    n1 = np.asarray(modes1, dtype=np.float64)
    n2 = np.asarray(modes2, dtype=np.float64)
    x, sw = acc.x, acc.s * acc.w
    dx = x[:, None, :] - x[None, :, :]  # x_i - x_k
    npart = len(x)
    mask = np.ones((npart, npart, npart), dtype=bool)
    ii = np.arange(npart)
    mask[ii, ii, :] = False
    mask[ii, :, ii] = False
    mask[:, ii, ii] = False
    tot = 0j
    for m1, m2, M, c3 in _m_terms(l1, l2, L, glob):
        y1 = _yk(params, l1, m1, n1)
        y2 = _yk(params, l2, m2, n2)
        A1 = np.exp(-1j * acc.kF * np.einsum("ikd,nd->ikn", dx, n1)) @ y1 / len(n1)
        A2 = np.exp(-1j * acc.kF * np.einsum("ikd,nd->ikn", dx, n2)) @ y2 / len(n2)
        c = sw * acc.yc(L, M)
        T = (sw[:, None, None] * A1[:, None, :]) * (sw[None, :, None] * A2[None, :, :]) * c[None, None, :]
        tot += c3 * np.sum(T[mask])
    return n_lll(l1, l2, L) * h_lll(l1, l2, L) / I * tot.real
