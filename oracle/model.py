"""FP64 oracle of the window-convolved model (Sec. 6.2): the Wigner 9j symbol, the masked
three-point multipoles (Eq. zetaMask) with the integral constraint (Eq. IC), and the Hankel
transforms between three-point and bispectrum multipoles (Eq. HankelTransform,
Eq. masked_bispectrum).

TEST INFRASTRUCTURE ONLY.  Plain sums over the definitions; shares no code with the library.
Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may import it.

* the 9j symbol from the five-3j identity of App. A (Eq. Wigner9j), solved for the 9j with one
  choice of (m1, m2, m3) whose 3j symbol is not zero;
* the masked model sums the printed formula over the theory multipoles l' and the window
  multipoles l'' it is given; the integral constraint is Eq. IC over the multipoles present in
  both sets; the radial integrals are sums with caller-given weights w (int dr r^2 f ~ sum_i w_i
  r_i^2 f(r_i));
* the spherical Bessel functions are scipy's (a library primitive).
"""
from __future__ import annotations

import itertools

import numpy as np
from scipy.special import spherical_jn

from .sph import h_lll, n_lll, wigner3j


def wigner9j(j):
    """{j1 j2 j3; j4 j5 j6; j7 j8 j9} from Eq. Wigner9j (integer j).  The projections of the five
    3j symbols on its left are fixed by (m1, m2, m3), m7 and m5 through their zero sums."""
    l1, l2, l3, l4, l5, l6, l7, l8, l9 = (int(v) for v in j)
    best = (0.0, 0, 0)
    for m1, m2 in itertools.product(range(-l1, l1 + 1), range(-l2, l2 + 1)):
        if abs(m1 + m2) <= l3:
            c = wigner3j(l1, l2, l3, m1, m2, -m1 - m2)
            if abs(c) > abs(best[0]):
                best = (c, m1, m2)
    c, m1, m2 = best
    if c == 0.0:
        return 0.0  # (l1, l2, l3) violates the triangle rule
    m3 = -m1 - m2
    tot = 0.0
    for m7 in range(-l7, l7 + 1):
        m4 = m1 - m7          # (l4 l1 l7; m4 -m1 m7)
        if abs(m4) > l4:
            continue
        a = wigner3j(l4, l1, l7, m4, -m1, m7)
        if a == 0.0:
            continue
        for m5 in range(-l5, l5 + 1):
            m6 = -m5 - m4     # (l5 l4 l6; -m5 -m4 -m6)
            m9 = m3 - m6      # (l6 l3 l9; m6 -m3 m9)
            m8 = -m7 - m9     # (l7 l9 l8; -m7 -m9 -m8)
            if abs(m6) > l6 or abs(m9) > l9 or abs(m8) > l8 or m8 - m2 + m5 != 0:
                continue
            t = (a * wigner3j(l5, l4, l6, -m5, -m4, -m6) * wigner3j(l6, l3, l9, m6, -m3, m9)
                 * wigner3j(l7, l9, l8, -m7, -m9, -m8) * wigner3j(l8, l2, l5, m8, -m2, m5))
            ph = (-1) ** ((l4 - m4) + (l5 - m5) + (l6 - m6) + (l7 - m7) + (l8 - m8) + (l9 - m9))
            tot += ph * t
    return tot / ((-1) ** (l2 + l5 + l8) * c)


def masked_coefficient(ell, ellp, ellpp):
    """Coefficient of Q_{l''} zeta_{l'} in <zeta_l>_model (Eq. zetaMask)."""
    l1, l2, L = ell
    a1, a2, A = ellp
    b1, b2, B = ellpp
    den = h_lll(a1, a2, A) * h_lll(b1, b2, B)
    if den == 0.0:
        return 0.0
    num = h_lll(l1, l2, L) * h_lll(l1, a1, b1) * h_lll(l2, a2, b2) * h_lll(L, A, B)
    if num == 0.0:
        return 0.0
    return n_lll(l1, l2, L) * wigner9j((b1, b2, B, a1, a2, A, l1, l2, L)) * num / den


def integral_constraint(theory, window, w_r):
    """zeta_bar of Eq. IC; theory, window: dict l -> [nr, nr] arrays; w_r: weights w_i r_i^2."""
    W = np.outer(w_r, w_r)
    num = 0.0
    for ell, z in theory.items():
        if ell in window:
            num += np.sum(W * window[ell] * z) / (h_lll(*ell) ** 2 * n_lll(*ell))
    return num / np.sum(W * window[(0, 0, 0)])


def masked_zeta(ells_out, theory, window, w_r, ic=True):
    """<zeta_l>_model for every l in ells_out (Eq. zetaMask), and zeta_bar."""
    zb = integral_constraint(theory, window, w_r) if ic else 0.0
    out = {}
    for ell in ells_out:
        acc = 0.0
        for lp, z in theory.items():
            for lpp, q in window.items():
                c = masked_coefficient(ell, lp, lpp)
                if c != 0.0:
                    acc = acc + c * q * z
        if ell in window:
            acc = acc - window[ell] * zb
        out[ell] = acc
    return out, zb


def zeta_to_bk(l1, l2, r, w, zeta, k1, k2):
    """B(k1, k2) = (-i)^{l1+l2} (4 pi)^2 sum_ij w_i r_i^2 w_j r_j^2 j_l1(k1 r_i) j_l2(k2 r_j) zeta_ij
    (Eq. masked_bispectrum; l1 + l2 even, so the factor is real)."""
    ph = (-1) ** ((l1 + l2) // 2)
    J1 = spherical_jn(l1, np.outer(k1, r)) * (w * r * r)[None, :]
    J2 = spherical_jn(l2, np.outer(k2, r)) * (w * r * r)[None, :]
    return ph * (4 * np.pi) ** 2 * J1 @ zeta @ J2.T


def bk_to_zeta(l1, l2, k, wk, B, r1, r2):
    """zeta(r1, r2) = i^{l1+l2} sum_ij wk_i k_i^2/(2 pi^2) wk_j k_j^2/(2 pi^2) j_l1(r1 k_i) j_l2(r2 k_j) B_ij
    (Eq. HankelTransform)."""
    ph = (-1) ** ((l1 + l2) // 2)
    J1 = spherical_jn(l1, np.outer(r1, k)) * (wk * k * k / (2 * np.pi ** 2))[None, :]
    J2 = spherical_jn(l2, np.outer(r2, k)) * (wk * k * k / (2 * np.pi ** 2))[None, :]
    return ph * J1 @ B @ J2.T


# --------------------------------------------------------------------------------------
# tree-level bispectrum multipoles (App. F)
# --------------------------------------------------------------------------------------


def power_loglog(k_tab, p_tab):
    """P(k) by log-log interpolation of a table (a power law is reproduced exactly)."""
    lk, lp = np.log(np.asarray(k_tab, float)), np.log(np.asarray(p_tab, float))
    return lambda k: np.exp(np.interp(np.log(k), lk, lp))


def tree_bispectrum(P, b1, b2, f, k1v, k2v, n=(0.0, 0.0, 1.0)):
    """B(k1, k2, k3 = -k1 - k2; n) = 2 Z2(k1, k2) Z1(k1) Z1(k2) P1 P2 + cyc. (App. F) for arrays of
    wave vectors [..., 3]."""
    n = np.asarray(n, float)
    k3v = -(k1v + k2v)

    def Z1(kv):
        k = np.linalg.norm(kv, axis=-1)
        mu = (kv @ n) / k
        return b1 + f * mu * mu

    def Z2(av, bv):
        a = np.linalg.norm(av, axis=-1)
        b = np.linalg.norm(bv, axis=-1)
        mab = np.sum(av * bv, axis=-1) / (a * b)
        F2 = 5.0 / 7.0 + 0.5 * mab * (a / b + b / a) + 2.0 / 7.0 * mab * mab
        G2 = 3.0 / 7.0 + 0.5 * mab * (a / b + b / a) + 4.0 / 7.0 * mab * mab
        kv = av + bv
        k = np.linalg.norm(kv, axis=-1)
        mu = np.where(k > 0, (kv @ n) / np.where(k > 0, k, 1.0), 0.0)
        mua, mub = (av @ n) / a, (bv @ n) / b
        return (b1 * F2 + 0.5 * b2 + f * mu * mu * G2
                + 0.5 * f * mu * k * (mua / a * Z1(bv) + mub / b * Z1(av)))

    def term(av, bv):
        return 2.0 * Z2(av, bv) * Z1(av) * Z1(bv) * P(np.linalg.norm(av, axis=-1)) * P(np.linalg.norm(bv, axis=-1))

    return term(k1v, k2v) + term(k2v, k3v) + term(k3v, k1v)


def tree_multipole(P, b1, b2, f, ell, k1, k2, n_mu=24, n_phi=48, n=(0.0, 0.0, 1.0)):
    """B_{l1 l2 L}(k1, k2) = N H sum_m 3j int d^2k1/4pi int d^2k2/4pi y_l1^{m1*} y_l2^{m2*} y_L^{M*}(n)
    B(k1, k2; n) (Eq. reduced_ones with the expansion of Eq. TripoSH_J0), over both directions on a
    Gauss-Legendre x uniform grid for one line of sight n (the integrand is rotation invariant, so
    any n gives the same multipole)."""
    from .sph import ylm
    l1, l2, L = ell
    mu, wmu = np.polynomial.legendre.leggauss(n_mu)
    ph = 2 * np.pi * (np.arange(n_phi) + 0.5) / n_phi
    MU1, PH1, MU2, PH2 = np.meshgrid(mu, ph, mu, ph, indexing="ij")
    W = (wmu[:, None, None, None] * wmu[None, None, :, None]) / (4.0 * n_phi * n_phi)
    s1, s2 = np.sqrt(1 - MU1 ** 2), np.sqrt(1 - MU2 ** 2)
    u1 = np.stack([s1 * np.cos(PH1), s1 * np.sin(PH1), MU1], axis=-1)
    u2 = np.stack([s2 * np.cos(PH2), s2 * np.sin(PH2), MU2], axis=-1)
    n = np.asarray(n, float) / np.linalg.norm(n)
    B = tree_bispectrum(P, b1, b2, f, k1 * u1, k2 * u2, n)
    tot = 0.0 + 0.0j
    for m1 in range(-l1, l1 + 1):
        for m2 in range(-l2, l2 + 1):
            M = -m1 - m2
            if abs(M) > L:
                continue
            c = wigner3j(l1, l2, L, m1, m2, M)
            if c == 0.0:
                continue
            yM = np.conj(ylm(L, M, n[0], n[1], n[2]))
            if yM == 0:
                continue
            y1 = np.conj(ylm(l1, m1, u1[..., 0], u1[..., 1], u1[..., 2]))
            y2 = np.conj(ylm(l2, m2, u2[..., 0], u2[..., 1], u2[..., 2]))
            tot += c * yM * np.sum(W * y1 * y2 * B)
    return n_lll(l1, l2, L) * h_lll(l1, l2, L) * tot.real
