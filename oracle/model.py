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
