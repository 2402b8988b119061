"""Angular algebra of the FP64 oracle: Wigner 3j symbols and normalised spherical harmonics.

TEST INFRASTRUCTURE ONLY: this package is the slow, plain reference that the CUDA
path is checked against.  Only tests/, __graft_entry__.smoke() and bench.py's CPU
baseline leg may import it; the product never does.

Paper conventions (Sec. 2, App. A):
* y_l^m = sqrt(4 pi / (2l+1)) Y_l^m, so y_0^0 = 1 (App. A, Eq. YL);
* N_{l1 l2 L} = (2l1+1)(2l2+1)(2L+1) and H_{l1 l2 L} = 3j(l1 l2 L; 0 0 0) (Sec. 2,
  Eq. SH_coefficients and Eq. reduced_ones).

Reading: the associated Legendre functions carry the Condon-Shortley phase.  Every
estimator term contains y_{l1}^{m1} y_{l2}^{m2} y_L^M with m1+m2+M = 0, so the choice
of phase cancels (a test flips it).
"""
from __future__ import annotations

from fractions import Fraction
from math import factorial, sqrt

import numpy as np


def wigner3j(j1, j2, j3, m1, m2, m3):
    """Wigner 3j symbol (j1 j2 j3; m1 m2 m3) for integer arguments, Racah's closed form.

    Evaluated with exact rational arithmetic; one square root at the end.
    """
    if m1 + m2 + m3 != 0:
        return 0.0
    if abs(m1) > j1 or abs(m2) > j2 or abs(m3) > j3:
        return 0.0
    if j3 < abs(j1 - j2) or j3 > j1 + j2:
        return 0.0
    f = factorial
    tri = Fraction(f(j1 + j2 - j3) * f(j1 - j2 + j3) * f(-j1 + j2 + j3), f(j1 + j2 + j3 + 1))
    pref2 = tri * f(j1 + m1) * f(j1 - m1) * f(j2 + m2) * f(j2 - m2) * f(j3 + m3) * f(j3 - m3)
    tmin = max(0, j2 - j3 - m1, j1 - j3 + m2)
    tmax = min(j1 + j2 - j3, j1 - m1, j2 + m2)
    s = Fraction(0)
    for t in range(tmin, tmax + 1):
        den = (f(t) * f(j3 - j2 + t + m1) * f(j3 - j1 + t - m2) * f(j1 + j2 - j3 - t)
               * f(j1 - t - m1) * f(j2 - t + m2))
        s += Fraction((-1) ** t, den)
    sign = -1.0 if (j1 - j2 - m3) % 2 else 1.0
    return sign * sqrt(float(pref2)) * float(s)


def n_lll(l1, l2, L):
    """N_{l1 l2 L} = (2l1+1)(2l2+1)(2L+1)."""
    return (2 * l1 + 1) * (2 * l2 + 1) * (2 * L + 1)


def h_lll(l1, l2, L):
    """H_{l1 l2 L} = 3j(l1 l2 L; 0 0 0)."""
    return wigner3j(l1, l2, L, 0, 0, 0)


def _legendre_deriv_coeffs(l, m):
    """Coefficients (highest power first) of d^m/dmu^m P_l(mu), P_l from Rodrigues' formula
    P_l(mu) = 1/(2^l l!) d^l/dmu^l (mu^2 - 1)^l."""
    base = np.polynomial.polynomial.polypow([-1.0, 0.0, 1.0], l)  # (mu^2-1)^l, low->high
    c = np.polynomial.polynomial.polyder(base, l + m) if l + m > 0 else base
    c = c / (2.0 ** l * factorial(l))
    return c  # low -> high


def ylm(l, m, x, y, z, condon_shortley=True):
    """Normalised spherical harmonic y_l^m of the direction (x, y, z) (need not be unit).

    y_l^m = sqrt((l-|m|)!/(l+|m|)!) P_l^{|m|}(mu) e^{i m phi} for m >= 0, with
    P_l^m(mu) = (-1)^m (1-mu^2)^{m/2} d^m P_l/dmu^m, and y_l^{-m} = (-1)^m conj(y_l^m)
    (App. A, Eq. YL).  (1-mu^2)^{m/2} e^{i m phi} is ((x + i y)/r)^m.
    Direction (0,0,0) returns 0 for l > 0 and 1 for l = 0.
    """
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    z = np.asarray(z, dtype=np.float64)
    r = np.sqrt(x * x + y * y + z * z)
    rs = np.where(r > 0, r, 1.0)
    mu = z / rs
    am = abs(m)
    if am > l:
        return np.zeros(np.broadcast(x, y, z).shape, dtype=np.complex128)
    c = _legendre_deriv_coeffs(l, am)
    poly = np.polynomial.polynomial.polyval(mu, c)
    phase = ((x + 1j * y) / rs) ** am
    norm = sqrt(factorial(l - am) / factorial(l + am))
    cs = (-1.0) ** am if condon_shortley else 1.0
    val = cs * norm * poly * phase
    if l > 0:
        val = np.where(r > 0, val, 0.0)
    if m < 0:
        val = (-1.0) ** am * np.conj(val)
    return val.astype(np.complex128)


def legendre(l, mu):
    """Legendre polynomial P_l(mu)."""
    return np.polynomial.polynomial.polyval(np.asarray(mu, dtype=np.float64), _legendre_deriv_coeffs(l, 0))


def allowed_multipole(l1, l2, L):
    """Selection rules of Table 1: l1 >= l2, L even, |l1-l2| <= L <= l1+l2, l1+l2+L even."""
    return (l1 >= l2 >= 0 and L % 2 == 0 and abs(l1 - l2) <= L <= l1 + l2 and (l1 + l2 + L) % 2 == 0)
