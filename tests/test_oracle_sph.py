"""Pins of the oracle's angular algebra (3j symbols, y_l^m) against closed forms,
identities of App. A and the tables the paper prints."""
import os
from math import sqrt

import numpy as np
import pytest

from oracle.estimator import _m_terms
from oracle.sph import allowed_multipole, legendre, wigner3j, ylm

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    with open(os.path.join(GOLD, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


def test_wigner3j_closed_forms():
    for r in _rows("wigner3j_closed_forms.txt"):
        j = list(map(int, r[:6]))
        want = eval(r[6], {"sqrt": sqrt})
        assert wigner3j(*j) == pytest.approx(want, rel=1e-14, abs=1e-15)


@pytest.mark.parametrize("j1,j2", [(1, 1), (2, 0), (2, 2), (3, 1), (4, 2)])
def test_wigner3j_orthogonality(j1, j2):
    # sum_{m1 m2} (2j3+1) 3j(j1 j2 j3; m1 m2 m3) 3j(j1 j2 j3'; m1 m2 m3') = delta delta
    for j3 in range(abs(j1 - j2), j1 + j2 + 1):
        for j3p in range(abs(j1 - j2), j1 + j2 + 1):
            for m3 in range(-min(j3, j3p), min(j3, j3p) + 1):
                s = sum(wigner3j(j1, j2, j3, m1, m2, m3) * wigner3j(j1, j2, j3p, m1, m2, m3)
                        for m1 in range(-j1, j1 + 1) for m2 in range(-j2, j2 + 1))
                want = 1.0 / (2 * j3 + 1) if j3 == j3p else 0.0
                assert s == pytest.approx(want, abs=1e-14)


def test_wigner3j_symmetries():
    rng = np.random.default_rng(0)
    for _ in range(50):
        j1, j2 = rng.integers(0, 5, 2)
        j3 = rng.integers(abs(j1 - j2), j1 + j2 + 1)
        m1 = rng.integers(-j1, j1 + 1)
        m2 = rng.integers(-j2, j2 + 1)
        m3 = -m1 - m2
        if abs(m3) > j3:
            continue
        v = wigner3j(j1, j2, j3, m1, m2, m3)
        sgn = (-1) ** int(j1 + j2 + j3)
        assert wigner3j(j2, j1, j3, m2, m1, m3) == pytest.approx(sgn * v, abs=1e-15)
        assert wigner3j(j1, j2, j3, -m1, -m2, -m3) == pytest.approx(sgn * v, abs=1e-15)
        assert wigner3j(j2, j3, j1, m2, m3, m1) == pytest.approx(v, abs=1e-15)


def _dirs(n=200, seed=1):
    v = np.random.default_rng(seed).standard_normal((n, 3))
    return v[:, 0], v[:, 1], v[:, 2]


def test_ylm_low_orders():
    x, y, z = _dirs()
    r = np.sqrt(x * x + y * y + z * z)
    mu = z / r
    assert np.allclose(ylm(0, 0, x, y, z), 1.0)
    assert np.allclose(ylm(1, 0, x, y, z), mu, atol=1e-15)
    assert np.allclose(ylm(2, 0, x, y, z), 0.5 * (3 * mu * mu - 1), atol=1e-15)
    # y_1^1 = -sqrt(1/2) (x + i y)/r with the Condon-Shortley phase
    assert np.allclose(ylm(1, 1, x, y, z), -np.sqrt(0.5) * (x + 1j * y) / r, atol=1e-15)
    # y_2^2 = sqrt(3/8) ((x + i y)/r)^2
    assert np.allclose(ylm(2, 2, x, y, z), np.sqrt(3.0 / 8.0) * ((x + 1j * y) / r) ** 2, atol=1e-15)


@pytest.mark.parametrize("l", [0, 1, 2, 3, 4, 6])
def test_ylm_unit_sum_and_conjugation(l):
    x, y, z = _dirs()
    s = sum(np.abs(ylm(l, m, x, y, z)) ** 2 for m in range(-l, l + 1))
    assert np.allclose(s, 1.0, atol=1e-13)
    for m in range(1, l + 1):
        assert np.allclose(ylm(l, -m, x, y, z), (-1) ** m * np.conj(ylm(l, m, x, y, z)), atol=1e-14)
    # parity y(-n) = (-1)^l y(n)
    for m in range(-l, l + 1):
        assert np.allclose(ylm(l, m, -x, -y, -z), (-1) ** l * ylm(l, m, x, y, z), atol=1e-14)


@pytest.mark.parametrize("l", [1, 2, 3, 4])
def test_addition_theorem(l):
    # App. A, Eq. LYlm: L_l(x.y) = sum_m y_l^m(x) y_l^{m*}(y)
    a = _dirs(100, 2)
    b = _dirs(100, 3)
    na = np.sqrt(a[0] ** 2 + a[1] ** 2 + a[2] ** 2)
    nb = np.sqrt(b[0] ** 2 + b[1] ** 2 + b[2] ** 2)
    cosg = (a[0] * b[0] + a[1] * b[1] + a[2] * b[2]) / (na * nb)
    s = sum(ylm(l, m, *a) * np.conj(ylm(l, m, *b)) for m in range(-l, l + 1))
    assert np.allclose(s, legendre(l, cosg), atol=1e-13)


def test_ylm_orthogonality_quadrature():
    # int dOmega/4pi y_l^m y_l'^m'* = delta/(2l+1), Gauss-Legendre x uniform phi (exact for l <= 8)
    mu, wmu = np.polynomial.legendre.leggauss(12)
    phi = np.arange(24) * 2 * np.pi / 24
    MU, PHI = np.meshgrid(mu, phi, indexing="ij")
    W = (wmu[:, None] / 2.0) * np.full_like(PHI, 1.0 / 24)
    s = np.sqrt(1 - MU ** 2)
    x, y, z = s * np.cos(PHI), s * np.sin(PHI), MU
    for l in range(0, 5):
        for lp in range(0, 5):
            for m in range(-l, l + 1):
                for mp in range(-lp, lp + 1):
                    v = np.sum(W * ylm(l, m, x, y, z) * np.conj(ylm(lp, mp, x, y, z)))
                    want = 1.0 / (2 * l + 1) if (l, m) == (lp, mp) else 0.0
                    assert abs(v - want) < 1e-13


def test_table1_allowed_multipoles():
    rows = _rows("paper_table1_allowed_multipoles.txt")
    for L, l1, l2 in (map(int, r) for r in rows):
        assert allowed_multipole(l1, l2, L)
    # the table lists, per L, the first combinations in order of l1 + l2; check that the
    # selection rules admit nothing with a smaller l1 + l2 that the table skips
    for L in (0, 2, 4):
        listed = {(int(r[1]), int(r[2])) for r in rows if int(r[0]) == L}
        top = max(a + b for a, b in listed)
        for l1 in range(0, 8):
            for l2 in range(0, l1 + 1):
                if l1 + l2 < top and allowed_multipole(l1, l2, L):
                    assert (l1, l2) in listed, (L, l1, l2)
    assert not allowed_multipole(1, 0, 1)
    assert not allowed_multipole(0, 2, 2)  # l1 >= l2
    assert not allowed_multipole(2, 1, 2)  # l1 + l2 + L odd
    assert not allowed_multipole(3, 0, 2)  # triangle rule


def test_nmultipole_cost_table():
    # number of non-zero (m1, m2, M) terms = the paper's N_multipole (mock: local, box: global)
    for r in _rows("paper_nmultipole_cost.txt"):
        l1, l2, L, mock, box = map(int, r)
        assert len(_m_terms(l1, l2, L, False)) == mock
        assert len(_m_terms(l1, l2, L, True)) == box
