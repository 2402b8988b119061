"""Window-convolved model (Sec. 6.2): 9j symbols, masked three-point multipoles (Eq. zetaMask,
Eq. IC) and Hankel transforms (Eq. HankelTransform, Eq. masked_bispectrum).  The oracle against
library routines, printed values and closed forms; the host functions of the C ABI against the
oracle.  No GPU."""
import os
import itertools

import numpy as np
import pytest

import paper_1803_02132_gb300 as bisp
from oracle import model as Mo
from oracle.sph import h_lll, n_lll

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _tri(a, b, c):
    return abs(a - b) <= c <= a + b


def _nine(seed, n, jmax=4):
    """n random 9j arguments whose rows and columns all satisfy the triangle rule."""
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < n:
        m = rng.integers(0, jmax + 1, (3, 3))
        if all(_tri(*m[i]) for i in range(3)) and all(_tri(*m[:, i]) for i in range(3)):
            out.append(tuple(int(v) for v in m.reshape(-1)))
    return out


def test_oracle_9j_matches_sympy():
    wig = pytest.importorskip("sympy.physics.wigner")
    cases = _nine(1, 150) + [(1, 1, 0, 1, 1, 0, 0, 0, 0), (2, 2, 2, 2, 2, 2, 2, 2, 2), (2, 0, 2, 1, 1, 2, 1, 1, 0)]
    nz = 0
    for j in cases:
        ref = float(wig.wigner_9j(*j, prec=30))
        assert Mo.wigner9j(j) == pytest.approx(ref, abs=1e-14)
        nz += ref != 0.0
    assert nz >= 100


def test_oracle_9j_symmetries():
    for j in [(2, 1, 1, 1, 2, 1, 1, 1, 2), (2, 2, 2, 1, 2, 1, 1, 2, 1), (3, 2, 1, 2, 2, 2, 1, 2, 3)]:
        v = Mo.wigner9j(j)
        m = np.array(j).reshape(3, 3)
        assert Mo.wigner9j(m.T.reshape(-1)) == pytest.approx(v, abs=1e-14)  # transposition
        ph = (-1) ** int(m.sum())
        assert Mo.wigner9j(m[[1, 0, 2]].reshape(-1)) == pytest.approx(ph * v, abs=1e-14)  # odd row swap
        assert Mo.wigner9j(m[:, [0, 2, 1]].reshape(-1)) == pytest.approx(ph * v, abs=1e-14)  # odd column swap


def test_masked_coefficients_printed_in_the_paper():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "masked_monopole_coefficients.txt")) if l.strip() and l[0] != "#"]
    assert len(rows) == 3
    for r in rows:
        v = [int(x) for x in r]
        assert Mo.masked_coefficient(tuple(v[0:3]), tuple(v[3:6]), tuple(v[6:9])) == pytest.approx(v[9] / v[10], rel=1e-13)


def test_masked_coefficients_of_eq_maskzeta2():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "masked_zeta_coefficients_eq_maskzeta2.txt"))
            if l.strip() and l[0] != "#"]
    assert len(rows) == 14
    for r in rows:
        v = [int(x) for x in r]
        assert Mo.masked_coefficient(tuple(v[0:3]), tuple(v[3:6]), tuple(v[6:9])) == pytest.approx(v[9] / v[10], rel=1e-13)
    # terms the printed expressions do not contain (and that are not products of two L = 2 modes)
    assert Mo.masked_coefficient((2, 0, 2), (1, 1, 0), (1, 1, 0)) == pytest.approx(0.0, abs=1e-14)
    assert Mo.masked_coefficient((1, 1, 2), (1, 1, 0), (1, 1, 0)) == pytest.approx(0.0, abs=1e-14)
    assert Mo.masked_coefficient((1, 1, 0), (2, 0, 2), (0, 0, 0)) == pytest.approx(0.0, abs=1e-14)


def _grid(nr=24, rmax=150.0):
    r = np.linspace(rmax / nr, rmax, nr)
    w = np.full(nr, rmax / nr)
    return r, w


def _fields(seed, ells, nr):
    rng = np.random.default_rng(seed)
    return {e: rng.normal(size=(nr, nr)) + (3.0 if e == (0, 0, 0) else 0.0) for e in ells}


def test_isotropic_unit_window_is_the_identity():
    # only Q_000 (no anisotropic window): <zeta_l> = Q_000 zeta_l for every l, without the constraint
    r, w = _grid()
    ells = [(0, 0, 0), (1, 1, 0), (2, 0, 2), (1, 1, 2), (2, 2, 2)]
    th = _fields(2, ells, len(r))
    q0 = {(0, 0, 0): 0.5 + np.random.default_rng(3).random((len(r), len(r)))}
    out, zb = Mo.masked_zeta(ells, th, q0, w * r * r, ic=False)
    for e in ells:
        assert np.allclose(out[e], q0[(0, 0, 0)] * th[e], rtol=1e-12, atol=1e-14)


def test_integral_constraint_nulls_the_monopole_integral():
    # Eq. IC makes int dr1 r1^2 int dr2 r2^2 <zeta_000>_model = 0
    r, w = _grid()
    ells = [(0, 0, 0), (1, 1, 0), (2, 2, 0), (2, 0, 2), (1, 1, 2)]
    th = _fields(4, ells, len(r))
    win = _fields(5, ells + [(0, 2, 2), (2, 2, 2)], len(r))
    out, zb = Mo.masked_zeta([(0, 0, 0)], th, win, w * r * r)
    W = np.outer(w * r * r, w * r * r)
    assert abs(np.sum(W * out[(0, 0, 0)])) < 1e-10 * np.sum(W * np.abs(out[(0, 0, 0)]))
    assert zb != 0.0


@pytest.mark.parametrize("l1,l2", [(0, 0), (1, 1), (2, 0), (2, 2), (3, 1)])
def test_hankel_gaussian_closed_form(l1, l2):
    # int_0^inf dr r^(l+2) exp(-r^2/(2 s^2)) j_l(k r) = sqrt(pi/2) s^(2l+3) k^l exp(-k^2 s^2/2)
    s1, s2 = 20.0, 35.0
    r = np.linspace(0.0, 12 * s2, 3001)
    w = np.full(len(r), r[1] - r[0])
    w[0] = w[-1] = 0.5 * (r[1] - r[0])
    z = np.outer(r ** l1 * np.exp(-r * r / (2 * s1 ** 2)), r ** l2 * np.exp(-r * r / (2 * s2 ** 2)))
    k1 = np.array([0.005, 0.02, 0.05, 0.09])
    k2 = np.array([0.003, 0.01, 0.03])
    g = lambda k, l, s: np.sqrt(np.pi / 2) * s ** (2 * l + 3) * k ** l * np.exp(-k * k * s * s / 2)
    ref = (-1) ** ((l1 + l2) // 2) * (4 * np.pi) ** 2 * np.outer(g(k1, l1, s1), g(k2, l2, s2))
    B = Mo.zeta_to_bk(l1, l2, r, w, z, k1, k2)
    assert np.allclose(B, ref, rtol=1e-8, atol=1e-10 * np.abs(ref).max())
    Bl = bisp.zeta_to_bk(l1, l2, r, w, z, k1, k2)
    assert np.allclose(Bl, B, rtol=1e-10, atol=1e-12 * np.abs(B).max())


def test_hankel_round_trip():
    # zeta -> B -> zeta for a smooth zeta (both transforms on dense grids)
    s = 25.0
    r = np.linspace(0.0, 300.0, 1201)
    w = np.gradient(r)
    w[0] = w[-1] = 0.5 * (r[1] - r[0])
    z = np.outer(r * r * np.exp(-r * r / (2 * s * s)), np.exp(-r * r / (2 * s * s)))
    k = np.linspace(0.0, 0.4, 1601)
    wk = np.full(len(k), k[1] - k[0])
    wk[0] = wk[-1] = 0.5 * (k[1] - k[0])
    B = Mo.zeta_to_bk(2, 0, r, w, z, k, k)
    rr = np.array([10.0, 30.0, 60.0])
    back = Mo.bk_to_zeta(2, 0, k, wk, B, rr, rr)
    ref = np.outer(rr * rr * np.exp(-rr * rr / (2 * s * s)), np.exp(-rr * rr / (2 * s * s)))
    assert np.allclose(back, ref, rtol=1e-6, atol=1e-8 * np.abs(ref).max())
    assert np.allclose(bisp.bk_to_zeta(2, 0, k, wk, B, rr, rr), back, rtol=1e-10, atol=1e-12 * np.abs(back).max())


def test_library_matches_oracle():
    for j in _nine(6, 200, jmax=5):
        assert bisp.wigner9j(j) == pytest.approx(Mo.wigner9j(j), abs=1e-13)
    r, w = _grid(18)
    ells = [(0, 0, 0), (1, 1, 0), (2, 0, 2), (1, 1, 2), (2, 2, 2)]
    th = _fields(7, ells, len(r))
    win = _fields(8, ells + [(0, 2, 2), (2, 2, 0), (4, 2, 2)], len(r))
    ref, zb = Mo.masked_zeta(ells, th, win, w * r * r)
    got, zb2 = bisp.masked_zeta(th, win, ells, r, w)
    assert zb2 == pytest.approx(zb, rel=1e-12)
    for e in ells:
        assert np.allclose(got[e], ref[e], rtol=1e-11, atol=1e-12 * np.abs(ref[e]).max())


def test_library_errors():
    with pytest.raises(bisp.BispError, match="Q_000"):
        r, w = _grid(4)
        bisp.masked_zeta({(0, 0, 0): np.ones((4, 4))}, {(2, 0, 2): np.ones((4, 4))}, [(0, 0, 0)], r, w)
    with pytest.raises(bisp.BispError) as e:
        bisp.zeta_to_bk(1, 0, np.ones(3), np.ones(3), np.ones((3, 3)), np.ones(2), np.ones(2))
    assert e.value.status == bisp.BISP_EUNSUPPORTED
    with pytest.raises(bisp.BispError):
        bisp.wigner9j([1, 1, 1, 1, 1, 1, 1, 1, 99])


def _plaw():
    kt = np.array([1e-4, 10.0])
    return kt, 2e4 * (kt / 0.05) ** -1.5


def test_tree_real_space_is_isotropic_and_follows_the_legendre_route():
    # f = 0: B depends on the triangle only, so every L > 0 multipole vanishes and
    # B_{l l 0}(k1, k2) = (2l+1) int dmu/2 L_l(mu) B(k1, k2, mu)   (mu = k1_hat . k2_hat)
    from oracle.sph import legendre
    kt, pt = _plaw()
    P = Mo.power_loglog(kt, pt)
    k1, k2 = 0.05, 0.08
    mu, w = np.polynomial.legendre.leggauss(64)
    v1 = np.stack([np.zeros_like(mu), np.zeros_like(mu), np.full_like(mu, k1)], axis=-1)
    v2 = k2 * np.stack([np.sqrt(1 - mu * mu), np.zeros_like(mu), mu], axis=-1)
    B = Mo.tree_bispectrum(P, 1.7, 0.9, 0.0, v1, v2)
    for l in (0, 1, 2):
        ref = (2 * l + 1) * np.sum(w / 2 * legendre(l, mu) * B)
        assert Mo.tree_multipole(P, 1.7, 0.9, 0.0, (l, l, 0), k1, k2) == pytest.approx(ref, rel=1e-8)
    for ell in [(2, 0, 2), (1, 1, 2), (2, 2, 2)]:
        assert abs(Mo.tree_multipole(P, 1.7, 0.9, 0.0, ell, k1, k2)) < 1e-8 * abs(ref)


def test_tree_multipoles_do_not_depend_on_the_line_of_sight_direction():
    kt, pt = _plaw()
    P = Mo.power_loglog(kt, pt)
    for ell in [(0, 0, 0), (2, 0, 2), (1, 1, 2)]:
        a = Mo.tree_multipole(P, 2.0, 1.0, 0.7, ell, 0.05, 0.08)
        b = Mo.tree_multipole(P, 2.0, 1.0, 0.7, ell, 0.05, 0.08, n=(1.0, 0.3, 0.2))
        assert a == pytest.approx(b, rel=1e-7)
    # the redshift-space boost makes the quadrupole positive
    assert Mo.tree_multipole(P, 2.0, 1.0, 0.7, (2, 0, 2), 0.05, 0.08) > 0


def test_library_tree_multipoles_match_oracle():
    kt, pt = _plaw()
    P = Mo.power_loglog(kt, pt)
    ells = [(0, 0, 0), (1, 1, 0), (2, 0, 2), (1, 1, 2)]
    k1, k2 = np.array([0.04, 0.09]), np.array([0.06])
    lib = bisp.tree_multipoles(kt, pt, 2.0, 1.0, 0.7, ells, k1, k2)
    for i, e in enumerate(ells):
        for a, kk1 in enumerate(k1):
            ref = Mo.tree_multipole(P, 2.0, 1.0, 0.7, e, kk1, k2[0])
            assert lib[i, a, 0] == pytest.approx(ref, rel=1e-7)
    with pytest.raises(bisp.BispError):
        bisp.tree_multipoles(kt[::-1], pt, 1.0, 0.0, 0.0, ells, k1, k2)
