"""Pins of the oracle's estimator (Eq. bi_estimator_FFTs) and shot noise (Eq. ShotNoise)
against the triangle-sum definition (Eq. bi_estimator), brute force over particle
triplets, the Legendre reduction (Sec. 3.1), and symmetries the paper states."""
import numpy as np
import pytest

from oracle import estimator as E
from oracle.sph import legendre

L_BOX = 1000.0
KF = 2 * np.pi / L_BOX


def _cats(seed, ngal=300, nran=900, weights=True):
    rng = np.random.default_rng(seed)
    gal = {"xyz": (rng.random((ngal, 3)) * L_BOX).astype(np.float32)}
    ran = {"xyz": (rng.random((nran, 3)) * L_BOX).astype(np.float32)}
    if weights:
        gal["w"] = (0.5 + rng.random(ngal)).astype(np.float32)
        ran["w"] = (0.5 + rng.random(nran)).astype(np.float32)
    # a clustered galaxy component so that B is not pure noise
    gal["xyz"][: ngal // 3] = (gal["xyz"][: ngal // 3] * 0.3 + 200.0).astype(np.float32)
    return gal, ran


def _params(**kw):
    base = dict(N=16, L=L_BOX, edges=[1.5 * KF, 2.5 * KF, 3.5 * KF, 4.6 * KF],
                ells=[(0, 0, 0), (1, 1, 0), (2, 0, 2), (1, 1, 2), (2, 2, 2)],
                los="local", observer=(500.0, 400.0, -900.0), mas=3, interlace=True)
    base.update(kw)
    return E.Params(**base)


@pytest.mark.parametrize("los,mas,interlace", [("local", 3, True), ("global", 2, False), ("global", 3, True)])
def test_fft_mode_equals_triangle_sum(los, mas, interlace):
    gal, ran = _cats(1)
    p = _params(los=los, mas=mas, interlace=interlace)
    specs = E.catalogue_spectra(p, gal, ran)
    sd = specs["data"]
    pairs = [(0, 1), (1, 2), (2, 2), (2, 0)]
    raw = E.bispectrum_raw_fft(p, sd, pairs)
    shot, parts = E.shot_noise_fft(p, sd, pairs, parts=True)
    acc = E.MeshSpectrumAccess(p, sd)
    bins = E.bin_grid(p)
    for im, (l1, l2, L) in enumerate(p.ells):
        for b1, b2 in pairs:
            m1, m2 = E.shell_modes(p, b1, bins), E.shell_modes(p, b2, bins)
            d = E.bispectrum_raw_direct(p, acc, sd.I, l1, l2, L, b1, b2, m1, m2)
            assert raw[im, b1, b2] == pytest.approx(d, rel=1e-10, abs=1e-10 * np.nanmax(abs(raw[im])))
            ds = E.shot_noise_direct(p, acc, sd.I, l1, l2, L, m1, m2)
            for k in ds:
                scale = max(np.nanmax(abs(parts[k][im])), 1e-300)
                assert parts[k][im, b1, b2] == pytest.approx(ds[k], rel=1e-10, abs=1e-10 * scale)


def test_window_fft_mode_equals_triangle_sum():
    gal, ran = _cats(2)
    p = _params(window=True, ells=[(0, 0, 0), (2, 0, 2)])
    sw = E.catalogue_spectra(p, gal, ran)["window"]
    assert sw.D[(0, 0)][0, 0, 0] != 0.0  # k = 0 kept for the window
    raw = E.bispectrum_raw_fft(p, sw, [(0, 0), (0, 2)])
    acc = E.MeshSpectrumAccess(p, sw)
    bins = E.bin_grid(p)
    for im, (l1, l2, L) in enumerate(p.ells):
        for b1, b2 in [(0, 0), (0, 2)]:
            d = E.bispectrum_raw_direct(p, acc, sw.I, l1, l2, L, b1, b2,
                                        E.shell_modes(p, b1, bins), E.shell_modes(p, b2, bins))
            assert raw[im, b1, b2] == pytest.approx(d, rel=1e-10)


@pytest.mark.parametrize("los", ["local", "global"])
def test_shot_noise_equals_distinct_triplets(los):
    # particle-exact mode: hat B - (four shot terms) = sum over distinct triplets i != j != k
    gal, ran = _cats(3, ngal=30, nran=60)
    gal["xyz"] = gal["xyz"].astype(np.float64)
    p = _params(los=los, edges=[1.5 * KF, 2.5 * KF, 3.2 * KF],
                ells=[(0, 0, 0), (2, 0, 2), (1, 1, 2), (2, 2, 0), (4, 0, 4)])
    alpha = float(gal["w"].astype(np.float64).sum() / ran["w"].astype(np.float64).sum())
    acc = E.ExactSpectrumAccess(p, gal, ran, alpha)
    bins = E.bin_grid(p)
    for (l1, l2, L) in p.ells:
        for b1, b2 in [(0, 0), (0, 1), (1, 0)]:
            m1, m2 = E.shell_modes(p, b1, bins), E.shell_modes(p, b2, bins)
            raw = E.bispectrum_raw_direct(p, acc, 1.0, l1, l2, L, b1, b2, m1, m2)
            shot = sum(E.shot_noise_direct(p, acc, 1.0, l1, l2, L, m1, m2).values())
            bf = E.distinct_triplet_sum(p, acc, 1.0, l1, l2, L, m1, m2)
            assert raw - shot == pytest.approx(bf, rel=1e-10, abs=1e-12 * abs(raw))


@pytest.mark.parametrize("ell", [0, 1, 2])
def test_legendre_route(ell):
    # B_{l l 0} = (2l+1)/I <L_l(k1.k2) D D D> (Sec. 3.1, Eq. Legendre)
    gal, ran = _cats(4)
    p = _params(ells=[(ell, ell, 0)])
    sd = E.catalogue_spectra(p, gal, ran)["data"]
    raw = E.bispectrum_raw_fft(p, sd, [(0, 2), (1, 1)])
    acc = E.MeshSpectrumAccess(p, sd)
    bins = E.bin_grid(p)
    for b1, b2 in [(0, 2), (1, 1)]:
        n1, n2 = E.shell_modes(p, b1, bins), E.shell_modes(p, b2, bins)
        u1 = n1 / np.linalg.norm(n1, axis=1)[:, None]
        u2 = n2 / np.linalg.norm(n2, axis=1)[:, None]
        s = 0j
        for i in range(len(n1)):
            n3 = -(n1[i][None, :] + n2)
            s += acc.D(0, 0, n1[i]) * np.sum(legendre(ell, u2 @ u1[i]) * acc.D(0, 0, n2) * acc.D(0, 0, n3))
        want = (2 * ell + 1) / sd.I * (s / (len(n1) * len(n2))).real
        assert raw[0, b1, b2] == pytest.approx(want, rel=1e-10)


def test_k1_k2_symmetry_and_l1_l2_exchange():
    # B_{l l L}(k1,k2) = B_{l l L}(k2,k1) and B_{l1 l2 L}(k1,k2) = B_{l2 l1 L}(k2,k1) (Sec. 2)
    gal, ran = _cats(5)
    p = _params(ells=[(1, 1, 2), (2, 0, 2), (0, 2, 2)], ells_all_orders=True)
    res = E.measure(p, gal, ran, pairs=[(0, 1), (1, 0), (0, 2), (2, 0)])
    B = res["B"]
    for b1, b2 in [(0, 1), (0, 2)]:
        assert B[0, b1, b2] == pytest.approx(B[0, b2, b1], rel=1e-10)
        assert B[1, b1, b2] == pytest.approx(B[2, b2, b1], rel=1e-10)


def test_isotropy_sum_over_axes_vanishes():
    # global LOS along x, y, z (cyclic relabelling of the catalogue): sum of L=2 multipoles = 0
    rng = np.random.default_rng(6)
    xyz = (rng.random((3000, 3)) * L_BOX).astype(np.float32)
    xyz[:1000] = (xyz[:1000] * 0.25 + 300.0).astype(np.float32)
    p = _params(los="global", ells=[(2, 0, 2), (1, 1, 2), (2, 2, 2), (0, 0, 0)])
    tot = 0
    ref = None
    for perm in ([0, 1, 2], [1, 2, 0], [2, 0, 1]):
        r = E.measure(p, {"xyz": xyz[:, perm]}, None, pairs=[(0, 1), (1, 1), (2, 0)])["B"]
        tot = tot + r
        ref = r if ref is None else ref
    for im in range(3):
        for b1, b2 in [(0, 1), (1, 1), (2, 0)]:
            assert abs(tot[im, b1, b2]) < 1e-9 * abs(ref[3, b1, b2])


def test_polar_axis_invariance_local_los():
    # "the resulting multipoles do not depend on this axis choice" (Sec. 4)
    gal, ran = _cats(7)
    pz = _params(ells=[(2, 0, 2), (1, 1, 2), (2, 2, 2)])
    px = _params(ells=[(2, 0, 2), (1, 1, 2), (2, 2, 2)], polar_axis="x")
    pairs = [(0, 1), (2, 2)]
    bz = E.measure(pz, gal, ran, pairs)["B"]
    bx = E.measure(px, gal, ran, pairs)["B"]
    for b1, b2 in pairs:
        assert np.allclose(bx[:, b1, b2], bz[:, b1, b2], rtol=1e-9, atol=1e-9 * abs(bz[:, b1, b2]).max())


def test_condon_shortley_phase_cancels():
    gal, ran = _cats(8)
    pairs = [(0, 1), (2, 2)]
    a = E.measure(_params(), gal, ran, pairs)["B"]
    b = E.measure(_params(condon_shortley=False), gal, ran, pairs)["B"]
    for b1, b2 in pairs:
        assert np.allclose(a[:, b1, b2], b[:, b1, b2], rtol=1e-11)


def test_far_observer_limit_is_global_los():
    gal, ran = _cats(9)
    pairs = [(0, 1), (1, 2)]
    ells = [(0, 0, 0), (2, 0, 2), (1, 1, 2)]
    loc = E.measure(_params(ells=ells, observer=(500.0, 500.0, -1e9)), gal, ran, pairs)["B"]
    glo = E.measure(_params(ells=ells, los="global"), gal, ran, pairs)["B"]
    for b1, b2 in pairs:
        assert np.allclose(loc[:, b1, b2], glo[:, b1, b2], rtol=1e-6, atol=1e-6 * abs(glo[:, b1, b2]).max())


def test_normalisation_I_and_fkp_weights():
    # Eq. normalization: I = int nbar^3 d^3x.  Randoms one per mesh node (CIC deposits each
    # on its own node) give nbar = alpha w / H^3 exactly, so I = V (alpha w / H^3)^3.
    N, Lb = 8, 80.0
    H = Lb / N
    g = (np.arange(N) * H).astype(np.float32)
    nodes = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    ran = {"xyz": nodes, "w": np.full(len(nodes), 0.5, np.float32)}
    gal = {"xyz": nodes[:100] + np.float32(1.0)}
    p = E.Params(N=N, L=Lb, edges=[0.1, 0.2], ells=[(0, 0, 0)], los="local", mas=2)
    sd = E.catalogue_spectra(p, gal, ran)["data"]
    alpha = 100.0 / (0.5 * len(nodes))
    assert sd.alpha == pytest.approx(alpha, rel=1e-14)
    assert sd.I == pytest.approx(Lb ** 3 * (alpha * 0.5 / H ** 3) ** 3, rel=1e-12)
    # periodic box: I = Np^3 / V^2 (Sec. 4.4)
    pb = E.Params(N=N, L=Lb, edges=[0.1, 0.2], ells=[(0, 0, 0)], los="global", mas=2)
    sb = E.catalogue_spectra(pb, gal, None)["data"]
    assert sb.I == pytest.approx(100.0 ** 3 / Lb ** 6, rel=1e-14)
    # FKP weight w / (1 + nbar P0) (Sec. 5.2)
    cat = {"xyz": nodes[:3], "w": np.array([1.0, 2.0, 0.5], np.float32),
           "nbar": np.array([1e-4, 3e-4, 0.0], np.float32)}
    w = E.object_weights(cat, 1e4)
    assert np.allclose(w, [1.0 / 2.0, 2.0 / (1.0 + np.float32(3e-4) * 1e4), 0.5], rtol=1e-7)
