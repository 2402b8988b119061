"""Pins of the three-point-function oracle (Sec. 4.3, Eq. reduced_xi_estimator; window
multipoles Q, Sec. 6.1, Eq. Q) against routes that share none of its filter arithmetic."""
import numpy as np
import pytest

from oracle import estimator as E
from oracle import threept as T
from oracle.sph import legendre as legendre_p

L_BOX = 800.0


def _cats(seed, N, ngal=400, nran=1200):
    rng = np.random.default_rng(seed)
    gal = {"xyz": (rng.random((ngal, 3)) * L_BOX).astype(np.float32),
           "w": (0.5 + rng.random(ngal)).astype(np.float32)}
    ran = {"xyz": (rng.random((nran, 3)) * L_BOX).astype(np.float32),
           "w": (0.5 + rng.random(nran)).astype(np.float32)}
    gal["xyz"][: ngal // 3] = (gal["xyz"][: ngal // 3] * 0.3 + 250.0).astype(np.float32)
    return gal, ran


def _params(N=12, **kw):
    H = L_BOX / N
    base = dict(N=N, L=L_BOX, edges=[0.9 * H, 1.5 * H, 2.05 * H, 2.95 * H],
                ells=[(0, 0, 0), (1, 1, 0), (2, 0, 2), (1, 1, 2), (2, 2, 2)],
                los="local", observer=(400.0, 300.0, -700.0), mas=3, interlace=True)
    base.update(kw)
    return E.Params(**base)


def test_r_bins_are_separation_shells():
    p = _params(N=12)
    bins = T.offset_bins(p)
    # bin 0 = [0.9 H, 1.5 H): the 6 nearest and 12 second-nearest separations (|s|^2 = 1, 2)
    s0 = T.shell_offsets(p, 0, bins)
    assert len(s0) == 18 and set(np.sum(s0 * s0, axis=1)) == {1, 2}
    # bin 1 = [1.5 H, 2.05 H): |s|^2 = 3 (8) and 4 (6)
    s1 = T.shell_offsets(p, 1, bins)
    assert len(s1) == 14 and set(np.sum(s1 * s1, axis=1)) == {3, 4}
    # every shell is symmetric under s -> -s and excludes the Nyquist separation
    for a in range(3):
        s = T.shell_offsets(p, a, bins)
        assert {tuple(v) for v in s} == {tuple(-v) for v in s}
        assert np.all(np.abs(s) < p.N // 2)
    # a bin that starts at 0 holds s = 0 only when it ends below one cell
    p0 = _params(N=12, edges=[0.0, 0.5 * p.H, 1.2 * p.H])
    assert [tuple(v) for v in T.shell_offsets(p0, 0)] == [(0, 0, 0)]


@pytest.mark.parametrize("los,mas,interlace", [("local", 3, True), ("global", 2, False)])
def test_fft_mode_equals_separation_sums(los, mas, interlace):
    # F by the k-space filter K_a(k) == F by explicit sums over the separations of the bin
    gal, ran = _cats(1, 12)
    p = _params(los=los, mas=mas, interlace=interlace)
    sd = E.catalogue_spectra(p, gal, ran)["data"]
    raw = T.threept_raw_fft(p, sd)
    for im, (l1, l2, L) in enumerate(p.ells):
        for a, b in [(0, 0), (0, 2), (2, 1)]:
            d = T.threept_raw_direct(p, sd, l1, l2, L, a, b)
            assert raw[im, a, b] == pytest.approx(d, rel=1e-10, abs=1e-12 * np.abs(raw[im]).max())


@pytest.mark.parametrize("los", ["local", "global"])
def test_shot_noise_equals_distinct_triplets(los):
    # objects on mesh nodes, exact DFTs (W = C = 1): hat zeta - S_{i=j!=k} equals the sum over
    # distinct triplets with separations in the two bins (none of the bins holds s = 0)
    rng = np.random.default_rng(5)
    N = 8
    p = _params(N=N, los=los, edges=[0.9 * L_BOX / N, 1.5 * L_BOX / N, 2.05 * L_BOX / N],
                ells=[(0, 0, 0), (1, 1, 0), (2, 0, 2), (1, 1, 2), (2, 2, 2)])
    g = rng.integers(0, N, size=(25, 3))
    g[5:12] = g[0]  # several objects on one node
    r = rng.integers(0, N, size=(40, 3))
    wg = 0.5 + rng.random(25)
    wr = 0.5 + rng.random(40)
    spec = T.node_spectra(p, g, wg, r, wr)
    ones = np.ones((N,) * 3)
    raw = T.threept_raw_fft(p, spec)
    shot = T.threept_shot_fft(p, spec, cw=ones)
    for im, (l1, l2, L) in enumerate(p.ells):
        for a, b in [(0, 0), (0, 1), (1, 0), (1, 1)]:
            bf = T.distinct_triplet_sum(p, g, wg, l1, l2, L, a, b, r, wr)
            got = raw[im, a, b] - shot[im, a, b]
            assert got == pytest.approx(bf, rel=1e-9, abs=1e-10 * np.abs(raw[im]).max())
    assert np.all(shot[:, 0, 1] == 0) and np.any(shot[:, 0, 0] != 0)


@pytest.mark.parametrize("ell", [0, 1, 2])
def test_legendre_route(ell):
    # zeta_{l l 0}(a, b) = (2l+1)/I (V/Ng) sum_x delta(x) (1/(N_a N_b))
    #     sum_{s1 in a, s2 in b} L_l(s1_hat . s2_hat) delta(x + s1) delta(x + s2)
    gal, ran = _cats(2, 8, ngal=200, nran=600)
    N = 8
    H = L_BOX / N
    p = _params(N=N, los="global", edges=[0.9 * H, 1.5 * H, 2.05 * H], ells=[(ell, ell, 0)], mas=2,
                interlace=False)
    sd = E.catalogue_spectra(p, gal, ran)["data"]
    raw = T.threept_raw_fft(p, sd)
    d = E.g_field(p, sd.D[(0, 0)]).real
    for a, b in [(0, 0), (0, 1)]:
        s1, s2 = T.shell_offsets(p, a), T.shell_offsets(p, b)
        u1 = s1 / np.linalg.norm(s1, axis=1)[:, None]
        u2 = s2 / np.linalg.norm(s2, axis=1)[:, None]
        sh1 = [np.roll(d, tuple(-v), axis=(0, 1, 2)) for v in s1]
        sh2 = [np.roll(d, tuple(-v), axis=(0, 1, 2)) for v in s2]
        tot = 0.0
        for i in range(len(s1)):
            for j in range(len(s2)):
                tot += legendre_p(ell, float(u1[i] @ u2[j])) * np.sum(d * sh1[i] * sh2[j])
        ref = (2 * ell + 1) / sd.I * p.V / p.Ng * tot / (len(s1) * len(s2))
        assert raw[0, a, b] == pytest.approx(ref, rel=1e-10)


def test_exchange_symmetry():
    # zeta_{l1 l2 L}(r_a, r_b) = zeta_{l2 l1 L}(r_b, r_a)
    gal, ran = _cats(3, 12)
    p = _params(ells=[(2, 0, 2), (0, 2, 2), (2, 1, 1), (1, 2, 1)], ells_all_orders=True)
    sd = E.catalogue_spectra(p, gal, ran)["data"]
    raw = T.threept_raw_fft(p, sd)
    shot = T.threept_shot_fft(p, sd)
    for i, j in [(0, 1), (2, 3)]:
        assert np.allclose(raw[i], raw[j].T, rtol=1e-10, atol=1e-12 * np.abs(raw[i]).max())
        assert np.allclose(shot[i], shot[j].T, rtol=1e-10, atol=1e-12 * np.abs(shot[i]).max())


def _smooth_window_spectra(p, sigma):
    """Spectra of a smooth mean density on the mesh (no particles, W = 1)."""
    c = (np.arange(p.N) + 0.5) * p.H - 0.5 * p.L
    x, y, z = np.meshgrid(c, c, c, indexing="ij")
    nbar = 1.0 + 5.0 * np.exp(-(x * x + 1.3 * y * y + 0.8 * z * z) / (2 * sigma ** 2))
    D = {(0, 0): np.fft.fftn(nbar)}
    I = float(np.sum(nbar ** 3)) / p.H ** 6
    return E.Spectra(D, {(0, 0): np.zeros_like(D[(0, 0)])}, {(0, 0): 0.0}, I, None, "window")


def test_window_q000_small_separation_limit():
    # Q_000(0, 0) = 1 exactly; Q_000(0, r) -> 1 as r -> 0 for a smooth nbar, the faster the
    # smoother; Q_{l1 l2 L}(0, r) = 0 for l1 > 0 (y_l(0) = 0)
    N = 24
    H = L_BOX / N
    p = E.Params(N=N, L=L_BOX, edges=[0.0, 0.5 * H, 1.2 * H, 1.5 * H], ells=[(0, 0, 0), (1, 1, 0)], los="global")
    dev = []
    for sigma in (0.12 * L_BOX, 0.24 * L_BOX):
        q = T.threept_raw_fft(p, _smooth_window_spectra(p, sigma))
        assert q[0, 0, 0] == pytest.approx(1.0, rel=1e-12)
        assert q[0, 1, 0] == pytest.approx(q[0, 0, 1], rel=1e-12)
        dev.append(abs(q[0, 0, 1] - 1.0))
        assert abs(q[0, 0, 2] - 1.0) < 0.1
        assert np.all(np.abs(q[1, 0, :]) < 1e-12)
    assert dev[1] < 0.4 * dev[0] and dev[1] < 0.01
