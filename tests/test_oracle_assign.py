"""Pins of the oracle's mass assignment, mass-assignment window, alias sums and binning."""
import numpy as np
import pytest

from oracle import estimator as E


def test_assignment_conserves_weight_and_is_local():
    rng = np.random.default_rng(5)
    xyz = (rng.random((500, 3)) * 100.0).astype(np.float32)
    w = rng.random(500)
    for p in (1, 2, 3):
        for shift in (0.0, 0.5):
            m = E.assign(xyz, w, 8, 100.0, p, shift)
            assert m.sum() == pytest.approx(w.sum(), rel=1e-13)
            assert np.all(m >= 0)


def test_kernels_1d_values():
    # CIC (1-d, d); TSC (1/2 (1/2-d)^2, 3/4 - d^2, 1/2 (1/2+d)^2) (Hockney & Eastwood)
    d = np.array([-0.5, -0.25, 0.0, 0.3, 0.49])
    t = [E._kernel_1d(d, s, 3) for s in (-1, 0, 1)]
    assert np.allclose(sum(t), 1.0)
    assert np.allclose(t[1], 0.75 - d * d)
    assert E._kernel_1d(np.array([0.0]), 0, 3)[0] == 0.75
    assert E._kernel_1d(np.array([0.0]), -1, 3)[0] == 0.125
    c = [E._kernel_1d(np.array([0.3]), s, 2)[0] for s in (0, 1)]
    assert c == pytest.approx([0.7, 0.3])


def test_single_particle_on_node_and_between_nodes():
    N, L = 8, 8.0  # H = 1
    xyz = np.array([[3.0, 4.0, 5.0]], np.float32)
    assert E.assign(xyz, [1.0], N, L, 2)[3, 4, 5] == 1.0
    m = E.assign(xyz, [1.0], N, L, 3)
    assert m[3, 4, 5] == pytest.approx(0.75 ** 3)
    assert m[2, 4, 5] == pytest.approx(0.125 * 0.75 ** 2)
    # periodic wrap: a particle just below L deposits onto node 0
    xyz = np.array([[7.9, 0.1, 0.0]], np.float32)
    m = E.assign(xyz, [1.0], N, L, 3)
    assert m.sum() == pytest.approx(1.0)
    assert m[0, 0, 0] == pytest.approx((0.75 - 0.1 ** 2) ** 2 * 0.75, rel=1e-6)


def test_cell_keys_and_stable_order():
    N, L = 4, 4.0
    xyz = np.array([[0.2, 0.2, 0.2], [3.9, 0, 0], [0.4, 0.1, 0.3], [1.6, 0, 0]], np.float32)
    # TSC home = round(u) mod N: (0,0,0), (0 after wrap), (0,0,0), (2,0,0)
    k = E.cell_keys(xyz, N, L, 3)
    assert list(k) == [0, 0, 0, 32]
    assert list(E.stable_cell_order(xyz, N, L, 3)) == [0, 1, 2, 3]
    # CIC home = floor(u): (0,0,0), (3,0,0), (0,0,0), (1,0,0)
    assert list(E.cell_keys(xyz, N, L, 2)) == [0, 48, 0, 16]
    assert list(E.stable_cell_order(xyz, N, L, 2)) == [0, 2, 3, 1]


def test_mas_window_shape():
    # W_mass (Sec. 4.2): 1 at k = 0, sinc^p along an axis, even in k.
    N = 16
    for p in (1, 2, 3):
        W = E.mas_window(N, p)
        assert W[0, 0, 0] == 1.0
        n = np.arange(1, N // 2)
        assert np.allclose(W[n, 0, 0], (np.sin(np.pi * n / N) / (np.pi * n / N)) ** p)
        neg = (-np.arange(N)) % N
        assert np.array_equal(W, W[neg][:, neg][:, :, neg])


@pytest.mark.parametrize("p", [2, 3])
def test_cshot_closed_forms(p):
    # Jing (2005) Eq. 20 closed forms of the alias sum of W^2, no interlacing
    N = 16
    C = E.c_shot(N, p, False)
    n = E.signed_modes(N)
    s = np.sin(np.pi * n / N) ** 2
    f = 1 - 2.0 / 3.0 * s if p == 2 else 1 - s + 2.0 / 15.0 * s * s
    want = f[:, None, None] * f[None, :, None] * f[None, None, :]
    assert np.allclose(C, want, rtol=0, atol=1e-9)


def _avg_power_1d(N, p, n, interlace, npts=40000):
    """<Delta(n) Delta2(n)^*> over a uniformly distributed particle position (1D), from the
    assignment weights themselves: returns (<|a|^2>, <|b|^2>, <a b^*>)."""
    u = (np.arange(npts) + 0.5) / npts * N  # positions over the whole line (periodic)
    a = np.zeros(npts, complex)
    b = np.zeros(npts, complex)
    for shift, arr in ((0.0, a), (0.5, b)):
        uu = u - shift
        hf = E.home_cells(uu, p)
        d = uu - hf
        for s in E._offsets(p):
            c = (hf.astype(int) + s) % N
            arr += E._kernel_1d(d, s, p) * np.exp(-2j * np.pi * n * c / N)
    b *= np.exp(-1j * np.pi * n / N)  # interlacing phase of the shifted mesh
    return np.mean(np.abs(a) ** 2), np.mean(np.abs(b) ** 2), np.mean(a * np.conj(b))


@pytest.mark.parametrize("p", [2, 3])
def test_cshot_interlaced_equals_position_average(p):
    # For one particle at a uniform random position, <|(D1 + phase D2)/2|^2> is the alias sum
    # with even images only.  The 3D average factorises into 1D averages along each axis.
    N = 8
    C = E.c_shot(N, p, True)
    for nvec in [(1, 0, 0), (2, 1, 0), (3, 2, 1), (1, 1, 1), (3, 3, 3)]:
        aa, bb, ab = zip(*[_avg_power_1d(N, p, n, True) for n in nvec])
        val = 0.25 * (np.prod(aa) + np.prod(bb) + 2 * np.real(np.prod(ab)))
        assert val == pytest.approx(C[nvec], rel=2e-6)
    # and without interlacing it is the product of the 1D mean powers
    C0 = E.c_shot(N, p, False)
    for nvec in [(1, 0, 0), (3, 2, 1)]:
        aa = [_avg_power_1d(N, p, n, False)[0] for n in nvec]
        assert np.prod(aa) == pytest.approx(C0[nvec], rel=2e-6)


def test_bins_and_mode_counts_brute_force():
    N, L = 16, 1000.0
    kF = 2 * np.pi / L
    edges = [1.0 * kF, 2.0 * kF, 3.7 * kF, 5.0 * kF, 7.9 * kF]
    p = E.Params(N=N, L=L, edges=edges, ells=[(0, 0, 0)])
    b = E.bin_grid(p)
    counts = np.bincount(b[b >= 0].ravel(), minlength=4)
    want = np.zeros(4, int)
    for i in range(N):
        for j in range(N):
            for k in range(N):
                n = [(t if t < N // 2 else t - N) for t in (i, j, k)]
                if any(abs(t) == N // 2 for t in n):
                    continue
                kk = kF * np.sqrt(n[0] ** 2 + n[1] ** 2 + n[2] ** 2)
                for bb in range(4):
                    if edges[bb] <= kk < edges[bb + 1]:
                        want[bb] += 1
    assert list(counts) == list(want)
    # shells are symmetric under k -> -k
    assert np.array_equal(b, np.roll(b[::-1, ::-1, ::-1], 1, axis=(0, 1, 2)))


def test_interlacing_phase_single_particle():
    # For one particle, the interlaced and deconvolved D(k) approximates exp(-i k.x) at
    # low k; a wrong interlacing phase sign gives an O(1) error.
    N, L = 32, 32.0
    p = E.Params(N=N, L=L, edges=[0.1, 0.2], ells=[(0, 0, 0)], mas=3, interlace=True)
    x = np.array([[10.3, 5.7, 20.1]], np.float32)
    D = E.spectrum(p, x, np.array([1.0]))
    for n in [(1, 0, 0), (0, 2, 1), (2, 1, 1)]:
        want = np.exp(-1j * 2 * np.pi / L * np.dot(n, x[0].astype(float)))
        assert abs(D[n] - want) < 2e-3
    p.interlace = False
    D0 = E.spectrum(p, x, np.array([1.0]))
    n = (2, 1, 1)
    want = np.exp(-1j * 2 * np.pi / L * np.dot(n, x[0].astype(float)))
    assert abs(D[n] - want) < abs(D0[n] - want)
