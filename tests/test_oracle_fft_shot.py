"""More pins of the oracle: its FFT against a naive DFT and Parseval, the box shot noise against
the textbook form assembled from an explicit triangle enumeration, and y_l^m parity."""
import numpy as np
import pytest

from oracle import estimator as E
from oracle.sph import ylm


def _naive_dft3(m):
    """X(k) = sum_x m(x) exp(-2 pi i k.x / N), written out as one sum over all cells."""
    N = m.shape[0]
    j = np.arange(N)
    x = np.stack(np.meshgrid(j, j, j, indexing="ij"), -1).reshape(-1, 3)
    ph = np.exp(-2j * np.pi * (x @ x.T) / N)  # k and x run over the same index set
    return (ph @ m.reshape(-1)).reshape(N, N, N)


def test_fft_equals_naive_dft_and_parseval():
    N, L = 8, 800.0
    rng = np.random.default_rng(3)
    xyz = (rng.random((60, 3)) * L).astype(np.float32)
    vals = 0.5 + rng.random(60)
    p = E.Params(N=N, L=L, edges=[0.01, 0.02], ells=[(0, 0, 0)], los="global", mas=2, interlace=False)
    m = E.assign(xyz, vals, N, L, 2)
    X = _naive_dft3(m)
    F = np.fft.fftn(m)
    assert np.max(np.abs(F - X)) <= 1e-12 * np.max(np.abs(X))
    # Parseval: sum |m|^2 = sum |X|^2 / N^3
    assert np.sum(np.abs(m) ** 2) == pytest.approx(np.sum(np.abs(X) ** 2) / N ** 3, rel=1e-12)
    # the oracle's spectrum is that DFT over W_mass, zero on the Nyquist planes
    D = E.spectrum(p, xyz, vals)
    ref = X / E.mas_window(N, 2)
    ref[E.nyquist_mask(N)] = 0.0
    assert np.max(np.abs(D - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("mas,interlace", [(2, False), (3, True)])
def test_box_shot_noise_textbook_limit(mas, interlace):
    """Global line of sight, B000: shot = [<P>_1 + <P>_2 + <P(k3)>_triangles]/nbar + 1/nbar^2,
    P(k) = V |D(k)|^2 / Np^2 - V C(k) / (W(k)^2 Np), the triangle average taken over all ordered
    mode pairs (k1, k2) of the two shells with k3 = -k1-k2 (mod N)."""
    N, L, Np = 16, 1000.0, 400
    kf = 2 * np.pi / L
    rng = np.random.default_rng(5)
    xyz = (rng.random((Np, 3)) * L).astype(np.float32)
    xyz[: Np // 4] = (xyz[: Np // 4] * 0.2 + 300.0).astype(np.float32)  # some clustering
    edges = [1.5 * kf, 2.5 * kf, 3.5 * kf, 4.6 * kf]
    p = E.Params(N=N, L=L, edges=edges, ells=[(0, 0, 0)], los="global", mas=mas, interlace=interlace)
    res = E.measure(p, {"xyz": xyz})
    V = L ** 3
    nbar = Np / V
    D = E.spectrum(p, xyz, np.ones(Np))
    D[0, 0, 0] = 0.0  # the data pass removes the mean
    Pk = V * np.abs(D) ** 2 / Np ** 2 - V * E.cw2(p) / Np
    Pk[E.nyquist_mask(N)] = 0.0
    bins = E.bin_grid(p)
    nb = len(edges) - 1
    sh = [E.shell_modes(p, b, bins) for b in range(nb)]
    avg = [np.mean(Pk[bins == b]) for b in range(nb)]
    for b1 in range(nb):
        for b2 in range(nb):
            k3 = np.mod(-(sh[b1][:, None, :] + sh[b2][None, :, :]), N)
            tri = np.mean(Pk[k3[..., 0], k3[..., 1], k3[..., 2]])
            expect = (avg[b1] + avg[b2] + tri) / nbar + 1.0 / nbar ** 2
            assert res["shot"][0, b1, b2] == pytest.approx(expect, rel=1e-10)


def test_ylm_parity():
    rng = np.random.default_rng(9)
    v = rng.normal(size=(200, 3))
    for l in range(5):
        for m in range(-l, l + 1):
            a = ylm(l, m, v[:, 0], v[:, 1], v[:, 2])
            b = ylm(l, m, -v[:, 0], -v[:, 1], -v[:, 2])
            assert np.max(np.abs(b - (-1) ** l * a)) <= 1e-13
