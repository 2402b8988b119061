"""Pins of the line-of-sight variants of the oracle (App. B): the y_L^{M*} weight on x1 or x2."""
import numpy as np
import pytest

from oracle import estimator as E
from oracle import los as LS

L_BOX = 1000.0
KF = 2 * np.pi / L_BOX


def _cats(seed, ngal=300, nran=900):
    rng = np.random.default_rng(seed)
    gal = {"xyz": (rng.random((ngal, 3)) * L_BOX).astype(np.float32), "w": (0.5 + rng.random(ngal)).astype(np.float32)}
    ran = {"xyz": (rng.random((nran, 3)) * L_BOX).astype(np.float32), "w": (0.5 + rng.random(nran)).astype(np.float32)}
    gal["xyz"][: ngal // 3] = (gal["xyz"][: ngal // 3] * 0.3 + 200.0).astype(np.float32)
    return gal, ran


def _params(**kw):
    base = dict(N=16, L=L_BOX, edges=[1.5 * KF, 2.5 * KF, 3.5 * KF, 4.6 * KF],
                ells=[(0, 0, 0), (1, 1, 0), (2, 0, 2), (1, 1, 2), (2, 2, 2)],
                los="local", observer=(500.0, 400.0, -900.0), mas=3, interlace=True)
    base.update(kw)
    return E.Params(**base)


def test_los_on_x3_is_the_main_estimator():
    gal, ran = _cats(1)
    p = _params()
    sd = E.catalogue_spectra(p, gal, ran)["data"]
    assert np.allclose(LS.bispectrum_raw_fft(p, sd, 3), E.bispectrum_raw_fft(p, sd), rtol=1e-12, atol=0)
    assert np.allclose(LS.shot_noise_fft(p, sd, 3), E.shot_noise_fft(p, sd), rtol=1e-12, atol=0)


def test_l0_modes_do_not_depend_on_the_los_object():
    # y_0^0 = 1: the L = 0 multipoles are the same for every choice (App. B)
    gal, ran = _cats(2)
    p = _params(ells=[(0, 0, 0), (1, 1, 0), (2, 2, 0)])
    sd = E.catalogue_spectra(p, gal, ran)["data"]
    r3, s3 = LS.bispectrum_raw_fft(p, sd, 3), LS.shot_noise_fft(p, sd, 3)
    for q in (1, 2):
        assert np.allclose(LS.bispectrum_raw_fft(p, sd, q), r3, rtol=1e-12, atol=1e-14 * np.abs(r3).max())
        assert np.allclose(LS.shot_noise_fft(p, sd, q), s3, rtol=1e-12, atol=1e-14 * np.abs(s3).max())


def test_x1_x2_exchange():
    # B^{(x1)}_{l1 l2 L}(k1, k2) = B^{(x2)}_{l2 l1 L}(k2, k1)
    gal, ran = _cats(3)
    p = _params(ells=[(2, 0, 2), (0, 2, 2), (3, 1, 2), (1, 3, 2)], ells_all_orders=True)
    sd = E.catalogue_spectra(p, gal, ran)["data"]
    r1, r2 = LS.bispectrum_raw_fft(p, sd, 1), LS.bispectrum_raw_fft(p, sd, 2)
    s1, s2 = LS.shot_noise_fft(p, sd, 1), LS.shot_noise_fft(p, sd, 2)
    for i, j in [(0, 1), (2, 3)]:
        assert np.allclose(r1[i], r2[j].T, rtol=1e-11, atol=1e-13 * np.abs(r1[i]).max())
        assert np.allclose(s1[i], s2[j].T, rtol=1e-11, atol=1e-13 * np.abs(s1[i]).max())
    # and the choice matters for L = 2 on a survey
    assert not np.allclose(r1[0], LS.bispectrum_raw_fft(p, sd, 3)[0], rtol=1e-3)


@pytest.mark.parametrize("q", [1, 2])
def test_fft_mode_equals_triangle_sum(q):
    gal, ran = _cats(4)
    p = _params()
    sd = E.catalogue_spectra(p, gal, ran)["data"]
    raw = LS.bispectrum_raw_fft(p, sd, q)
    acc = E.MeshSpectrumAccess(p, sd)
    bins = E.bin_grid(p)
    for im, (l1, l2, L) in enumerate(p.ells):
        for b1, b2 in [(0, 0), (0, 2), (1, 2)]:
            d = LS.raw_direct(p, acc, sd.I, q, l1, l2, L, E.shell_modes(p, b1, bins), E.shell_modes(p, b2, bins))
            assert raw[im, b1, b2] == pytest.approx(d, rel=1e-10, abs=1e-12 * np.abs(raw[im]).max())


@pytest.mark.parametrize("q", [1, 2])
def test_fft_shot_noise_equals_mode_sums(q):
    gal, ran = _cats(6)
    p = _params(ells=[(2, 0, 2), (1, 1, 2), (2, 2, 2)])
    sd = E.catalogue_spectra(p, gal, ran)["data"]
    shot = LS.shot_noise_fft(p, sd, q)
    acc = E.MeshSpectrumAccess(p, sd)
    bins = E.bin_grid(p)
    for im, (l1, l2, L) in enumerate(p.ells):
        for b1, b2 in [(0, 0), (0, 2)]:
            d = LS.shot_direct(p, acc, sd.I, q, l1, l2, L, E.shell_modes(p, b1, bins), E.shell_modes(p, b2, bins))
            assert shot[im, b1, b2] == pytest.approx(d, rel=1e-10, abs=1e-12 * np.abs(shot[im]).max())


@pytest.mark.parametrize("q", [1, 2, 3])
def test_shot_noise_equals_distinct_triplets(q):
    # particle-exact mode: hat B - (four shot terms) = sum over distinct triplets, the y_L^{M*}
    # weight on the object of slot q
    gal, ran = _cats(5, ngal=30, nran=60)
    gal["xyz"] = gal["xyz"].astype(np.float64)
    p = _params(edges=[1.5 * KF, 2.5 * KF, 3.2 * KF], ells=[(0, 0, 0), (2, 0, 2), (1, 1, 2), (2, 2, 2)])
    alpha = float(gal["w"].astype(np.float64).sum() / ran["w"].astype(np.float64).sum())
    acc = E.ExactSpectrumAccess(p, gal, ran, alpha)
    bins = E.bin_grid(p)
    for (l1, l2, L) in p.ells:
        for b1, b2 in [(0, 0), (0, 1), (1, 0)]:
            m1, m2 = E.shell_modes(p, b1, bins), E.shell_modes(p, b2, bins)
            raw = LS.raw_direct(p, acc, 1.0, q, l1, l2, L, m1, m2)
            shot = LS.shot_direct(p, acc, 1.0, q, l1, l2, L, m1, m2)
            bf = LS.distinct_triplet_sum(p, acc, 1.0, q, l1, l2, L, m1, m2)
            assert raw - shot == pytest.approx(bf, rel=1e-10, abs=1e-12 * abs(raw))
