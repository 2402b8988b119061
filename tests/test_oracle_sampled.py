"""The memory-bounded oracle path (oracle/sampled.py) gives the same numbers as the plain oracle:
spectra built one channel at a time into files are the catalogue_spectra arrays bit for bit, and
the per-pair evaluation equals estimator.measure at the same pairs (local line of sight with the
window pass, and a periodic box with the global line of sight)."""
import numpy as np

import synthcat
from oracle import estimator as E
from oracle import sampled as S


def _survey():
    N, L = 16, 2000.0
    obs = (0.5 * L, 0.5 * L, -0.3 * L)
    gal, ran = synthcat.survey_catalogs(N, L, obs, 3000, 12_000, 5, r_min=0.35 * L, r_max=1.25 * L,
                                        half_angle_deg=40.0, r_mean=0.8 * L, sigma=0.2 * L)
    kf = 2 * np.pi / L
    p = E.Params(N=N, L=L, edges=kf * np.array([1.0, 2.5, 4.0, 5.5, 7.0]),
                 ells=[(0, 0, 0), (2, 0, 2), (1, 1, 2)], los="local", observer=obs, mas=3, interlace=True,
                 P0=1e4, window=True)
    return p, gal, ran


def test_on_disk_spectra_equal_catalogue_spectra(tmp_path):
    p, gal, ran = _survey()
    ref = E.catalogue_spectra(p, gal, ran)
    got = S.catalogue_spectra_on_disk(p, gal, ran, str(tmp_path))
    for pas in ("data", "window"):
        a, b = ref[pas], got[pas]
        assert a.I == b.I and a.alpha == b.alpha
        assert set(a.D) == set(b.D) and set(a.Nk) == set(b.Nk)
        for k in a.D:
            assert np.array_equal(a.D[k], np.asarray(b.D[k])), (pas, k)
            assert np.array_equal(a.Nk[k], np.asarray(b.Nk[k])), (pas, k)
            assert a.Sbar[k] == b.Sbar[k]


def test_pairs_equal_full_oracle(tmp_path):
    p, gal, ran = _survey()
    pairs = {(0, 0, 0): [(0, 3), (2, 2)], (2, 0, 2): [(1, 3), (3, 1)], (1, 1, 2): [(0, 2)]}
    specs = S.catalogue_spectra_on_disk(p, gal, ran, str(tmp_path))
    got = S.measure_pairs(p, specs, pairs)
    ref = E.measure(p, gal, ran)
    for mult, prs in pairs.items():
        im = p.ells.index(mult)
        for b1, b2 in prs:
            rec = got[mult + (b1, b2)]
            for k in ("B", "shot", "window", "window_shot"):
                assert np.isclose(rec[k], ref[k][im, b1, b2], rtol=1e-12, atol=0), (mult, b1, b2, k)


def test_pairs_equal_full_oracle_box(tmp_path):
    N, L = 16, 1000.0
    gal = {"xyz": synthcat.periodic_catalog(N, L, 5000, seed=9)}
    kf = 2 * np.pi / L
    p = E.Params(N=N, L=L, edges=kf * np.array([1.0, 2.5, 4.0, 5.5, 7.0]), ells=[(0, 0, 0), (2, 2, 2)],
                 los="global", mas=2, interlace=False)
    specs = S.catalogue_spectra_on_disk(p, gal, None, str(tmp_path))
    got = S.measure_pairs(p, specs, {(2, 2, 2): [(1, 3)], (0, 0, 0): [(2, 2)]})
    ref = E.measure(p, gal, None)
    assert np.isclose(got[(2, 2, 2, 1, 3)]["B"], ref["B"][1, 1, 3], rtol=1e-12, atol=0)
    assert np.isclose(got[(0, 0, 0, 2, 2)]["shot"], ref["shot"][0, 2, 2], rtol=1e-12, atol=0)
