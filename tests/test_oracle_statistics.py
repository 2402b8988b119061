"""Statistical pins of the oracle on the synthetic generator (64^3, 2e5 particles, CIC, global
line of sight): an isotropic field has no quadrupole, a Kaiser-boosted one a positive B_202.

For a field whose law is symmetric under the cube's rotations (the unboosted generator, CIC
assignment and deconvolution are) E[B_202] = 0 exactly on the mesh: the L = 2 weight averages to
zero over the rotated copies of every triangle.  A mistake that leaks B_000 into B_202 (a wrong
constant in y_2^0 or in a 3j symbol) shows up as a mean many standard errors from zero.  The
generator's redshift-space boost (1 + 0.7 mu^2) along z makes B_202 positive."""
import numpy as np

import synthcat
from oracle import estimator as E

N, L = 64, 1000.0
EDGES = [0.03, 0.05, 0.07, 0.09]


def _runs(seeds, kaiser):
    p = E.Params(N=N, L=L, edges=EDGES, ells=[(0, 0, 0), (2, 0, 2)], los="global", mas=2)
    out = []
    for s in seeds:
        gal = {"xyz": synthcat.periodic_catalog(N, L, 200_000, s, kaiser=kaiser)}
        out.append(E.measure(p, gal, None)["B"])
    v = np.array(out)
    return v.mean(axis=0), v.std(axis=0, ddof=1) / np.sqrt(len(v))


def test_isotropic_field_has_no_quadrupole():
    mean, se = _runs(range(700, 724), 0.0)
    t = mean[1] / se[1]
    assert np.all(np.abs(t) < 4.0), t
    assert np.all(mean[0] / se[0] > 20.0)  # the monopole is measured with high significance


def test_kaiser_boost_gives_a_positive_quadrupole():
    mean, se = _runs(range(900, 906), 0.7)
    assert np.all(mean[1] / se[1] > 3.0), mean[1] / se[1]
