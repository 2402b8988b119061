"""Covariance statistics of batches of measurements (Sec. 5.5, Eq. Covariance; App. E): the
oracle against library routines and statistical facts, and the host functions of the C ABI
against the oracle.  No GPU: these functions do no device work."""
import numpy as np
import pytest

import paper_1803_02132_gb300 as bisp
from oracle import stats as S


def _batch(seed, nm=40, nb=7):
    rng = np.random.default_rng(seed)
    A = rng.normal(size=(nb, nb))
    cov = A @ A.T + nb * np.eye(nb)
    mean = rng.normal(size=nb) * 10
    return rng.multivariate_normal(mean, cov, size=nm), mean, cov


def test_oracle_covariance_matches_numpy():
    X, _, _ = _batch(1)
    mean, C, r = S.covariance(X)
    assert np.allclose(mean, X.mean(axis=0), rtol=1e-13)
    assert np.allclose(C, np.cov(X, rowvar=False, ddof=1), rtol=1e-12)
    assert np.allclose(r, np.corrcoef(X, rowvar=False), rtol=1e-12)
    assert np.allclose(np.diag(r), 1.0)


def test_oracle_chi2_matches_solve():
    X, mean, cov = _batch(2)
    _, C, _ = S.covariance(X)
    x = X[0] + 0.3
    ref = (x - mean) @ np.linalg.solve(C, x - mean) * S.hartlap(len(X), C.shape[0])
    assert S.chi2(C, len(X), x, mean) == pytest.approx(ref, rel=1e-10)


def test_factors_limits():
    # both factors tend to 1 for infinitely many realisations; the Percival factor inflates
    # parameter variances (M > 1) when the bins outnumber the parameters well (Nb > 2 Np + 1 + A/B)
    for nb in (5, 40):
        assert S.hartlap(10 ** 9, nb) == pytest.approx(1.0, abs=1e-7)
        assert S.percival_m(10 ** 7, nb, 2) == pytest.approx(1.0, abs=1e-5)
    assert S.percival_m(140, 40, 2) > 1.0
    assert S.percival_m(140, 5, 2) < 1.0
    assert S.hartlap(600, 11) == pytest.approx(587 / 599)


def test_hartlap_makes_chi2_unbiased():
    # E[chi^2] of an independent Gaussian vector against the true mean, with the inverse of a
    # covariance estimated from Nm realisations, is Nb after the Hartlap factor (and
    # Nb (Nm - 1)/(Nm - Nb - 2) without it)
    rng = np.random.default_rng(3)
    nb, nm, trials = 6, 24, 3000
    L = np.tril(rng.normal(size=(nb, nb))) + 3 * np.eye(nb)
    cov = L @ L.T
    vals = []
    for _ in range(trials):
        X = rng.normal(size=(nm, nb)) @ L.T
        C = np.cov(X, rowvar=False, ddof=1)
        x = rng.normal(size=nb) @ L.T
        vals.append(x @ np.linalg.solve(C, x) * S.hartlap(nm, nb))
    m = float(np.mean(vals))
    se = float(np.std(vals)) / np.sqrt(trials)
    assert abs(m - nb) < 4 * se
    assert abs(m / S.hartlap(nm, nb) - nb) > 8 * se  # the uncorrected value is visibly biased


def test_library_matches_oracle():
    X, mean, _ = _batch(4, nm=37, nb=9)
    out = bisp.covariance(X, n_par=2)
    m, C, r = S.covariance(X)
    assert np.allclose(out["mean"], m, rtol=1e-13)
    assert np.allclose(out["cov"], C, rtol=1e-12)
    assert np.allclose(out["corr"], r, rtol=1e-12)
    assert out["hartlap"] == S.hartlap(37, 9)
    assert out["percival_m"] == pytest.approx(S.percival_m(37, 9, 2), rel=1e-14)
    x = X[3] * 1.01
    assert bisp.chi2(C, 37, x, mean) == pytest.approx(S.chi2(C, 37, x, mean), rel=1e-10)


def test_library_errors():
    with pytest.raises(bisp.BispError) as e:
        bisp.covariance(np.zeros((1, 3)))
    assert e.value.status == bisp.BISP_EINVAL
    with pytest.raises(bisp.BispError, match="Percival"):
        bisp.covariance(np.random.default_rng(0).normal(size=(8, 5)), n_par=1)
    with pytest.raises(bisp.BispError, match="positive definite"):
        bisp.chi2(np.zeros((3, 3)), 10, np.ones(3), np.zeros(3))
