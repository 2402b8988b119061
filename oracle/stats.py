"""FP64 oracle of the covariance statistics of a batch of measurements (Sec. 5.5,
Eq. Covariance; App. E, the Hartlap and Percival factors).

TEST INFRASTRUCTURE ONLY.  Plain loops over the definitions; shares no code with the
library.  Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may import it.

Reading: App. E prints the Percival factors with square roots in the denominators of A and B.
With them B -> 1 as Nm -> infinity and M tends to (1 + Nb - Np)/(2 + Np) instead of 1, although M
propagates the noise of an estimated covariance, which vanishes for infinitely many mocks.  Both
sides take the form of the reference the appendix cites, without square roots:
A = 2 / ((Nm - Nb - 1)(Nm - Nb - 4)), B = (Nm - Nb - 2) / ((Nm - Nb - 1)(Nm - Nb - 4)), for which
M -> 1.
"""
from __future__ import annotations

import math

import numpy as np


def covariance(X):
    """mean [nb], C [nb, nb] = 1/(Nm - 1) sum_n (X_n - mean)^T (X_n - mean), r_ij = C_ij / sqrt(C_ii C_jj)."""
    X = np.asarray(X, dtype=np.float64)
    nm, nb = X.shape
    mean = np.zeros(nb)
    for n in range(nm):
        mean += X[n]
    mean /= nm
    C = np.zeros((nb, nb))
    for n in range(nm):
        d = X[n] - mean
        for i in range(nb):
            for j in range(nb):
                C[i, j] += d[i] * d[j]
    C /= nm - 1
    r = np.zeros((nb, nb))
    for i in range(nb):
        for j in range(nb):
            r[i, j] = C[i, j] / math.sqrt(C[i, i] * C[j, j])
    return mean, C, r


def hartlap(n_mock, n_bin):
    """(Nm - Nb - 2) / (Nm - 1), the factor on the inverse covariance."""
    return (n_mock - n_bin - 2) / (n_mock - 1)


def percival_m(n_mock, n_bin, n_par):
    """M = (1 + B (Nb - Np)) / (1 + A + B (Np + 1)) (App. E, A and B without square roots)."""
    den = (n_mock - n_bin - 1) * (n_mock - n_bin - 4)
    A = 2.0 / den
    B = (n_mock - n_bin - 2) / den
    return (1.0 + B * (n_bin - n_par)) / (1.0 + A + B * (n_par + 1))


def chi2(C, n_mock, x_obs, x_theory):
    """(x_obs - x_theory)^T C_Hartlap^{-1} (x_obs - x_theory), C^{-1} by Gauss-Jordan elimination."""
    C = np.asarray(C, dtype=np.float64)
    nb = C.shape[0]
    aug = np.concatenate([C.copy(), np.eye(nb)], axis=1)
    for c in range(nb):
        p = c + int(np.argmax(np.abs(aug[c:, c])))
        aug[[c, p]] = aug[[p, c]]
        aug[c] /= aug[c, c]
        for r in range(nb):
            if r != c:
                aug[r] -= aug[r, c] * aug[c]
    inv = aug[:, nb:] * hartlap(n_mock, nb)
    d = np.asarray(x_obs, dtype=np.float64) - np.asarray(x_theory, dtype=np.float64)
    return float(d @ inv @ d)
