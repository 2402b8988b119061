"""Seeded synthetic galaxy catalogues (inputs only).

This module draws the random inputs that both the CUDA path and the FP64 oracle
consume.  It holds none of the estimator's arithmetic: it only makes particle
positions, weights and expected number densities.  The recipe follows the
workloads of the paper (periodic simulation boxes with a global line of sight,
Sec. 4.4, and survey-like catalogues with a local line of sight and a random
catalogue, Sec. 4.1 and Sec. 5.2):

* a Gaussian field with power spectrum P(k) = 2e4 (k/0.05)^-1.5 (Mpc/h)^3 for
  k > 0.005 h/Mpc (zero below), drawn as white noise on a generator mesh;
* a local quadratic term, delta = dG + (dG^2 - <dG^2>)/2, which gives the field a
  tree-level-like bispectrum;
* a Kaiser-like boost delta(k) *= (1 + 0.7 mu^2), mu measured from the z axis;
* Poisson sampling of particles with cell intensity proportional to
  max(1 + delta, 0) (times the survey selection for survey catalogues), with
  positions uniform inside the generator cell.

All draws come from numpy's PCG64 generator seeded with the given seed.
Positions are float32 in [0, L).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "power_law_pk",
    "clustered_field",
    "periodic_catalog",
    "survey_catalogs",
    "uniform_catalog",
]


def power_law_pk(k):
    """P(k) = 2e4 (k/0.05)^-1.5 for k > 0.005 h/Mpc, else 0."""
    k = np.asarray(k, dtype=np.float64)
    out = np.zeros_like(k)
    m = k > 0.005
    out[m] = 2.0e4 * (k[m] / 0.05) ** -1.5
    return out


def _kgrid(n, box):
    kf = 2.0 * np.pi / box
    k1 = np.fft.fftfreq(n, d=1.0 / n) * kf
    kz = np.fft.rfftfreq(n, d=1.0 / n) * kf
    return k1, kz


def clustered_field(n, box, seed, kaiser=0.7, quadratic=True):
    """Density contrast delta on an n^3 generator mesh (float32, C order x,y,z).

    <|dG(k)|^2> = V P(k) with the continuous Fourier convention; the quadratic term
    and the (1 + kaiser mu^2) boost are applied as described in the module doc.
    """
    rng = np.random.default_rng(seed)
    vol = float(box) ** 3
    white = rng.standard_normal((n, n, n), dtype=np.float32)
    wk = np.fft.rfftn(white)
    del white
    k1, kz = _kgrid(n, box)
    kk = np.sqrt(k1[:, None, None] ** 2 + k1[None, :, None] ** 2 + kz[None, None, :] ** 2)
    # discrete amplitude: DFT of a field with <|delta(k)|^2> = V P has variance n^6 P / V,
    # white noise DFT has variance n^3.
    amp = np.sqrt(power_law_pk(kk) * n ** 3 / vol).astype(np.float32)
    dk = wk * amp
    del wk, amp
    dg = np.fft.irfftn(dk, s=(n, n, n), axes=(0, 1, 2)).astype(np.float32)
    del dk
    if quadratic:
        dg = dg + 0.5 * (dg * dg - np.mean(dg.astype(np.float64) ** 2)).astype(np.float32)
    if kaiser:
        dk = np.fft.rfftn(dg)
        with np.errstate(invalid="ignore", divide="ignore"):
            mu2 = np.where(kk > 0, (kz[None, None, :] / np.where(kk > 0, kk, 1.0)) ** 2, 0.0)
        dk *= (1.0 + kaiser * mu2).astype(np.float32)
        dg = np.fft.irfftn(dk, s=(n, n, n), axes=(0, 1, 2)).astype(np.float32)
        del dk
    return dg


def _sample_cells(rng, lam, cell, box):
    """Poisson counts per cell with intensity lam, uniform positions in each cell."""
    counts = rng.poisson(lam.ravel())
    idx = np.repeat(np.arange(counts.size, dtype=np.int64), counts)
    n = lam.shape[0]
    ix = idx // (n * n)
    iy = (idx // n) % n
    iz = idx % n
    off = rng.random((idx.size, 3))
    pos = np.empty((idx.size, 3), dtype=np.float64)
    pos[:, 0] = (ix + off[:, 0]) * cell
    pos[:, 1] = (iy + off[:, 1]) * cell
    pos[:, 2] = (iz + off[:, 2]) * cell
    pos = pos.astype(np.float32)
    pos[pos >= np.float32(box)] -= np.float32(box)
    pos[pos < 0] += np.float32(box)
    return pos


def periodic_catalog(n_gen, box, n_particles, seed, kaiser=0.7, quadratic=True):
    """Periodic-box catalogue: float32 positions (n, 3) Poisson-sampled from max(1+delta, 0)."""
    delta = clustered_field(n_gen, box, seed, kaiser=kaiser, quadratic=quadratic)
    rho = np.maximum(1.0 + delta, 0.0).astype(np.float64)
    del delta
    lam = rho * (n_particles / rho.sum())
    rng = np.random.default_rng(seed + 7919)
    return _sample_cells(rng, lam, box / n_gen, box)


def uniform_catalog(box, n_particles, seed):
    """Unclustered uniform positions in [0, box)^3 (float32)."""
    rng = np.random.default_rng(seed)
    pos = (rng.random((n_particles, 3)) * box).astype(np.float32)
    pos[pos >= np.float32(box)] = 0.0
    return pos


def survey_nbar_shape(r, r_mean=1350.0, sigma=200.0):
    return np.exp(-0.5 * ((r - r_mean) / sigma) ** 2)


def _survey_mask(pos, observer, r_min, r_max, half_angle_deg):
    d = pos.astype(np.float64) - np.asarray(observer, dtype=np.float64)[None, :]
    r = np.sqrt(np.sum(d * d, axis=1))
    u = d / np.where(r > 0, r, 1.0)[:, None]
    ra = np.degrees(np.arctan2(u[:, 0], u[:, 2]))
    dec = np.degrees(np.arcsin(np.clip(u[:, 1], -1.0, 1.0)))
    m = (r >= r_min) & (r <= r_max) & (np.abs(ra) <= half_angle_deg) & (np.abs(dec) <= half_angle_deg)
    return m, r


def survey_catalogs(n_gen, box, observer, n_gal, n_ran, seed, r_min=1000.0, r_max=1700.0,
                    half_angle_deg=30.0, r_mean=1350.0, sigma=200.0, kaiser=0.7):
    """Survey-like galaxies and randoms with a radial selection n(r) and an angular cap.

    Returns (gal, ran), each a dict with float32 'xyz' (n,3) and float32 'nbar' (n,):
    the expected galaxy number density at the object's position, normalised so that
    its integral over the selected volume equals the requested galaxy count.
    """
    cell = box / n_gen
    c = (np.arange(n_gen) + 0.5) * cell
    # selection evaluated at cell centres (x, y planes are broadcast lazily per x slab)
    sel = np.empty((n_gen, n_gen, n_gen), dtype=np.float32)
    yy, zz = np.meshgrid(c, c, indexing="ij")
    for i in range(n_gen):
        p = np.stack([np.full(yy.size, c[i]), yy.ravel(), zz.ravel()], axis=1)
        m, r = _survey_mask(p, observer, r_min, r_max, half_angle_deg)
        sel[i] = (m * survey_nbar_shape(r, r_mean, sigma)).reshape(n_gen, n_gen)
    sel_sum = float(sel.sum(dtype=np.float64))
    # amplitude A of nbar(x) = A * shape(r) inside the selection, with integral = n_gal
    amp = n_gal / (sel_sum * cell ** 3)

    delta = clustered_field(n_gen, box, seed, kaiser=kaiser)
    lam_g = sel * np.maximum(1.0 + delta, 0.0)
    del delta
    lam_g = lam_g.astype(np.float64)
    lam_g *= n_gal / lam_g.sum()
    rng = np.random.default_rng(seed + 104729)
    gal = _sample_cells(rng, lam_g, cell, box)
    del lam_g
    lam_r = sel.astype(np.float64) * (n_ran / sel_sum)
    ran = _sample_cells(rng, lam_r, cell, box)
    del lam_r, sel

    def nbar_of(pos):
        _, r = _survey_mask(pos, observer, r_min, r_max, half_angle_deg)
        return (amp * survey_nbar_shape(r, r_mean, sigma)).astype(np.float32)

    return ({"xyz": gal, "nbar": nbar_of(gal)}, {"xyz": ran, "nbar": nbar_of(ran)})
