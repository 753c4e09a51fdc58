"""Plain CPU oracle for Gaussian random fields by direct matrix decomposition
(Sec. 5, Algorithm 2) -- the fourth application of the paper's generator.

TEST INFRASTRUCTURE ONLY, like the rest of this package: nothing in the
product imports it.  Everything is float64 numpy; the modified Bessel
function K (as the exponentially scaled kve times e^-x) and the gamma
function come from scipy.special and the Cholesky factor from numpy.linalg
as library steps.  The standard normals Z are an
input (the GPU path draws them from its streams).

What the functions compute:
  * matern(dist, shape, range_, variance): the Matern covariance of Sec. 5,
    variance * 2^(1-kappa) / Gamma(kappa) * x^kappa * K_kappa(x) with
    x = sqrt(8 kappa) |d| / phi, and the variance itself at d = 0 (the limit
    of x^kappa K_kappa(x) is 2^(kappa-1) Gamma(kappa)).  The printed formula
    reads 2^(kappa-1); only 2^(1-kappa) gives var(U_i) = variance, which the
    paper states, so that is the reading taken.
  * aniso_dist(dx, dy, ratio, angle): |d| for d = diag(1, omega) R(theta) dx
    with R(theta) = [[cos, -sin], [sin, cos]] (Sec. 5).
  * matern_cov(points, params): the covariance matrix of one parameter set
    (shape, range, variance, anisoRatio, anisoAngleRadians) -- Algorithm 2
    step 1.
  * ldl(sigma): Sigma = L D L^T with L unit lower triangular -- step 2
    (from the Cholesky factor C: D = diag(C)^2, L = C diag(C)^-1).
  * simulate(L, D, Z): U = L D^(1/2) Z -- step 4.
  * square_grid(nrow, ncol, cell): centres of an nrow x ncol raster of square
    cells (the stand-in for the paper's 62 x 90 raster over Switzerland).
"""
from __future__ import annotations

import numpy as np
from scipy.special import gamma, kve

# The four parameter sets of the paper's example (Sec. 5, step 2):
# (shape kappa, range phi [m], variance sigma^2, anisoRatio omega, anisoAngleRadians theta)
PAPER_PARAMS = (
    (1.25, 50e3, 1.5, 1.0, 0.0),
    (2.15, 60e3, 2.0, 4.0, np.pi / 7),
    (0.60, 30e3, 2.0, 2.0, np.pi / 5),
    (3.00, 30e3, 2.0, 2.0, np.pi / 7),
)
# The paper's raster: 62 rows x 90 columns (5580 cells).
PAPER_GRID = (62, 90)


def matern(dist, shape: float, range_: float, variance: float) -> np.ndarray:
    """Matern covariance at distances |d| >= 0 (Sec. 5)."""
    d = np.asarray(dist, dtype=np.float64)
    x = np.sqrt(8.0 * shape) * d / range_
    out = np.full(d.shape, float(variance))
    pos = x > 0
    xp = x[pos]
    # K_kappa(x) = kve(kappa, x) e^-x: scipy's unscaled kv returns 0 from
    # x ~ 700 on, where K is still a representable positive number
    out[pos] = (variance * 2.0 ** (1.0 - shape) / gamma(shape) * xp ** shape * np.exp(-xp)
                * kve(shape, xp))
    return out


def aniso_dist(dx, dy, ratio: float, angle: float) -> np.ndarray:
    """|diag(1, omega) R(theta) (dx, dy)| (Sec. 5)."""
    c, s = np.cos(angle), np.sin(angle)
    u = c * np.asarray(dx, dtype=np.float64) - s * np.asarray(dy, dtype=np.float64)
    v = ratio * (s * np.asarray(dx, dtype=np.float64) + c * np.asarray(dy, dtype=np.float64))
    return np.hypot(u, v)


def matern_cov(points: np.ndarray, params) -> np.ndarray:
    """Covariance matrix of the points (n x 2, metres) for one parameter set
    (Algorithm 2, step 1)."""
    shape, range_, variance, ratio, angle = params
    p = np.asarray(points, dtype=np.float64)
    dx = p[:, None, 0] - p[None, :, 0]
    dy = p[:, None, 1] - p[None, :, 1]
    return matern(aniso_dist(dx, dy, ratio, angle), shape, range_, variance)


def ldl(sigma: np.ndarray):
    """Sigma = L D L^T, L unit lower triangular, D > 0 (Algorithm 2, step 2)."""
    c = np.linalg.cholesky(np.asarray(sigma, dtype=np.float64))
    dc = np.diag(c)
    return c / dc[None, :], dc * dc


def simulate(L: np.ndarray, D: np.ndarray, Z: np.ndarray) -> np.ndarray:
    """U = L D^(1/2) Z for standard normal columns Z (Algorithm 2, step 4)."""
    return L @ (np.sqrt(D)[:, None] * np.asarray(Z, dtype=np.float64))


def square_grid(nrow: int, ncol: int, cell: float) -> np.ndarray:
    """Centres of an nrow x ncol raster of square cells, row-major, as n x 2
    (x, y) coordinates in the units of `cell`."""
    yy, xx = np.meshgrid((np.arange(nrow) + 0.5) * cell, (np.arange(ncol) + 0.5) * cell,
                         indexing="ij")
    return np.stack([xx.ravel(), yy.ravel()], axis=1)
