"""Pins of the Gaussian-random-field oracle (oracle/grf.py; Sec. 5,
Algorithm 2) against what the mathematics and the paper fix -- each chosen
so that a plausible mistake fails one of them:

* half-integer shapes, where x^kappa K_kappa(x) has a closed form
  (kappa = 1/2: e^-x; 3/2: (1 + x) e^-x; 5/2: (1 + x + x^2/3) e^-x) -- pins
  the normalisation 2^(1-kappa)/Gamma(kappa) and the sqrt(8 kappa)/phi scale;
* the variance on the diagonal and continuity at d -> 0;
* the paper's statement that phi is the distance beyond which the
  correlation is below 0.14 (true of the sqrt(8 kappa) form only);
* anisotropy: omega = 1 is rotation invariant; with omega > 1 the direction
  theta is the slowest decay and its normal omega times faster;
* K_kappa itself against its integral representation (independent of
  scipy's routine), at the paper's non-half-integer shapes;
* L D L^T reconstructs Sigma (L unit lower triangular, D > 0) for the
  paper's four parameter sets on a grid of the paper's cell size;
* the sample covariance of simulated fields U = L D^(1/2) Z matches Sigma.
"""
import numpy as np
import pytest

pytest.importorskip("scipy")

from oracle import grf  # noqa: E402


@pytest.mark.parametrize("shape,closed", [
    (0.5, lambda x: np.exp(-x)),
    (1.5, lambda x: (1 + x) * np.exp(-x)),
    (2.5, lambda x: (1 + x + x * x / 3) * np.exp(-x)),
])
def test_half_integer_shapes_closed_forms(shape, closed):
    phi, var = 30e3, 1.7
    d = np.concatenate([np.linspace(1.0, 3 * phi, 400), [1e-3, 0.5 * phi, phi, 2 * phi]])
    x = np.sqrt(8 * shape) * d / phi
    got = grf.matern(d, shape, phi, var)
    assert np.allclose(got, var * closed(x), rtol=1e-12, atol=0)


def test_far_tail_stays_positive():
    # kappa = 1/2 at x = 700: variance e^-700, far below any covariance that
    # matters but representable -- the oracle must not underflow to 0 early
    x = 700.0
    got = grf.matern(np.array([x / 2.0]), 0.5, 1.0, 1.3)[0]      # x = sqrt(4) d / phi
    assert got > 0 and got == pytest.approx(1.3 * np.exp(-x), rel=1e-12)


@pytest.mark.parametrize("shape", [0.6, 1.25, 2.15, 3.0])
def test_variance_on_diagonal_and_continuity(shape):
    assert grf.matern(np.array([0.0]), shape, 50e3, 2.0)[0] == 2.0
    near = grf.matern(np.array([1e-6, 1e-3]), shape, 50e3, 2.0)
    assert np.all(np.abs(near - 2.0) < 1e-5)
    assert np.all(near <= 2.0 * (1 + 1e-13))          # the maximum, up to rounding


@pytest.mark.parametrize("shape", [0.5, 0.6, 1.25, 2.15, 3.0])
def test_range_is_where_correlation_falls_below_0_14(shape):
    rho = grf.matern(np.array([0.95, 1.0]), shape, 1.0, 1.0)
    assert rho[0] > 0.14 > rho[1] > 0.13


def test_anisotropy_directions():
    rng = np.random.default_rng(3)
    dx, dy = rng.normal(size=50) * 1e4, rng.normal(size=50) * 1e4
    base = grf.aniso_dist(dx, dy, 1.0, 0.0)
    for theta in (0.3, np.pi / 7, 2.0):
        assert np.allclose(grf.aniso_dist(dx, dy, 1.0, theta), base, rtol=1e-14)
    omega, theta, r = 4.0, np.pi / 7, 1234.5
    c, s = np.cos(theta), np.sin(theta)
    # R(theta) maps (c, -s) onto the x-axis and (s, c) onto the y-axis
    assert np.isclose(grf.aniso_dist(r * c, -r * s, omega, theta), r, rtol=1e-14)
    assert np.isclose(grf.aniso_dist(r * s, r * c, omega, theta), omega * r, rtol=1e-14)


@pytest.mark.parametrize("shape", [0.6, 1.25, 2.15, 3.0])
def test_bessel_k_against_integral_representation(shape):
    from scipy.integrate import quad
    from scipy.special import kv
    for x in (0.05, 0.7, 2.0, 6.0):
        # K_nu(x) = int_0^inf exp(-x cosh t) cosh(nu t) dt; beyond t_max the
        # integrand is below e^-700 of its start
        t_max = np.arccosh(700.0 / x + 1.0)
        f = lambda t: 0.5 * (np.exp(shape * t - x * np.cosh(t)) + np.exp(-shape * t - x * np.cosh(t)))
        ref, _ = quad(f, 0.0, t_max, epsabs=0, epsrel=1e-13, limit=400)
        assert abs(kv(shape, x) - ref) <= 1e-11 * ref


def test_ldl_reconstructs_covariance_for_the_papers_parameters():
    pts = grf.square_grid(12, 15, 4000.0)            # the paper's cell size, 180 cells
    for params in grf.PAPER_PARAMS:
        S = grf.matern_cov(pts, params)
        assert np.allclose(S, S.T, rtol=0, atol=0)
        assert np.allclose(np.diag(S), params[2])
        L, D = grf.ldl(S)
        assert np.allclose(np.diag(L), 1.0, rtol=0, atol=1e-15)
        assert np.allclose(np.triu(L, 1), 0.0)
        assert (D > 0).all()
        assert np.abs(L @ (D[:, None] * L.T) - S).max() <= 1e-12 * params[2]


def test_simulated_fields_have_the_covariance():
    pts = grf.square_grid(5, 6, 4000.0)
    params = grf.PAPER_PARAMS[1]                      # anisotropic, shape 2.15
    S = grf.matern_cov(pts, params)
    L, D = grf.ldl(S)
    nsim = 40000
    Z = np.random.default_rng(11).standard_normal((len(pts), nsim))
    U = grf.simulate(L, D, Z)
    C = U @ U.T / nsim
    sd = np.sqrt((np.outer(np.diag(S), np.diag(S)) + S * S) / nsim)
    assert (np.abs(C - S) <= 5 * sd).all()
