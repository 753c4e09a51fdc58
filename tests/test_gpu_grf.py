"""Gaussian random fields on the GPU (Sec. 5, Algorithm 2) against the
oracle (oracle/grf.py), through the C ABI:

* step 1 -- covariance entries element by element (raster and arbitrary
  points), relative 1e-12 (the device Bessel K is accurate to ~1e-13);
* step 2 -- the factor's reconstruction ||L D L^T - Sigma||_max <= 1e-12
  sigma^2, L unit lower triangular, D > 0, and L, D against the oracle's
  (LAPACK Cholesky) factor within a bound scaled by the conditioning of the
  matrices; sizes span several 128-column panels with a ragged tail, one
  panel exactly, and n = 1; a matrix that is not positive definite is
  reported through info;
* step 4 -- U = L D^(1/2) Z element by element against the oracle's product
  with the same L, D and Z (1e-13 relative to sum |L_ij| sqrt(D_j) |Z_j|),
  and against the oracle's own factor within the factor's tolerance;
* the paper's size (four 5580 x 5580 matrices on the 62 x 90 raster of 4 km
  cells, the paper's four parameter sets) in the launch configuration the
  benchmark times: sampled entries of Sigma, of L D L^T - Sigma and of U.
"""
import numpy as np
import pytest
import torch

from oracle import grf as G

pytestmark = pytest.mark.gpu

CELL = 4000.0
PARAMS = np.array(G.PAPER_PARAMS)


@pytest.fixture(scope="module")
def R():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2201_06604_gb300 import grf
    return grf


def oracle_cov(nrow, ncol, cell, params):
    pts = G.square_grid(nrow, ncol, cell)
    return np.stack([G.matern_cov(pts, p) for p in params])


def test_raster_covariance_matches_oracle(R):
    nrow, ncol = 9, 13
    got = R.matern_raster(PARAMS, nrow, ncol, CELL).cpu().numpy()
    ref = oracle_cov(nrow, ncol, CELL, PARAMS)
    assert got.shape == ref.shape
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-300)
    assert np.array_equal(got, np.transpose(got, (0, 2, 1)))          # symmetric exactly


@pytest.mark.parametrize("nrow,ncol,pad", [(4, 1, 0), (2, 3, 0), (5, 8, 0), (6, 10, 4), (12, 25, 3),
                                            (1, 7, 1), (33, 2, 0)])
def test_raster_covariance_layouts(R, nrow, ncol, pad):
    # one-column rasters, rows that wrap inside a thread's four columns, the
    # 32-byte store path (n and ld multiples of 4) and padded leading
    # dimensions (the padding stays untouched)
    n = nrow * ncol
    out = torch.full((len(PARAMS), n, n + pad), -7.0, dtype=torch.float64, device="cuda")
    R.matern_raster(PARAMS, nrow, ncol, CELL, out=out[:, :, :n])
    got = out.cpu().numpy()
    ref = oracle_cov(nrow, ncol, CELL, PARAMS)
    np.testing.assert_allclose(got[:, :, :n], ref, rtol=1e-12, atol=1e-300)
    assert (got[:, :, n:] == -7.0).all()


def test_points_covariance_matches_oracle(R):
    rng = np.random.default_rng(5)
    pts = rng.uniform(0, 60e3, size=(70, 2))
    xy = torch.tensor(pts, dtype=torch.float64, device="cuda")
    got = R.matern_points(PARAMS, xy).cpu().numpy()
    ref = np.stack([G.matern_cov(pts, p) for p in PARAMS])
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-300)


def check_factor(sigma, L, D, tol_rel=1e-12):
    """L unit lower (strict lower part read), D > 0, ||L D L^T - Sigma|| small."""
    n = sigma.shape[-1]
    Lu = np.tril(L, -1) + np.eye(n)
    rec = (Lu * D[None, :]) @ Lu.T
    s2 = np.abs(np.diag(sigma)).max()
    err = np.abs(np.tril(rec - sigma)).max()
    assert (D > 0).all()
    assert err <= tol_rel * s2, err / s2
    return err / s2


@pytest.mark.parametrize("nrow,ncol", [(15, 20), (8, 16), (1, 1), (3, 43)])
def test_ldl_reconstructs_sigma(R, nrow, ncol):
    # n = 300 (two panels + a 44-column tail), 128 (one panel exactly), 1, 129
    cov = R.matern_raster(PARAMS, nrow, ncol, CELL)
    sigma = cov.cpu().numpy()
    a, d, info = R.ldl(cov)
    assert info == [0, 0, 0, 0]
    L, D = a.cpu().numpy(), d.cpu().numpy()
    for b in range(len(PARAMS)):
        assert np.array_equal(np.diag(L[b]), D[b])              # D on the diagonal too
        check_factor(sigma[b], L[b], D[b])
        Lo, Do = G.ldl(sigma[b])
        # forward error of a backward-stable factor: ~ n u cond(Sigma) relative
        cond = np.linalg.cond(sigma[b]) if sigma.shape[-1] > 1 else 1.0
        tol = max(1e-12, 64 * sigma.shape[-1] * 2.0 ** -52 * cond)
        assert np.abs(np.tril(L[b], -1) - np.tril(Lo, -1)).max() <= tol
        assert np.abs(D[b] - Do).max() <= tol * np.abs(Do).max()


def test_ldl_random_spd_spans_scales(R):
    # a random SPD matrix (not a covariance of the raster) whose diagonal
    # spans six orders of magnitude: the row scaling of the slices and the
    # power-of-two scaling of the diagonal blocks
    rng = np.random.default_rng(11)
    n = 333
    q = rng.standard_normal((n, n))
    s = q @ q.T / n + np.eye(n)
    sc = 10.0 ** rng.uniform(-3, 3, n)
    s = s * sc[:, None] * sc[None, :]
    a = torch.tensor(s[None], device="cuda")
    a, d, info = R.ldl(a)
    assert info == [0]
    L, D = a[0].cpu().numpy(), d[0].cpu().numpy()
    Lu = np.tril(L, -1) + np.eye(n)
    rec = (Lu * D[None, :]) @ Lu.T
    # componentwise backward error relative to sqrt(s_ii s_jj)
    den = np.sqrt(np.outer(np.diag(s), np.diag(s)))
    assert np.abs(np.tril(rec - s) / den).max() <= 1e-12


def test_ldl_reports_non_positive_pivot(R):
    n = 200
    s = np.eye(n)
    s[150, 150] = -1.0                                   # pivot 150 is negative
    a = torch.tensor(np.stack([np.eye(n), s]), device="cuda")
    _, _, info = R.ldl(a)
    assert info == [0, 151]


def test_simulate_matches_oracle(R):
    from paper_2201_06604_gb300 import mrg
    nrow, ncol, nsim = 12, 25, 3
    cov = R.matern_raster(PARAMS, nrow, ncol, CELL)
    sigma = cov.cpu().numpy()
    a, d, info = R.ldl(cov)
    assert info == [0] * 4
    n = nrow * ncol
    s = mrg.create_streams(len(PARAMS) * nsim, seed=(12345,) * 6)
    z = mrg.generate(s, n, "normal", torch.float64).view(len(PARAMS), nsim, n)
    u = R.simulate(a, d, z).cpu().numpy()
    L, D, Z = a.cpu().numpy(), d.cpu().numpy(), z.cpu().numpy()
    for b in range(len(PARAMS)):
        Lu = np.tril(L[b], -1) + np.eye(n)
        ref = G.simulate(Lu, D[b], Z[b].T).T                       # same L, D, Z
        mag = (np.abs(Lu) @ (np.sqrt(D[b])[:, None] * np.abs(Z[b].T))).T
        assert (np.abs(u[b] - ref) <= 1e-13 * mag + 1e-300).all()
        Lo, Do = G.ldl(sigma[b])
        ref_o = G.simulate(Lo, Do, Z[b].T).T                        # the oracle's own factor
        cond = np.linalg.cond(sigma[b])
        assert np.abs(u[b] - ref_o).max() <= max(1e-10, 64 * n * 2.0 ** -52 * cond) * mag.max()


def test_paper_size_sampled(R):
    """The paper's example: four 5580 x 5580 matrices (62 x 90 raster, 4 km
    cells, the four printed parameter sets), two simulations each."""
    from paper_2201_06604_gb300 import mrg
    nrow, ncol = G.PAPER_GRID
    n = nrow * ncol
    cov = R.matern_raster(PARAMS, nrow, ncol, CELL)
    rng = np.random.default_rng(3)
    rows = np.unique(np.concatenate([[0, 1, 127, 128, 129, n - 1], rng.integers(0, n, 24)]))
    pts = G.square_grid(nrow, ncol, CELL)
    sig_rows = cov[:, rows, :].cpu().numpy()
    for b, p in enumerate(PARAMS):
        dx = pts[rows][:, None, 0] - pts[None, :, 0]
        dy = pts[rows][:, None, 1] - pts[None, :, 1]
        ref = G.matern(G.aniso_dist(dx, dy, p[3], p[4]), p[0], p[1], p[2])
        np.testing.assert_allclose(sig_rows[b], ref, rtol=1e-12, atol=1e-300)
    a, d, info = R.ldl(cov)
    assert info == [0] * 4
    D = d.cpu().numpy()
    assert (D > 0).all()
    # (L D L^T)_ij for sampled rows i and every j <= i, from L's rows on the host
    Lr = a[:, rows, :].cpu().numpy()
    below = np.arange(n)[None, :] < rows[:, None]         # column j < row i: L's strict lower part

    def unit_lower(m):
        out = np.where(below, m, 0.0)
        out[np.arange(len(rows)), rows] = 1.0
        return out

    for b in range(4):
        Lb = unit_lower(Lr[b])
        full_rows = {int(r): k for k, r in enumerate(rows)}
        for k, i in enumerate(rows):
            # row j of L for the sampled j: reuse the sampled rows themselves
            for j in rows[rows <= i]:
                lj = Lb[full_rows[int(j)]]
                v = np.dot(Lb[k] * D[b], lj)
                assert abs(v - sig_rows[b][k, j]) <= 1e-12 * 2.0, (b, i, j, v - sig_rows[b][k, j])
    # U for two simulations, sampled rows against L_i. D^(1/2) Z on the host
    s = mrg.create_streams(8, seed=(12345,) * 6)
    z = mrg.generate(s, n, "normal", torch.float64).view(4, 2, n)
    u = R.simulate(a, d, z).cpu().numpy()
    Z = z.cpu().numpy()
    for b in range(4):
        Lb = unit_lower(Lr[b])
        y = np.sqrt(D[b])[None, :] * Z[b]
        ref = (Lb @ y.T).T
        mag = (np.abs(Lb) @ np.abs(y.T)).T
        assert (np.abs(u[b][:, rows] - ref) <= 1e-13 * mag).all()


def test_padded_rows_single_matrix_and_many_simulations(R):
    """lda > n with rows that are not 32-byte aligned (the element-wise
    epilogue path), one matrix, an odd order, and nine simulations (two passes
    of the product kernel) -- through the C ABI directly."""
    import ctypes
    from paper_2201_06604_gb300 import mrg
    rng = np.random.default_rng(9)
    n, lda, nsim = 211, 215, 9
    pts = rng.uniform(0, 80e3, size=(n, 2))
    p = PARAMS[1]
    sigma = G.matern_cov(pts, p)
    buf = torch.zeros((1, n, lda), dtype=torch.float64, device="cuda")
    buf[0, :, :n] = torch.tensor(sigma, device="cuda")
    d = torch.empty((1, n), dtype=torch.float64, device="cuda")
    ws = R.ldl_workspace(n, 1, buf.device)
    wp, wn = R._aligned(ws)
    info = (ctypes.c_int32 * 1)()
    st = torch.cuda.current_stream().cuda_stream
    assert mrg.lib.mrg_grf_ldl(buf.data_ptr(), n, lda, 1, d.data_ptr(), wp, wn, info, st) == mrg.OK
    assert list(info) == [0]
    L = buf[0, :, :n].cpu().numpy()
    D = d[0].cpu().numpy()
    check_factor(sigma, L, D)
    s = mrg.create_streams(nsim, seed=(12345,) * 6)
    z = mrg.generate(s, n, "normal", torch.float64).view(1, nsim, n)
    u = torch.empty_like(z)
    nb = int(mrg.lib.mrg_grf_simulate_scratch_bytes(n, nsim, 1))
    scratch = torch.empty(nb, dtype=torch.uint8, device="cuda")
    assert mrg.lib.mrg_grf_simulate(buf.data_ptr(), d.data_ptr(), n, lda, 1, z.data_ptr(), nsim,
                                    u.data_ptr(), scratch.data_ptr(), nb, st) == mrg.OK
    Lu = np.tril(L, -1) + np.eye(n)
    Z = z[0].cpu().numpy()
    ref = G.simulate(Lu, D, Z.T).T
    mag = (np.abs(Lu) @ (np.sqrt(D)[:, None] * np.abs(Z.T))).T
    assert (np.abs(u[0].cpu().numpy() - ref) <= 1e-13 * mag + 1e-300).all()
