"""The paper's matrix layout (runifGpu / rexpGpu with Nglobal, Sec. 2.2 and
3.2) as a compatibility mode, through the C ABI.

* The paper's printed examples, reproduced through this layout on MRG31k3p
  streams created from 12345 x 6: runifGpu(n = 8, Nglobal = c(2, 2)) and then
  rexpGpu(c(2, 4), rate = 1, Nglobal = c(2, 2)) on the same streams.
* Parity with a plain restatement of the layout on the oracle's draws for
  ragged shapes, both generators: the same values (bit-exact uniforms and
  integers, exponentials within tolerance) and the same final states.
"""
import numpy as np
import pytest
import torch

import oracle as O

pytestmark = pytest.mark.gpu

SEED = (12345,) * 6
GENS = {"mrg32k3a": O.MRG32K3A, "mrg31k3p": O.MRG31K3P}


@pytest.fixture(scope="module")
def M():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2201_06604_gb300 import mrg
    return mrg


def test_printed_runif_and_rexp_through_the_matrix_layout(M, golden):
    s = M.create_streams(4, seed=SEED, generator="mrg31k3p")
    u = M.generate_matrix(s, 8, (2, 2), "uniform", torch.float64).cpu().numpy()
    want = [float(v) for v in golden("mrg31k3p_runif.txt")[0]]
    assert np.abs(u - np.array(want)).max() <= 0.0005 + 1e-12, (u, want)
    e = M.generate_matrix(s, (2, 4), (2, 2), "exponential", torch.float64, rate=1.0).cpu().numpy()
    rows = golden("mrg31k3p_rexp.txt")
    for r in range(2):
        for c in range(4):
            dec = len(rows[r][c].split(".")[1])
            assert abs(e[r, c] - float(rows[r][c])) <= 0.5 * 10 ** -dec + 1e-12


def layout_reference(states, nrow, ncol, g0, g1, dist, f32, rate, gen):
    """The layout written out: work item t = i0 * g1 + i1 takes stream t's
    draws in its visiting order over the column-padded matrix."""
    npad = -(-ncol // g1) * g1
    out = np.zeros((nrow, ncol), np.float64 if dist != O.RAW else np.uint32)
    after = states.copy()
    for t in range(g0 * g1):
        i0, i1 = divmod(t, g1)
        pos = [(r, c) for r in range(i0, nrow, g0) for c in range(i1, npad, g1)]
        vals, st = O.generate_streams(states[t:t + 1], len(pos), dist, f32=f32, rate=rate, gen=gen)
        after[t] = st[0]
        for k, (r, c) in enumerate(pos):
            if c < ncol:
                out[r, c] = vals[0, k]
    return out, after


@pytest.mark.parametrize("generator", list(GENS))
@pytest.mark.parametrize("dist,dtype", [("uniform", torch.float64), ("uniform", torch.float32),
                                        ("raw", torch.int32), ("exponential", torch.float64),
                                        ("exponential", torch.float32)])
@pytest.mark.parametrize("nrow,ncol,g", [(37, 13, (4, 3)), (5, 1, (2, 2)), (8, 64, (1, 7))])
def test_layout_matches_reference(M, generator, dist, dtype, nrow, ncol, g):
    gen = GENS[generator]
    ns = g[0] * g[1] + 3
    s = M.create_streams(ns, seed=(7, 7, 7, 7, 7, 7), generator=generator)
    st0 = M.get_state(s)[0].T.copy()
    got = M.generate_matrix(s, (nrow, ncol), g, dist, dtype, rate=1.5).cpu().numpy()
    dcode = {"uniform": O.UNIFORM, "raw": O.RAW, "exponential": O.EXPONENTIAL}[dist]
    ref, after = layout_reference(st0, nrow, ncol, g[0], g[1], dcode, dtype == torch.float32, 1.5,
                                  gen)
    if dist == "raw":
        assert np.array_equal(got.view(np.uint32), ref)
    elif dist == "uniform":
        assert np.array_equal(got.astype(np.float64), ref)
    elif dtype == torch.float64:
        assert np.abs(got - ref).max() <= 1e-12 / 1.5 + 1e-12
    else:
        ulp = np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64)
        assert (np.abs(got.astype(np.float64) - ref) <= 2 * ulp).all()
    st = M.get_state(s)[0].T
    assert np.array_equal(st[: g[0] * g[1]], after[: g[0] * g[1]])
    assert np.array_equal(st[g[0] * g[1]:], st0[g[0] * g[1]:])     # unused streams untouched


def test_matrix_errors(M):
    s = M.create_streams(4, seed=SEED)
    with pytest.raises(M.MrgError):
        M.generate_matrix(s, (4, 4), (2, 2), "normal")            # normals refused
    with pytest.raises(M.MrgError):
        M.generate_matrix(s, (4, 4), (4, 2), "uniform")           # 8 work items, 4 streams
