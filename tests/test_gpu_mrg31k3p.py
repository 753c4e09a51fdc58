"""MRG31k3p, the paper's own generator, on the GPU through the C ABI.

The paper prints this generator's output, so these tests pin the CUDA path
to the paper directly (not only to the oracle):

* the four stream starts of Sec. 2.1 (createStreamsGpu after setBaseCreator
  with 12345 x 6), exact;
* the runifGpu uniforms of Sec. 2.2 and the rexpGpu exponentials of Sec. 3.2,
  to the printed three decimals (same work-item -> stream / draw mapping as
  the fixtures state).

Then parity with the oracle run with MRG31k3p parameters: stream starts and
states bit-exact, raw integers and uniforms bit-exact, normals and
exponentials within 1e-12 (fp64) or 2 ulp of fp32.
"""
import numpy as np
import pytest
import torch

import oracle as O

pytestmark = pytest.mark.gpu

SEED = (12345,) * 6
G = O.MRG31K3P
DISTS = {"raw": O.RAW, "uniform": O.UNIFORM, "normal": O.NORMAL, "exponential": O.EXPONENTIAL}


@pytest.fixture(scope="module")
def M():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2201_06604_gb300 import mrg
    return mrg


def states(M, s):
    return M.get_state(s)[0].T.copy()


def test_stream_starts_match_paper(M, golden):
    want = np.array(golden("mrg31k3p_stream_starts.txt"), dtype=np.uint64)
    s = M.create_streams(4, seed=SEED, generator="mrg31k3p")
    st = M.get_state(s)
    for a in range(3):                                   # cur = start = sub
        assert np.array_equal(st[a].T.astype(np.uint64), want)
    _, nxt = O.create_streams(SEED, 4, gen=G)
    assert tuple(s.next_seed) == tuple(int(v) for v in nxt)


def test_runif_and_rexp_match_paper(M, golden):
    s = M.create_streams(4, seed=SEED, generator="mrg31k3p")
    u = M.generate(s, 4, "uniform", torch.float64).cpu().numpy()
    want = [float(v) for v in golden("mrg31k3p_runif.txt")[0]]
    got = [u[2 * (r % 2), r // 2] for r in range(8)]
    for g, w in zip(got, want):
        assert abs(g - w) <= 0.0005 + 1e-12, (got, want)
    # every stream has now produced four draws; the next two are the
    # exponentials of the Sec. 3.2 printout
    e = M.generate(s, 2, "exponential", torch.float64, rate=1.0).cpu().numpy()
    rows = golden("mrg31k3p_rexp.txt")
    for r in range(2):
        for c in range(4):
            w = float(rows[r][c])
            dec = len(rows[r][c].split(".")[1])
            assert abs(e[2 * (r % 2) + (c % 2), c // 2] - w) <= 0.5 * 10 ** -dec + 1e-12


@pytest.mark.parametrize("n", [1, 33, 1000, 4099])
def test_create_streams_bit_exact(M, n):
    seed = (1, 2, 3, 4, 5, 6)
    s = M.create_streams(n, seed=seed, generator="mrg31k3p")
    want, nxt = O.create_streams(seed, n, gen=G)
    assert np.array_equal(states(M, s), want)
    assert tuple(s.next_seed) == tuple(int(v) for v in nxt)


def f32_ulp(ref):
    return np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64)


@pytest.mark.parametrize("dist,dtype", [("raw", torch.int32), ("uniform", torch.float64),
                                        ("uniform", torch.float32), ("normal", torch.float64),
                                        ("normal", torch.float32), ("exponential", torch.float64),
                                        ("exponential", torch.float32)])
@pytest.mark.parametrize("ns,n", [(37, 1003), (64, 4096), (3, 17)])
def test_generate_matches_oracle(M, dist, dtype, ns, n):
    s = M.create_streams(ns, seed=SEED, generator="mrg31k3p")
    M.skip(s, 12345)                                     # start mid-stream
    st0 = states(M, s)
    rate = 2.5
    got = M.generate(s, n, dist, dtype, rate=rate).cpu().numpy()
    ref, after = O.generate_streams(st0, n, DISTS[dist], f32=dtype == torch.float32, rate=rate,
                                    nthreads=8, gen=G)
    if dist == "raw":
        assert np.array_equal(got.view(np.uint32), ref)
    elif dist == "uniform":
        assert np.array_equal(got, ref)
    elif dtype == torch.float64:
        assert np.abs(got - ref).max() <= 1e-12
    else:
        assert (np.abs(got.astype(np.float64) - ref) <= 2 * f32_ulp(ref)).all()
    assert np.array_equal(states(M, s), after)


def test_calls_continue_the_streams(M):
    s = M.create_streams(50, seed=SEED, generator="mrg31k3p")
    st0 = states(M, s)
    a = M.generate(s, 300, "uniform", torch.float64)
    b = M.generate(s, 301, "uniform", torch.float64)
    ref, _ = O.generate_streams(st0, 601, O.UNIFORM, gen=G)
    assert np.array_equal(torch.cat([a, b], 1).cpu().numpy(), ref)


def test_skip_matches_oracle(M):
    s = M.create_streams(8, seed=SEED, generator="mrg31k3p")
    st0 = states(M, s)
    k = (1 << 63) + 987654321
    M.skip(s, k)
    for i in range(8):
        assert np.array_equal(states(M, s)[i], O.jump(st0[i], k, gen=G))


def test_mrg32k3a_only_calls_refuse_mrg31k3p_streams(M):
    s = M.create_streams(4, seed=SEED, generator="mrg31k3p")
    with pytest.raises(ValueError):
        M.substream_next(s)
    with pytest.raises(ValueError):
        M.fused_pi_normsum(s, 16)
    with pytest.raises(ValueError):
        M.Batch(s)
    with pytest.raises(M.MrgError):                      # a word >= 2^31 - 1 is not a state
        M.create_streams(1, seed=(2147483647, 1, 1, 1, 1, 1), generator="mrg31k3p")


@pytest.mark.parametrize("dist,dtype", [("uniform", torch.float64), ("normal", torch.float64),
                                        ("uniform", torch.float32)])
def test_materialised_full_size_sampled(M, dist, dtype):
    from paper_2201_06604_gb300 import workloads as W
    ns, n = W.MATERIALISED["streams"], W.MATERIALISED["draws"]
    s = M.create_streams(ns, seed=SEED, generator="mrg31k3p")
    out = M.generate(s, n, dist, dtype)
    torch.cuda.synchronize()
    sample = [0, 1, 31, 32, 4095, 40000, ns - 1]
    st0, _ = O.create_streams(SEED, ns, gen=G)
    got = out.index_select(0, torch.tensor(sample, device="cuda")).cpu().numpy()
    ref, after = O.generate_streams(st0[sample], n, DISTS[dist], f32=dtype == torch.float32,
                                    nthreads=8, gen=G)
    if dist == "uniform":
        assert np.array_equal(got, ref)
    else:
        assert np.abs(got - ref).max() <= 1e-12
    assert np.array_equal(states(M, s)[sample], after)
    del out


@pytest.mark.parametrize("dist,dt", [("normal", torch.float64), ("normal", torch.float32),
                                     ("exponential", torch.float32), ("exponential", torch.float64)])
@pytest.mark.parametrize("ns,n", [(300, 4096), (33, 1002)])
def test_packed_equals_scalar(M, ns, n, dist, dt):
    # rows aligned for 16- or 32-byte stores take the packed two-at-a-time
    # evaluation, a pitch of one element more the one-at-a-time one: same
    # streams, same bits
    a = M.create_streams(ns, seed=SEED, generator="mrg31k3p")
    b = M.create_streams(ns, seed=SEED, generator="mrg31k3p")
    got_a = M.generate(a, n, dist, dt, rate=0.6)
    big = torch.zeros((ns, n + 1), dtype=dt, device="cuda")
    got_b = M.generate(b, n, dist, dt, rate=0.6, out=big[:, 1:])
    torch.cuda.synchronize()
    iv = np.uint64 if dt == torch.float64 else np.uint32
    x = got_a[:ns, :n].cpu().numpy().view(iv)
    y = got_b[:ns, :n].cpu().numpy().view(iv)
    assert np.array_equal(x, y), np.argwhere(x != y)[:5]
    assert np.array_equal(states(M, a), states(M, b))
