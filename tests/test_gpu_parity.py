"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Bars: raw integers, stream states and uniforms bit-exact; normals and
exponentials within 1e-12 absolute (fp64 outputs) or 2 ulp of the fp32
spacing at the reference value (fp32 outputs), the reference being the
oracle's double evaluation of the exact transform of the same integers.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2201_06604_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SEED = W.PAPER_SEED


@pytest.fixture(scope="module")
def M():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2201_06604_gb300 import mrg
    return mrg


def host_states(M, s, which=0):
    """[n, 6] uint32 states (which: 0 cur, 1 start, 2 sub) of a Streams."""
    return M.get_state(s)[which].T.copy()


def f32_ulp(ref):
    return np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64)


def assert_close(got, ref, dtype):
    got = got.astype(np.float64)
    if dtype == torch.float64:
        err = np.abs(got - ref).max() if ref.size else 0.0
        assert err <= 1e-12, err
    else:
        bad = np.abs(got - ref) > 2 * f32_ulp(ref)
        assert not bad.any(), (np.argwhere(bad)[:5], got[bad][:5], ref[bad][:5])


def oracle_rows(states, n, dist, dtype, rate=1.0):
    f32 = dtype == torch.float32
    out, after = O.generate_streams(states, n, {"raw": O.RAW, "uniform": O.UNIFORM,
                                                "normal": O.NORMAL,
                                                "exponential": O.EXPONENTIAL}[dist],
                                    f32=f32, rate=rate, nthreads=8)
    return out, after


def check_dist(M, s, n, dist, dtype, rate=1.0, out=None):
    st0 = host_states(M, s)
    got = M.generate(s, n, dist, dtype, rate=rate, out=out)
    torch.cuda.synchronize()
    got = got[: s.n, :n].cpu().numpy()
    ref, after = oracle_rows(st0, n, dist, dtype, rate)
    if dist == "raw":
        assert np.array_equal(got.view(np.uint32), ref)
    elif dist == "uniform":
        assert np.array_equal(got, ref), np.argwhere(got != ref)[:5]
    else:
        assert_close(got, ref, dtype)
    assert np.array_equal(host_states(M, s), after)


# ---------------------------------------------------------------------------


@pytest.mark.parametrize("n", [1, 31, 1000, 1024, 4099])
def test_create_streams_bit_exact(M, n):
    s = M.create_streams(n, seed=SEED)
    want, nxt = O.create_streams(SEED, n)
    st = M.get_state(s)
    for a in range(3):
        assert np.array_equal(st[a].T, want)
    assert tuple(s.next_seed) == tuple(int(v) for v in nxt)


def test_creator_state_advances_like_sequential_creation(M):
    M.set_base_creator(SEED)
    a = M.create_streams(5)
    b = M.create_streams(7)
    want, _ = O.create_streams(SEED, 12)
    assert np.array_equal(host_states(M, a), want[:5])
    assert np.array_equal(host_states(M, b), want[5:])
    M.set_base_creator(SEED)


def test_plain_1024x1024_f64_uniform_bit_exact(M):
    # 1024 streams from the paper's default seed by successive 2^127 jumps,
    # 1024 fp64 uniforms each (2^20) and the final states.
    cfg = W.PLAIN
    s = M.create_streams(cfg["streams"], seed=SEED)
    got = M.generate(s, cfg["draws"], "uniform", torch.float64).cpu().numpy()
    st0, _ = O.create_streams(SEED, cfg["streams"])
    ref, after = O.generate_streams(st0, cfg["draws"], O.UNIFORM, nthreads=8)
    assert np.array_equal(got, ref)
    assert np.array_equal(host_states(M, s), after)


CASES = [(33, 1000), (1, 4097), (100, 17), (7, 1), (64, 2048), (5, 3333), (9, 1002), (40, 998)]
DISTS = [("raw", torch.int32), ("uniform", torch.float64), ("uniform", torch.float32),
         ("normal", torch.float64), ("normal", torch.float32),
         ("exponential", torch.float64), ("exponential", torch.float32)]


@pytest.mark.parametrize("ns,n", CASES)
@pytest.mark.parametrize("dist,dtype", DISTS)
def test_generate_ragged(M, ns, n, dist, dtype):
    s = M.create_streams(ns, seed=SEED)
    M.skip(s, 12345)  # start away from the stream starts
    check_dist(M, s, n, dist, dtype, rate=1.7)


@pytest.mark.parametrize("dist,dtype", DISTS)
def test_generate_unaligned_output(M, dist, dtype):
    # odd leading dimension and a 4-byte shifted base pointer: no 16-byte
    # alignment, so the kernel's direct-store path runs
    ns, n = 37, 301
    s = M.create_streams(ns, seed=(1, 2, 3, 4, 5, 6))
    dt = torch.int32 if dist == "raw" else dtype
    big = torch.zeros((ns, n + 3), dtype=dt, device="cuda")
    out = big[:, 1:n + 2]
    check_dist(M, s, n, dist, dtype, out=out)
    assert (big[:, 0] == 0).all() and (big[:, n + 1:] == 0).all()


def test_output_does_not_touch_padding(M):
    ns, n = 40, 1001
    s = M.create_streams(ns, seed=SEED)
    big = torch.full((ns + 2, n + 16), -7.0, dtype=torch.float64, device="cuda")
    M.generate(s, n, "uniform", torch.float64, out=big)
    b = big.cpu().numpy()
    assert (b[:, n:] == -7.0).all() and (b[ns:] == -7.0).all()


@pytest.mark.parametrize("dist,dtype", DISTS)
def test_continuation_equals_one_long_call(M, dist, dtype):
    ns = 50
    s = M.create_streams(ns, seed=SEED)
    st0 = host_states(M, s)
    parts = [M.generate(s, k, dist, dtype).cpu().numpy() for k in (100, 257, 1)]
    torch.cuda.synchronize()
    # The normal transform consumes whole pairs: an odd call discards its last
    # sine, so the oracle is called with the same split.
    pos = st0.copy()
    for k, got in zip((100, 257, 1), parts):
        ref, pos = oracle_rows(pos, k, dist, dtype)
        if dist in ("raw", "uniform"):
            assert np.array_equal(got.view(ref.dtype), ref)
        else:
            assert_close(got, ref, dtype)
    assert np.array_equal(host_states(M, s), pos)


@pytest.mark.parametrize("k", [1, 2**20 + 3, 2**64 - 1, 2**64, 2**100 + 5, 2**128 - 1])
def test_skip_matches_oracle_jump(M, k):
    s = M.create_streams(9, seed=SEED)
    st0 = host_states(M, s)
    M.skip(s, k)
    want = np.stack([O.jump(x, k) for x in st0])
    assert np.array_equal(host_states(M, s), want)
    assert np.array_equal(host_states(M, s, 1), st0)


def test_substreams_and_resets(M):
    s = M.create_streams(17, seed=SEED)
    st0 = host_states(M, s)
    M.generate(s, 55, "uniform", torch.float64)
    M.substream_next(s)
    sub1 = np.stack([O.jump(x, 1 << 76) for x in st0])
    assert np.array_equal(host_states(M, s, 2), sub1)
    assert np.array_equal(host_states(M, s, 0), sub1)
    M.substream_next(s)
    sub2 = np.stack([O.jump(x, 2 << 76) for x in st0])
    assert np.array_equal(host_states(M, s, 2), sub2)
    M.generate(s, 10, "raw")
    M.reset_substream(s)
    assert np.array_equal(host_states(M, s, 0), sub2)
    M.reset_stream(s)
    for a in range(3):
        assert np.array_equal(host_states(M, s, a), st0)


def test_checkpoint_restore_identical_bytes(M):
    s = M.create_streams(64, seed=(11, 22, 33, 44, 55, 66))
    M.generate(s, 1000, "normal", torch.float64)
    ck = M.get_state(s)
    a = M.generate(s, 777, "exponential", torch.float32, rate=3.0).cpu().numpy()
    M.set_state(s, ck)
    b = M.generate(s, 777, "exponential", torch.float32, rate=3.0).cpu().numpy()
    assert a.tobytes() == b.tobytes()


def test_set_state_rejects_invalid(M):
    s = M.create_streams(4, seed=SEED)
    ck = M.get_state(s)
    bad = ck.copy()
    bad[0, :3, 2] = 0  # all-zero first component of stream 2
    with pytest.raises(M.MrgError) as e:
        M.set_state(s, bad)
    assert e.value.code == M.EINVAL
    assert np.array_equal(M.get_state(s), ck)


def test_argument_errors(M):
    s = M.create_streams(4, seed=SEED)
    with pytest.raises(M.MrgError):
        M.generate(s, 10, "exponential", torch.float32, rate=0.0)
    with pytest.raises(M.MrgError):
        M.create_streams(3, seed=(0, 0, 0, 1, 1, 1))
    out = torch.empty((4, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        M.generate(s, 10, "uniform", torch.float64, out=out)


def test_views_generate_subsets(M):
    s = M.create_streams(100, seed=SEED)
    st0 = host_states(M, s)
    v = s.view(40, 25)
    got = M.generate(v, 300, "raw").cpu().numpy().view(np.uint32)
    ref, after = O.generate_streams(st0[40:65], 300, O.RAW)
    assert np.array_equal(got, ref)
    full = host_states(M, s)
    assert np.array_equal(full[40:65], after)
    assert np.array_equal(full[:40], st0[:40]) and np.array_equal(full[65:], st0[65:])


@pytest.mark.parametrize("ns,draws", [(256, 4096), (77, 1001), (3, 2)])
def test_fused_small(M, ns, draws):
    s = M.create_streams(ns, seed=SEED)
    st0 = host_states(M, s)
    cnt, sm = M.fused_pi_normsum(s, draws)
    cnt, sm = cnt.cpu().numpy(), sm.cpu().numpy()
    rc, rs, after = O.fused(st0, draws, nthreads=8)
    assert np.array_equal(cnt, rc)
    x, _ = O.generate_streams(st0, draws + (draws & 1), O.NORMAL, nthreads=8)
    scale = np.abs(x).sum(axis=1)
    print(f"fused sum: max error {(np.abs(sm - rs) / scale).max():.2e} of sum |x| (bar 1e-9)")
    assert (np.abs(sm - rs) <= 1e-9 * scale).all()
    assert np.array_equal(host_states(M, s), after)


# ---------------------------------------------------------------------------
# Full-size workloads, checked on sampled streams
# ---------------------------------------------------------------------------

SAMPLE = [0, 1, 31, 32, 1000, 32767, 40000, 65534, 65535]


@pytest.mark.parametrize("dist,dt", [("uniform", "f64"), ("uniform", "f32"), ("normal", "f64"),
                                     ("normal", "f32"), ("exponential", "f32")])
def test_materialised_full_size_sampled(M, dist, dt):
    cfg = W.MATERIALISED
    dtype = torch.float64 if dt == "f64" else torch.float32
    s = M.create_streams(cfg["streams"], seed=SEED)
    out = M.generate(s, cfg["draws"], dist, dtype)
    torch.cuda.synchronize()
    st0, _ = O.create_streams(SEED, cfg["streams"])
    idx = torch.tensor(SAMPLE, device="cuda")
    got = out.index_select(0, idx).cpu().numpy()
    ref, after = oracle_rows(st0[SAMPLE], cfg["draws"], dist, dtype)
    if dist == "uniform":
        assert np.array_equal(got, ref)
    else:
        assert_close(got, ref, dtype)
    cur = host_states(M, s)
    assert np.array_equal(cur[SAMPLE], after)
    # every state stays in range; sampled output rows are finite and in range
    assert np.isfinite(out.float().sum().item())
    del out


def test_fused_full_size_sampled(M):
    cfg = W.FUSED
    s = M.create_streams(cfg["streams"], seed=SEED)
    st0 = host_states(M, s)
    cnt, sm = M.fused_pi_normsum(s, cfg["draws"])
    cnt, sm = cnt.cpu().numpy(), sm.cpu().numpy()
    sample = [0, 1, 5, 1 << 10, 777777, (1 << 20) - 1]
    rc, rs, after = O.fused(st0[sample], cfg["draws"], nthreads=8)
    assert np.array_equal(cnt[sample], rc)
    x, _ = O.generate_streams(st0[sample], cfg["draws"], O.NORMAL, nthreads=8)
    assert (np.abs(sm[sample] - rs) <= 1e-9 * np.abs(x).sum(axis=1)).all()
    assert np.array_equal(host_states(M, s)[sample], after)
    # statistical sanity of the whole run: fraction inside within 5 sigma of pi/4
    n = cfg["streams"] * cfg["draws"] // 2
    p = cnt.sum() / n
    assert abs(p - np.pi / 4) < 5 * np.sqrt(np.pi / 4 * (1 - np.pi / 4) / n)


@pytest.mark.parametrize("dist,dtype", [("uniform", torch.float64), ("normal", torch.float32),
                                        ("raw", torch.int32)])
def test_generate_host_matches_device(M, dist, dtype):
    ns, n = 77, 1003
    a = M.create_streams(ns, seed=SEED)
    b = M.create_streams(ns, seed=SEED)
    want = M.generate(a, n, dist, dtype).cpu().numpy()
    es = 8 if dtype == torch.float64 else 4
    scratch = torch.empty(2 * 3 * n * es + 100, dtype=torch.uint8, device="cuda")  # 3 rows a half
    dt = torch.int32 if dist == "raw" else dtype
    out = torch.full((ns, n + 5), -1, dtype=dt).pin_memory()
    M.generate_host(b, n, dist, dtype, out=out, scratch=scratch)
    got = out.numpy()
    assert np.array_equal(got[:, :n], want)
    assert (got[:, n:] == -1).all()
    assert np.array_equal(M.get_state(a), M.get_state(b))


@pytest.mark.parametrize("n", [8, 4096, 8 * 1000, 8 * 12345, 8 * (152 * 8 * 8 * 32 + 7), 1 << 24])
def test_fill_writes_every_word(M, n):
    # sizes below, at and above one 1 KiB chunk per warp, ragged chunk counts
    t = torch.zeros(n + 64, dtype=torch.int32, device="cuda")
    M.fill_u32(t[8:8 + n], 0x12345678)
    torch.cuda.synchronize()
    h = t.cpu().numpy()
    assert (h[8:8 + n] == 0x12345678).all() and (h[:8] == 0).all() and (h[8 + n:] == 0).all()
    with pytest.raises(M.MrgError):
        M.fill_u32(t[1:9])                       # not 32-byte aligned
    with pytest.raises(M.MrgError):
        M.fill_u32(t[8:12])                      # not a whole 32-byte unit


def test_unaddressable_extent_is_rejected(M):
    # 4 streams with a row pitch of 2^60 fp64 elements would span 2^65 bytes:
    # refused before any device work
    s = M.create_streams(4, seed=SEED)
    out = torch.empty(64, dtype=torch.float64, device="cuda")
    rc = M.lib.mrg_generate(s.ptr(), 8, M.UNIFORM, M.F64, 1.0, out.data_ptr(), 1 << 60,
                            torch.cuda.current_stream().cuda_stream)
    assert rc == M.ERANGE


@pytest.mark.parametrize("dist,dt", [("normal", torch.float64), ("normal", torch.float32),
                                     ("exponential", torch.float32), ("exponential", torch.float64)])
@pytest.mark.parametrize("ns,n", [(300, 4096), (33, 1002), (1, 9)])
def test_packed_equals_scalar(M, ns, n, dist, dt):
    # normals and exponentials into rows aligned for 16- or 32-byte
    # stores are evaluated two draws (two pairs) at a time with packed fp32x2
    # instructions; a row pitch of one element more selects the one-at-a-time
    # evaluation.  Same streams, same bits.
    a = M.create_streams(ns, seed=SEED)
    b = M.create_streams(ns, seed=SEED)
    M.skip(a, 999)
    M.skip(b, 999)
    got_a = M.generate(a, n, dist, dt, rate=1.7)
    big = torch.zeros((ns, n + 1), dtype=dt, device="cuda")
    got_b = M.generate(b, n, dist, dt, rate=1.7, out=big[:, 1:])
    torch.cuda.synchronize()
    iv = np.uint64 if dt == torch.float64 else np.uint32
    x = got_a[:ns, :n].cpu().numpy().view(iv)
    y = got_b[:ns, :n].cpu().numpy().view(iv)
    assert np.array_equal(x, y), np.argwhere(x != y)[:5]
    assert np.array_equal(host_states(M, a), host_states(M, b))
