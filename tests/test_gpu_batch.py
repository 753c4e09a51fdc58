"""Batched requests (one persistent, graph-captured launch): each request's
output equals the oracle at the same absolute stream position, equals what
the plain entry point writes for a single stream positioned there (bit for
bit), and does not depend on the other requests or their order."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2201_06604_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SEED = W.PAPER_SEED
DISTS = {"raw": O.RAW, "uniform": O.UNIFORM, "normal": O.NORMAL, "exponential": O.EXPONENTIAL}


@pytest.fixture(scope="module")
def M():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2201_06604_gb300 import mrg
    return mrg


def make_requests(ns, count, seed, nmax=20000):
    rng = np.random.default_rng(seed)
    reqs = []
    for r in range(count):
        dist = ["raw", "uniform", "normal", "exponential"][rng.integers(0, 4)]
        dtype = "u32" if dist == "raw" else ["f32", "f64"][rng.integers(0, 2)]
        n = int(rng.choice([0, 1, 2, 3, 7, 8, 9, 31, 255, 256, 257, 1000, 4097,
                            int(rng.integers(1, nmax))]))
        reqs.append(dict(stream=int(rng.integers(0, ns)), substream=int(rng.integers(0, 3)),
                         offset=int(rng.integers(0, 1 << 40)) if rng.integers(0, 2) else 0,
                         n=n, dist=dist, dtype=dtype, rate=float(rng.choice([1.0, 2.5]))))
    return reqs


def oracle_request(start_states, q):
    st = O.jump(start_states[q["stream"]], (q["substream"] << 76) + q["offset"])
    out, _ = O.generate_streams(st[None, :], q["n"], DISTS[q["dist"]],
                                f32=q["dtype"] == "f32", rate=q["rate"])
    return out[0]


def check_close(got, ref, q):
    if q["dist"] in ("raw", "uniform"):
        assert np.array_equal(got.astype(ref.dtype) if q["dist"] == "uniform" else got.view(np.uint32),
                              ref), q
    elif q["dtype"] == "f64":
        tol = 1e-12 / min(q["rate"], 1.0)
        assert np.abs(got - ref).max() <= tol, q
    else:
        ulp = np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64)
        assert (np.abs(got.astype(np.float64) - ref) <= 2 * ulp).all(), q


def test_batch_matches_oracle(M):
    ns = 300
    s = M.create_streams(ns, seed=SEED)
    start, _ = O.create_streams(SEED, ns)
    reqs = make_requests(ns, 120, seed=11)
    buf = M.alloc_outputs(reqs)
    b = M.Batch(s, max_requests=256, max_tiles=4096)
    b.run(reqs)
    torch.cuda.synchronize()
    assert b.last_tiles >= sum(1 for q in reqs if q["n"] > 0)
    for q in reqs:
        if q["n"] == 0:
            continue
        got = q["out"].cpu().numpy()
        check_close(got, oracle_request(start, q), q)
    b.close()
    del buf


def test_batch_equals_plain_and_is_order_independent(M):
    ns = 64
    s = M.create_streams(ns, seed=(1, 2, 3, 4, 5, 6))
    reqs = make_requests(ns, 80, seed=12)
    buf1 = M.alloc_outputs(reqs)
    b = M.Batch(s, max_requests=128, max_tiles=4096)
    b.run(reqs)
    torch.cuda.synchronize()
    first = [q["out"].clone() for q in reqs]
    # same requests, reversed order, in a fresh output buffer
    rev = [dict(q) for q in reversed(reqs)]
    buf2 = M.alloc_outputs(rev)
    b.run(rev)
    torch.cuda.synchronize()
    for q, a in zip(reversed(rev), first):
        assert torch.equal(q["out"], a)
    # plain generate on a single stream positioned at the request's draw
    for q, a in zip(reqs, first):
        if q["n"] == 0:
            continue
        one = M.create_streams(1, seed=tuple(int(v) for v in M.get_state(s)[1][:, q["stream"]]))
        for _ in range(q["substream"]):
            M.substream_next(one)
        M.skip(one, q["offset"])
        dt = {"f32": torch.float32, "f64": torch.float64, "u32": torch.int32}[q["dtype"]]
        p = M.generate(one, q["n"], q["dist"], dt, rate=q["rate"])[0]
        assert torch.equal(p, a), q
    b.close()
    del buf1, buf2


def test_batch_alone_equals_in_mix(M):
    ns = 32
    s = M.create_streams(ns, seed=SEED)
    reqs = make_requests(ns, 40, seed=13)
    M.alloc_outputs(reqs)
    b = M.Batch(s, max_requests=64, max_tiles=2048)
    b.run(reqs)
    torch.cuda.synchronize()
    for q in reqs[::7]:
        alone = dict(q)
        M.alloc_outputs([alone])
        b.run([alone])
        torch.cuda.synchronize()
        assert torch.equal(alone["out"], q["out"])
    b.close()


def test_batch_errors(M):
    s = M.create_streams(4, seed=SEED)
    b = M.Batch(s, max_requests=2, max_tiles=4)
    out = torch.empty(64, dtype=torch.float64, device="cuda")
    with pytest.raises(M.MrgError):
        b.run([dict(stream=4, n=8, dist="uniform", dtype="f64", out=out)])        # bad stream
    with pytest.raises(M.MrgError):
        b.run([dict(stream=0, n=8, dist="uniform", dtype="f64", out=out[1:])])    # misaligned
    with pytest.raises(M.MrgError):
        b.run([dict(stream=0, n=8, dist="uniform", dtype="u32", out=out)])        # no u32 uniform
    with pytest.raises(M.MrgError):
        b.run([dict(stream=0, n=8, dist="uniform", dtype="f64", out=out)] * 3)   # too many
    big = torch.empty(600000, dtype=torch.float64, device="cuda")
    with pytest.raises(M.MrgError):
        b.run([dict(stream=0, n=600000, dist="uniform", dtype="f64", out=big)])  # too many tiles
    b.run([dict(stream=1, n=8, dist="uniform", dtype="f64", out=out)])           # still usable
    torch.cuda.synchronize()
    b.close()


TILINGS = [dict(seg_min=8, seg_max=8, target_segments=1),
           dict(seg_min=8, seg_max=2048, target_segments=32),
           dict(seg_min=64, seg_max=512, target_segments=2048),
           dict(seg_min=8, seg_max=1 << 20, target_segments=1),
           dict(seg_min=256, seg_max=8192, target_segments=7)]


def test_every_tiling_writes_the_same_bytes(M):
    ns = 50
    s = M.create_streams(ns, seed=SEED)
    reqs = make_requests(ns, 60, seed=21)
    M.alloc_outputs(reqs)
    b = M.Batch(s, max_requests=64, max_tiles=1 << 14)
    b.run(reqs)
    torch.cuda.synchronize()
    assert b.get_tiling() == dict(seg_min=8, seg_max=256, target_segments=32)
    ref = [q["out"].clone() for q in reqs]
    tiles = set()
    for t in TILINGS:
        b.set_tiling(t)
        assert b.get_tiling() == t
        again = [dict(q) for q in reqs]
        M.alloc_outputs(again)
        b.run(again)
        torch.cuda.synchronize()
        tiles.add(b.last_tiles)
        for q, a in zip(again, ref):
            assert torch.equal(q["out"], a), (t, q)
    assert len(tiles) >= 3          # the tilings really cut the work differently
    b.set_tiling(None)
    assert b.get_tiling()["seg_max"] == 256
    for bad in (dict(seg_min=4, seg_max=64, target_segments=1),
                dict(seg_min=64, seg_max=32, target_segments=1),
                dict(seg_min=8, seg_max=100, target_segments=1),
                dict(seg_min=8, seg_max=64, target_segments=0)):
        with pytest.raises(M.MrgError):
            b.set_tiling(bad)
    b.close()


def test_batch_tuner_keeps_the_fastest_tiling(M):
    ns = 256
    s = M.create_streams(ns, seed=SEED)
    start, _ = O.create_streams(SEED, ns)
    rng = np.random.default_rng(5)
    reqs = [dict(stream=r, substream=1, offset=0, n=int(10 ** rng.uniform(2, 5)),
                 dist=["uniform", "normal", "exponential"][r % 3], dtype=["f32", "f64"][r % 2],
                 rate=1.0) for r in range(ns)]
    M.alloc_outputs(reqs)
    b = M.Batch(s, max_requests=ns, max_tiles=1 << 15)
    best, table = b.tune(reqs, reps=2)
    torch.cuda.synchronize()
    assert len(table) >= 5
    assert table[0][0] == dict(seg_min=8, seg_max=256, target_segments=32)    # current first
    fastest = min(table, key=lambda e: e[2])
    assert best == fastest[0] and b.get_tiling() == best
    # outputs written by the tuner are the requests' outputs
    for q in reqs[::17]:
        check_close(q["out"].cpu().numpy(), oracle_request(start, q), q)
    ref = [q["out"].clone() for q in reqs]
    again = [dict(q) for q in reqs]
    M.alloc_outputs(again)
    b.run(again)
    torch.cuda.synchronize()
    for q, a in zip(again, ref):
        assert torch.equal(q["out"], a)
    b.close()


def test_back_to_back_runs_without_sync(M):
    """Runs issued back to back (host tables double-buffered, device tables
    shared) on one stream and then alternating between two streams give the
    same outputs as runs issued one at a time."""
    ns = 128
    s = M.create_streams(ns, seed=SEED)
    sets = [make_requests(ns, 50, seed=40 + k, nmax=200000) for k in range(4)]
    b = M.Batch(s, max_requests=64, max_tiles=1 << 14)
    refs = []
    for reqs in sets:
        M.alloc_outputs(reqs)
        b.run(reqs)
        torch.cuda.synchronize()
        refs.append([q["out"].clone() for q in reqs])
    streams = [torch.cuda.current_stream(), torch.cuda.Stream()]
    for mode in ("one stream", "two streams"):
        again = [[dict(q) for q in reqs] for reqs in sets]
        for k, reqs in enumerate(again):
            M.alloc_outputs(reqs)
            st = streams[k % 2] if mode == "two streams" else streams[0]
            b.run(M.Batch.prepare(reqs) if k % 2 else reqs, stream=st)
        torch.cuda.synchronize()
        for reqs, ref in zip(again, refs):
            for q, a in zip(reqs, ref):
                assert torch.equal(q["out"], a), (mode, q)
    b.close()


def test_full_size_batch_sampled(M):
    """The 4096-request workload (lengths log-uniform in [1e2, 1e6], mixed
    variants, request r on stream r, substream 1) in one tuned batched launch:
    sampled requests against the oracle, all of them against plain
    single-stream generation."""
    reqs = W.batched_requests(4096)
    for q in reqs:
        q["dist"] = {1: "uniform", 2: "normal", 3: "exponential"}[q["dist"]]
        q["offset"] = 0
    s = M.create_streams(len(reqs), seed=SEED)
    start, _ = O.create_streams(SEED, len(reqs))
    M.alloc_outputs(reqs)
    b = M.Batch(s, max_requests=len(reqs), max_tiles=1 << 17)
    b.tune(reqs, reps=1)
    b.run(reqs)
    torch.cuda.synchronize()
    rng = np.random.default_rng(9)
    for r in list(rng.choice(len(reqs), 24, replace=False)) + [int(np.argmax([q["n"] for q in reqs]))]:
        q = reqs[r]
        check_close(q["out"].cpu().numpy(), oracle_request(start, q), q)
    # every request equals plain generation from the same position
    dt = {"f32": torch.float32, "f64": torch.float64}
    M.substream_next(s)
    for r in range(0, len(reqs), 97):
        q = reqs[r]
        p = M.generate(s.view(r, 1), q["n"], q["dist"], dt[q["dtype"]])[0]
        assert torch.equal(p, q["out"]), q
    b.close()


def test_plain_host_loop_matches_batch_and_oracle(M):
    # mrg_batch_run_plain: the same requests, one position jump and one
    # generate launch each from the library's host loop
    ns = 200
    s = M.create_streams(ns, seed=SEED)
    start, _ = O.create_streams(SEED, ns)
    reqs = make_requests(ns, 90, seed=17)
    ref = [dict(q) for q in reqs]
    buf_b = M.alloc_outputs(ref)
    buf_p = M.alloc_outputs(reqs)
    b = M.Batch(s, max_requests=128, max_tiles=4096)
    b.run(ref)
    b.run_plain(reqs)
    torch.cuda.synchronize()
    for q, r in zip(reqs, ref):
        if q["n"] == 0:
            continue
        assert torch.equal(q["out"], r["out"]), q
        check_close(q["out"].cpu().numpy(), oracle_request(start, q), q)
    b.close()
    del buf_b, buf_p
