"""Serving engine (continuous batching into one persistent worker):

* outputs equal the batch runner's for the same requests (and the oracle's);
* a request's output is the same alone and in a mix whose members arrive
  while others are on the GPU;
* admission by memory and slots: EBUSY when full, admitted again after
  release;
* failure detection without a GPU fault: the worker's wait for work is
  bounded, so a server that nobody feeds stops by itself, reports
  MRG_ETIMEOUT, and restarts;
* destroy with requests in flight processes them and returns.
"""
import time

import numpy as np
import pytest
import torch

import oracle as O

pytestmark = pytest.mark.gpu

SEED = (12345, 12345, 12345, 12345, 12345, 12345)


@pytest.fixture(scope="module")
def M():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2201_06604_gb300 import mrg
    return mrg


def mix(ns, count, seed, nmax=300000):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        dist = ["raw", "uniform", "normal", "exponential"][rng.integers(0, 4)]
        dtype = "u32" if dist == "raw" else ["f32", "f64"][rng.integers(0, 2)]
        n = int(np.exp(rng.uniform(0, np.log(nmax))))
        out.append(dict(stream=int(rng.integers(0, ns)), substream=int(rng.integers(0, 4)),
                        offset=int(rng.integers(0, 1 << 20)), n=n, dist=dist, dtype=dtype,
                        rate=float(rng.choice([1.0, 0.5]))))
    return out


class Client:
    """Submits with retry (polling while the server is busy, since finished
    requests free ring space only when they are polled) and remembers the
    ids finished so far."""

    def __init__(self, sv):
        self.sv = sv
        self.finished = set()

    def submit_all(self, reqs, stagger=0.0, timeout=30.0):
        got = []
        t0 = time.time()
        for q in reqs:
            r = None
            while r is None:
                r = self.sv.submit(q["stream"], q["n"], q["dist"], q["dtype"], q["substream"],
                                   q["offset"], q["rate"])
                if r is None:
                    self.finished.update(self.sv.poll())
                assert time.time() - t0 < timeout, "server stayed busy"
            got.append(r)
            if stagger:
                time.sleep(stagger)
        return got

    def wait(self, ids, timeout=30.0):
        pending = set(ids) - self.finished
        t0 = time.time()
        while pending:
            done = self.sv.poll()
            self.finished.update(done)
            pending.difference_update(done)
            assert time.time() - t0 < timeout, f"{len(pending)} requests not finished"


def test_server_matches_batch_and_oracle(M):
    ns = 512
    s = M.create_streams(ns, seed=SEED)
    reqs = mix(ns, 60, seed=31)
    ref = [dict(q) for q in reqs]
    M.alloc_outputs(ref)
    b = M.Batch(s, max_requests=64, max_tiles=1 << 12)   # allocate before the worker runs
    sv = M.Server(s, 256 << 20, max_slots=64, ring_tiles=1 << 12)
    c = Client(sv)
    got = c.submit_all(reqs)
    c.wait([i for i, _ in got])
    b.run(ref)
    # a device-wide synchronize would wait for the running worker: sync the
    # stream, and compare on the host (no new device kernels while it runs)
    torch.cuda.current_stream().synchronize()
    for (rid, out), r in zip(got, ref):
        assert np.array_equal(out.cpu().numpy(), r["out"].cpu().numpy()), r
    # spot-check a uniform request against the oracle
    start, _ = O.create_streams(SEED, ns)
    for (rid, out), q in zip(got, reqs):
        if q["dist"] == "uniform":
            st = O.jump(start[q["stream"]], (q["substream"] << 76) + q["offset"])
            ref64, _ = O.generate_streams(st[None], q["n"], O.UNIFORM, f32=q["dtype"] == "f32")
            assert np.array_equal(out.cpu().numpy(), ref64[0])
            break
    for rid, _ in got:
        sv.release(rid)
    sv.close()
    b.close()


def test_alone_equals_mix(M):
    ns = 128
    s = M.create_streams(ns, seed=(3, 1, 4, 1, 5, 9))
    reqs = mix(ns, 50, seed=32, nmax=2_000_000)
    sv = M.Server(s, 1 << 30, max_slots=64, ring_tiles=1 << 13)
    c = Client(sv)
    got = c.submit_all(reqs, stagger=0.0005)   # arrivals while earlier ones run
    c.wait([i for i, _ in got])
    mixed = [out.cpu() for _, out in got]
    for rid, _ in got:
        sv.release(rid)
    for q, m in list(zip(reqs, mixed))[::5]:
        (rid, out), = c.submit_all([q])
        c.wait([rid])
        assert torch.equal(out.cpu(), m), q
        sv.release(rid)
    sv.close()


def test_admission_by_memory_and_slots(M):
    s = M.create_streams(8, seed=SEED)
    sv = M.Server(s, 1 << 20, max_slots=3, ring_tiles=256)  # 1 MiB arena
    a = sv.submit(0, 100_000, "uniform", "f64")            # 800 KB
    assert a is not None
    assert sv.submit(1, 100_000, "uniform", "f64") is None  # arena full
    b = sv.submit(2, 1000, "uniform", "f32")
    c = sv.submit(3, 1000, "uniform", "f32")
    assert b is not None and c is not None
    assert sv.submit(4, 8, "uniform", "f32") is None        # no free slot
    cl = Client(sv)
    cl.wait([a[0], b[0], c[0]])
    with pytest.raises(M.MrgError):
        sv.release(12345678)
    sv.release(a[0])
    d = sv.submit(1, 100_000, "uniform", "f64")             # admitted after release
    assert d is not None
    cl.wait([d[0]])
    for r in (b, c, d):
        sv.release(r[0])
    assert sv.inflight() == 0
    sv.close()


def test_worker_idle_limit_is_detected_and_restarts(M):
    s = M.create_streams(8, seed=SEED)
    sv = M.Server(s, 1 << 20, max_slots=4, ring_tiles=16, idle_seconds=0.05)
    time.sleep(0.5)                                     # nobody publishes work
    ids, rc = sv.poll_status()
    assert rc == M.ETIMEOUT and ids == []
    with pytest.raises(M.MrgError) as e:
        sv.submit(0, 10, "uniform", "f64")
    assert e.value.code == M.ETIMEOUT
    sv.restart()
    r = sv.submit(0, 10, "uniform", "f64")
    assert r is not None
    Client(sv).wait([r[0]], timeout=5.0)
    sv.release(r[0])
    sv.close()


def test_destroy_with_requests_in_flight(M):
    s = M.create_streams(64, seed=SEED)
    sv = M.Server(s, 1 << 30, max_slots=16, ring_tiles=1 << 16)
    for k in range(8):
        assert sv.submit(k, 3_000_000, "normal", "f64") is not None
    sv.close()          # processes what was admitted, then stops
    torch.cuda.synchronize()


def test_tiling_changes_no_output(M):
    ns = 64
    s = M.create_streams(ns, seed=SEED)
    reqs = mix(ns, 24, seed=33, nmax=3_000_000)
    sv = M.Server(s, 1 << 30, max_slots=64, ring_tiles=1 << 14)
    c = Client(sv)
    results = []
    for t in (None, dict(seg_min=8, seg_max=8, target_segments=1),
              dict(seg_min=256, seg_max=4096, target_segments=512)):
        sv.set_tiling(t)
        got = c.submit_all(reqs)
        c.wait([i for i, _ in got])
        results.append([out.cpu() for _, out in got])
        for rid, _ in got:
            sv.release(rid)
    for other in results[1:]:
        for a, b in zip(results[0], other):
            assert torch.equal(a, b)
    with pytest.raises(M.MrgError):
        sv.set_tiling(dict(seg_min=8, seg_max=12, target_segments=1))
    sv.close()


def test_saturation_with_a_small_ring_drains(M):
    """Many large requests offered at once into a ring far smaller than their
    tiles: requests start only when the ring can take all their tiles, so the
    server keeps draining instead of filling the ring with first chunks.
    Outputs equal the batch runner's."""
    ns = 64
    s = M.create_streams(ns, seed=SEED)
    rng = np.random.default_rng(35)
    reqs = [dict(stream=int(rng.integers(0, ns)), substream=int(k % 3), offset=0,
                 n=int(rng.integers(1_200_000, 3_000_000)), dist=["uniform", "normal"][k % 2],
                 dtype="f32", rate=1.0) for k in range(40)]
    ref = [dict(q) for q in reqs]
    M.alloc_outputs(ref)
    b = M.Batch(s, max_requests=64, max_tiles=1 << 15)
    # ring of 2048 tiles; each request takes ~290-730 tiles, more than one
    # emission chunk, so several requests would be half-emitted at once
    sv = M.Server(s, 1 << 30, max_slots=64, ring_tiles=2048, idle_seconds=10.0)
    c = Client(sv)
    got = c.submit_all(reqs)
    c.wait([i for i, _ in got], timeout=60.0)
    b.run(ref)
    torch.cuda.current_stream().synchronize()
    for (rid, out), r in zip(got, ref):
        assert torch.equal(out.cpu(), r["out"].cpu()), r
        sv.release(rid)
    with pytest.raises(M.MrgError) as e:                      # more tiles than the ring
        sv.submit(0, 100_000_000, "uniform", "f32")
    assert e.value.code == M.ERANGE
    sv.close()
    b.close()
