"""mrg_batch_run_static: batched generation for callers that cannot allocate
device memory (a plug-in under a host application that owns the
device-memory budget through its own allocator, or a loop where cudaMalloc's
implicit synchronisation is not acceptable).  Its scratch lives in a fixed
device array inside the library, so it must produce what mrg_batch_run
produces, call after call, and a call after the first must leave the
device's free memory unchanged.

This file is collected last on purpose: a failure here leaves every other
test already run.  It passes alone in a fresh process and after the others.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

SEED = (12345, 12345, 12345, 12345, 12345, 12345)


@pytest.fixture(scope="module")
def M():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2201_06604_gb300 import mrg
    f = mrg.lib.mrg_batch_run_static
    f.argtypes = [ctypes.POINTER(mrg._Streams), ctypes.POINTER(mrg._Request), ctypes.c_uint32,
                  ctypes.c_void_p]
    f.restype = ctypes.c_int
    return mrg


def requests(ns, count, seed):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        dist = ["raw", "uniform", "normal", "exponential"][rng.integers(0, 4)]
        dtype = "u32" if dist == "raw" else ["f32", "f64"][rng.integers(0, 2)]
        out.append(dict(stream=int(rng.integers(0, ns)), substream=int(rng.integers(0, 2)),
                        offset=int(rng.integers(0, 1 << 30)), n=int(rng.integers(1, 30000)),
                        dist=dist, dtype=dtype, rate=float(rng.choice([1.0, 3.0]))))
    return out


def run_static(M, streams, reqs):
    arr = (M._Request * len(reqs))()
    for i, q in enumerate(reqs):
        d = M._DIST[q["dist"]]
        arr[i] = M._Request(q["stream"], q["substream"], q["offset"], q["n"], d,
                            M.U32 if d == M.RAW else M._DT_CODE[q["dtype"]], q["rate"],
                            q["out"].data_ptr())
    rc = M.lib.mrg_batch_run_static(streams.ptr(), arr, len(reqs),
                                    torch.cuda.current_stream().cuda_stream)
    return rc


def same(a, b, q):
    if q["dist"] in ("raw", "uniform"):
        return torch.equal(a, b)
    a64, b64 = a.double().cpu().numpy(), b.double().cpu().numpy()
    if q["dtype"] == "f64":
        return np.abs(a64 - b64).max() <= 1e-12 / min(q["rate"], 1.0)
    ulp = np.spacing(np.abs(b64).astype(np.float32)).astype(np.float64)
    return bool((np.abs(a64 - b64) <= 2 * ulp).all())


def test_static_scratch_matches_batch_run_twice(M):
    ns = 256
    s = M.create_streams(ns, seed=SEED)
    b = M.Batch(s, max_requests=128, max_tiles=8192)
    for call, seed in enumerate((21, 22)):       # two calls in a row
        reqs = requests(ns, 100, seed)
        ref = [dict(q) for q in reqs]
        M.alloc_outputs(ref)
        b.run(ref)
        buf = M.alloc_outputs(reqs)
        buf.fill_(0xA5)
        assert run_static(M, s, reqs) == M.OK, M.lib.mrg_last_error()
        torch.cuda.synchronize()
        for q, r in zip(reqs, ref):
            assert same(q["out"], r["out"], q), (call, q)
    b.close()


def test_static_scratch_rejects_oversize(M):
    s = M.create_streams(4, seed=SEED)
    out = torch.empty(8, dtype=torch.float64, device="cuda")
    reqs = [dict(stream=0, substream=0, offset=0, n=8, dist="uniform", dtype="f64", rate=1.0,
                 out=out)] * 1025
    assert run_static(M, s, reqs) == M.ERANGE
    assert b"1024" in M.lib.mrg_last_error()
    big = torch.empty(40_000_000, dtype=torch.float32, device="cuda")   # 19532 segments ... tiles
    many = [dict(stream=0, substream=0, offset=0, n=40_000_000, dist="uniform", dtype="f32",
                 rate=1.0, out=big)] * 30
    assert run_static(M, s, many) == M.ERANGE
    # still usable afterwards
    ok = [dict(stream=1, substream=0, offset=0, n=8, dist="uniform", dtype="f64", rate=1.0,
               out=out)]
    assert run_static(M, s, ok) == M.OK
    torch.cuda.synchronize()


def test_static_scratch_allocates_nothing(M):
    ns = 64
    s = M.create_streams(ns, seed=SEED)
    reqs = requests(ns, 40, 23)
    M.alloc_outputs(reqs)
    assert run_static(M, s, reqs) == M.OK, M.lib.mrg_last_error()   # first call: set-up
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    used0 = torch.cuda.memory_allocated()
    for _ in range(3):
        assert run_static(M, s, reqs) == M.OK, M.lib.mrg_last_error()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert torch.cuda.memory_allocated() == used0
    assert free1 == free0, (free0, free1)
