"""The C ABI's documented argument errors, decided on the host before any
device work (no GPU needed): every case below must be refused by the
entry point's validation, which runs before the library touches a device.

The stream descriptors here carry non-null placeholder addresses that are
never dereferenced -- so the module runs only where no CUDA device exists
(on a machine with one, a validation regression must not become a launch).
"""
import ctypes

import pytest
import torch

from paper_2201_06604_gb300 import mrg

pytestmark = pytest.mark.skipif(torch.cuda.is_available(),
                                reason="placeholder device addresses: host-only checks")

L = mrg.lib
GOOD = (12345,) * 6
FAKE = 0x100000                                  # 1 MiB: aligned, never dereferenced


def seed(v):
    return (ctypes.c_uint32 * 6)(*v)


def fake_streams(n=16, stride=16):
    return mrg._Streams(FAKE, FAKE, FAKE, n, stride)


def test_create_streams_errors():
    nxt = (ctypes.c_uint32 * 6)()
    assert L.mrg_create_streams(seed((0, 0, 0, 1, 2, 3)), 1, None, nxt, None) == mrg.EINVAL
    assert L.mrg_create_streams(seed(GOOD), (1 << 63) + 1, None, nxt, None) == mrg.ERANGE
    assert L.mrg_create_streams(seed(GOOD), 5, None, nxt, None) == mrg.EINVAL
    s = fake_streams(n=4, stride=4)
    assert L.mrg_create_streams(seed(GOOD), 5, ctypes.byref(s), nxt, None) == mrg.EINVAL
    assert b"exceeds" in L.mrg_last_error()
    # n = 0 creates nothing and only reports the creator (no device work)
    assert L.mrg_create_streams(seed(GOOD), 0, None, nxt, None) == mrg.OK
    assert tuple(nxt) == GOOD


def test_generate_errors():
    s = fake_streams()
    sp = ctypes.byref(s)
    g = L.mrg_generate
    assert g(None, 8, mrg.UNIFORM, mrg.F64, 1.0, FAKE, 8, None) == mrg.EINVAL
    bad = mrg._Streams(FAKE, None, FAKE, 16, 16)
    assert g(ctypes.byref(bad), 8, mrg.UNIFORM, mrg.F64, 1.0, FAKE, 8, None) == mrg.EINVAL
    narrow = mrg._Streams(FAKE, FAKE, FAKE, 16, 8)                 # stride < n
    assert g(ctypes.byref(narrow), 8, mrg.UNIFORM, mrg.F64, 1.0, FAKE, 8, None) == mrg.EINVAL
    assert g(sp, 8, mrg.NORMAL, mrg.U32, 1.0, FAKE, 8, None) == mrg.EINVAL
    assert g(sp, 8, mrg.RAW, mrg.F64, 1.0, FAKE, 8, None) == mrg.EINVAL
    for rate in (0.0, -1.0, 2.0 ** -65, 2.0 ** 65, float("nan")):
        assert g(sp, 8, mrg.EXPONENTIAL, mrg.F64, rate, FAKE, 8, None) == mrg.EINVAL
    assert g(sp, 8, mrg.UNIFORM, mrg.F64, 1.0, None, 8, None) == mrg.EINVAL
    assert g(sp, 8, mrg.UNIFORM, mrg.F64, 1.0, FAKE, 7, None) == mrg.EINVAL
    assert g(sp, 8, mrg.UNIFORM, mrg.F64, 1.0, FAKE + 4, 8, None) == mrg.EINVAL
    assert g(sp, 8, mrg.UNIFORM, mrg.F32, 1.0, FAKE + 2, 8, None) == mrg.EINVAL
    assert g(sp, 8, mrg.UNIFORM, mrg.F64, 1.0, FAKE, 1 << 61, None) == mrg.ERANGE
    assert g(sp, (1 << 62) + 1, mrg.RAW, mrg.U32, 1.0, FAKE, (1 << 62) + 1, None) == mrg.ERANGE
    # an empty request is a no-op
    assert g(sp, 0, mrg.UNIFORM, mrg.F64, 1.0, None, 0, None) == mrg.OK


def test_transform_and_matrix_errors():
    t = L.mrg_transform
    assert t(FAKE, 8, mrg.RAW, mrg.U32, 1.0, FAKE, None) == mrg.EINVAL
    assert t(FAKE, 8, mrg.EXPONENTIAL, mrg.F32, 0.0, FAKE, None) == mrg.EINVAL
    assert t(None, 8, mrg.UNIFORM, mrg.F64, 1.0, FAKE, None) == mrg.EINVAL
    assert t(FAKE + 2, 8, mrg.UNIFORM, mrg.F64, 1.0, FAKE, None) == mrg.EINVAL
    assert t(FAKE, 8, mrg.UNIFORM, mrg.F64, 1.0, FAKE + 4, None) == mrg.EINVAL
    assert t(None, 0, mrg.UNIFORM, mrg.F64, 1.0, None, None) == mrg.OK
    s = fake_streams(n=16, stride=16)
    sp = ctypes.byref(s)
    m = L.mrg_generate_matrix
    assert m(sp, 7, 4, 4, 2, 2, mrg.UNIFORM, mrg.F64, 1.0, FAKE, 4, None) == mrg.EINVAL
    assert m(sp, 0, 4, 4, 2, 2, mrg.NORMAL, mrg.F64, 1.0, FAKE, 4, None) == mrg.EINVAL
    assert m(sp, 0, 4, 4, 0, 2, mrg.UNIFORM, mrg.F64, 1.0, FAKE, 4, None) == mrg.EINVAL
    assert m(sp, 0, 4, 4, 8, 4, mrg.UNIFORM, mrg.F64, 1.0, FAKE, 4, None) == mrg.EINVAL  # 32 > 16 streams
    assert m(sp, 0, 4, 4, 2, 2, mrg.UNIFORM, mrg.F64, 1.0, FAKE, 3, None) == mrg.EINVAL  # ld < ncol


def test_fill_and_fisher_errors():
    assert L.mrg_fill_u32(FAKE + 16, 8, 0, None) == mrg.EINVAL
    assert L.mrg_fill_u32(FAKE, 12, 0, None) == mrg.EINVAL
    assert L.mrg_fill_u32(None, 8, 0, None) == mrg.EINVAL
    assert L.mrg_fill_u32(None, 0, 0, None) == mrg.OK
    assert L.mrg_fisher_scratch_bytes(100) == 1024 + 8 * 101
    s = fake_streams()
    sp = ctypes.byref(s)
    cnt = ctypes.c_uint64()
    f = L.mrg_fisher_sim

    def table(vals):
        return (ctypes.c_int32 * len(vals))(*vals)

    ok2x2 = table([3, 1, 1, 3])
    scratch = FAKE
    nbytes = L.mrg_fisher_scratch_bytes(8)
    assert f(sp, ok2x2, 1, 4, 100, scratch, nbytes, None, ctypes.byref(cnt), None, None, None) == mrg.EINVAL
    assert f(sp, ok2x2, 2, 65, 100, scratch, nbytes, None, ctypes.byref(cnt), None, None, None) == mrg.EINVAL
    assert f(sp, table([3, -1, 1, 3]), 2, 2, 100, scratch, nbytes, None, ctypes.byref(cnt), None, None,
             None) == mrg.EINVAL
    big = table([1 << 23, 1 << 23, 1, 1])
    assert f(sp, big, 2, 2, 100, scratch, 1 << 30, None, ctypes.byref(cnt), None, None,
             None) == mrg.ERANGE
    assert f(sp, ok2x2, 2, 2, 100, scratch, nbytes - 8, None, ctypes.byref(cnt), None, None,
             None) == mrg.EINVAL                                        # scratch too small
    assert f(sp, None, 2, 2, 100, scratch, nbytes, None, ctypes.byref(cnt), None, None, None) == mrg.EINVAL


def test_mrg31k3p_errors():
    nxt = (ctypes.c_uint32 * 6)()
    assert L.mrg31k3p_create_streams(seed((2147483647, 1, 1, 1, 1, 1)), 1, None, nxt,
                                     None) == mrg.EINVAL
    assert L.mrg31k3p_create_streams(seed(GOOD), 3, None, nxt, None) == mrg.EINVAL
    s = fake_streams()
    assert L.mrg31k3p_generate(ctypes.byref(s), 8, mrg.NORMAL, mrg.U32, 1.0, FAKE, 8,
                               None) == mrg.EINVAL


def _static_call(reqs):
    f = L.mrg_batch_run_static
    f.argtypes = [ctypes.POINTER(mrg._Streams), ctypes.POINTER(mrg._Request), ctypes.c_uint32,
                  ctypes.c_void_p]
    f.restype = ctypes.c_int
    arr = (mrg._Request * len(reqs))(*reqs)
    s = fake_streams()
    return f(ctypes.byref(s), arr, len(reqs), None)


def test_static_batch_refuses_requests_before_any_device_work():
    # 2^43 + 2048 draws at 2048 draws per segment is 2^32 + 1 segments: more
    # than a request record counts, refused (it once wrapped to one segment)
    huge = mrg._Request(0, 0, 0, (1 << 43) + 2048, mrg.UNIFORM, mrg.F64, 1.0, FAKE)
    assert _static_call([huge]) == mrg.ERANGE
    assert b"2^32" in L.mrg_last_error()
    # the same checks as mrg_batch_run: stream index, dist/dtype, alignment, rate
    assert _static_call([mrg._Request(16, 0, 0, 8, mrg.UNIFORM, mrg.F64, 1.0, FAKE)]) == mrg.EINVAL
    assert _static_call([mrg._Request(0, 0, 0, 8, mrg.RAW, mrg.F64, 1.0, FAKE)]) == mrg.EINVAL
    assert _static_call([mrg._Request(0, 0, 0, 8, mrg.UNIFORM, mrg.F64, 1.0, FAKE + 16)]) == mrg.EINVAL
    assert _static_call([mrg._Request(0, 1 << 51, 0, 8, mrg.UNIFORM, mrg.F64, 1.0, FAKE)]) == mrg.ERANGE
    assert _static_call([mrg._Request(0, 0, 0, 8, mrg.EXPONENTIAL, mrg.F32, 0.0, FAKE)]) == mrg.EINVAL
    # a request of 2^26 draws takes 1024 tiles (2048-draw segments, 32 per
    # tile): 17 of them pass the 16384-tile limit
    big = [mrg._Request(0, 0, 0, 1 << 26, mrg.UNIFORM, mrg.F32, 1.0, FAKE)] * 17
    assert _static_call(big) == mrg.ERANGE
    assert b"16384" in L.mrg_last_error()
    # an empty call is a no-op that touches nothing
    assert _static_call([mrg._Request(0, 0, 0, 0, mrg.UNIFORM, mrg.F64, 1.0, None)]) == mrg.OK


def test_grf_argument_errors():
    P = mrg.MaternParams
    good = (P * 1)(P(1.25, 50e3, 1.5, 1.0, 0.0))
    nb = L.mrg_grf_matern_scratch_bytes(1, 4, 5)
    assert nb == 4096 + 7 * 9 * 8
    r = L.mrg_grf_matern_raster
    assert r(None, 1, 4, 5, 4000.0, FAKE, 20, FAKE, nb, None) == mrg.EINVAL
    assert r(good, 0, 4, 5, 4000.0, FAKE, 20, FAKE, nb, None) == mrg.EINVAL       # empty batch
    assert r(good, 65, 4, 5, 4000.0, FAKE, 20, FAKE, 1 << 30, None) == mrg.EINVAL  # batch > 64
    assert r(good, 1, 4, 5, 4000.0, FAKE, 19, FAKE, nb, None) == mrg.EINVAL       # ld < n
    assert r(good, 1, 4, 5, 0.0, FAKE, 20, FAKE, nb, None) == mrg.EINVAL          # cell
    assert r(good, 1, 4, 5, 4000.0, FAKE, 20, FAKE, nb - 8, None) == mrg.EINVAL   # scratch
    assert r(good, 1, 4, 5, 4000.0, FAKE + 8, 20, FAKE + 64, nb, None) == mrg.EINVAL  # alignment
    assert r(good, 1, 1025, 1025, 4000.0, FAKE, 1 << 21, FAKE, 1 << 40, None) == mrg.ERANGE
    for bad in (P(0.0, 50e3, 1.5, 1.0, 0.0), P(1.0, -1.0, 1.5, 1.0, 0.0),
                P(1.0, 50e3, 0.0, 1.0, 0.0), P(1.0, 50e3, 1.5, 0.5, 0.0),
                P(11.0, 50e3, 1.5, 1.0, 0.0), P(1.0, 50e3, 1.5, 1.0, float("nan"))):
        assert r((P * 1)(bad), 1, 4, 5, 4000.0, FAKE, 20, FAKE, nb, None) == mrg.EINVAL
    # the factorisation
    ws = L.mrg_grf_ldl_workspace_bytes(300, 2)
    assert ws > L.mrg_grf_ldl_workspace_bytes(300, 1) > 0
    f = L.mrg_grf_ldl
    assert f(None, 300, 300, 1, FAKE, FAKE, ws, None, None) == mrg.EINVAL
    assert f(FAKE, 300, 299, 1, FAKE, FAKE, ws, None, None) == mrg.EINVAL         # lda < n
    assert f(FAKE, 300, 300, 0, FAKE, FAKE, ws, None, None) == mrg.EINVAL         # batch 0
    assert f(FAKE, 300, 300, 256, FAKE, FAKE, 1 << 40, None, None) == mrg.EINVAL  # batch > 255
    assert f(FAKE, 300, 300, 2, FAKE, FAKE, ws - 1, None, None) == mrg.EINVAL     # workspace
    assert f(FAKE, 300, 300, 2, FAKE, FAKE + 512, ws, None, None) == mrg.EINVAL   # 1024-byte alignment
    assert f(FAKE, (1 << 20) + 1, (1 << 20) + 1, 1, FAKE, FAKE, 1 << 50, None, None) == mrg.ERANGE
    assert f(FAKE, 0, 0, 1, FAKE, FAKE, 0, None, None) == mrg.OK                   # empty: no-op
    # U = L D^(1/2) Z
    sb = L.mrg_grf_simulate_scratch_bytes(300, 2, 4)
    assert sb == 300 * 2 * 4 * 8
    s = L.mrg_grf_simulate
    assert s(FAKE, FAKE, 300, 300, 4, FAKE, 2, FAKE, FAKE, sb - 8, None) == mrg.EINVAL
    assert s(FAKE, FAKE, 300, 299, 4, FAKE, 2, FAKE, FAKE, sb, None) == mrg.EINVAL
    assert s(FAKE, FAKE + 4, 300, 300, 4, FAKE, 2, FAKE, FAKE, sb, None) == mrg.EINVAL
    assert s(FAKE, FAKE, 300, 300, 4, FAKE, (1 << 16) + 1, FAKE, FAKE, 1 << 50, None) == mrg.ERANGE
    assert s(FAKE, FAKE, 300, 300, 4, FAKE, 0, FAKE, FAKE, sb, None) == mrg.OK
