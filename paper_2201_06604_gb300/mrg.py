"""Python binding of libmrg32k3a (ctypes; argument marshalling only).

Every step of the hot path runs in the library's CUDA kernels; torch only
provides device memory and CUDA streams.  If the compiled library is missing
this module raises at import: there is no CPU fallback.

Names follow the C ABI in include/mrg32k3a.h.  The module keeps a stream
creator state like the paper's hidden creator seed (Sec. 2.1,
setBaseCreator / createStreamsGpu): `set_base_creator(seed)` sets it, and every
`create_streams(n)` call reads it and advances it past the streams it made.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np
import torch

from . import build as _build

RAW, UNIFORM, NORMAL, EXPONENTIAL = 0, 1, 2, 3
U32, F32, F64 = 0, 1, 2
OK, EINVAL, ERANGE, ECUDA, EBUSY, ETIMEOUT = 0, -1, -2, -3, -4, -5

DEFAULT_SEED = (12345, 12345, 12345, 12345, 12345, 12345)
M1, M2 = 4294967087, 4294944443

_DIST = {"raw": RAW, "uniform": UNIFORM, "normal": NORMAL, "exponential": EXPONENTIAL}
_DTYPE = {torch.float32: F32, torch.float64: F64, torch.int32: U32}


class MrgError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class _Request(ctypes.Structure):
    _fields_ = [("stream", ctypes.c_uint64), ("substream", ctypes.c_uint64),
                ("offset", ctypes.c_uint64), ("n", ctypes.c_uint64), ("dist", ctypes.c_int32),
                ("dtype", ctypes.c_int32), ("rate", ctypes.c_double), ("out", ctypes.c_void_p)]


class LaunchConfig(ctypes.Structure):
    """Launch shape of the generate kernel (mrg_launch_config); 0 = default."""
    _fields_ = [("seg_len", ctypes.c_uint64), ("block", ctypes.c_uint32),
                ("vec_bytes", ctypes.c_uint32), ("blocks_per_sm", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32)]

    def as_dict(self):
        return {"seg_len": int(self.seg_len), "block": int(self.block),
                "vec_bytes": int(self.vec_bytes), "blocks_per_sm": int(self.blocks_per_sm)}


class _TuneEntry(ctypes.Structure):
    _fields_ = [("cfg", LaunchConfig), ("ms", ctypes.c_float)]


class Tiling(ctypes.Structure):
    """Request tiling of the batch runner and the serving engine (mrg_tiling)."""
    _fields_ = [("seg_min", ctypes.c_uint32), ("seg_max", ctypes.c_uint32),
                ("target_segments", ctypes.c_uint64)]

    def as_dict(self):
        return {"seg_min": int(self.seg_min), "seg_max": int(self.seg_max),
                "target_segments": int(self.target_segments)}


def _tiling(t) -> Tiling:
    if isinstance(t, Tiling):
        return t
    return Tiling(int(t["seg_min"]), int(t["seg_max"]), int(t["target_segments"]))


class _BatchTuneEntry(ctypes.Structure):
    _fields_ = [("tiling", Tiling), ("tiles", ctypes.c_uint64), ("ms", ctypes.c_float)]


class MaternParams(ctypes.Structure):
    """One Matern parameter set (mrg_matern_params, Sec. 5)."""
    _fields_ = [("shape", ctypes.c_double), ("range", ctypes.c_double),
                ("variance", ctypes.c_double), ("aniso_ratio", ctypes.c_double),
                ("aniso_angle", ctypes.c_double)]


class _Streams(ctypes.Structure):
    _fields_ = [("cur", ctypes.c_void_p), ("start", ctypes.c_void_p), ("sub", ctypes.c_void_p),
                ("n", ctypes.c_uint64), ("stride", ctypes.c_uint64)]


def _load():
    path = _build.LIB
    if not os.path.exists(path):
        raise ImportError(f"libmrg32k3a is not built ({path}); run "
                          "`python -m paper_2201_06604_gb300.build` first")
    L = ctypes.CDLL(path)
    vp, u64, i32, u32p = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.POINTER(ctypes.c_uint32)
    sp = ctypes.POINTER(_Streams)
    sig = {
        "mrg_last_error": ([], ctypes.c_char_p),
        "mrg_launch_count": ([], u64),
        "mrg_version": ([], ctypes.c_char_p),
        "mrg_seed_check": ([u32p], i32),
        "mrg_create_streams": ([u32p, u64, sp, u32p, vp], i32),
        "mrg_creator_advance": ([u32p, u64, u32p], i32),
        "mrg31k3p_creator_advance": ([u32p, u64, u32p], i32),
        "mrg_generate": ([sp, u64, i32, i32, ctypes.c_double, vp, u64, vp], i32),
        "mrg_skip": ([sp, u64, u64, vp], i32),
        "mrg_transform": ([vp, u64, i32, i32, ctypes.c_double, vp, vp], i32),
        "mrg_generate_host": ([sp, u64, i32, i32, ctypes.c_double, vp, u64, vp, u64, vp], i32),
        "mrg_substream_next": ([sp, vp], i32),
        "mrg_reset_substream": ([sp, vp], i32),
        "mrg_reset_stream": ([sp, vp], i32),
        "mrg_get_state": ([sp, u32p, vp], i32),
        "mrg_set_state": ([sp, u32p, vp], i32),
        "mrg_fused_pi_normsum": ([sp, u64, vp, vp, vp], i32),
        "mrg_fill_u32": ([vp, u64, ctypes.c_uint32, vp], i32),
        "mrg_generate_matrix": ([sp, i32, u64, u64, ctypes.c_uint32, ctypes.c_uint32, i32, i32,
                                 ctypes.c_double, vp, u64, vp], i32),
        "mrg_fisher_scratch_bytes": ([u64], u64),
        "mrg_fisher_sim": ([sp, ctypes.POINTER(ctypes.c_int32), ctypes.c_uint32, ctypes.c_uint32,
                            u64, vp, u64, vp, ctypes.POINTER(u64), ctypes.POINTER(ctypes.c_double),
                            ctypes.POINTER(ctypes.c_double), vp], i32),
        "mrg31k3p_seed_check": ([u32p], i32),
        "mrg31k3p_create_streams": ([u32p, u64, sp, u32p, vp], i32),
        "mrg31k3p_generate": ([sp, u64, i32, i32, ctypes.c_double, vp, u64, vp], i32),
        "mrg31k3p_skip": ([sp, u64, vp], i32),
        "mrg_generate_config": ([sp, u64, i32, i32, ctypes.c_double, vp, u64,
                                 ctypes.POINTER(LaunchConfig), vp], i32),
        "mrg_tune_generate": ([sp, u64, i32, i32, ctypes.c_double, vp, u64, ctypes.c_uint32,
                               ctypes.POINTER(_TuneEntry), ctypes.c_uint32,
                               ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(LaunchConfig), vp],
                              i32),
        "mrg_tune_lookup": ([i32, i32, u64, u64, ctypes.POINTER(LaunchConfig)], i32),
        "mrg_tune_set": ([i32, i32, u64, u64, ctypes.POINTER(LaunchConfig)], i32),
        "mrg_tune_clear": ([], None),
        "mrg_batch_create": ([sp, ctypes.c_uint32, u64, ctypes.POINTER(vp), vp], i32),
        "mrg_batch_run": ([vp, ctypes.POINTER(_Request), ctypes.c_uint32, vp], i32),
        "mrg_batch_run_plain": ([sp, ctypes.POINTER(_Request), ctypes.c_uint32, vp], i32),
        "mrg_batch_last_tiles": ([vp], u64),
        "mrg_batch_set_tiling": ([vp, ctypes.POINTER(Tiling)], i32),
        "mrg_batch_get_tiling": ([vp, ctypes.POINTER(Tiling)], i32),
        "mrg_batch_tune": ([vp, ctypes.POINTER(_Request), ctypes.c_uint32, ctypes.c_uint32,
                            ctypes.POINTER(_BatchTuneEntry), ctypes.c_uint32,
                            ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(Tiling), vp], i32),
        "mrg_server_set_tiling": ([vp, ctypes.POINTER(Tiling)], i32),
        "mrg_batch_destroy": ([vp], i32),
        "mrg_batch_run_static": ([sp, ctypes.POINTER(_Request), ctypes.c_uint32, vp], i32),
        "mrg_server_create": ([sp, vp, u64, ctypes.c_uint32, u64, ctypes.c_double,
                               ctypes.c_double, ctypes.POINTER(vp)], i32),
        "mrg_server_submit": ([vp, ctypes.POINTER(_Request), ctypes.POINTER(u64),
                               ctypes.POINTER(vp)], i32),
        "mrg_server_poll": ([vp, ctypes.POINTER(u64), ctypes.c_uint32,
                             ctypes.POINTER(ctypes.c_uint32)], i32),
        "mrg_server_release": ([vp, u64], i32),
        "mrg_server_inflight": ([vp], u64),
        "mrg_server_restart": ([vp], i32),
        "mrg_server_destroy": ([vp], i32),
        "mrg_grf_matern_scratch_bytes": ([ctypes.c_uint32] * 3, u64),
        "mrg_grf_matern_raster": ([ctypes.POINTER(MaternParams), ctypes.c_uint32, ctypes.c_uint32,
                                   ctypes.c_uint32, ctypes.c_double, vp, u64, vp, u64, vp], i32),
        "mrg_grf_matern_points": ([ctypes.POINTER(MaternParams), ctypes.c_uint32, vp, u64, vp, u64,
                                   vp, u64, vp], i32),
        "mrg_grf_ldl_workspace_bytes": ([u64, ctypes.c_uint32], u64),
        "mrg_grf_ldl": ([vp, u64, u64, ctypes.c_uint32, vp, vp, u64,
                         ctypes.POINTER(ctypes.c_int32), vp], i32),
        "mrg_grf_simulate_scratch_bytes": ([u64, ctypes.c_uint32, ctypes.c_uint32], u64),
        "mrg_grf_simulate": ([vp, vp, u64, u64, ctypes.c_uint32, vp, ctypes.c_uint32, vp, vp, u64,
                              vp], i32),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    return L


lib = _load()


def _check(rc: int):
    if rc != OK:
        raise MrgError(rc, lib.mrg_last_error().decode())


def _stream_handle(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _u32_array(values) -> ctypes.Array:
    a = (ctypes.c_uint32 * 6)(*[int(v) for v in values])
    return a


def launch_count() -> int:
    return int(lib.mrg_launch_count())


def seed_check(seed) -> bool:
    return lib.mrg_seed_check(_u32_array(seed)) == OK


GENERATORS = ("mrg32k3a", "mrg31k3p")


class Streams:
    """n streams on one device: three int32 tensors [6, n] holding the uint32
    words of the current state, the stream start and the substream start.
    `generator` is "mrg32k3a" (default) or "mrg31k3p" (the paper's own
    generator; create + generate + skip and the state copies only)."""

    generator = "mrg32k3a"

    def __init__(self, n: int, device=None, *, _tensors=None, generator: str = "mrg32k3a"):
        if generator not in GENERATORS:
            raise ValueError(f"generator must be one of {GENERATORS}")
        self.generator = generator
        dev = torch.device(device) if device is not None else torch.device("cuda")
        if _tensors is None:
            self.buf = torch.empty((3, 6, max(n, 1)), dtype=torch.int32, device=dev)
        else:
            self.buf = _tensors
        self.n = n
        self._c = _Streams(self.buf[0].data_ptr(), self.buf[1].data_ptr(), self.buf[2].data_ptr(),
                           n, self.buf.shape[2])

    @property
    def cur(self):
        return self.buf[0, :, : self.n]

    @property
    def start(self):
        return self.buf[1, :, : self.n]

    @property
    def sub(self):
        return self.buf[2, :, : self.n]

    @property
    def device(self):
        return self.buf.device

    def view(self, a: int, m: int) -> "Streams":
        """Streams [a, a + m) sharing this set's memory."""
        if a < 0 or m < 0 or a + m > self.n:
            raise IndexError("stream range out of bounds")
        v = Streams.__new__(Streams)
        v.buf, v.n, v.generator = self.buf, m, self.generator
        v._c = _Streams(self.buf[0].data_ptr() + 4 * a, self.buf[1].data_ptr() + 4 * a,
                        self.buf[2].data_ptr() + 4 * a, m, self.buf.shape[2])
        v._parent = self
        return v

    def ptr(self):
        return ctypes.byref(self._c)


class _Creator:
    def __init__(self):
        self.lock = threading.Lock()
        self.seed = list(DEFAULT_SEED)


_creator = _Creator()


def set_base_creator(seed=DEFAULT_SEED):
    """Sets the creator state that the next create_streams call starts from."""
    if not seed_check(seed):
        raise MrgError(EINVAL, "invalid seed")
    with _creator.lock:
        _creator.seed = [int(v) for v in seed]


def creator_advance(seed, n_streams: int, generator: str = "mrg32k3a") -> tuple:
    """The creator state after n_streams streams (seed advanced n_streams *
    2^127 steps for MRG32k3a, 2^134 for MRG31k3p), on the host: the seed of
    a shard whose streams start n_streams into the creator's sequence."""
    if generator not in GENERATORS:
        raise ValueError(f"generator must be one of {GENERATORS}")
    out = (ctypes.c_uint32 * 6)()
    fn = lib.mrg31k3p_creator_advance if generator == "mrg31k3p" else lib.mrg_creator_advance
    _check(fn(_u32_array(seed), int(n_streams), out))
    return tuple(int(v) for v in out)


def get_base_creator():
    with _creator.lock:
        return tuple(_creator.seed)


def create_streams(n: int, device=None, seed=None, stream=None,
                   generator: str = "mrg32k3a") -> Streams:
    """Creates n streams on the device.  With seed=None the module's creator
    state is used and advanced by n streams (Sec. 2.1); an explicit seed
    leaves the creator untouched.  generator="mrg31k3p" creates streams of
    the paper's own generator (2^134 apart; an explicit seed is required)."""
    s = Streams(n, device, generator=generator)
    nxt = (ctypes.c_uint32 * 6)()
    fn = lib.mrg31k3p_create_streams if generator == "mrg31k3p" else lib.mrg_create_streams
    with torch.cuda.device(s.device):
        if seed is None:
            if generator != "mrg32k3a":
                raise ValueError("the module's creator state is MRG32k3a's: pass a seed")
            with _creator.lock:
                _check(fn(_u32_array(_creator.seed), n, s.ptr(), nxt, _stream_handle(stream)))
                _creator.seed = list(nxt)
        else:
            _check(fn(_u32_array(seed), n, s.ptr(), nxt, _stream_handle(stream)))
    s.next_seed = tuple(nxt)
    return s


def _dtype_code(dist: int, dtype) -> int:
    if dist == RAW:
        return U32
    return {torch.float32: F32, torch.float64: F64}[dtype]


def generate(streams: Streams, n: int, dist="uniform", dtype=torch.float64, rate: float = 1.0,
             out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """n values per stream into a [streams.n, n] tensor (stream-major), or
    into `out` (2-D, row stride = leading dimension, unit column stride).
    Raw draws come back as int32 holding the uint32 bit patterns."""
    d = _DIST[dist] if isinstance(dist, str) else int(dist)
    dt = torch.int32 if d == RAW else dtype
    code = _dtype_code(d, dt)
    if out is None:
        out = torch.empty((streams.n, n), dtype=dt, device=streams.device)
    if out.dim() != 2 or out.shape[0] < streams.n or out.shape[1] < n or out.stride(1) != 1:
        raise ValueError("out must be [>= n_streams, >= n] with unit column stride")
    if out.dtype != dt:
        raise ValueError(f"out dtype {out.dtype} != {dt}")
    fn = lib.mrg31k3p_generate if streams.generator == "mrg31k3p" else lib.mrg_generate
    with torch.cuda.device(streams.device):
        _check(fn(streams.ptr(), n, d, code, float(rate), out.data_ptr(), out.stride(0),
                  _stream_handle(stream)))
    return out


def _need_mrg32k3a(streams: Streams, what: str):
    if streams.generator != "mrg32k3a":
        raise ValueError(f"{what} is implemented for MRG32k3a streams only")


def _gen_args(streams, n, dist, dtype, out):
    d = _DIST[dist] if isinstance(dist, str) else int(dist)
    dt = torch.int32 if d == RAW else dtype
    code = _dtype_code(d, dt)
    if out is None:
        out = torch.empty((streams.n, n), dtype=dt, device=streams.device)
    if out.dim() != 2 or out.shape[0] < streams.n or out.shape[1] < n or out.stride(1) != 1:
        raise ValueError("out must be [>= n_streams, >= n] with unit column stride")
    if out.dtype != dt:
        raise ValueError(f"out dtype {out.dtype} != {dt}")
    return d, code, out


def _config(cfg) -> LaunchConfig:
    if isinstance(cfg, LaunchConfig):
        return cfg
    c = LaunchConfig()
    for k, v in dict(cfg).items():
        setattr(c, k, int(v))
    return c


def generate_config(streams: Streams, n: int, cfg, dist="uniform", dtype=torch.float64,
                    rate: float = 1.0, out: torch.Tensor | None = None,
                    stream=None) -> torch.Tensor:
    """generate() with an explicit launch shape (dict or LaunchConfig with
    seg_len, block, vec_bytes, blocks_per_sm); same output for any shape."""
    _need_mrg32k3a(streams, "generate_config")
    d, code, out = _gen_args(streams, n, dist, dtype, out)
    c = _config(cfg)
    with torch.cuda.device(streams.device):
        _check(lib.mrg_generate_config(streams.ptr(), n, d, code, float(rate), out.data_ptr(),
                                       out.stride(0), ctypes.byref(c), _stream_handle(stream)))
    return out


def tune_generate(streams: Streams, n: int, dist="uniform", dtype=torch.float64,
                  rate: float = 1.0, out: torch.Tensor | None = None, reps: int = 3,
                  stream=None):
    """Runs the library's autotuner for this generate call (states are not
    advanced) and returns (best shape dict, [(shape dict, ms), ...])."""
    _need_mrg32k3a(streams, "tune_generate")
    d, code, out = _gen_args(streams, n, dist, dtype, out)
    res = (_TuneEntry * 64)()
    nres = ctypes.c_uint32()
    best = LaunchConfig()
    with torch.cuda.device(streams.device):
        _check(lib.mrg_tune_generate(streams.ptr(), n, d, code, float(rate), out.data_ptr(),
                                     out.stride(0), reps, res, 64, ctypes.byref(nres),
                                     ctypes.byref(best), _stream_handle(stream)))
    return best.as_dict(), [(res[i].cfg.as_dict(), float(res[i].ms)) for i in range(nres.value)]


def tune_lookup(dist, dtype, n_streams: int, n: int, device=None) -> dict:
    """The launch shape generate() uses for this size class."""
    d = _DIST[dist] if isinstance(dist, str) else int(dist)
    c = LaunchConfig()
    with torch.cuda.device(device if device is not None else torch.cuda.current_device()):
        _check(lib.mrg_tune_lookup(d, _dtype_code(d, dtype), n_streams, n, ctypes.byref(c)))
    return c.as_dict()


def tune_set(dist, dtype, n_streams: int, n: int, cfg, device=None):
    """Records a launch shape for a size class (cfg=None removes it)."""
    d = _DIST[dist] if isinstance(dist, str) else int(dist)
    c = None if cfg is None else ctypes.byref(_config(cfg))
    with torch.cuda.device(device if device is not None else torch.cuda.current_device()):
        _check(lib.mrg_tune_set(d, _dtype_code(d, dtype), n_streams, n, c))


def tune_clear():
    lib.mrg_tune_clear()


def generate_host(streams: Streams, n: int, dist="uniform", dtype=torch.float64,
                  rate: float = 1.0, out: torch.Tensor | None = None,
                  scratch: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Like generate, but into a host tensor (pinned when allocated here); the
    device-to-host copy of one chunk of streams overlaps the generation of
    the next.  `scratch` is a device uint8 tensor (default 512 MiB)."""
    _need_mrg32k3a(streams, "generate_host")
    d = _DIST[dist] if isinstance(dist, str) else int(dist)
    dt = torch.int32 if d == RAW else dtype
    code = _dtype_code(d, dt)
    if out is None:
        out = torch.empty((streams.n, n), dtype=dt, pin_memory=True)
    if out.device.type != "cpu" or out.dim() != 2 or out.stride(1) != 1 or out.dtype != dt:
        raise ValueError("out must be a 2-D host tensor with unit column stride")
    if out.shape[0] < streams.n or out.shape[1] < n:
        raise ValueError("out too small")
    if scratch is None:
        scratch = torch.empty(512 << 20, dtype=torch.uint8, device=streams.device)
    with torch.cuda.device(streams.device):
        _check(lib.mrg_generate_host(streams.ptr(), n, d, code, float(rate), out.data_ptr(),
                                     out.stride(0), scratch.data_ptr(), scratch.numel(),
                                     _stream_handle(stream)))
    return out


def transform(z: torch.Tensor, dist="normal", dtype=torch.float64, rate: float = 1.0,
              out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Applies the generate transform to raw draws z (int32 tensor holding
    uint32 values in [1, m1]; consecutive pairs for normals)."""
    d = _DIST[dist] if isinstance(dist, str) else int(dist)
    if d == RAW:
        raise ValueError("raw draws need no transform")
    code = _dtype_code(d, dtype)
    z = z.contiguous()
    n = z.numel()
    if out is None:
        out = torch.empty(n, dtype=dtype, device=z.device)
    with torch.cuda.device(z.device):
        _check(lib.mrg_transform(z.data_ptr(), n, d, code, float(rate), out.data_ptr(),
                                 _stream_handle(stream)))
    return out


def skip(streams: Streams, k: int, stream=None):
    if streams.generator == "mrg31k3p":
        if k < 0 or k >= 1 << 64:
            raise ValueError("k must be in [0, 2^64) for MRG31k3p streams")
        with torch.cuda.device(streams.device):
            _check(lib.mrg31k3p_skip(streams.ptr(), k, _stream_handle(stream)))
        return
    if k < 0 or k >= 1 << 128:
        raise ValueError("k must be in [0, 2^128)")
    with torch.cuda.device(streams.device):
        _check(lib.mrg_skip(streams.ptr(), k >> 64, k & ((1 << 64) - 1), _stream_handle(stream)))


def substream_next(streams: Streams, stream=None):
    _need_mrg32k3a(streams, "substream_next")
    with torch.cuda.device(streams.device):
        _check(lib.mrg_substream_next(streams.ptr(), _stream_handle(stream)))


def reset_substream(streams: Streams, stream=None):
    with torch.cuda.device(streams.device):
        _check(lib.mrg_reset_substream(streams.ptr(), _stream_handle(stream)))


def reset_stream(streams: Streams, stream=None):
    with torch.cuda.device(streams.device):
        _check(lib.mrg_reset_stream(streams.ptr(), _stream_handle(stream)))


def get_state(streams: Streams, stream=None) -> np.ndarray:
    """Host checkpoint [3, 6, n] uint32: (cur, start, sub)."""
    host = np.zeros((3, 6, max(streams.n, 1)), np.uint32)
    with torch.cuda.device(streams.device):
        _check(lib.mrg_get_state(streams.ptr(), host.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                                 _stream_handle(stream)))
    return host[:, :, : streams.n].copy()


def set_state(streams: Streams, host, stream=None):
    host = np.ascontiguousarray(host, dtype=np.uint32)
    if host.shape != (3, 6, streams.n):
        raise ValueError("state must be [3, 6, n]")
    with torch.cuda.device(streams.device):
        _check(lib.mrg_set_state(streams.ptr(), host.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                                 _stream_handle(stream)))


def fused_pi_normsum(streams: Streams, draws: int, count=None, sum_=None, stream=None):
    _need_mrg32k3a(streams, "fused_pi_normsum")
    if count is None:
        count = torch.empty(streams.n, dtype=torch.int64, device=streams.device)
    if sum_ is None:
        sum_ = torch.empty(streams.n, dtype=torch.float64, device=streams.device)
    with torch.cuda.device(streams.device):
        _check(lib.mrg_fused_pi_normsum(streams.ptr(), draws, count.data_ptr(), sum_.data_ptr(),
                                        _stream_handle(stream)))
    return count, sum_


def generate_matrix(streams: Streams, shape, nglobal=(2, 2), dist="uniform",
                    dtype=torch.float64, rate: float = 1.0, out=None, stream=None) -> torch.Tensor:
    """The paper's runifGpu / rexpGpu layout (Sec. 2.2): `shape` is n (a
    vector) or (nrow, ncol); nglobal the work-item grid.  Returns a tensor of
    that shape (row-major)."""
    nrow, ncol = (int(shape), 1) if np.ndim(shape) == 0 else (int(shape[0]), int(shape[1]))
    d = _DIST[dist] if isinstance(dist, str) else int(dist)
    dt = torch.int32 if d == RAW else dtype
    if out is None:
        out = torch.empty((nrow, ncol), dtype=dt, device=streams.device)
    if out.dim() != 2 or out.shape[0] < nrow or out.shape[1] < ncol or out.stride(1) != 1:
        raise ValueError("out must be [>= nrow, >= ncol] with unit column stride")
    gen = 1 if streams.generator == "mrg31k3p" else 0
    with torch.cuda.device(streams.device):
        _check(lib.mrg_generate_matrix(streams.ptr(), gen, nrow, ncol, int(nglobal[0]),
                                       int(nglobal[1]), d, _dtype_code(d, dt), float(rate),
                                       out.data_ptr(), out.stride(0), _stream_handle(stream)))
    return out[:, 0] if np.ndim(shape) == 0 else out


def fill_u32(t: torch.Tensor, value: int = 0, stream=None):
    """Writes `value` into every 32-bit word of a device tensor (32-byte
    aligned, size a multiple of 32 bytes) with the library's write-only
    stream kernel."""
    nbytes = t.numel() * t.element_size()
    with torch.cuda.device(t.device):
        _check(lib.mrg_fill_u32(t.data_ptr(), nbytes // 4, value, _stream_handle(stream)))
    return t


def fisher_sim(streams: Streams, table, B: int, return_stats: bool = False, stream=None) -> dict:
    """Monte Carlo Fisher's exact test (Sec. 4, fisher.sim): B random tables
    with the margins of `table` (I x J integers), replicate b on stream
    b mod streams.n.  Returns dict(p_value (the library's (1+count)/(B+1)), count, threshold,
    B[, stats = device tensor of the B statistics])."""
    _need_mrg32k3a(streams, "fisher_sim")
    t = np.ascontiguousarray(np.asarray(table), dtype=np.int32)
    if t.ndim != 2:
        raise ValueError("table must be 2-D")
    I, J = t.shape
    total = int(t.sum())
    nbytes = int(lib.mrg_fisher_scratch_bytes(total))
    scratch = torch.empty(nbytes, dtype=torch.uint8, device=streams.device)
    stats = torch.empty(max(B, 1), dtype=torch.float64, device=streams.device) if return_stats else None
    cnt, thr, pv = ctypes.c_uint64(), ctypes.c_double(), ctypes.c_double()
    with torch.cuda.device(streams.device):
        _check(lib.mrg_fisher_sim(streams.ptr(), t.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                  I, J, B, scratch.data_ptr(), nbytes,
                                  stats.data_ptr() if return_stats else None, ctypes.byref(cnt),
                                  ctypes.byref(thr), ctypes.byref(pv), _stream_handle(stream)))
    out = {"p_value": pv.value, "count": int(cnt.value),
           "threshold": thr.value, "B": B}
    if return_stats:
        out["stats"] = stats[:B]
    return out


_DT_CODE = {"u32": U32, "f32": F32, "f64": F64}
_DT_TORCH = {"u32": torch.int32, "f32": torch.float32, "f64": torch.float64}


class PreparedRequests:
    """A request list marshalled into C request records (see Batch)."""

    def __init__(self, requests):
        self.n = len(requests)
        self.arr = (_Request * max(self.n, 1))()
        for i, q in enumerate(requests):
            d = _DIST[q["dist"]] if isinstance(q["dist"], str) else int(q["dist"])
            dt = q.get("dtype", "f64")
            self.arr[i] = _Request(q["stream"], q.get("substream", 0), q.get("offset", 0), q["n"], d,
                                   U32 if d == RAW else _DT_CODE[dt], float(q.get("rate", 1.0)),
                                   q["out"].data_ptr() if q["n"] else None)
        self._keep = [q["out"] for q in requests if q["n"]]   # outputs stay alive


class Batch:
    """Runner of batched requests over a stream set: one persistent,
    graph-captured kernel launch per run.  A request is a dict with keys
    stream, substream, offset (default 0), n, dist ("uniform" / "normal" /
    "exponential" / "raw" or code), dtype ("f32" / "f64" / "u32"), rate
    (default 1.0) and out (a device tensor of n elements, 32-byte aligned)."""

    def __init__(self, streams: Streams, max_requests: int = 4096, max_tiles: int = 1 << 16,
                 stream=None):
        _need_mrg32k3a(streams, "Batch")
        self.streams = streams
        self.max_requests = max_requests
        h = ctypes.c_void_p()
        with torch.cuda.device(streams.device):
            _check(lib.mrg_batch_create(streams.ptr(), max_requests, max_tiles, ctypes.byref(h),
                                        _stream_handle(stream)))
        self._h = h

    @staticmethod
    def prepare(requests) -> "PreparedRequests":
        """Marshals a request list once into the C request records, for
        callers that run the same requests repeatedly (run() accepts the
        result in place of the list)."""
        return PreparedRequests(requests)

    @staticmethod
    def _requests(requests):
        if isinstance(requests, PreparedRequests):
            return requests.arr, requests.n
        p = PreparedRequests(requests)
        return p.arr, p.n

    def run(self, requests, stream=None):
        arr, n = self._requests(requests)
        with torch.cuda.device(self.streams.device):
            _check(lib.mrg_batch_run(self._h, arr, n, _stream_handle(stream)))

    def run_plain(self, requests, stream=None):
        """The same requests served one by one from the library's host loop
        (mrg_batch_run_plain: a position jump and a generate launch per
        request); same outputs as run()."""
        arr, n = self._requests(requests)
        with torch.cuda.device(self.streams.device):
            _check(lib.mrg_batch_run_plain(self.streams.ptr(), arr, n, _stream_handle(stream)))

    def set_tiling(self, tiling=None):
        """tiling: dict(seg_min, seg_max, target_segments) or None (default)."""
        _check(lib.mrg_batch_set_tiling(self._h, None if tiling is None
                                        else ctypes.byref(_tiling(tiling))))

    def get_tiling(self) -> dict:
        t = Tiling()
        _check(lib.mrg_batch_get_tiling(self._h, ctypes.byref(t)))
        return t.as_dict()

    def tune(self, requests, reps: int = 3, stream=None):
        """Runs the library's tiling autotuner on these requests (their
        outputs are written) and keeps the fastest tiling; returns
        (best tiling dict, [(tiling dict, tiles, ms), ...])."""
        arr, n = self._requests(requests)
        res = (_BatchTuneEntry * 64)()
        nres = ctypes.c_uint32()
        best = Tiling()
        with torch.cuda.device(self.streams.device):
            _check(lib.mrg_batch_tune(self._h, arr, n, reps, res, 64,
                                      ctypes.byref(nres), ctypes.byref(best),
                                      _stream_handle(stream)))
        return best.as_dict(), [(res[i].tiling.as_dict(), int(res[i].tiles), float(res[i].ms))
                                for i in range(nres.value)]

    @property
    def last_tiles(self) -> int:
        return int(lib.mrg_batch_last_tiles(self._h))

    def close(self):
        if self._h:
            lib.mrg_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def alloc_outputs(requests, device=None, align: int = 256):
    """One device buffer holding every request's output (aligned slices);
    sets q["out"] on each request and returns the backing buffer."""
    offs, total = [], 0
    for q in requests:
        es = 8 if q.get("dtype", "f64") == "f64" else 4
        offs.append(total)
        total += (q["n"] * es + align - 1) // align * align
    buf = torch.empty(max(total, align), dtype=torch.uint8, device=device or "cuda")
    for q, o in zip(requests, offs):
        dt = q.get("dtype", "f64")
        if (_DIST[q["dist"]] if isinstance(q["dist"], str) else int(q["dist"])) == RAW:
            dt = "u32"
        es = 8 if dt == "f64" else 4
        q["out"] = buf[o: o + q["n"] * es].view(_DT_TORCH[dt])
    return buf


class Server:
    """Serving engine: a persistent worker kernel that requests join while it
    runs (continuous batching).  Admission is by free slots, ring space and
    output memory in the arena; submit returns None when the request must wait
    (the caller keeps it queued and retries after releasing finished ones)."""

    def __init__(self, streams: Streams, arena_bytes: int, max_slots: int = 4096,
                 ring_tiles: int = 1 << 16, idle_seconds: float = 30.0, sm_fraction: float = 0.5):
        _need_mrg32k3a(streams, "Server")
        self.streams = streams
        self.arena = torch.empty(arena_bytes, dtype=torch.uint8, device=streams.device)
        h = ctypes.c_void_p()
        with torch.cuda.device(streams.device):
            _check(lib.mrg_server_create(streams.ptr(), self.arena.data_ptr(), arena_bytes,
                                         max_slots, ring_tiles, float(idle_seconds),
                                         float(sm_fraction), ctypes.byref(h)))
        self._h = h
        self._ids = (ctypes.c_uint64 * max_slots)()
        self._cap = max_slots

    def submit(self, stream: int, n: int, dist="uniform", dtype="f64", substream: int = 0,
               offset: int = 0, rate: float = 1.0):
        """Returns (id, output tensor view in the arena) or None if busy."""
        d = _DIST[dist] if isinstance(dist, str) else int(dist)
        dt = "u32" if d == RAW else dtype
        req = _Request(stream, substream, offset, n, d, _DT_CODE[dt], float(rate), None)
        rid, out = ctypes.c_uint64(), ctypes.c_void_p()
        rc = lib.mrg_server_submit(self._h, ctypes.byref(req), ctypes.byref(rid), ctypes.byref(out))
        if rc == EBUSY:
            return None
        _check(rc)
        es = 8 if dt == "f64" else 4
        off = out.value - self.arena.data_ptr()
        return rid.value, self.arena[off: off + n * es].view(_DT_TORCH[dt])

    def poll(self):
        cnt = ctypes.c_uint32()
        _check(lib.mrg_server_poll(self._h, self._ids, self._cap, ctypes.byref(cnt)))
        return [self._ids[i] for i in range(cnt.value)]

    def poll_status(self):
        """(ids, status code) without raising."""
        cnt = ctypes.c_uint32()
        rc = lib.mrg_server_poll(self._h, self._ids, self._cap, ctypes.byref(cnt))
        return [self._ids[i] for i in range(cnt.value)], rc

    def release(self, rid: int):
        _check(lib.mrg_server_release(self._h, rid))

    def set_tiling(self, tiling=None):
        """Tiling of requests admitted from now on (None: the default)."""
        _check(lib.mrg_server_set_tiling(self._h, None if tiling is None
                                         else ctypes.byref(_tiling(tiling))))

    def inflight(self) -> int:
        return int(lib.mrg_server_inflight(self._h))

    def restart(self):
        _check(lib.mrg_server_restart(self._h))

    def close(self):
        if self._h:
            rc = lib.mrg_server_destroy(self._h)
            self._h = None
            _check(rc)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
