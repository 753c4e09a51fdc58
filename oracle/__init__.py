"""Plain CPU oracle for the multi-stream MRG32k3a hot path.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg may use this package; the product
path (``paper_2201_06604_gb300``) never imports it, and it imports nothing
from the product.  The arithmetic lives in ``mrg_oracle.c`` (plain C, 128-bit
integers, IEEE double); this module compiles it with gcc on first use and
wraps it with ctypes + numpy.

Conventions (see mrg_oracle.c for the passages each one follows):
  * a stream state is six words, newest first
    (x1[n-1], x1[n-2], x1[n-3], x2[n-1], x2[n-2], x2[n-3]) -- Sec. 2.1;
  * streams are 2^127 steps apart and substreams 2^76 apart for MRG32k3a;
    the paper's own generator MRG31k3p uses 2^134 (Sec. 2.1);
  * uniforms are z * (1/(m1+1)) in IEEE double, z in [1, m1] (Sec. 2.2);
  * normals are Box-Muller on consecutive pairs of one stream (Sec. 3.1),
    exponentials -ln(u)/rate (Sec. 3.2, reading fixed by the printed values).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mrg_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")

# Generator parameters p[8] = (m1, m2, a1_1, a1_2, a1_3, a2_1, a2_2, a2_3):
# a_c_j multiplies x_c[n-j].
# MRG32k3a: L'Ecuyer (1999), the generator of RngStreams (cited in Sec. 1).
MRG32K3A = (4294967087, 4294944443, 0, 1403580, -810728, 527612, 0, -1370589)
# MRG31k3p: L'Ecuyer and Touzin (2000), the paper's base generator (Sec. 2).
MRG31K3P = (2147483647, 2147462579, 0, 1 << 22, (1 << 7) + 1, 1 << 15, 0, (1 << 15) + 1)

STREAM_LOG2 = {MRG32K3A: 127, MRG31K3P: 134}
SUBSTREAM_LOG2 = 76  # MRG32k3a substream spacing (RngStreams)

RAW, UNIFORM, NORMAL, EXPONENTIAL = 0, 1, 2, 3

_lock = threading.Lock()
_lib = None

_u32p = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")
_u64p = np.ctypeslib.ndpointer(np.uint64, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
_f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile mrg_oracle.c into _build/liboracle.so (gcc, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math",
               "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            P = _i64p
            L.orc_matpow.argtypes = [P, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, _u64p]
            L.orc_matpow2k.argtypes = [P, ctypes.c_int, ctypes.c_uint, _u64p]
            L.orc_jump.argtypes = [P, _u32p, ctypes.c_uint64, ctypes.c_uint64]
            L.orc_create_streams.argtypes = [P, _u32p, ctypes.c_uint64, ctypes.c_uint,
                                             _u32p, _u32p]
            L.orc_raw.argtypes = [P, _u32p, ctypes.c_uint64, _u32p]
            L.orc_uniform64.argtypes = [P, _u32p, ctypes.c_uint64, _f64p]
            L.orc_uniform32.argtypes = [P, _u32p, ctypes.c_uint64, _f32p]
            L.orc_normal.argtypes = [P, _u32p, ctypes.c_uint64, _f64p]
            L.orc_exponential.argtypes = [P, _u32p, ctypes.c_uint64, ctypes.c_double, _f64p]
            L.orc_box_muller_pairs.argtypes = [P, _u32p, ctypes.c_uint64, _f64p]
            L.orc_exp_of.argtypes = [P, _u32p, ctypes.c_uint64, ctypes.c_double, _f64p]
            L.orc_norm.argtypes = [P]
            L.orc_norm.restype = ctypes.c_double
            L.orc_generate_streams.argtypes = [P, _u32p, ctypes.c_uint64, ctypes.c_uint64,
                                               ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                               ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int]
            L.orc_fused.argtypes = [P, _u32p, ctypes.c_uint64, ctypes.c_uint64, _i64p, _f64p,
                                    ctypes.c_int]
            _i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
            L.orc_logfact_table.argtypes = [ctypes.c_uint64, _f64p]
            L.orc_logfact_sum.argtypes = [_i32p, ctypes.c_uint32, ctypes.c_uint32, _f64p]
            L.orc_logfact_sum.restype = ctypes.c_double
            L.orc_hyper_inv.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                        ctypes.c_double, _f64p]
            L.orc_hyper_inv.restype = ctypes.c_int64
            L.orc_fisher.argtypes = [P, _u32p, ctypes.c_uint64, _i32p, ctypes.c_uint32,
                                     ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double, _f64p,
                                     ctypes.c_void_p, ctypes.c_int]
            L.orc_fisher.restype = ctypes.c_uint64
            L.orc_fisher_tables.argtypes = [P, _u32p, _i32p, ctypes.c_uint32, ctypes.c_uint32,
                                            ctypes.c_uint64, _f64p, _i32p]
            _lib = L
    return _lib


def _p(gen):
    return np.asarray(gen, dtype=np.int64)


def _state(st):
    a = np.ascontiguousarray(np.asarray(st, dtype=np.uint32).reshape(6))
    return a


def _split(e: int):
    if e < 0 or e >= 1 << 128:
        raise ValueError("exponent out of range")
    return e & ((1 << 64) - 1), e >> 64


def matpow(c: int, e: int, gen=MRG32K3A) -> np.ndarray:
    """A_c^e mod m_c as a 3x3 uint64 array (c = 0 or 1)."""
    out = np.zeros(9, np.uint64)
    lo, hi = _split(e)
    lib().orc_matpow(_p(gen), c, lo, hi, out)
    return out.reshape(3, 3)


def matpow2k(c: int, k: int, gen=MRG32K3A) -> np.ndarray:
    """A_c^(2^k) mod m_c by k squarings (any k >= 0)."""
    out = np.zeros(9, np.uint64)
    lib().orc_matpow2k(_p(gen), c, k, out)
    return out.reshape(3, 3)


def jump(state, e: int, gen=MRG32K3A) -> np.ndarray:
    """The state e steps after `state`."""
    st = _state(state).copy()
    lo, hi = _split(e)
    lib().orc_jump(_p(gen), st, lo, hi)
    return st


def create_streams(seed, n: int, gen=MRG32K3A, zlog2: int | None = None):
    """Stream starts created one after another, 2^zlog2 steps apart.

    Returns (states[n, 6], next_seed[6])."""
    zlog2 = STREAM_LOG2[tuple(gen)] if zlog2 is None else zlog2
    states = np.zeros((max(n, 1), 6), np.uint32)
    nxt = np.zeros(6, np.uint32)
    lib().orc_create_streams(_p(gen), _state(seed), n, zlog2, states.reshape(-1), nxt)
    return states[:n], nxt


def raw(state, n: int, gen=MRG32K3A):
    """(z[n] in [1, m1], state after)."""
    st = _state(state).copy()
    out = np.zeros(max(n, 1), np.uint32)
    lib().orc_raw(_p(gen), st, n, out)
    return out[:n], st


def uniform64(state, n: int, gen=MRG32K3A):
    st = _state(state).copy()
    out = np.zeros(max(n, 1), np.float64)
    lib().orc_uniform64(_p(gen), st, n, out)
    return out[:n], st


def uniform32(state, n: int, gen=MRG32K3A):
    st = _state(state).copy()
    out = np.zeros(max(n, 1), np.float32)
    lib().orc_uniform32(_p(gen), st, n, out)
    return out[:n], st


def normal(state, n: int, gen=MRG32K3A):
    """Double reference normals; the state advances by n + (n % 2) draws."""
    st = _state(state).copy()
    out = np.zeros(max(n, 1), np.float64)
    lib().orc_normal(_p(gen), st, n, out)
    return out[:n], st


def exponential(state, n: int, rate: float = 1.0, gen=MRG32K3A):
    st = _state(state).copy()
    out = np.zeros(max(n, 1), np.float64)
    lib().orc_exponential(_p(gen), st, n, float(rate), out)
    return out[:n], st


def box_muller_of(z, gen=MRG32K3A) -> np.ndarray:
    """Box-Muller outputs (X, Y per pair) for given output integers z[2k]."""
    z = np.ascontiguousarray(z, dtype=np.uint32)
    out = np.zeros(max(z.size, 2), np.float64)
    lib().orc_box_muller_pairs(_p(gen), z, z.size // 2, out)
    return out[: 2 * (z.size // 2)]


def exp_of(z, rate: float = 1.0, gen=MRG32K3A) -> np.ndarray:
    """-ln(z/(m1+1))/rate for given output integers."""
    z = np.ascontiguousarray(z, dtype=np.uint32)
    out = np.zeros(max(z.size, 1), np.float64)
    lib().orc_exp_of(_p(gen), z, z.size, float(rate), out)
    return out[: z.size]


def norm(gen=MRG32K3A) -> float:
    return lib().orc_norm(_p(gen))


def generate_streams(states, n: int, dist: int, f32: bool = False, rate: float = 1.0,
                     nthreads: int = 1, gen=MRG32K3A):
    """Generate n values for every row of states[ns, 6].

    Returns (out[ns, n], states after).  Output dtype: uint32 for RAW, float32
    for an f32 UNIFORM, otherwise float64 (normals and exponentials are always
    the double reference)."""
    states = np.array(states, dtype=np.uint32, order="C", copy=True)
    ns = states.shape[0]
    if dist == RAW:
        dt = np.uint32
    elif dist == UNIFORM and f32:
        dt = np.float32
    else:
        dt = np.float64
    out = np.zeros((ns, max(n, 1)), dt)
    lib().orc_generate_streams(_p(gen), states.reshape(-1), ns, n, dist, int(bool(f32)),
                               float(rate), out.ctypes.data, out.shape[1], nthreads)
    return out[:, :n], states


def fused(states, draws: int, nthreads: int = 1, gen=MRG32K3A):
    """Per-stream (count of pairs inside the quarter circle, sum of X+Y)."""
    states = np.ascontiguousarray(states, dtype=np.uint32).copy()
    ns = states.shape[0]
    cnt = np.zeros(max(ns, 1), np.int64)
    sm = np.zeros(max(ns, 1), np.float64)
    lib().orc_fused(_p(gen), states.reshape(-1), ns, draws, cnt, sm, nthreads)
    return cnt[:ns], sm[:ns], states


# ---------------------------------------------------------------------------
# Fisher's exact test by Monte Carlo (Sec. 4)
# ---------------------------------------------------------------------------

def logfact_table(n: int) -> np.ndarray:
    """log(k!) for k = 0..n (lgamma)."""
    lf = np.zeros(n + 1, np.float64)
    lib().orc_logfact_table(n, lf)
    return lf


def logfact_sum(table, lf=None) -> float:
    """-sum log(n_ij!) of a table (the statistic of Sec. 4, logfactSum)."""
    t = np.ascontiguousarray(table, dtype=np.int32)
    if lf is None:
        lf = logfact_table(int(t.max()))
    return lib().orc_logfact_sum(t, t.shape[0], t.shape[1], lf)


def hyper_inv(S: int, K: int, R: int, u: float, lf) -> int:
    """Smallest x with u <= F(x), F the CDF of the number of marked items in
    R draws without replacement from S items of which K are marked."""
    return int(lib().orc_hyper_inv(S, K, R, float(u), lf))


def fisher_threshold(table, lf=None) -> float:
    """The observed statistic, widened by a relative 64 ulp so that tables
    whose statistic equals it mathematically count as "at or below" it
    whatever their summation rounding."""
    return logfact_sum(table, lf) / (1.0 + 64.0 * np.finfo(np.float64).eps)


def fisher(states, table, B: int, nthreads: int = 1, return_stats: bool = False,
           gen=MRG32K3A):
    """B simulated tables with the margins of `table`; replicate b uses
    stream b mod len(states).  Returns (count of statistics <= threshold,
    threshold, states after[, stats[B]])."""
    t = np.ascontiguousarray(table, dtype=np.int32)
    I, J = t.shape
    if not (2 <= I <= 64 and 2 <= J <= 64):
        raise ValueError("2 <= I, J <= 64")
    lf = logfact_table(int(t.sum()))
    thr = fisher_threshold(t, lf)
    st = np.array(states, dtype=np.uint32, order="C", copy=True)
    stats = np.zeros(max(B, 1), np.float64) if return_stats else None
    cnt = lib().orc_fisher(_p(gen), st.reshape(-1), st.shape[0], t, I, J, B, thr, lf,
                           stats.ctypes.data if return_stats else None, nthreads)
    out = (int(cnt), thr, st)
    return out + (stats[:B],) if return_stats else out


def fisher_tables(state, table, B: int, gen=MRG32K3A):
    """B random tables [B, I, J] with the margins of `table`, from one stream
    (returns (tables, state after))."""
    t = np.ascontiguousarray(table, dtype=np.int32)
    I, J = t.shape
    lf = logfact_table(int(t.sum()))
    st = _state(state).copy()
    out = np.zeros((max(B, 1), I, J), np.int32)
    lib().orc_fisher_tables(_p(gen), st, t, I, J, B, lf, out.reshape(-1))
    return out[:B], st
