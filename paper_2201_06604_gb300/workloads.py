"""Seeded synthetic workloads shared by the tests and the benchmark.

This module holds no arithmetic of the method: only the sizes, mixes and
arrival processes of the workloads, drawn with numpy's seeded generator.
The generator seed 12345 x 6 is the paper's default creator seed (Sec. 2.1).
"""
from __future__ import annotations

import numpy as np

PAPER_SEED = (12345, 12345, 12345, 12345, 12345, 12345)

# Plain check: 1024 streams x 1024 fp64 uniforms (2^20) plus final states.
PLAIN = dict(streams=1024, draws=1024)
# Materialised generation: 65536 streams (the paper's 512 x 128 work items,
# Sec. 3.1 timing example) x 16384 draws = 2^30 outputs per variant.
MATERIALISED = dict(streams=65536, draws=16384)
MATERIALISED_VARIANTS = (("uniform", "f64"), ("uniform", "f32"), ("normal", "f64"),
                         ("normal", "f32"), ("exponential", "f32"))
# Fused consumer: 2^20 streams x 4096 draws.
FUSED = dict(streams=1 << 20, draws=4096)
# Gaussian random fields (Sec. 5): the paper's four Matern parameter sets
# (shape, range [m], variance, anisoRatio, anisoAngleRadians), its 62 x 90
# raster (the swissRain extent is not available: 4 km square cells stand in
# for it) and two simulations per parameter set.
GRF_PARAMS = ((1.25, 50e3, 1.5, 1.0, 0.0),
              (2.15, 60e3, 2.0, 4.0, np.pi / 7),
              (0.60, 30e3, 2.0, 2.0, np.pi / 5),
              (3.00, 30e3, 2.0, 2.0, np.pi / 7))
GRF_GRID = (62, 90)
GRF_CELL = 4000.0
GRF_NSIM = 2


def random_states(n: int, seed: int = 0) -> np.ndarray:
    """n valid MRG32k3a states [n, 6] (uniform words below each modulus; an
    all-zero triple, probability ~2^-96, is replaced)."""
    rng = np.random.default_rng(seed)
    st = np.empty((n, 6), np.uint32)
    st[:, :3] = rng.integers(0, 4294967087, size=(n, 3), dtype=np.uint64)
    st[:, 3:] = rng.integers(0, 4294944443, size=(n, 3), dtype=np.uint64)
    st[(st[:, :3] == 0).all(axis=1), 0] = 1
    st[(st[:, 3:] == 0).all(axis=1), 3] = 1
    return st


def batched_requests(nreq: int = 4096, lo: float = 1e2, hi: float = 1e6, seed: int = 1):
    """Uneven requests: lengths log-uniform in [lo, hi], dist uniform over
    {uniform, normal, exponential}, dtype uniform over {f32, f64}; request r
    runs on stream r, substream 1."""
    rng = np.random.default_rng(seed)
    n = np.exp(rng.uniform(np.log(lo), np.log(hi), nreq)).astype(np.int64)
    dist = rng.integers(1, 4, nreq)   # 1 uniform, 2 normal, 3 exponential
    f64 = rng.integers(0, 2, nreq).astype(bool)
    return [dict(stream=r, substream=1, n=int(n[r]), dist=int(dist[r]),
                 dtype="f64" if f64[r] else "f32", rate=1.0) for r in range(nreq)]


def serving_trace(rate_hz: float = 2000.0, seconds: float = 10.0, lo: float = 1e3,
                  hi: float = 1e8, n_streams: int = 1 << 20, seed: int = 2):
    """Poisson arrivals at rate_hz over `seconds`, sizes log-uniform in
    [lo, hi] draws, mixed dist/dtype, stream id uniform in [0, n_streams)."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t >= seconds:
            break
        out.append(dict(t=t, stream=int(rng.integers(0, n_streams)),
                        n=int(np.exp(rng.uniform(np.log(lo), np.log(hi)))),
                        dist=int(rng.integers(1, 4)),
                        dtype="f64" if rng.integers(0, 2) else "f32", rate=1.0))
    return out
