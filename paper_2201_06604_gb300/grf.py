"""Gaussian random fields by direct matrix decomposition (Sec. 5, Algorithm
2) through the library's C ABI: Matern covariance matrices, their LDL^T
factorisation on the tensor cores, and U = L D^(1/2) Z with Z drawn from the
generator's own normals.  Argument marshalling only: every step runs in the
library's kernels; device memory comes from torch."""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import mrg
from .workloads import GRF_CELL, GRF_GRID, GRF_NSIM, GRF_PARAMS  # noqa: F401 (re-exported)
from .mrg import MaternParams, _check, _stream_handle, lib



def _params(params):
    p = np.atleast_2d(np.asarray(params, dtype=np.float64))
    if p.shape[1] != 5:
        raise ValueError("params: rows of (shape, range, variance, aniso_ratio, aniso_angle)")
    arr = (MaternParams * len(p))()
    for i, row in enumerate(p):
        arr[i] = MaternParams(*[float(v) for v in row])
    return arr, len(p)


def matern_raster(params, nrow: int, ncol: int, cell: float, device=None, out=None,
                  stream=None) -> torch.Tensor:
    """Covariance matrices [batch, n, n] (n = nrow ncol) of a raster of square
    cells (mrg_grf_matern_raster)."""
    arr, batch = _params(params)
    n = nrow * ncol
    dev = torch.device(device) if device is not None else torch.device("cuda")
    if out is None:
        out = torch.empty((batch, n, n), dtype=torch.float64, device=dev)
    nb = int(lib.mrg_grf_matern_scratch_bytes(batch, nrow, ncol))
    scratch = torch.empty(nb, dtype=torch.uint8, device=out.device)
    with torch.cuda.device(out.device):
        _check(lib.mrg_grf_matern_raster(arr, batch, nrow, ncol, float(cell), out.data_ptr(),
                                         out.stride(1), scratch.data_ptr(), nb,
                                         _stream_handle(stream)))
    return out


def matern_points(params, xy: torch.Tensor, out=None, stream=None) -> torch.Tensor:
    """Covariance matrices [batch, n, n] of arbitrary locations xy [n, 2]
    (device, fp64) (mrg_grf_matern_points)."""
    arr, batch = _params(params)
    xy = xy.contiguous()
    n = xy.shape[0]
    if out is None:
        out = torch.empty((batch, n, n), dtype=torch.float64, device=xy.device)
    scratch = torch.empty(4096, dtype=torch.uint8, device=xy.device)
    with torch.cuda.device(xy.device):
        _check(lib.mrg_grf_matern_points(arr, batch, xy.data_ptr(), n, out.data_ptr(),
                                         out.stride(1), scratch.data_ptr(), 4096,
                                         _stream_handle(stream)))
    return out


def ldl_workspace(n: int, batch: int, device=None) -> torch.Tensor:
    nb = int(lib.mrg_grf_ldl_workspace_bytes(n, batch))
    return torch.empty(nb + 1024, dtype=torch.uint8, device=device)


def _aligned(ws: torch.Tensor, align: int = 1024):
    p = ws.data_ptr()
    off = (-p) % align
    return p + off, ws.numel() - off


def ldl(a: torch.Tensor, d: torch.Tensor | None = None, workspace: torch.Tensor | None = None,
        check: bool = True, stream=None):
    """Sigma = L D L^T in place for a [batch, n, n] fp64 device tensor
    (mrg_grf_ldl).  Returns (a, d, info); info is None when check is False
    (no synchronisation)."""
    if a.dim() == 2:
        a = a.unsqueeze(0)
    batch, n, _ = a.shape
    if not a.is_contiguous():
        raise ValueError("a must be contiguous [batch, n, n]")
    if d is None:
        d = torch.empty((batch, n), dtype=torch.float64, device=a.device)
    if workspace is None:
        workspace = ldl_workspace(n, batch, a.device)
    wp, wn = _aligned(workspace)
    info = (ctypes.c_int32 * batch)() if check else None
    with torch.cuda.device(a.device):
        _check(lib.mrg_grf_ldl(a.data_ptr(), n, a.stride(1), batch, d.data_ptr(), wp, wn, info,
                               _stream_handle(stream)))
    return a, d, (list(info) if check else None)


def simulate(l: torch.Tensor, d: torch.Tensor, z: torch.Tensor, out=None, scratch=None,
             stream=None) -> torch.Tensor:
    """U = L D^(1/2) Z (mrg_grf_simulate): l [batch, n, n] from ldl(), d
    [batch, n], z [batch, nsim, n] standard normals; returns [batch, nsim, n]."""
    if l.dim() == 2:
        l = l.unsqueeze(0)
    batch, n, _ = l.shape
    nsim = z.shape[-2] if z.dim() == 3 else 1
    z = z.reshape(batch, nsim, n).contiguous()
    if out is None:
        out = torch.empty_like(z)
    nb = int(lib.mrg_grf_simulate_scratch_bytes(n, nsim, batch))
    if scratch is None:
        scratch = torch.empty(nb, dtype=torch.uint8, device=l.device)
    with torch.cuda.device(l.device):
        _check(lib.mrg_grf_simulate(l.data_ptr(), d.data_ptr(), n, l.stride(1), batch, z.data_ptr(),
                                    nsim, out.data_ptr(), scratch.data_ptr(), nb,
                                    _stream_handle(stream)))
    return out


def simulate_fields(streams: "mrg.Streams", params, nrow: int, ncol: int, cell: float,
                    nsim: int = 2):
    """Algorithm 2 end to end on a raster: covariance matrices of every
    parameter set, their LDL^T, Z from the first batch * nsim streams of
    `streams` (n normals each, fp64), U = L D^(1/2) Z.  Returns (U, Z, L, D)
    with U and Z [batch, nsim, n]."""
    cov = matern_raster(params, nrow, ncol, cell, device=streams.device)
    batch, n, _ = cov.shape
    l, d, info = ldl(cov)
    if any(info):
        raise mrg.MrgError(mrg.EINVAL, f"covariance matrix not positive definite: info {info}")
    need = batch * nsim
    if streams.n < need:
        raise ValueError(f"need {need} streams")
    z = mrg.generate(streams.view(0, need), n, "normal", torch.float64)
    u = simulate(l, d, z.view(batch, nsim, n))
    return u, z.view(batch, nsim, n), l, d


def _example(repeats: int = 1) -> None:
    """The paper's example (Sec. 5): four Matern parameter sets on the 62 x 90
    raster, two simulations each, end to end on cuda:0; prints each stage's
    time (CUDA events) and the factorisation's info."""
    dev = torch.device("cuda", 0)
    params = np.array(GRF_PARAMS)
    nrow, ncol = GRF_GRID
    n, batch = nrow * ncol, len(params)
    streams = mrg.create_streams(batch * GRF_NSIM, device=dev, seed=(12345,) * 6)
    cov = torch.empty((batch, n, n), dtype=torch.float64, device=dev)
    d = torch.empty((batch, n), dtype=torch.float64, device=dev)
    ws = ldl_workspace(n, batch, dev)
    for _ in range(repeats):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
        ev[0].record()
        matern_raster(params, nrow, ncol, GRF_CELL, out=cov)
        ev[1].record()
        _, _, info = ldl(cov, d, ws, check=True)
        ev[2].record()
        z = mrg.generate(streams, n, "normal", torch.float64).view(batch, GRF_NSIM, n)
        ev[3].record()
        u = simulate(cov, d, z)
        ev[4].record()
        torch.cuda.synchronize()
        t = [ev[i].elapsed_time(ev[i + 1]) for i in range(4)]
        print(f"covariance {t[0]:.3f} ms, LDL^T {t[1]:.3f} ms, normals {t[2]:.3f} ms, "
              f"U = L D^1/2 Z {t[3]:.3f} ms; info {info}; U[0, 0, :3] = {u[0, 0, :3].tolist()}")


if __name__ == "__main__":
    import sys
    _example(int(sys.argv[1]) if len(sys.argv) > 1 else 1)
