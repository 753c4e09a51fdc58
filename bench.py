"""Benchmark of the MRG32k3a multi-stream hot path on GB300.

Step = one pass of the materialised-generation workload: create 65536 streams
from the paper's default seed (12345 x 6) by successive 2^127 jumps, then
generate 16384 draws per stream (2^30 outputs) of each of fp64 uniform, fp32
uniform, fp64 normal, fp32 normal and fp32 exponential(1), each stream's state
written back after every call.  Outputs (4-8 GiB per variant) are larger than
L2, so no flush is needed between steps.

Prints ONE JSON line (rank 0).  `--impl reference` times the CPU oracle on the
host cores over a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "MRG32k3a draws/s & GB/s vs HBM peak; batched/plain speedup; p99 latency"
VARIANTS = (("uniform", "f64"), ("uniform", "f32"), ("normal", "f64"), ("normal", "f32"),
            ("exponential", "f32"))
ES = {"f64": 8, "f32": 4, "u32": 4}
DTYPE_NOTE = ("exact 32-bit integer recurrence; uniforms formed in integers; normals and "
              "exponentials in double-float (fp32 pairs); fp64 and fp32 outputs")

# Warp-level instructions issued per output by generate_kernel, measured with
# ncu (smsp__inst_executed.sum x 32 / outputs) on 65536 streams x 2048 draws
# (profiles/generate_pipe_balance_65536x2048.txt, fp64 exponentials from a
# capture of their own at the same size, listed there).
# These kernels are bound by instruction issue or by the IMAD (fmaheavy) pipe
# (the FP64 pipe is not used and the recurrence is integer multiply-add work),
# so beside the HBM roofline the bench reports issue slots: 4
# warp-instructions per cycle per SM.
INSTR_PER_OUTPUT = {("raw", "u32"): 28.1, ("uniform", "f64"): 43.8, ("uniform", "f32"): 38.2,
                    ("normal", "f64"): 115.1, ("normal", "f32"): 83.7,
                    ("exponential", "f32"): 58.0, ("exponential", "f64"): 93.9}


def env_rank():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]
        return False

    def summary(self):
        sms, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sms.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sms:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        return {"sm_mhz": float(np.median(sms)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sms)}


# ---------------------------------------------------------------------------
# Reference arm: the CPU oracle on the host cores
# ---------------------------------------------------------------------------

def load_table(name):
    """A contingency table printed in the paper (test fixture, Sec. 4)."""
    rows = []
    with open(os.path.join(ROOT, "tests", "golden", name)) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([int(v) for v in line.split()])
    return np.array(rows, np.int32)


def cpu_oracle_sample(streams: int, draws: int, nthreads: int):
    """Times the oracle on `streams` streams x `draws` draws of every variant
    (same seed, same transforms).  Returns (draws/s, seconds, draws done)."""
    import oracle as O
    st, _ = O.create_streams((12345,) * 6, streams)
    codes = {"uniform": O.UNIFORM, "normal": O.NORMAL, "exponential": O.EXPONENTIAL}
    t0 = time.perf_counter()
    total = 0
    for dist, dt in VARIANTS:
        _, st = O.generate_streams(st, draws, codes[dist], f32=(dt == "f32"), nthreads=nthreads)
        total += streams * draws
    sec = time.perf_counter() - t0
    return total / sec, sec, total


def run_reference(args):
    rank, _, world = env_rank()
    if rank != 0:
        return
    import oracle
    oracle.build()
    cores = len(os.sched_getaffinity(0))
    streams, draws = 4096, 16384   # bounded sample of the 65536 x 16384 workload
    for _ in range(args.warmup):
        cpu_oracle_sample(streams, draws, cores)
    times, total = [], 0
    for _ in range(args.steps):
        v, sec, total = cpu_oracle_sample(streams, draws, cores)
        times.append(sec)
    value = total / float(np.mean(times))
    sample = (f"{streams} of 65536 streams x {draws} draws x {len(VARIANTS)} variants per step "
              f"({total} draws), OpenMP over streams")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "draws/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * float(np.mean(times)), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32+fp64/fp32",
            "dtype_note": DTYPE_NOTE, "data": "synthetic",
            "config": {"workload": "materialised generation, 65536 streams x 16384 draws x 5 "
                                   "variants (fp64/fp32 uniform, fp64/fp32 normal, fp32 Exp(1))",
                       "sample": sample},
            "cpu_baseline": {"value": value, "unit": "draws/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "draws/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

# DRAM bytes (read + write) per output of generate_kernel, from an ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum) on 65536 streams x 4096 draws
# (profiles/generate_dram_traffic_65536x4096.txt).
TRAFFIC_PER_OUTPUT = {("uniform", "f64"): 7.829, ("uniform", "f32"): 3.809,
                      ("normal", "f64"): 7.822, ("normal", "f32"): 3.813,
                      ("exponential", "f32"): 3.812}


def roofline(dom, hbm, peak_kind, issue_peak, total_out, sm_count):
    """The dominant kernel against the HBM roofline: algorithmic bytes (8 or 4
    B written per draw + 24 B of state read per stream) per launch over its
    CUDA-event duration, against the measured copy bandwidth.  The issue-slot
    fraction (instructions per output from ncu x outputs / duration, against
    4 warp-instructions per cycle per SM) sits beside it: it is what holds
    the transform kernels below the HBM line on a part with weak FP64."""
    key = (dom["dist"], dom["dtype"])
    traffic = TRAFFIC_PER_OUTPUT.get(key)
    traffic = traffic * total_out if traffic else None
    out = {"kernel": f"generate_kernel<{dom['dist']},{dom['dtype']}>", "bound": "hbm",
           "achieved": dom["gbs"], "peak": hbm, "unit": "GB/s", "frac": dom["hbm_frac"],
           "traffic": traffic, "algo_bytes_per_launch": dom["algo_bytes"],
           "ms_per_launch": dom["ms"], "peak_source": f"{peak_kind} hbm_gbs (MEASURED_PEAKS.json)"}
    if "issue_tinst_s" in dom:
        out.update({"issue_achieved_tinst_s": dom["issue_tinst_s"], "issue_peak_tinst_s": issue_peak,
                    "issue_frac": dom["issue_tinst_s"] / issue_peak,
                    "issue_peak_source": f"4 warp-instructions/cycle/SM x {sm_count} SMs x "
                                         "sm_max_mhz (MEASURED_PEAKS.json) x 32 threads"})
    return out


def run_batched(mrg, W, dev, stream, seed, quick=False, reps=3, tune=True):
    """4096 requests, lengths log-uniform in [1e2, 1e6], mixed dist/dtype,
    request r on stream r, substream 1: one persistent graph-captured launch
    vs 4096 plain mrg_generate calls (each followed by its state advance)."""
    import torch
    reqs = W.batched_requests(1024 if quick else 4096)
    for q in reqs:
        q["dist"] = {1: "uniform", 2: "normal", 3: "exponential"}[q["dist"]]
    nst = len(reqs)
    s = mrg.create_streams(nst, device=dev, seed=seed)
    buf_b = mrg.alloc_outputs(reqs, device=dev)
    outs_b = [q["out"] for q in reqs]
    b = mrg.Batch(s, max_requests=nst, max_tiles=1 << 17)
    b.run(reqs)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    prepared = b.prepare(reqs)   # requests marshalled once (a C caller has none of this)

    def time_batch(r):
        b.run(r)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            b.run(r)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps
    t_default = time_batch(prepared)
    tiling, tiles_default = b.get_tiling(), b.last_tiles
    if tune:
        # the library's tiling autotuner on this request mix (untimed)
        tiling, table = b.tune(prepared, reps=3)
    t_batch = time_batch(prepared)
    t_python = time_batch(reqs)  # the same runs with the request list marshalled every time
    # plain: position every stream at substream 1, then one call per request
    plain = [dict(q) for q in reqs]
    buf_p = mrg.alloc_outputs(plain, device=dev)
    views = [s.view(r, 1) for r in range(nst)]
    tdt = {"f32": torch.float32, "f64": torch.float64}
    mrg.substream_next(s)

    def plain_pass():
        mrg.reset_substream(s)
        for r, q in enumerate(plain):
            mrg.generate(views[r], q["n"], q["dist"], tdt[q["dtype"]], out=q["out"].view(1, -1))
    plain_pass()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        plain_pass()
    e1.record(stream)
    torch.cuda.synchronize()
    t_plain = e0.elapsed_time(e1) / reps
    identical = all(torch.equal(a, q["out"]) for a, q in zip(outs_b, plain))
    # plain launches issued from the library's own host loop
    # (mrg_batch_run_plain: per request one position jump + one generate
    # launch): launch against launch, without the interpreter in between
    plain_c = [dict(q) for q in reqs]
    buf_c = mrg.alloc_outputs(plain_c, device=dev)
    prepared_c = b.prepare(plain_c)
    b.run_plain(prepared_c)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        b.run_plain(prepared_c)
    e1.record(stream)
    torch.cuda.synchronize()
    t_plain_c = e0.elapsed_time(e1) / reps
    identical_c = all(torch.equal(a, q["out"]) for a, q in zip(outs_b, plain_c))
    draws = sum(q["n"] + (q["n"] & 1 if q["dist"] == "normal" else 0) for q in reqs)
    nbytes = sum(q["n"] * (8 if q["dtype"] == "f64" else 4) for q in reqs)
    res = {"workload": f"{nst} requests, n log-uniform [1e2, 1e6], mixed dist/dtype, "
                       "request r on stream r substream 1",
           "draws": draws, "bytes": nbytes, "tiles": b.last_tiles, "tiling": tiling,
           "untuned_ms": t_default, "untuned_tiles": tiles_default,
           "batched_ms_python_marshalling": t_python,
           "batched_ms": t_batch, "plain_ms_c": t_plain_c, "speedup_c": t_plain_c / t_batch,
           "plain_ms_python": t_plain, "speedup_python": t_plain / t_batch,
           "batched_draws_per_s": draws / (t_batch / 1e3), "batched_gbs": nbytes / (t_batch / 1e3) / 1e9,
           "plain_launches": 2 * nst, "identical_output": bool(identical and identical_c)}
    b.close()
    del buf_b, buf_p, buf_c
    return res


def run_serving(mrg, W, dev, seed, seconds=10.0, arena_gb=40):
    """Poisson arrivals (2000 req/s), sizes log-uniform in [1e3, 1e8] draws,
    mixed dist/dtype, 2^20 resident streams, request -> uniform stream id (its
    next substream), outputs in a 40 GB arena released on completion: the
    serving engine vs the same trace served by serial plain calls."""
    import collections
    import torch
    trace = W.serving_trace(seconds=seconds)
    for q in trace:
        q["dist"] = {1: "uniform", 2: "normal", 3: "exponential"}[q["dist"]]
    ns = 1 << 20
    streams = mrg.create_streams(ns, device=dev, seed=seed)
    next_sub = collections.defaultdict(int)
    for q in trace:
        q["substream"] = next_sub[q["stream"]]
        next_sub[q["stream"]] += 1
    draws = sum(q["n"] + (q["n"] & 1 if q["dist"] == "normal" else 0) for q in trace)

    def pct(lat):
        a = np.array(lat) * 1e3
        return {"p50_ms": float(np.percentile(a, 50)), "p99_ms": float(np.percentile(a, 99)),
                "p999_ms": float(np.percentile(a, 99.9)), "mean_ms": float(a.mean())}

    # serving engine
    sv = mrg.Server(streams, arena_gb << 30, max_slots=8192, ring_tiles=1 << 18, idle_seconds=60.0,
                    sm_fraction=1.0)
    lat, arrival, busy = [], {}, 0
    pending = collections.deque()
    i, n_req = 0, len(trace)
    t0 = time.perf_counter()
    while i < n_req or pending or arrival:
        now = time.perf_counter() - t0
        while i < n_req and trace[i]["t"] <= now:
            pending.append(trace[i])
            i += 1
        while pending:
            q = pending[0]
            r = sv.submit(q["stream"], q["n"], q["dist"], q["dtype"], q["substream"], 0, q["rate"])
            if r is None:
                busy += 1
                break
            arrival[r[0]] = q["t"]
            pending.popleft()
        done = sv.poll()
        if done:
            tc = time.perf_counter() - t0
            for rid in done:
                lat.append(tc - arrival.pop(rid))
                sv.release(rid)
        if now > seconds + 120:
            raise RuntimeError("serving run did not drain")
    t_end = time.perf_counter() - t0
    sv.close()
    served = {"requests": n_req, "draws": draws, "draws_per_s": draws / t_end,
              "wall_s": t_end, "busy_retries": busy, **pct(lat)}
    del sv
    torch.cuda.empty_cache()

    # saturation: the whole trace offered at once (admission by slots and
    # arena memory gates it), until every request has completed
    sv = mrg.Server(streams, arena_gb << 30, max_slots=8192, ring_tiles=1 << 18, idle_seconds=60.0,
                    sm_fraction=1.0)
    pending = collections.deque(trace)
    inflight = 0
    t0 = time.perf_counter()
    while pending or inflight:
        while pending:
            q = pending[0]
            r = sv.submit(q["stream"], q["n"], q["dist"], q["dtype"], q["substream"], 0, q["rate"])
            if r is None:
                break
            pending.popleft()
            inflight += 1
        for rid in sv.poll():
            sv.release(rid)
            inflight -= 1
        if time.perf_counter() - t0 > 120:
            raise RuntimeError("saturated serving run did not drain")
    sat_s = time.perf_counter() - t0
    sv.close()
    del sv
    torch.cuda.empty_cache()

    # serial plain calls (one request at a time, synchronous)
    maxn = max(q["n"] for q in trace)
    out = torch.empty(maxn * 8, dtype=torch.uint8, device=dev)
    tdt = {"f32": torch.float32, "f64": torch.float64}
    lat = []
    t0 = time.perf_counter()
    for q in trace:
        now = time.perf_counter() - t0
        if now < q["t"]:
            while time.perf_counter() - t0 < q["t"]:
                pass
        es = 8 if q["dtype"] == "f64" else 4
        o = out[: q["n"] * es].view(tdt[q["dtype"]]).view(1, -1)
        mrg.generate(streams.view(q["stream"], 1), q["n"], q["dist"], tdt[q["dtype"]], out=o)
        torch.cuda.synchronize()
        lat.append(time.perf_counter() - t0 - q["t"])
    t_end = time.perf_counter() - t0
    serial = {"draws_per_s": draws / t_end, "wall_s": t_end, **pct(lat)}
    # the same requests back to back as fast as plain calls go (no pacing)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for q in trace:
        es = 8 if q["dtype"] == "f64" else 4
        o = out[: q["n"] * es].view(tdt[q["dtype"]]).view(1, -1)
        mrg.generate(streams.view(q["stream"], 1), q["n"], q["dist"], tdt[q["dtype"]], out=o)
    torch.cuda.synchronize()
    plain_sat_s = time.perf_counter() - t0
    del out, streams
    torch.cuda.empty_cache()
    return {"workload": f"Poisson 2000 req/s for {seconds:g} s ({n_req} requests), n log-uniform "
                        "[1e3, 1e8], mixed dist/dtype, 2^20 resident streams, 40 GB arena",
            "offered_draws_per_s": draws / seconds, "server": served, "serial_plain": serial,
            "p99_speedup": serial["p99_ms"] / served["p99_ms"],
            "saturated": {"server_s": sat_s, "server_draws_per_s": draws / sat_s,
                          "plain_back_to_back_s": plain_sat_s,
                          "plain_draws_per_s": draws / plain_sat_s,
                          "speedup": plain_sat_s / sat_s}}


def grf_tensor_flops(n: int, batch: int, nb: int = 128, bm: int = 128, bn: int = 64,
                     slices: int = 8) -> float:
    """bf16 tensor-core FLOPs the factorisation issues: per 128-column panel
    step, the panel product (tiles of 128 x 64) and the lower-triangle tiles
    of the trailing product, each tile slices (slices + 1) / 2 digit products
    of bm x bn x nb multiply-adds."""
    per_tile = slices * (slices + 1) // 2 * 2.0 * bm * bn * nb
    tiles = 0
    for k0 in range(0, n, nb):
        kb = min(nb, n - k0)
        nt = n - k0 - kb
        if nt <= 0:
            break
        T = -(-nt // bm)
        tiles += T * (-(-kb // bn))                     # panel
        tiles += T * (T - 1) + (-(-nt // bn))           # trailing, lower tiles
    return per_tile * tiles * batch


def run_grf(dev, stream, peaks, steps=3):
    """Gaussian random fields on the paper's example (Sec. 5): the 62 x 90
    raster of 4 km cells, the four printed parameter sets, two simulations
    each -- covariance, LDL^T and U = L D^(1/2) Z, with Z from the
    generator's normals."""
    import torch
    from paper_2201_06604_gb300 import grf as R, mrg
    from paper_2201_06604_gb300 import workloads as W
    P = np.array(W.GRF_PARAMS)
    nrow, ncol = W.GRF_GRID
    cell = W.GRF_CELL
    n, batch, nsim = nrow * ncol, len(P), W.GRF_NSIM
    cov = torch.empty((batch, n, n), dtype=torch.float64, device=dev)
    d = torch.empty((batch, n), dtype=torch.float64, device=dev)
    ws = R.ldl_workspace(n, batch, dev)
    s = mrg.create_streams(batch * nsim, device=dev, seed=(12345,) * 6)
    z = torch.empty((batch, nsim, n), dtype=torch.float64, device=dev)
    u = torch.empty_like(z)

    def ev():
        return torch.cuda.Event(enable_timing=True)

    def one():
        e = [ev() for _ in range(5)]
        e[0].record(stream)
        R.matern_raster(P, nrow, ncol, cell, out=cov)
        e[1].record(stream)
        R.ldl(cov, d, ws, check=False)
        e[2].record(stream)
        mrg.generate(s, n, "normal", torch.float64, out=z.view(batch * nsim, n))
        e[3].record(stream)
        R.simulate(cov, d, z, out=u)
        e[4].record(stream)
        torch.cuda.synchronize()
        return [e[i].elapsed_time(e[i + 1]) for i in range(4)]
    one()
    _, _, info = R.ldl(R.matern_raster(P, nrow, ncol, cell, out=cov), d, ws, check=True)
    t = np.array([one() for _ in range(steps)]).mean(axis=0)
    # each parameter set alone (batch of one)
    alone = []
    for b in range(batch):
        c1 = cov[b:b + 1]
        R.matern_raster(P[b:b + 1], nrow, ncol, cell, out=c1)
        R.ldl(c1, d[b:b + 1], ws, check=False)
        torch.cuda.synchronize()
        R.matern_raster(P[b:b + 1], nrow, ncol, cell, out=c1)
        a0, a1 = ev(), ev()
        a0.record(stream)
        R.ldl(c1, d[b:b + 1], ws, check=False)
        a1.record(stream)
        torch.cuda.synchronize()
        alone.append(a0.elapsed_time(a1))
    tf = grf_tensor_flops(n, batch)
    fp64_flops = batch * n ** 3 / 3.0
    bf16 = float(peaks.get("bf16_tflops", 1887.0))
    bf16_s = float(peaks.get("bf16_tflops_sustained", bf16))
    ldl_s = t[1] / 1e3
    del cov, d, ws, s, z, u
    torch.cuda.empty_cache()
    return {"workload": f"62 x 90 raster of 4 km cells (n = {n}), the paper's {batch} Matern "
                        f"parameter sets, {nsim} simulations each",
            "covariance_ms": t[0], "ldl_ms": t[1], "normals_ms": t[2], "simulate_ms": t[3],
            "total_ms": float(t.sum()), "ldl_ms_per_parameter_set_alone": alone,
            "info": info,
            "ldl_tensor_tflops": tf / ldl_s / 1e12,
            "ldl_tensor_frac_of_bf16_burst": tf / ldl_s / 1e12 / bf16,
            "ldl_tensor_frac_of_bf16_sustained": tf / ldl_s / 1e12 / bf16_s,
            "ldl_tensor_flops": tf,
            "ldl_fp64_equivalent_tflops": fp64_flops / ldl_s / 1e12,
            "method": "blocked LDL^T, 128-column panels; panel and trailing products as 8-slice "
                      "bf16 Ozaki splits on tcgen05 (36 digit products per K = 128 block); "
                      "diagonal blocks in double-float"}


def run_gpu(args):
    import torch
    import torch.distributed as dist

    rank, local_rank, world = env_rank()
    torch.cuda.set_device(local_rank)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    from paper_2201_06604_gb300 import mrg, shard
    from paper_2201_06604_gb300 import workloads as W

    dev = torch.device("cuda", local_rank)
    ns, n = W.MATERIALISED["streams"], W.MATERIALISED["draws"]
    if args.quick:
        ns, n = 4096, 4096
    if args.streams:
        ns = args.streams
    if args.draws:
        n = args.draws
    variants_run = VARIANTS
    if args.only:
        variants_run = tuple(tuple(v.split(":")) for v in args.only.split(","))
    total_out = ns * n
    # Replicas: rank r owns streams [r ns, (r+1) ns) of the creator sequence.
    seed = shard.rank_seed(W.PAPER_SEED, rank, ns)
    s = mrg.Streams(ns, dev)
    buf = torch.empty(total_out * 8, dtype=torch.uint8, device=dev)
    outs = {"f64": buf.view(torch.float64).view(ns, n),
            "f32": buf[: total_out * 4].view(torch.float32).view(ns, n),
            "u32": buf[: total_out * 4].view(torch.int32).view(ns, n)}
    tdt = {"f64": torch.float64, "f32": torch.float32, "u32": torch.int32}
    stream = torch.cuda.current_stream()

    def create():
        nxt = (mrg.ctypes.c_uint32 * 6)()
        mrg._check(mrg.lib.mrg_create_streams(mrg._u32_array(seed), ns, s.ptr(), nxt,
                                              stream.cuda_stream))

    def step(events=None):
        create()
        for i, (d, dt) in enumerate(variants_run):
            if events is not None:
                events[i][0].record(stream)
            mrg.generate(s, n, d, tdt[dt], out=outs[dt])
            if events is not None:
                events[i][1].record(stream)

    # Autotune the generate kernel's launch shape for every variant of the
    # workload (untimed; the library then launches each variant with the
    # shape it recorded for this size class).
    tuned = {}
    if not args.no_tune:
        create()
        for d, dt in variants_run:
            best, table = mrg.tune_generate(s, n, d, tdt[dt], out=outs[dt], reps=2)
            default_ms = table[0][1]
            best_ms = min(ms for _, ms in table)
            tuned[f"{d}:{dt}"] = {"shape": best, "ms": best_ms, "default_ms": default_ms,
                                  "candidates": len(table)}

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    K = args.steps
    ev = [[[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in variants_run]
          for _ in range(K)]
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = mrg.launch_count()
    with ClockSampler(local_rank) as clk:
        t_start.record(stream)
        for k in range(K):
            step(ev[k])
        t_end.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    launches = mrg.launch_count() - launches0
    ms = shard.max_over_ranks(t_start.elapsed_time(t_end), dev)
    per_step_ms = ms / K

    # advance kernel cost (mrg_skip runs the same jump kernel the generate
    # call uses to write states back), to isolate generate_kernel
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(20):
        mrg.skip(s, n)
    e1.record(stream)
    torch.cuda.synchronize()
    adv_ms = e0.elapsed_time(e1) / 20

    # HBM write bandwidth measured live: the library's write-only stream
    # kernel (each warp fills its own contiguous chunk, 1 KiB per store --
    # the fastest write pattern measured) over the whole output buffer
    # (8 GiB), best of 5 -- the write ceiling of the materialised variants;
    # the roofline's peak stays the measured copy bandwidth
    write_gbs = None
    if not args.quick:
        fills = []
        for _ in range(6):
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            mrg.fill_u32(buf)
            a1.record(stream)
            torch.cuda.synchronize()
            fills.append(a0.elapsed_time(a1))
        write_gbs = buf.numel() / (min(fills[1:]) / 1e3) / 1e9

    peaks, peak_kind = load_peaks()
    hbm = float(peaks["hbm_gbs"])
    sm_max_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    issue_peak = 4 * sm_count * sm_max_mhz * 1e6 * 32 / 1e12   # thread-instr/s, in T
    variants = []
    for i, (d, dt) in enumerate(variants_run):
        t_call = float(np.mean([ev[k][i][0].elapsed_time(ev[k][i][1]) for k in range(K)]))
        t_kern = max(t_call - adv_ms, 1e-6)
        algo = total_out * ES[dt] + ns * 24  # outputs written + states read
        v = {"dist": d, "dtype": dt, "ms": t_kern, "draws_per_s": total_out / t_kern * 1e3,
             "algo_bytes": algo, "gbs": algo / t_kern / 1e6}
        v["hbm_frac"] = v["gbs"] / hbm
        if write_gbs:
            v["write_frac"] = v["gbs"] / write_gbs
        ipo = INSTR_PER_OUTPUT.get((d, dt))
        if ipo:
            v["issue_tinst_s"] = ipo * total_out / (t_kern * 1e-3) / 1e12
            v["issue_frac"] = v["issue_tinst_s"] / issue_peak
        variants.append(v)
    dom = max(variants, key=lambda v: v["ms"])

    draws_step = total_out * len(variants_run)
    bytes_step = sum(total_out * ES[dt] for _, dt in variants_run)
    value = shard.whole_job_rate(draws_step, world, per_step_ms)

    # e2e through the public API with host buffers: every variant generated
    # into pinned host memory by mrg_generate_host (chunked; the copy of one
    # chunk overlaps the generation of the next).  The only input is the
    # 24-byte creator seed, passed by value to the stream-creation kernel.
    e2e = None
    if not args.skip_e2e:
        host = torch.empty(total_out * 8, dtype=torch.uint8, pin_memory=True)
        hosts = {"f64": host.view(torch.float64).view(ns, n),
                 "f32": host[: total_out * 4].view(torch.float32).view(ns, n),
                 "u32": host[: total_out * 4].view(torch.int32).view(ns, n)}
        scratch = torch.empty(1 << 30, dtype=torch.uint8, device=dev)

        def e2e_step():
            create()
            for d, dt in variants_run:
                mrg.generate_host(s, n, d, tdt[dt], out=hosts[dt], scratch=scratch)
        e2e_step()
        torch.cuda.synchronize()
        KE = max(1, min(K, 3))
        t0 = time.perf_counter()
        for _ in range(KE):
            e2e_step()
        torch.cuda.synchronize()
        e2e_ms = (time.perf_counter() - t0) * 1e3 / KE
        # the box's device -> pinned host copy ceiling: plain 1 GiB copies
        # (cudaMemcpyAsync through torch) into the same pinned buffer
        ch = host[: 1 << 30]
        ch.copy_(scratch, non_blocking=True)
        torch.cuda.synchronize()
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        for _ in range(4):
            ch.copy_(scratch, non_blocking=True)
        c1.record(stream)
        torch.cuda.synchronize()
        ceiling = 4 * (1 << 30) / (c0.elapsed_time(c1) / 1e3) / 1e9
        # where pinned memory can live: the NUMA nodes this process sees and
        # the GPU's own node (sysfs)
        numa_nodes = len([n for n in os.listdir("/sys/devices/system/node")
                          if n.startswith("node") and n[4:].isdigit()]) \
            if os.path.isdir("/sys/devices/system/node") else None
        gpu_node = None
        try:
            bus = torch.cuda.get_device_properties(dev)
            path = (f"/sys/bus/pci/devices/{bus.pci_domain_id:04x}:{bus.pci_bus_id:02x}:"
                    f"{bus.pci_device_id:02x}.0/numa_node")
            with open(path) as f:
                gpu_node = int(f.read().strip())
        except (OSError, ValueError, AttributeError):
            pass
        e2e = {"value": draws_step * world / (e2e_ms / 1e3), "unit": "draws/s",
               "h2d_bytes_per_step": 24, "d2h_bytes_per_step": bytes_step, "ms_per_step": e2e_ms,
               "d2h_gbs": bytes_step / (e2e_ms / 1e3) / 1e9, "d2h_copy_ceiling_gbs": ceiling,
               "frac_of_copy_ceiling": bytes_step / (e2e_ms / 1e3) / 1e9 / ceiling,
               "numa_nodes_visible": numa_nodes, "gpu_numa_node": gpu_node}
        del host, scratch

    # fused no-store consumer: 2^20 streams x 4096 draws -> count and sum
    fused = None
    if not args.skip_fused:
        from paper_2201_06604_gb300 import workloads as Wl
        fs, fd = Wl.FUSED["streams"], Wl.FUSED["draws"]
        if args.quick:
            fs = 1 << 16
        f_st = mrg.create_streams(fs, device=dev, seed=seed)
        cnt = torch.empty(fs, dtype=torch.int64, device=dev)
        sm_ = torch.empty(fs, dtype=torch.float64, device=dev)
        mrg.fused_pi_normsum(f_st, fd, cnt, sm_)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(3):
            mrg.fused_pi_normsum(f_st, fd, cnt, sm_)
        b.record(stream)
        torch.cuda.synchronize()
        f_ms = a.elapsed_time(b) / 3
        pairs = fs * fd // 2
        fused = {"workload": f"{fs} streams x {fd} draws", "ms": f_ms,
                 "draws_per_s": fs * fd / (f_ms / 1e3),
                 "pi_estimate": 4.0 * cnt.sum().item() / pairs}
        del f_st, cnt, sm_

    # Monte Carlo Fisher's exact test on the paper's two tables at the
    # paper's replicate counts (one thread per stream, 2^20 streams)
    fisher = None
    if not args.skip_fisher:
        fisher = {}
        f_st = mrg.create_streams(1 << 20, device=dev, seed=seed)
        for name, fname, B in (("month 12x12", "fisher_month.txt", 1 << 20),
                               ("week 7x12", "fisher_week.txt", 10027008)):
            table = load_table(fname)
            mrg.fisher_sim(f_st, table, B)          # warm-up
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            res = mrg.fisher_sim(f_st, table, B)
            sec = time.perf_counter() - t0
            fisher[name] = {"B": B, "seconds": sec, "tables_per_s": B / sec,
                            "p_value": res["p_value"], "count": res["count"],
                            "threshold": res["threshold"]}
        del f_st

    # the paper's own generator (MRG31k3p) on the same materialised shape
    g31 = None
    if not args.skip_mrg31k3p:
        s31 = mrg.create_streams(ns, device=dev, seed=tuple(W.PAPER_SEED), generator="mrg31k3p")
        g31 = {"workload": f"{ns} streams x {n} draws, MRG31k3p (streams 2^134 apart)"}
        for d, dt in (("uniform", "f64"), ("normal", "f64"), ("uniform", "f32")):
            mrg.generate(s31, n, d, tdt[dt], out=outs[dt])
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(3):
                mrg.generate(s31, n, d, tdt[dt], out=outs[dt])
            b.record(stream)
            torch.cuda.synchronize()
            t = a.elapsed_time(b) / 3
            g31[f"{d}:{dt}"] = {"ms": t, "draws_per_s": total_out / (t / 1e3),
                                "gbs": total_out * ES[dt] / (t / 1e3) / 1e9}
        del s31

    # Gaussian random fields (Sec. 5, Algorithm 2) on the paper's example
    grf_res = None
    if not args.skip_grf:
        grf_res = run_grf(dev, stream, load_peaks()[0])

    # batched uneven requests vs back-to-back plain launches at identical output
    batched = None
    if not args.skip_batched:
        batched = run_batched(mrg, W, dev, stream, seed, quick=args.quick, tune=not args.no_tune)

    serving = None
    if not args.skip_serving:
        serving = run_serving(mrg, W, dev, seed, seconds=2.0 if args.quick else args.serve_seconds)

    cpu = None
    if rank == 0 and world == 1 and not args.skip_cpu:
        import oracle
        oracle.build()
        cores = len(os.sched_getaffinity(0))
        v, sec, tot = cpu_oracle_sample(16384, 16384, cores)
        cpu = {"value": v, "unit": "draws/s", "cores": cores, "kind": "oracle",
               "sample": f"16384 of 65536 streams x 16384 draws x 5 variants ({tot} draws) in "
                         f"{sec:.2f} s, OpenMP over streams"}
        if grf_res is not None:
            from oracle import grf as OG
            pts = OG.square_grid(*W.GRF_GRID, W.GRF_CELL)
            sig = OG.matern_cov(pts, W.GRF_PARAMS[0])
            t0 = time.perf_counter()
            OG.ldl(sig)
            gsec = time.perf_counter() - t0
            cpu["grf_ldl_ms_per_matrix"] = gsec * 1e3
            cpu["grf_sample"] = (f"oracle LDL^T (numpy Cholesky) of one 5580 x 5580 covariance matrix "
                                 f"in {gsec:.2f} s")
        if fisher is not None:
            month = load_table("fisher_month.txt")
            ost, _ = oracle.create_streams(tuple(W.PAPER_SEED), 4096)
            t0 = time.perf_counter()
            oracle.fisher(ost, month, 1 << 16, nthreads=cores)
            fsec = time.perf_counter() - t0
            cpu["fisher_month_tables_per_s"] = (1 << 16) / fsec
            cpu["fisher_sample"] = f"month table, 65536 replicates on 4096 streams in {fsec:.2f} s"

    line = {
        "metric": METRIC, "value": value, "unit": "draws/s", "n_gpus": world, "steps": K,
        "warmup": args.warmup, "ms_per_step": per_step_ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32+fp64/fp32", "dtype_note": DTYPE_NOTE,
        "data": "synthetic (paper default seed 12345x6)",
        "config": {"workload": f"materialised generation: {ns} streams x {n} draws x 5 variants "
                               "(fp64/fp32 uniform, fp64/fp32 normal, fp32 Exp(1)) + stream creation",
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "l2": "outputs (4-8 GiB per variant) larger than L2; no flush"},
        "gbs": bytes_step * world / (per_step_ms / 1e3) / 1e9,
        "hbm_write_gbs_measured": write_gbs,
        "roofline": roofline(dom, hbm, peak_kind, issue_peak, total_out, sm_count),
        "variants": variants,
        "tuned": tuned or None,
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
        "e2e": e2e,
        "fused": fused,
        "mrg31k3p": g31,
        "fisher": fisher,
        "grf": grf_res,
        "batched": batched,
        "serving": serving,
        "cpu_baseline": cpu,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--quick", action="store_true", help="small shapes (development only)")
    ap.add_argument("--no-tune", action="store_true", help="launch with the library defaults")
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-fused", action="store_true")
    ap.add_argument("--skip-batched", action="store_true")
    ap.add_argument("--skip-mrg31k3p", action="store_true")
    ap.add_argument("--skip-grf", action="store_true")
    ap.add_argument("--skip-fisher", action="store_true")
    ap.add_argument("--skip-serving", action="store_true")
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--streams", type=int, default=0, help="override the stream count (profiling)")
    ap.add_argument("--draws", type=int, default=0, help="override draws per stream (profiling)")
    ap.add_argument("--only", default="", help="comma list of dist:dtype variants (profiling)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
