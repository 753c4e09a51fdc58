"""The kernels' integer arithmetic, compiled for the host from the kernels'
own header and checked on the CPU (no GPU needed):

* the fp64 uniform built in integers equals the IEEE product z * norm for
  every z in [1, m1] (exhaustive), and the fp32 uniform equals its rounding;
* the folded modular step reproduces the oracle's plain `%` recurrence;
* the same for MRG31k3p, the paper's own generator: its exact fp64 uniform
  z / 2^31 and fp32 rounding for every z, and its step against the oracle;
* every entry of the transform tables the library builds on the host (1/C_k,
  sin and cos of the bucket angles in each of their eight copies,
  ln(C_k / (M 2^s)) for all shifts), as float pairs, against 50-digit values
  from mpmath;
* the device Matern correlation's Bessel function (matern.cuh, compiled for
  the host) against scipy's exponentially scaled K and the Matern
  correlation against the GRF oracle.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "host_harness", "uniform_exhaustive.cu")
HOST_JUMP = os.path.join(HERE, "..", "paper_2201_06604_gb300", "csrc", "host_jump.cpp")
BIN = os.path.join(HERE, "host_harness", "_build", "harness")


@pytest.fixture(scope="module")
def harness():
    if shutil.which("nvcc") is None:
        pytest.skip("nvcc not available")
    os.makedirs(os.path.dirname(BIN), exist_ok=True)
    csrc = os.path.join(HERE, "..", "paper_2201_06604_gb300", "csrc")
    if not os.path.exists(BIN) or os.path.getmtime(BIN) < max(
            os.path.getmtime(SRC), os.path.getmtime(HOST_JUMP),
            os.path.getmtime(os.path.join(csrc, "host_jump.h")),
            os.path.getmtime(os.path.join(csrc, "matern.cuh")),
            os.path.getmtime(os.path.join(csrc, "mrg32k3a_core.cuh")),
            os.path.getmtime(os.path.join(csrc, "mrg31k3p_core.cuh"))):
        subprocess.run(["nvcc", "-O2", "-std=c++17", "-Xcompiler", "-fopenmp",
                        "-Xcompiler", "-ffp-contract=off", "-o", BIN, SRC, HOST_JUMP], check=True)
    return BIN


def test_uniform_bits_exhaustive(harness):
    r = subprocess.run([harness, "uniform"], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "0 mismatches" in r.stdout


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_step_matches_oracle(harness, seed):
    from paper_2201_06604_gb300.workloads import random_states
    st = random_states(1, seed)[0]
    n = 20000
    r = subprocess.run([harness, "step", str(n), *map(str, st)], capture_output=True, text=True,
                       timeout=120, check=True)
    lines = r.stdout.split("\n")
    got = np.array([int(v) for v in lines[:n]], np.uint64)
    want, after = O.raw(st, n)
    assert np.array_equal(got, want.astype(np.uint64))
    assert [int(v) for v in lines[n].split()] == [int(v) for v in after]


def test_step_extreme_states(harness):
    # Words at the top of each range exercise the reductions' carries.
    m1, m2 = O.MRG32K3A[0], O.MRG32K3A[1]
    for st in ([m1 - 1] * 3 + [m2 - 1] * 3, [0, 0, 1, 0, 0, 1], [m1 - 1, 0, 0, 0, m2 - 1, 0],
               [1, m1 - 1, m1 - 1, m2 - 1, 1, m2 - 1]):
        n = 3000
        r = subprocess.run([harness, "step", str(n), *map(str, st)], capture_output=True,
                           text=True, timeout=120, check=True)
        lines = r.stdout.split("\n")
        want, after = O.raw(np.array(st, np.uint32), n)
        assert [int(v) for v in lines[:n]] == [int(v) for v in want]


def test_uniform31_bits_exhaustive(harness):
    r = subprocess.run([harness, "uniform31"], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "0 mismatches" in r.stdout


def test_step31_matches_oracle(harness):
    m1, m2 = O.MRG31K3P[0], O.MRG31K3P[1]
    rng = np.random.default_rng(7)
    states = [[12345] * 6, [m1 - 1] * 3 + [m2 - 1] * 3, [0, 0, 1, 0, 0, 1],
              [m1 - 1, 0, 0, 0, m2 - 1, 0], [1, m1 - 1, m1 - 1, m2 - 1, 1, m2 - 1],
              list(rng.integers(0, m1, 3)) + list(rng.integers(0, m2, 3))]
    for st in states:
        n = 5000
        r = subprocess.run([harness, "step31", str(n), *map(str, st)], capture_output=True,
                           text=True, timeout=120, check=True)
        lines = r.stdout.split("\n")
        want, after = O.raw(np.array(st, np.uint32), n, gen=O.MRG31K3P)
        assert [int(v) for v in lines[:n]] == [int(v) for v in want], st
        assert [int(v) for v in lines[n].split()] == [int(v) for v in after], st


def test_transform_tables_against_high_precision(harness):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    r = subprocess.run([harness, "tables"], capture_output=True, text=True, timeout=120, check=True)
    tabs = {0: {}, 1: {}}
    for line in r.stdout.split("\n"):
        if line:
            f = line.split()
            tabs[int(f[0])][int(f[1])] = [float.fromhex(v) for v in f[2:]]
    bound = mp.mpf(2) ** -47           # a float pair holds ~48 bits

    def close(hi, lo, want):
        got = mp.mpf(hi) + mp.mpf(lo)
        if want == 0:
            return hi == 0 and lo == 0
        return abs(got - want) <= bound * abs(want)

    for t, M in ((0, O.MRG32K3A[0] + 1), (1, 1 << 32)):
        tab = tabs[t]
        D = M // 4
        C = [M if k == 127 else (1 << 31) + (2 * k + 1) * (1 << 23) for k in range(128)]
        # layout in units of four floats: [0, 64) 1/C_k as 128 pairs;
        # [64, 584) 65 trig entries, 8 identical copies each; [584, 2632)
        # ln(C_k / (M 2^s)) as 4096 pairs
        assert len(tab) == 64 + 65 * 8 + 2048
        for k in range(128):
            e = tab[k // 2][2 * (k % 2):2 * (k % 2) + 2]
            assert close(e[0], e[1], mp.mpf(1) / C[k]), (t, k)
        for j in range(65):
            a = mp.pi / 2 * j * (1 << 23) / D
            e = tab[64 + 8 * j]
            assert close(e[0], e[1], mp.sin(a)), (t, j)
            assert close(e[2], e[3], mp.cos(a)), (t, j)
            assert all(tab[64 + 8 * j + c] == e for c in range(1, 8)), (t, j)
        for s in range(32):
            for k in range(128):
                i = 128 * s + k
                e = tab[584 + i // 2][2 * (i % 2):2 * (i % 2) + 2]
                assert close(e[0], e[1], mp.log(mp.mpf(C[k]) / (mp.mpf(M) * 2 ** s))), (t, s, k)


def test_matern_bessel_k_against_scipy_and_oracle(harness):
    special = pytest.importorskip("scipy.special")
    from oracle import grf
    r = subprocess.run([harness, "matern"], capture_output=True, text=True, timeout=120, check=True)
    rows = np.array([[float(v) for v in line.split()] for line in r.stdout.split("\n") if line])
    nu, x, ks, corr = rows.T
    ref = special.kve(nu, x)
    rel = np.abs(ks - ref) / ref
    assert rel.max() <= 1e-13, (rel.max(), rows[rel.argmax()])
    pos = nu > 0
    want = np.array([grf.matern(np.array([xi * 1.0]), n, np.sqrt(8 * n), 1.0)[0]
                     for n, xi in zip(nu[pos], x[pos])])      # phi = sqrt(8 nu): |d| = x
    assert np.allclose(corr[pos], want, rtol=2e-13, atol=1e-300)
