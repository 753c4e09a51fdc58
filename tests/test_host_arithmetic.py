"""The kernels' integer arithmetic, compiled for the host from the kernels'
own header and checked on the CPU (no GPU needed):

* the fp64 uniform built in integers equals the IEEE product z * norm for
  every z in [1, m1] (exhaustive), and the fp32 uniform equals its rounding;
* the folded modular step reproduces the oracle's plain `%` recurrence;
* the same for MRG31k3p, the paper's own generator: its exact fp64 uniform
  z / 2^31 and fp32 rounding for every z, and its step against the oracle.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "host_harness", "uniform_exhaustive.cu")
BIN = os.path.join(HERE, "host_harness", "_build", "harness")


@pytest.fixture(scope="module")
def harness():
    if shutil.which("nvcc") is None:
        pytest.skip("nvcc not available")
    os.makedirs(os.path.dirname(BIN), exist_ok=True)
    csrc = os.path.join(HERE, "..", "paper_2201_06604_gb300", "csrc")
    if not os.path.exists(BIN) or os.path.getmtime(BIN) < max(
            os.path.getmtime(SRC),
            os.path.getmtime(os.path.join(csrc, "mrg32k3a_core.cuh")),
            os.path.getmtime(os.path.join(csrc, "mrg31k3p_core.cuh"))):
        subprocess.run(["nvcc", "-O2", "-std=c++17", "-Xcompiler", "-fopenmp",
                        "-Xcompiler", "-ffp-contract=off", "-o", BIN, SRC], check=True)
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
