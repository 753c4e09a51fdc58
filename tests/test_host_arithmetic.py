"""The kernels' integer arithmetic, compiled for the host from the kernels'
own header and checked on the CPU (no GPU needed):

* the fp64 uniform built in integers equals the IEEE product z * norm for
  every z in [1, m1] (exhaustive), and the fp32 uniform equals its rounding;
* the folded modular step reproduces the oracle's plain `%` recurrence.
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
    if not os.path.exists(BIN) or os.path.getmtime(BIN) < max(
            os.path.getmtime(SRC),
            os.path.getmtime(os.path.join(HERE, "..", "paper_2201_06604_gb300", "csrc",
                                          "mrg32k3a_core.cuh"))):
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
