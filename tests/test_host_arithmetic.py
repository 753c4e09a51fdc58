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
* the GRF products' final rounding (ozaki_round.cuh): the exact level sum
  T = th 2^28 + tl times 2^E rounded once to fp64, against exact rational
  rounding, on level sums drawn at every magnitude, exact ties, the int64
  threshold and the flush below the normal range;
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
            os.path.getmtime(os.path.join(csrc, "ozaki_round.cuh")),
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


def _ozaki_cases(rng):
    """(th, tl, E) triples as the product kernels form them, and edge cases."""
    cases = []
    bound = [(l + 1) << 19 for l in range(8)]          # |acc_l| <= (l + 1) 2^19
    for _ in range(60000):
        shrink = int(rng.integers(0, 40))
        acc = [int(rng.integers(-b, b + 1)) >> min(shrink, 19 + l) for l, b in enumerate(bound)]
        if rng.random() < 0.05:                       # leading levels zero: small sums
            z = int(rng.integers(1, 8))
            acc[:z] = [0] * z
        p = [acc[2 * i] * 128 + acc[2 * i + 1] for i in range(4)]
        th, tl = p[0] * 16384 + p[1], p[2] * 16384 + p[3]
        cases.append((th, tl, int(rng.integers(-1080, 60))))
    # exact ties and their neighbours at every rounding position, both signs
    for s in range(1, 16):
        for m in (1 << 52, (1 << 52) + 1, (1 << 53) - 1, (1 << 53) - 2, int(rng.integers(1 << 52, 1 << 53))):
            for d in (-1, 0, 1):
                for sign in (1, -1):
                    T = sign * ((m << s) + (1 << (s - 1)) + d)
                    th, tl = T >> 28, T & ((1 << 28) - 1)
                    j = int(rng.integers(-4096, 4097))     # another split of the same T
                    cases.append((th - j, tl + (j << 28), int(rng.integers(-900, 0))))
                    cases.append((th, tl, -60))
    # around |T| = 2^62, where T stops fitting an int64 (T = 64 Th + Tl, |Th| = 2^56)
    for sign in (1, -1):
        for d in range(-130, 131):
            T = sign * ((1 << 62) + d)
            cases.append((T >> 28, T & ((1 << 28) - 1), -62))
    # the largest sums, zero, and results that fall below the normal range
    big = sum(b << (7 * (7 - l)) for l, b in enumerate(bound))
    for T in (big, -big, 0, 1, -1, 12345):
        for E in (-1200, -1136, -1075, -1074, -1023, -1022, -1021, -66, 0):
            cases.append((T >> 28, T & ((1 << 28) - 1), E))
    return cases


def _round_exact(T, E):
    """T 2^E rounded to nearest-even fp64, +0 below the normal range."""
    import math
    import struct
    if T == 0:
        return 0
    r = float(T)                                      # exact round-half-even of an integer
    m, e = math.frexp(r)                              # r = m 2^e, 0.5 <= |m| < 1
    biased = e - 1 + 1023 + E                         # exponent field of r 2^E
    if biased <= 0:
        return 0
    if biased >= 0x7FF:
        return struct.unpack("<Q", struct.pack("<d", math.copysign(math.inf, r)))[0]
    return struct.unpack("<Q", struct.pack("<d", math.ldexp(r, E)))[0]


def test_ozaki_round_against_exact_rounding(harness):
    rng = np.random.default_rng(2201)
    cases = _ozaki_cases(rng)
    for th, tl, E in cases:
        assert abs(tl) < 1 << 62 and abs(th * (1 << 28) + tl) < 1 << 69
    inp = "\n".join(f"{th} {tl} {E}" for th, tl, E in cases) + "\n"
    r = subprocess.run([harness, "ozround"], input=inp, capture_output=True, text=True, timeout=120,
                       check=True)
    got = [int(x, 16) for x in r.stdout.split()]
    assert len(got) == len(cases)
    bad = [(c, g) for c, g in zip(cases, got) if g != _round_exact(c[0] * (1 << 28) + c[1], c[2])]
    assert not bad, bad[:5]
