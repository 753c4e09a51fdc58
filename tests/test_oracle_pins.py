"""Pins of the CPU oracle to facts fixed outside the oracle itself.

* values the paper prints for its own generator MRG31k3p (Sec. 2.1, 2.2, 3.2),
  reproduced by the same generic code run with MRG31k3p parameters: they pin the
  jump-ahead, the state order, the output scaling and the exponential rule;
* brute force: a jump of k equals k single steps;
* algebra: composed jumps, the stream / substream relation, the full-period
  property of both MRG32k3a components (which a wrong multiplier breaks);
* exact arithmetic: the fp64 uniform is the correctly rounded product;
* high precision (mpmath) Box-Muller and -log values at extreme integers;
* statistics of long runs (mean, variance, KS).
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle as O

SEED = [12345] * 6
M1, M2 = O.MRG32K3A[0], O.MRG32K3A[1]


# --------------------------------------------------------------------------
# The paper's printed MRG31k3p examples
# --------------------------------------------------------------------------

def test_mrg31k3p_stream_starts_match_paper(golden):
    want = np.array(golden("mrg31k3p_stream_starts.txt"), dtype=np.uint64)
    got, _ = O.create_streams(SEED, 4, gen=O.MRG31K3P)
    assert np.array_equal(got.astype(np.uint64), want)


def test_mrg31k3p_stream_starts_reject_oldest_first(golden):
    # The printed order decides the convention: oldest-first words would be
    # the same numbers reversed within each component.
    want = np.array(golden("mrg31k3p_stream_starts.txt"), dtype=np.uint64)
    got, _ = O.create_streams(SEED, 4, gen=O.MRG31K3P)
    rev = got[:, [2, 1, 0, 5, 4, 3]].astype(np.uint64)
    assert not np.array_equal(rev[1:], want[1:])


def test_mrg31k3p_runif_matches_paper(golden):
    want = [float(v) for v in golden("mrg31k3p_runif.txt")[0]]
    st, _ = O.create_streams(SEED, 4, gen=O.MRG31K3P)
    u = {s: O.uniform64(st[s], 4, gen=O.MRG31K3P)[0] for s in range(4)}
    got = [u[2 * (r % 2)][r // 2] for r in range(8)]
    for g, w in zip(got, want):
        assert abs(g - w) <= 0.0005 + 1e-12, (got, want)


def test_mrg31k3p_rexp_matches_paper_as_minus_log_u(golden):
    rows = golden("mrg31k3p_rexp.txt")
    st, _ = O.create_streams(SEED, 4, gen=O.MRG31K3P)
    ex = {s: O.exponential(st[s], 6, 1.0, gen=O.MRG31K3P)[0] for s in range(4)}
    un = {s: O.uniform64(st[s], 6, gen=O.MRG31K3P)[0] for s in range(4)}
    alt_ok = True
    for r in range(2):
        for c in range(4):
            w = float(rows[r][c])
            dec = len(rows[r][c].split(".")[1])
            s, k = 2 * (r % 2) + (c % 2), 4 + c // 2
            assert abs(ex[s][k] - w) <= 0.5 * 10 ** -dec + 1e-12
            alt_ok &= abs(-np.log1p(-un[s][k]) - w) <= 0.5 * 10 ** -dec
    # The text's -log(1 - u) reading does not reproduce the printed numbers.
    assert not alt_ok


# --------------------------------------------------------------------------
# Jump-ahead: brute force and algebra
# --------------------------------------------------------------------------

@pytest.mark.parametrize("gen", [O.MRG32K3A, O.MRG31K3P])
@pytest.mark.parametrize("k", [0, 1, 2, 3, 4, 7, 64, 1000, 12345, 100000])
def test_jump_equals_k_steps(gen, k):
    st = np.array([11, 22, 33, 44, 55, 66], np.uint32)
    _, after = O.raw(st, k, gen=gen)
    assert np.array_equal(O.jump(st, k, gen=gen), after)


def test_jump_composition_random():
    rng = np.random.default_rng(7)
    st = np.array([1, 2, 3, 4, 5, 6], np.uint32)
    for _ in range(20):
        a = int(rng.integers(0, 2**62)) << int(rng.integers(0, 64))
        b = int(rng.integers(0, 2**62)) << int(rng.integers(0, 64))
        a &= (1 << 127) - 1
        b &= (1 << 127) - 1
        assert np.array_equal(O.jump(O.jump(st, a), b), O.jump(st, a + b))


def test_substream_power_equals_stream_jump():
    # (A^(2^76))^(2^51) = A^(2^127): 2^51 substreams tile one stream exactly.
    for c in (0, 1):
        T = O.matpow2k(c, 76)
        m = O.MRG32K3A[c]
        R = np.eye(3, dtype=object)
        B = T.astype(object)
        e = 1 << 51
        while e:
            if e & 1:
                R = (R.dot(B)) % m
            B = (B.dot(B)) % m
            e >>= 1
        assert np.array_equal(R.astype(np.uint64), O.matpow2k(c, 127))
        assert np.array_equal(O.matpow(c, 1 << 127), O.matpow2k(c, 127))


def test_matpow_matches_python_bigint():
    # Independent arbitrary-precision evaluation of A^e for a few exponents.
    for c in (0, 1):
        m = O.MRG32K3A[c]
        a = O.MRG32K3A[2 + 3 * c: 5 + 3 * c]
        A = [[a[0] % m, a[1] % m, a[2] % m], [1, 0, 0], [0, 1, 0]]

        def mul(X, Y):
            return [[sum(X[r][k] * Y[k][q] for k in range(3)) % m for q in range(3)]
                    for r in range(3)]

        for e in (1, 5, 2**40 + 3, 2**76, 2**127 + 2**76 + 9):
            R, B, x = [[1, 0, 0], [0, 1, 0], [0, 0, 1]], A, e
            while x:
                if x & 1:
                    R = mul(R, B)
                B = mul(B, B)
                x >>= 1
            assert O.matpow(c, e).tolist() == R


def test_streams_are_sequential_jumps():
    n = 37
    st, nxt = O.create_streams(SEED, n)
    x = np.array(SEED, np.uint32)
    for i in range(n):
        assert np.array_equal(st[i], x)
        x = O.jump(x, 1 << 127)
    assert np.array_equal(nxt, x)


def _has_full_period(c, gen):
    """Order of the companion matrix is exactly m^3 - 1 (primitive polynomial)."""
    sympy = pytest.importorskip("sympy")
    m = gen[c]
    N = m**3 - 1
    eye = np.eye(3, dtype=np.uint64)
    if not sympy.isprime(m) or not np.array_equal(O.matpow(c, N, gen=gen), eye):
        return False
    return all(not np.array_equal(O.matpow(c, N // q, gen=gen), eye)
               for q in sympy.factorint(N))


@pytest.mark.parametrize("c", [0, 1])
def test_full_period_of_components(c):
    # Each MRG32k3a component has a primitive characteristic polynomial, so
    # its companion matrix has order exactly m^3 - 1 (period of the pair ~2^191).
    assert _has_full_period(c, O.MRG32K3A)


@pytest.mark.parametrize("idx,delta", [(4, -1), (4, 1), (4, 2), (5, -1), (5, 1),
                                       (7, -1), (7, 1), (7, 2)])
def test_wrong_multiplier_breaks_period(idx, delta):
    # Planted mistakes in a multiplier caught by the full-period test.  For an
    # irreducible characteristic polynomial the period is full exactly when
    # its constant term is a primitive root mod m, so the test is sharp for
    # a13 and a23 and for some a21 changes; most small changes of a12 keep an
    # irreducible polynomial with the same constant term and are NOT caught:
    # a12 rests on the published constant alone.
    bad = list(O.MRG32K3A)
    bad[idx] += delta
    c = 0 if idx < 5 else 1
    assert not _has_full_period(c, tuple(bad))


# --------------------------------------------------------------------------
# Ranges and invariants
# --------------------------------------------------------------------------

def test_state_and_output_ranges_long_run():
    st, _ = O.create_streams(SEED, 8)
    for s in range(8):
        z, after = O.raw(st[s], 200000)
        assert z.min() >= 1 and z.max() <= M1
        assert (after[:3] < M1).all() and (after[3:] < M2).all()
        assert after[:3].any() and after[3:].any()
    states, _ = O.create_streams(SEED, 4096)
    assert (states[:, :3] < M1).all() and (states[:, 3:] < M2).all()
    assert states[:, :3].any(axis=1).all() and states[:, 3:].any(axis=1).all()


def test_first_step_by_hand():
    # x1 = 1403580*12345 - 810728*12345 mod m1, x2 = 527612*12345 - 1370589*12345 mod m2
    x1 = (1403580 * 12345 - 810728 * 12345) % M1
    x2 = (527612 * 12345 - 1370589 * 12345) % M2
    z = (x1 - x2) % M1 or M1
    got, st = O.raw(SEED, 1)
    assert got[0] == z
    assert list(st) == [x1, 12345, 12345, x2, 12345, 12345]


# --------------------------------------------------------------------------
# Transforms
# --------------------------------------------------------------------------

def test_norm_is_rounded_reciprocal():
    assert O.norm() == float(Fraction(1, M1 + 1))


def test_uniform64_is_correctly_rounded_product():
    st = np.array([987654321, 123456789, 55, 4000000000, 77, 1], np.uint32)
    z, _ = O.raw(st, 20000)
    u, _ = O.uniform64(st, 20000)
    nm = Fraction(O.norm())
    for zi, ui in zip(z[:3000], u[:3000]):
        assert ui == float(Fraction(int(zi)) * nm)
    assert (u > 0).all() and (u < 1).all()
    # extremes
    for zi in (1, 2, M1 // 2, M1 - 1, M1):
        assert float(zi) * O.norm() == float(Fraction(zi) * nm)


def test_uniform32_is_rounded_uniform64():
    st = np.array([5, 6, 7, 8, 9, 10], np.uint32)
    u64, _ = O.uniform64(st, 50000)
    u32, _ = O.uniform32(st, 50000)
    assert np.array_equal(u32, u64.astype(np.float32))
    # The top of the range rounds to 1.0f: fp32 uniforms lie in (0, 1].
    assert np.float32(M1 * O.norm()) == np.float32(1.0)


def _mp_box_muller(z1, z2):
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 50
    M = mpmath.mpf(M1 + 1)
    R = mpmath.sqrt(-2 * mpmath.log(mpmath.mpf(z1) / M))
    th = 2 * mpmath.pi * mpmath.mpf(z2) / M
    return R * mpmath.cos(th), R * mpmath.sin(th)


def test_box_muller_against_mpmath_on_stream():
    st = np.array([31, 41, 59, 26, 53, 58], np.uint32)
    z, _ = O.raw(st, 4000)
    x, _ = O.normal(st, 4000)
    assert np.array_equal(x, O.box_muller_of(z))
    for k in range(0, 4000, 2):
        X, Y = _mp_box_muller(int(z[k]), int(z[k + 1]))
        for got, ref in ((x[k], X), (x[k + 1], Y)):
            ref = float(ref)
            assert abs(got - ref) <= 4 * np.spacing(abs(ref)), (k, got, ref)


# Integers at the ends of the log's range and at the quarter-turn / octant
# boundaries of the angle reduction (M = m1 + 1 = 4294967088 = 16 * 268435443).
M = M1 + 1
EXTREME_Z = [1, 2, 3, M1, M1 - 1, M // 8, M // 8 + 1, M // 4 - 1, M // 4, M // 4 + 1,
             3 * M // 8, M // 2 - 1, M // 2, M // 2 + 1, 3 * M // 4 - 1, 3 * M // 4,
             3 * M // 4 + 1, 7 * M // 8, M1 - 2]


def test_box_muller_extreme_integers():
    z = np.array([(a, b) for a in EXTREME_Z for b in EXTREME_Z], np.uint32).reshape(-1)
    got = O.box_muller_of(z)
    for k in range(0, z.size, 2):
        X, Y = _mp_box_muller(int(z[k]), int(z[k + 1]))
        for g, ref in ((got[k], float(X)), (got[k + 1], float(Y))):
            # relative accuracy is kept even where cos or sin vanishes; at
            # z2 = M/4 and 3M/4 the exact value is 0 (mpmath leaves ~1e-51)
            exact_zero = abs(ref) < 1e-40 and g == 0.0
            assert exact_zero or abs(g - ref) <= 4 * np.spacing(abs(ref)), \
                (z[k], z[k + 1], g, ref)


def test_exponential_against_mpmath():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 50
    st = np.array([2, 7, 1, 8, 2, 8], np.uint32)
    z, _ = O.raw(st, 3000)
    assert np.array_equal(O.exponential(st, 3000)[0], O.exp_of(z))
    z = np.concatenate([z, np.array(EXTREME_Z, np.uint32)])
    for rate in (1.0, 2.5):
        e = O.exp_of(z, rate)
        for zi, ei in zip(z, e):
            ref = float(-mpmath.log(mpmath.mpf(int(zi)) / (M1 + 1)) / rate)
            assert abs(ei - ref) <= 3 * np.spacing(ref), (zi, ei, ref)


def test_odd_normal_count_advances_one_more():
    st = np.array([9, 8, 7, 6, 5, 4], np.uint32)
    x5, after5 = O.normal(st, 5)
    x6, after6 = O.normal(st, 6)
    assert np.array_equal(after5, after6)
    assert np.array_equal(x5, x6[:5])


# --------------------------------------------------------------------------
# Statistics of long runs
# --------------------------------------------------------------------------

def test_uniform_statistics():
    stats = pytest.importorskip("scipy.stats")
    st, _ = O.create_streams(SEED, 16)
    u, _ = O.generate_streams(st, 125000, O.UNIFORM)
    u = u.reshape(-1)
    n = u.size
    assert abs(u.mean() - 0.5) < 5 * np.sqrt(1 / 12 / n)
    assert abs(u.var() - 1 / 12) < 5 * np.sqrt(1 / 180 / n)
    assert stats.kstest(u, "uniform").pvalue > 1e-4
    # chi-square on the top 8 bits of the raw outputs
    z, _ = O.generate_streams(O.create_streams(SEED, 16)[0], 125000, O.RAW)
    h = np.bincount((z.reshape(-1) >> 24).astype(np.int64), minlength=256)
    assert stats.chisquare(h).pvalue > 1e-4


def test_normal_statistics():
    stats = pytest.importorskip("scipy.stats")
    st, _ = O.create_streams(SEED, 8)
    x, _ = O.generate_streams(st, 100000, O.NORMAL)
    pairs = x.reshape(-1, 2)
    x = x.reshape(-1)
    assert abs(x.mean()) < 5 / np.sqrt(x.size)
    assert abs(x.var() - 1) < 5 * np.sqrt(2 / x.size)
    assert stats.kstest(x, "norm").pvalue > 1e-4
    assert abs(np.corrcoef(pairs[:, 0], pairs[:, 1])[0, 1]) < 5 / np.sqrt(pairs.shape[0])


def test_exponential_statistics():
    stats = pytest.importorskip("scipy.stats")
    st, _ = O.create_streams(SEED, 8)
    e, _ = O.generate_streams(st, 100000, O.EXPONENTIAL, rate=2.0)
    e = e.reshape(-1)
    assert abs(e.mean() - 0.5) < 5 * 0.5 / np.sqrt(e.size)
    assert stats.kstest(e, "expon", args=(0, 0.5)).pvalue > 1e-4


def test_fused_consistent_and_near_pi_over_4():
    st, _ = O.create_streams(SEED, 64)
    draws = 4096
    cnt, sm, after = O.fused(st, draws)
    z, after2 = O.generate_streams(st, draws, O.RAW)
    x, _ = O.generate_streams(st, draws, O.NORMAL)
    assert np.array_equal(after, after2)
    M = M1 + 1
    za = z[:, 0::2].astype(object)
    zb = z[:, 1::2].astype(object)
    want = np.array([sum(1 for a, b in zip(ra, rb) if a * a + b * b < M * M)
                     for ra, rb in zip(za, zb)])
    assert np.array_equal(cnt, want)
    assert np.allclose(sm, x.sum(axis=1), rtol=0, atol=1e-9)
    p = cnt.sum() / (64 * draws / 2)
    n = 64 * draws / 2
    assert abs(p - np.pi / 4) < 5 * np.sqrt(np.pi / 4 * (1 - np.pi / 4) / n)


def test_generate_streams_matches_single_stream_calls():
    st, _ = O.create_streams(SEED, 5)
    for dist, f32 in ((O.RAW, False), (O.UNIFORM, False), (O.UNIFORM, True),
                      (O.NORMAL, False), (O.EXPONENTIAL, False)):
        many, after = O.generate_streams(st.copy(), 33, dist, f32, rate=1.5, nthreads=2)
        for s in range(5):
            if dist == O.RAW:
                one, a1 = O.raw(st[s], 33)
            elif dist == O.UNIFORM:
                one, a1 = (O.uniform32 if f32 else O.uniform64)(st[s], 33)
            elif dist == O.NORMAL:
                one, a1 = O.normal(st[s], 33)
            else:
                one, a1 = O.exponential(st[s], 33, 1.5)
            assert np.array_equal(many[s], one)
            assert np.array_equal(after[s], a1)
