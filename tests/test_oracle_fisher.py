"""Pins of the oracle's Monte Carlo Fisher test (Sec. 4) against what the
paper and the mathematics fix:

* the paper's printed observed statistics (thresholds) of its two tables;
* the hypergeometric inversion against exact rational CDFs (smallest x with
  u <= F(x)), including u just below and above a CDF step;
* simulated tables keep the margins, and their distribution matches the
  exact multivariate hypergeometric law (enumeration of every table with the
  margins of a small table, chi-square);
* the simulated p-value of a small table against its exact p-value, and of
  the paper's month table against the printed p-value, within 5 sigma.
"""
import itertools
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))
SEED = (12345,) * 6


def load(name):
    rows = []
    with open(os.path.join(HERE, "golden", name)) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([int(v) for v in line.split()])
    return np.array(rows, np.int32)


def test_observed_statistics_match_paper():
    month, week = load("fisher_month.txt"), load("fisher_week.txt")
    assert month.shape == (12, 12) and week.shape == (7, 12)
    assert abs(O.logfact_sum(month) - (-47954.798)) <= 0.0005
    assert abs(O.logfact_sum(week) - (-54989.556980)) <= 5e-7


def exact_cdf(S, K, R):
    lo, hi = max(0, R - (S - K)), min(R, K)
    tot = math.comb(S, R)
    F, out = Fraction(0), {}
    for x in range(lo, hi + 1):
        F += Fraction(math.comb(K, x) * math.comb(S - K, R - x), tot)
        out[x] = F
    return out


@pytest.mark.parametrize("S,K,R", [(20, 7, 10), (50, 3, 40), (100, 60, 55), (9, 9, 4),
                                   (300, 120, 150), (13, 1, 1), (1000, 37, 500)])
def test_hyper_inv_is_standard_inversion(S, K, R):
    lf = O.logfact_table(S)
    cdf = exact_cdf(S, K, R)
    xs = sorted(cdf)
    steps = [float(cdf[x]) for x in xs]
    # grid points, except those within rounding of a step (e.g. F = 1/2
    # exactly for a symmetric law), where fp64 cannot decide the side
    us = [u for u in np.linspace(1e-9, 1 - 1e-9, 257)
          if min(abs(u - f) for f in steps) > 1e-12]
    for x in xs[:-1]:                      # just below / above every step
        f = float(cdf[x])
        us += [f * (1 - 1e-9), min(f * (1 + 1e-9), 1 - 1e-12)]
    for u in us:
        want = next(x for x in xs if Fraction(u) <= cdf[x])
        assert O.hyper_inv(S, K, R, u, lf) == want, (u, want)


def all_tables(r, c):
    """Every table with row sums r and column sums c (small cases)."""
    I, J = len(r), len(c)

    def rows(i, cols_left):
        if i == I - 1:
            yield [list(cols_left)]
            return
        for first in itertools.product(*[range(min(r[i], cl) + 1) for cl in cols_left[:-1]]):
            last = r[i] - sum(first)
            if 0 <= last <= cols_left[-1]:
                row = list(first) + [last]
                for rest in rows(i + 1, [cl - v for cl, v in zip(cols_left, row)]):
                    yield [row] + rest

    yield from (np.array(t, np.int32) for t in rows(0, list(c)))


def table_prob(t, r, c, n):
    num = math.prod(math.factorial(v) for v in r) * math.prod(math.factorial(v) for v in c)
    den = math.factorial(n) * math.prod(math.factorial(int(v)) for v in t.reshape(-1))
    return Fraction(num, den)


SMALL = np.array([[3, 1, 2], [1, 4, 0], [2, 0, 3]], np.int32)


def test_tables_keep_margins_and_follow_the_exact_law():
    r, c, n = SMALL.sum(1), SMALL.sum(0), int(SMALL.sum())
    tabs = list(all_tables(list(r), list(c)))
    probs = {t.tobytes(): table_prob(t, r, c, n) for t in tabs}
    assert sum(probs.values()) == 1
    B = 60000
    sim, _ = O.fisher_tables(SEED, SMALL, B)
    assert (sim.sum(2) == r).all() and (sim.sum(1) == c).all() and (sim >= 0).all()
    counts = {}
    for t in sim:
        counts[t.tobytes()] = counts.get(t.tobytes(), 0) + 1
    assert set(counts) <= set(probs)
    # chi-square over tables with expected count >= 5 (the rest pooled)
    chi, dof, pooled_e, pooled_o = 0.0, -1, 0.0, 0
    for k, p in probs.items():
        e = float(p) * B
        o = counts.get(k, 0)
        if e >= 5:
            chi += (o - e) ** 2 / e
            dof += 1
        else:
            pooled_e += e
            pooled_o += o
    if pooled_e > 0:
        chi += (pooled_o - pooled_e) ** 2 / pooled_e
        dof += 1
    from scipy.stats import chi2
    assert chi2.sf(chi, dof) > 1e-4, (chi, dof)


def test_simulated_p_value_of_small_table_matches_exact():
    r, c, n = SMALL.sum(1), SMALL.sum(0), int(SMALL.sum())
    lf = O.logfact_table(n)
    thr = O.fisher_threshold(SMALL, lf)
    p_exact = float(sum(table_prob(t, r, c, n) for t in all_tables(list(r), list(c))
                        if O.logfact_sum(t, lf) <= thr))
    st, _ = O.create_streams(SEED, 64)
    B = 100000
    cnt, _, _ = O.fisher(st, SMALL, B, nthreads=8)
    p = (1 + cnt) / (B + 1)
    assert abs(p - p_exact) <= 5 * math.sqrt(p_exact * (1 - p_exact) / B) + 1 / B


def test_month_p_value_matches_paper():
    month = load("fisher_month.txt")
    st, _ = O.create_streams(SEED, 512)
    B = 1 << 14
    cnt, thr, _ = O.fisher(st, month, B, nthreads=os.cpu_count() or 1)
    p = (1 + cnt) / (B + 1)
    p_paper = 0.403507
    assert abs(p - p_paper) <= 5 * math.sqrt(p_paper * (1 - p_paper) / B)
