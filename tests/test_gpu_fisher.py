"""Monte Carlo Fisher's exact test (Sec. 4) on the GPU through the C ABI.

Parity with the oracle: the same replicate -> stream -> draws mapping gives
the same tables, so every replicate's statistic is bit-identical (the same
log-factorials summed in the same order), the count is identical and the
streams end in the same states.  Then the paper's two tables at the paper's
replicate counts: the simulated p-values agree with the printed ones within
5 sigma.
"""
import math
import os

import numpy as np
import pytest
import torch

import oracle as O

pytestmark = pytest.mark.gpu

SEED = (12345,) * 6
HERE = os.path.dirname(os.path.abspath(__file__))


def load(name):
    rows = []
    with open(os.path.join(HERE, "golden", name)) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([int(v) for v in line.split()])
    return np.array(rows, np.int32)


@pytest.fixture(scope="module")
def M():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2201_06604_gb300 import mrg
    return mrg


def random_table(rng, I, J, scale):
    t = rng.poisson(scale, size=(I, J)).astype(np.int32)
    return t


TABLES = {
    "small": np.array([[3, 1, 2], [1, 4, 0], [2, 0, 3]], np.int32),
    "2x2": np.array([[3, 9], [7, 1]], np.int32),
    "zero row/col": np.array([[0, 0, 0, 0], [5, 0, 2, 9], [1, 0, 7, 3]], np.int32),
    "2x64": random_table(np.random.default_rng(1), 2, 64, 4.0),
    "64x3": random_table(np.random.default_rng(2), 64, 3, 6.0),
    "9x13 large": random_table(np.random.default_rng(3), 9, 13, 400.0),
}


@pytest.mark.parametrize("name", list(TABLES))
def test_matches_oracle_per_replicate(M, name):
    table = TABLES[name]
    ns, B = 257, 1000                      # ragged: replicates per stream differ
    s = M.create_streams(ns, seed=SEED)
    st0 = M.get_state(s)[0].T.copy()
    res = M.fisher_sim(s, table, B, return_stats=True)
    cnt, thr, after, stats = O.fisher(st0, table, B, nthreads=8, return_stats=True)
    assert res["threshold"] == thr
    got = res["stats"].cpu().numpy()
    assert np.array_equal(got, stats), np.argwhere(got != stats)[:5]
    assert res["count"] == cnt
    assert np.array_equal(M.get_state(s)[0].T, after)


def test_month_table_matches_oracle(M):
    month = load("fisher_month.txt")
    ns, B = 1024, 4099
    s = M.create_streams(ns, seed=SEED)
    st0 = M.get_state(s)[0].T.copy()
    res = M.fisher_sim(s, month, B, return_stats=True)
    cnt, thr, after, stats = O.fisher(st0, month, B, nthreads=os.cpu_count() or 1,
                                      return_stats=True)
    assert abs(res["threshold"] - (-47954.798)) <= 0.0005
    assert np.array_equal(res["stats"].cpu().numpy(), stats)
    assert res["count"] == cnt
    assert np.array_equal(M.get_state(s)[0].T, after)


def test_calls_continue_the_streams(M):
    table = TABLES["small"]
    s = M.create_streams(64, seed=SEED)
    st0 = M.get_state(s)[0].T.copy()
    a = M.fisher_sim(s, table, 640, return_stats=True)["stats"].cpu().numpy()
    b = M.fisher_sim(s, table, 640, return_stats=True)["stats"].cpu().numpy()
    _, _, _, both = O.fisher(st0, table, 1280, nthreads=8, return_stats=True)
    # replicate b of the second call is replicate 640 + b of one long run
    assert np.array_equal(np.concatenate([a, b]), both)


@pytest.mark.parametrize("name,B,p_paper", [("fisher_month.txt", 1048576, 0.403507),
                                            ("fisher_week.txt", 10027008, 0.0001274)])
def test_p_values_match_paper(M, name, B, p_paper):
    table = load(name)
    s = M.create_streams(1 << 20, seed=SEED)
    res = M.fisher_sim(s, table, B)
    sigma = math.sqrt(p_paper * (1 - p_paper) / B)
    assert abs(res["p_value"] - p_paper) <= 5 * sigma, (res, sigma)


def test_errors(M):
    s = M.create_streams(4, seed=SEED)
    with pytest.raises(M.MrgError):
        M.fisher_sim(s, np.ones((1, 5), np.int32), 10)          # one row
    with pytest.raises(M.MrgError):
        M.fisher_sim(s, np.ones((2, 65), np.int32), 10)         # too many columns
    with pytest.raises(M.MrgError):
        M.fisher_sim(s, np.array([[1, -1], [2, 3]], np.int32), 10)
    r = M.fisher_sim(s, TABLES["2x2"], 0)                       # no replicates
    assert r["count"] == 0 and r["p_value"] == 1.0
