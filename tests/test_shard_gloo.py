"""The multi-rank path on the CPU (no GPU): replicas shard the creator's
stream sequence, rank r starting at the creator state after r n streams
(Sec. 2.1), with no collective on the data path; timing is the maximum over
ranks.

* `creator_advance` (host only) against the oracle's stream matrix raised
  to the n-th power (n 2^127 steps, n 2^134 for MRG31k3p), its composition
  law and its errors;
* two `gloo` ranks in separate processes: their seeds tile the sequence the
  oracle creates in one go, and the timing reduction and whole-job rate are
  the same on every rank.
"""
import multiprocessing
import os
import socket

import numpy as np
import pytest

import oracle as O
from paper_2201_06604_gb300 import mrg, shard
from paper_2201_06604_gb300 import workloads as W

SEED = tuple(W.PAPER_SEED)


def _creator_after(seed, n, gen):
    """The oracle's stream matrix S_c = A_c^(2^log2) raised to the n-th power in
    exact integers, applied to each component of the seed."""
    log2 = O.STREAM_LOG2[gen]
    out = []
    for c in range(2):
        m = gen[c]
        S = [[int(v) for v in row] for row in O.matpow2k(c, log2, gen)]
        P = [[int(i == j) for j in range(3)] for i in range(3)]
        e = n
        while e:
            if e & 1:
                P = [[sum(P[i][k] * S[k][j] for k in range(3)) % m for j in range(3)] for i in range(3)]
            S = [[sum(S[i][k] * S[k][j] for k in range(3)) % m for j in range(3)] for i in range(3)]
            e >>= 1
        x = [int(v) for v in seed[3 * c:3 * c + 3]]
        out += [sum(P[i][k] * x[k] for k in range(3)) % m for i in range(3)]
    return tuple(out)


def test_stream_matrix_reference_matches_the_oracle():
    # against the oracle's own creator (one stream) and, for MRG32k3a, its
    # jump by 2^127 (the jump takes exponents below 2^128)
    for gen in (O.MRG32K3A, O.MRG31K3P):
        for n in (1, 3):
            _, nxt = O.create_streams(SEED, n, gen=gen)
            assert _creator_after(SEED, n, gen) == tuple(int(v) for v in nxt)
    want = O.jump(np.array(SEED, np.uint32), 1 << 127)
    assert _creator_after(SEED, 1, O.MRG32K3A) == tuple(int(v) for v in want)


@pytest.mark.parametrize("n", [0, 1, 2, 1000, 65536, (1 << 40) + 12345, 1 << 63])
def test_creator_advance_matches_oracle(n):
    assert mrg.creator_advance(SEED, n) == _creator_after(SEED, n, O.MRG32K3A)
    assert mrg.creator_advance(SEED, n, "mrg31k3p") == _creator_after(SEED, n, O.MRG31K3P)


def test_creator_advance_composes_and_matches_creation():
    a, b = 7777, 123456789
    assert mrg.creator_advance(mrg.creator_advance(SEED, a), b) == mrg.creator_advance(SEED, a + b)
    _, nxt = O.create_streams(SEED, 1000)
    assert mrg.creator_advance(SEED, 1000) == tuple(int(v) for v in nxt)


def test_creator_advance_errors():
    with pytest.raises(mrg.MrgError):
        mrg.creator_advance((0, 0, 0, 1, 2, 3), 5)
    with pytest.raises(mrg.MrgError):
        mrg.creator_advance((2147483647, 1, 1, 1, 1, 1), 5, "mrg31k3p")
    with pytest.raises(mrg.MrgError) as e:
        mrg.creator_advance(SEED, (1 << 63) + 1)
    assert e.value.code == mrg.ERANGE
    with pytest.raises(ValueError):
        mrg.creator_advance(SEED, 1, "philox")


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, ns, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    from paper_2201_06604_gb300 import shard as sh
    from paper_2201_06604_gb300 import workloads as Wl
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seed = sh.rank_seed(Wl.PAPER_SEED, rank, ns)
        seeds = [None] * world
        dist.all_gather_object(seeds, seed)
        ms = sh.max_over_ranks(1.5 * (rank + 1))          # rank r "took" 1.5 (r + 1) ms
        rate = sh.whole_job_rate(1000.0, world, ms)
        q.put((rank, seeds, ms, rate))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_tile_the_creator_sequence():
    world, ns = 2, 1000
    ctx = multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, ns, q)) for r in range(world)]
    for p in procs:
        p.start()
    try:
        results = sorted(q.get(timeout=240) for _ in range(world))
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert all(p.exitcode == 0 for p in procs)
    seeds = results[0][1]
    assert results[1][1] == seeds                          # every rank sees the same list
    assert tuple(seeds[0]) == SEED
    # the two shards together are the sequence created in one go
    all_starts, _ = O.create_streams(SEED, world * ns)
    for r in range(world):
        starts, _ = O.create_streams(tuple(seeds[r]), ns)
        assert np.array_equal(starts, all_starts[r * ns:(r + 1) * ns])
    for rank, _, ms, rate in results:
        assert ms == 3.0                                   # the slowest rank's time
        assert rate == pytest.approx(1000.0 * world / 3e-3)


def test_single_process_has_no_reduction():
    assert shard.max_over_ranks(2.5) == 2.5
    assert shard.whole_job_rate(10.0, 1, 2.0) == pytest.approx(5000.0)
