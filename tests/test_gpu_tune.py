"""Launch shapes and the autotuner: every shape writes the same bytes.

The generate kernel cuts each stream into lane segments that start with a
jump to their absolute offset (Sec. 2.1 jump-ahead), so the segment length,
block size, store width and grid size may change only the speed.  These tests
check that property on ragged sizes, that the tuner leaves the stream states
alone, and that what it records is what generate() then uses.
"""
import itertools

import numpy as np
import pytest
import torch

import oracle as O
from paper_2201_06604_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SEED = W.PAPER_SEED
VARIANTS = [("raw", torch.int32), ("uniform", torch.float64), ("uniform", torch.float32),
            ("normal", torch.float64), ("normal", torch.float32),
            ("exponential", torch.float32), ("exponential", torch.float64)]


@pytest.fixture(scope="module")
def M():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2201_06604_gb300 import mrg
    return mrg


def padded_out(ns, n, ld, dtype, shift):
    """A [ns, n] view with row pitch ld whose first element sits `shift`
    elements past a 256-byte boundary (lowers the usable store width)."""
    base = torch.full((ns * ld + shift + 64,), -7, dtype=dtype, device="cuda")
    return base[shift: shift + ns * ld].view(ns, ld)[:, :n]


SHAPES = [dict(seg_len=s, block=b, vec_bytes=v, blocks_per_sm=p)
          for s, b, v, p in itertools.product([8, 24, 256, 1000, 1 << 20], [32, 128, 256],
                                              [4, 16, 32], [0, 1])]


@pytest.mark.parametrize("dist,dtype", VARIANTS)
@pytest.mark.parametrize("ns,n,ld,shift", [(37, 1003, 1011, 1), (64, 512, 512, 0), (5, 4099, 4100, 3)])
def test_every_shape_writes_the_same_bytes(M, dist, dtype, ns, n, ld, shift):
    s = M.create_streams(ns, seed=SEED)
    st0 = M.get_state(s)
    ref = padded_out(ns, n, ld, dtype, shift)
    M.generate(s, n, dist, dtype, rate=0.75, out=ref)
    after = M.get_state(s)[0]
    ref_h = np.ascontiguousarray(ref.cpu().numpy())
    for cfg in SHAPES:
        M.set_state(s, st0)
        out = padded_out(ns, n, ld, dtype, shift)
        M.generate_config(s, n, cfg, dist, dtype, rate=0.75, out=out)
        got = np.ascontiguousarray(out.cpu().numpy())
        assert np.array_equal(got.view(np.uint8), ref_h.view(np.uint8)), cfg
        assert np.array_equal(M.get_state(s)[0], after), cfg
    # the untouched padding between rows stays untouched
    full = padded_out(ns, n, ld, dtype, shift)
    M.set_state(s, st0)
    M.generate_config(s, n, SHAPES[-1], dist, dtype, rate=0.75, out=full)
    pad = full.as_strided((ns, ld - n), (ld, 1), full.storage_offset() + n).cpu().numpy()
    if pad.size:
        assert (pad == -7).all()


def test_shape_outputs_match_the_oracle(M):
    ns, n = 33, 777
    s = M.create_streams(ns, seed=SEED)
    st0 = M.get_state(s)[0].T.copy()
    got = M.generate_config(s, n, dict(seg_len=16, block=64, vec_bytes=8), "uniform",
                            torch.float64).cpu().numpy()
    ref, after = O.generate_streams(st0, n, O.UNIFORM)
    assert np.array_equal(got, ref)
    assert np.array_equal(M.get_state(s)[0].T, after)


def test_bad_shapes_are_rejected(M):
    s = M.create_streams(4, seed=SEED)
    for cfg in (dict(block=48), dict(block=512), dict(vec_bytes=12), dict(blocks_per_sm=65)):
        with pytest.raises(M.MrgError) as e:
            M.generate_config(s, 16, cfg)
        assert e.value.code == M.EINVAL


@pytest.mark.parametrize("dist,dtype", [("uniform", torch.float64), ("normal", torch.float32)])
def test_tuner_records_a_shape_and_leaves_states(M, dist, dtype):
    M.tune_clear()
    ns, n = 2048, 4096
    s = M.create_streams(ns, seed=SEED)
    st0 = M.get_state(s)
    assert M.tune_lookup(dist, dtype, ns, n)["seg_len"] == 0
    ref = M.generate(s, n, dist, dtype).clone()
    M.set_state(s, st0)
    out = torch.empty_like(ref)
    best, table = M.tune_generate(s, n, dist, dtype, out=out, reps=2)
    torch.cuda.synchronize()
    assert np.array_equal(M.get_state(s), st0)           # states untouched
    assert torch.equal(out, ref)                         # out holds what generate writes
    assert len(table) >= 2 and all(ms > 0 for _, ms in table)
    assert min(ms for _, ms in table) == pytest.approx(
        [ms for c, ms in table if c == best][0])
    assert M.tune_lookup(dist, dtype, ns, n) == best
    # the same size class uses it; a different class does not
    assert M.tune_lookup(dist, dtype, ns, n + 1) == best
    assert M.tune_lookup(dist, dtype, ns, 4 * n)["seg_len"] == 0
    got = M.generate(s, n, dist, dtype)
    assert torch.equal(got, ref)
    M.tune_clear()


def test_tune_set_and_clear(M):
    M.tune_clear()
    cfg = dict(seg_len=1024, block=128, vec_bytes=16, blocks_per_sm=2)
    M.tune_set("exponential", torch.float32, 1000, 5000, cfg)
    assert M.tune_lookup("exponential", torch.float32, 1000, 5000) == cfg
    assert M.tune_lookup("exponential", torch.float64, 1000, 5000)["seg_len"] == 0
    s = M.create_streams(1000, seed=SEED)
    st0 = M.get_state(s)
    a = M.generate(s, 5000, "exponential", torch.float32, rate=3.0)
    M.tune_set("exponential", torch.float32, 1000, 5000, None)
    assert M.tune_lookup("exponential", torch.float32, 1000, 5000)["seg_len"] == 0
    M.set_state(s, st0)
    b = M.generate(s, 5000, "exponential", torch.float32, rate=3.0)
    assert torch.equal(a, b)
    M.tune_set("uniform", torch.float64, 10, 10, cfg)
    M.tune_clear()
    assert M.tune_lookup("uniform", torch.float64, 10, 10)["seg_len"] == 0
