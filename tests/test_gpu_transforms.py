"""Accuracy of the double-float transforms on the GPU (through mrg_transform)
against the oracle's double evaluation of the exact transforms, on random
integers and on every boundary of the kernels' reductions and tables:
quarter turns and octants of the angle, the log table's bucket edges at every
exponent, powers of two and the ends of [1, m1].

Bars: fp64 normals |err| <= 1e-12; fp64 exponentials |err| <= 1e-12 / min(rate, 1);
fp32 outputs |err| <= 2 ulp of the fp32 spacing at the reference value.
"""
import numpy as np
import pytest
import torch

import oracle as O

pytestmark = pytest.mark.gpu

M1 = O.MRG32K3A[0]
M = M1 + 1
D = M // 4


@pytest.fixture(scope="module")
def mrg():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2201_06604_gb300 import mrg as m
    return m


def boundary_integers():
    z = set()
    for base in (1, 2, 3, D // 2, D, 2 * D, 3 * D, D + D // 2, 2 * D + D // 2, 3 * D + D // 2,
                 M1, M // 2, 1 << 31):
        for d in range(-3, 4):
            z.add(base + d)
    # angle table bucket edges inside each octant: w = j 2^23 (+ 2^22 centres)
    for q in range(4):
        for j in range(65):
            for off in (0, 1 << 22):
                for d in (-1, 0, 1):
                    w = j * (1 << 23) + off + d
                    z.add(q * D + w)
                    z.add(q * D + D - w)
    # log buckets at every exponent: zn = 2^31 + k 2^24 shifted right by s
    for s in range(32):
        for k in range(129):
            zn = (1 << 31) + k * (1 << 24)
            for d in (-1, 0, 1):
                z.add((zn >> s) + d)
        z.add((M - 208) >> s)
    for e in range(32):
        for d in (-2, -1, 0, 1, 2):
            z.add((1 << e) + d)
    z = np.array(sorted(v for v in z if 1 <= v <= M1), dtype=np.uint64)
    return z.astype(np.uint32)


def all_inputs(n_random=1 << 21, seed=5):
    rng = np.random.default_rng(seed)
    r = rng.integers(1, M1 + 1, size=n_random, dtype=np.uint64).astype(np.uint32)
    b = boundary_integers()
    # pair every boundary value with every role (first and second of a pair)
    rb = rng.integers(1, M1 + 1, size=b.size, dtype=np.uint64).astype(np.uint32)
    pairs = np.concatenate([np.stack([b, rb], 1).reshape(-1), np.stack([rb, b], 1).reshape(-1)])
    return np.concatenate([r, pairs])


def f32_ulp(ref):
    return np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64)


def run(mrg, z, dist, dtype, rate=1.0):
    zt = torch.from_numpy(z.view(np.int32)).cuda()
    return mrg.transform(zt, dist, dtype, rate=rate).cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_normal_transform_accuracy(mrg, dtype):
    z = all_inputs()
    got = run(mrg, z, "normal", dtype)
    ref = O.box_muller_of(z)
    err = np.abs(got - ref)
    # exact zeros (Theta on a multiple of pi/2) stay exact, with the sign the
    # oracle's quadrant negation gives them (R times a negated zero)
    nz = ref != 0
    assert (~nz).sum() > 0
    assert (got[~nz] == 0).all()
    assert (np.signbit(got[~nz]) == np.signbit(ref[~nz])).all()
    if dtype == torch.float64:
        print(f"fp64 normal: max abs err {err.max():.3e} over {z.size} values")
        assert err.max() <= 1e-12
        rel = (err[nz] / np.abs(ref[nz])).max()
        print(f"fp64 normal: max rel err {rel:.3e}")
        assert rel <= 1e-11
    else:
        ratio = (err / f32_ulp(ref)).max()
        print(f"fp32 normal: max err {ratio:.3f} ulp over {z.size} values")
        assert ratio <= 2.0


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("rate", [1.0, 0.37, 2.0 ** -64, 2.0 ** 64, 1e6])
def test_exponential_transform_accuracy(mrg, dtype, rate):
    z = all_inputs(n_random=1 << 19)
    got = run(mrg, z, "exponential", dtype, rate=rate)
    ref = O.exp_of(z, rate)
    err = np.abs(got - ref)
    if dtype == torch.float64:
        tol = 1e-12 / min(rate, 1.0)
        print(f"fp64 exponential rate={rate}: max abs err {err.max():.3e} (tol {tol:.1e})")
        assert err.max() <= tol
        # relative accuracy as well: an absolute bound cannot see wrong bits in
        # values of 1e-20 and below (rate 2^64 with u near 1)
        rel = (err / np.abs(ref)).max()
        print(f"fp64 exponential rate={rate}: max rel err {rel:.3e}")
        assert rel <= 4e-12
    else:
        ratio = (err / f32_ulp(ref)).max()
        print(f"fp32 exponential rate={rate}: max err {ratio:.3f} ulp")
        assert ratio <= 2.0


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_uniform_transform_bit_exact(mrg, dtype):
    z = all_inputs(n_random=1 << 18)
    got = run(mrg, z, "uniform", dtype)
    u = z.astype(np.float64) * O.norm()
    ref = u if dtype == torch.float64 else u.astype(np.float32).astype(np.float64)
    assert np.array_equal(got, ref)


def test_odd_normal_count_and_zero_crossings(mrg):
    # z2 = D and 3D put Theta exactly on pi/2 and 3 pi/2: X is exactly zero.
    z = np.array([12345, D, 777, 3 * D, 5], dtype=np.uint32)
    got = run(mrg, z, "normal", torch.float64)
    ref = O.box_muller_of(np.array([12345, D, 777, 3 * D, 5, 1], dtype=np.uint32))[:5]
    assert got[0] == 0.0 and got[2] == 0.0
    assert np.abs(got - ref).max() <= 1e-12


PACKED = [("normal", torch.float64), ("normal", torch.float32), ("exponential", torch.float32),
          ("exponential", torch.float64)]


@pytest.mark.parametrize("dist,dt", PACKED)
def test_packed_and_scalar_evaluations_identical(mrg, dist, dt):
    # An output aligned to four elements (32 bytes for fp64, 16 for fp32)
    # takes the packed two-at-a-time evaluation, a misaligned one the scalar
    # evaluation: bit-identical outputs on random draws and on every
    # reduction boundary (the accuracy tests above check the aligned path
    # against the oracle).
    z = all_inputs(n_random=1 << 20)
    zt = torch.from_numpy(z.view(np.int32)).cuda()
    n = z.size
    al = 8 * dt.itemsize if dt == torch.float64 else 4 * dt.itemsize
    aligned = mrg.transform(zt, dist, dt, rate=2.5)
    assert aligned.data_ptr() % al == 0
    big = torch.full((n + 5,), -7.0, dtype=dt, device="cuda")
    shifted = big[1:n + 1]
    assert shifted.data_ptr() % al != 0
    mrg.transform(zt, dist, dt, rate=2.5, out=shifted)
    iv = np.uint64 if dt == torch.float64 else np.uint32
    a = aligned.cpu().numpy().view(iv)
    b = shifted.cpu().numpy().view(iv)
    assert np.array_equal(a, b), np.argwhere(a != b)[:5]
    assert big[0].item() == -7.0 and (big[n + 1:] == -7.0).all()


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 7, 9, 1001, 4099])
def test_normal_f64_packed_tails(mrg, n):
    # counts that end inside a unit of four draws: the last pair (or the
    # lone last draw, whose pair partner is taken as 1) goes the scalar way
    z = all_inputs(n_random=4096, seed=n)[:n]
    zt = torch.from_numpy(z.view(np.int32)).cuda()
    big = torch.full((n + 8,), -7.0, dtype=torch.float64, device="cuda")
    got = mrg.transform(zt, "normal", torch.float64, out=big[:n])
    zz = np.concatenate([z, np.ones(n % 2, dtype=np.uint32)])
    ref = O.box_muller_of(zz)[:n]
    assert np.abs(got.cpu().numpy() - ref).max() <= 1e-12
    assert (big[n:] == -7.0).all()


@pytest.mark.parametrize("dist", ["normal", "exponential"])
@pytest.mark.parametrize("n", [1, 2, 3, 5, 7, 1001, 4099])
def test_f32_packed_tails(mrg, dist, n):
    # the same for fp32 outputs: a 16-byte aligned output whose count ends
    # inside a unit of four draws equals the misaligned (scalar) evaluation
    z = all_inputs(n_random=4096, seed=n)[:n]
    zt = torch.from_numpy(z.view(np.int32)).cuda()
    big = torch.full((n + 8,), -7.0, dtype=torch.float32, device="cuda")
    got = mrg.transform(zt, dist, torch.float32, rate=0.3, out=big[:n])
    assert big.data_ptr() % 16 == 0
    ref = mrg.transform(zt, dist, torch.float32, rate=0.3,
                        out=torch.empty(n + 1, dtype=torch.float32, device="cuda")[1:])
    a = got.cpu().numpy().view(np.uint32)
    b = ref.cpu().numpy().view(np.uint32)
    assert np.array_equal(a, b), np.argwhere(a != b)[:5]
    assert (big[n:] == -7.0).all()
