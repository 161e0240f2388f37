"""SGF_BF16X: the radix-16 DFTs of the FFT engine as split-BF16 tensor-core
tiles (tcgen05), FP32 everything else.

Bound: relative L-infinity 1e-4 against the FP64 oracle (tests/_gpu.py: tol).
Every N from 16 to 4096 is covered (one radix-16 stage at N = 16..128, two at
256..2048, three at 4096), nests with every pair case, the zero-rim merged path,
fused batches, and a check that the tensor-core path really ran (its rounding
differs from the FP32 path's).
"""
import numpy as np
import pytest

import oracle
from paper_1603_03142_gb300 import workloads as W
from tests._gpu import rel_linf_levels, run_gpu, sgf, tol, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    return sgf()


def _sigma(nest, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    return [rng.uniform(0.2, 1.5, (nest.n, nest.n)) for _ in range(nest.levels)]


NESTS = [
    (16, 1, [(0, 0)]),
    (32, 1, [(0, 0)]),
    (16, 2, [(0, 0), (8, 0)]),
    (16, 4, [(0, 0), (4, 4), (0, 8), (8, 2)]),
    (32, 3, [(0, 0), (5, 9), (4, 12)]),
    (64, 2, [(0, 0), (16, 16)]),
]


@pytest.mark.parametrize("case", NESTS, ids=[f"n{n}L{L}" for n, L, _ in NESTS])
def test_bf16x_nests_full_oracle(lib, case):
    n, L, off = case
    nest = W.Nest(n=n, levels=L, off=off)
    sigma = _sigma(nest, 300 + n + L)
    plan = lib.Plan(nest, "bf16x")
    gx, gy = run_gpu(plan, sigma)
    plan.check()
    ox, oy = oracle.force(nest, sigma)
    errs = rel_linf_levels(nest, gx, gy, ox, oy)
    assert max(errs) <= tol("bf16x", n), errs
    for l in range(L):
        cov = nest.covered_mask(l)
        assert np.all(gx[l][cov] == 0.0) and np.all(gy[l][cov] == 0.0)


@pytest.mark.parametrize("n", [128, 256, 512, 1024, 2048, 4096])
def test_bf16x_against_fp32_every_n(lib, n):
    """At sizes beyond the full oracle: BF16X within 1e-4 of the FP32 path (itself
    within 1e-5 of the oracle), and not equal to it (the tensor cores ran)."""
    nest = W.Nest(n=n, levels=2 if n <= 1024 else 1, off=[(0, 0), (n // 4, n // 4)])
    sigma = _sigma(nest, n)
    f32 = run_gpu(lib.Plan(nest, "fp32"), sigma)
    pb = lib.Plan(nest, "bf16x")
    b16 = run_gpu(pb, sigma)
    pb.check()
    worst, diff = 0.0, 0.0
    for l in range(nest.levels):
        scale = max(np.abs(f32[0][l]).max(), np.abs(f32[1][l]).max())
        d = max(np.abs(b16[0][l] - f32[0][l]).max(), np.abs(b16[1][l] - f32[1][l]).max())
        worst = max(worst, d / scale)
        diff = max(diff, d)
    assert worst <= tol("bf16x", n) - tol("fp32", n), worst
    assert diff > 0.0, "BF16X result identical to FP32: tensor-core path not taken"


def test_bf16x_4096_sampled_oracle(lib):
    """4096^2 lognormal tapered density, BF16X, sampled targets against the oracle."""
    nest, sigma = W.config3()
    for zero_rim in (False, True):
        plan = lib.Plan(nest, "bf16x", zero_rim=zero_rim)
        gx, gy = run_gpu(plan, sigma)
        plan.check()
        rng = np.random.Generator(np.random.PCG64(19))
        ii = np.concatenate([rng.integers(0, 4096, 24), [0, 4095, 2048, 200]])
        jj = np.concatenate([rng.integers(0, 4096, 24), [0, 4095, 2047, 3900]])
        ox, oy = oracle.force_at(nest, sigma, np.zeros_like(ii), ii, jj)
        scale = max(np.abs(ox).max(), np.abs(oy).max())
        err = max(np.abs(gx[0][jj, ii] - ox).max(), np.abs(gy[0][jj, ii] - oy).max()) / scale
        assert err <= tol("bf16x", 4096), (zero_rim, err)


def test_bf16x_batch_equals_single(lib):
    rng = np.random.Generator(np.random.PCG64(5))
    probs = [W.random_nest_problem(rng, n, L) for n, L in [(64, 2), (128, 1), (64, 3), (256, 2), (128, 2)]]
    plans = [lib.Plan(nest, "bf16x") for nest, _ in probs]
    batch = lib.Batch(plans)
    sig = [[torch.from_numpy(a).float().cuda() for a in s] for _, s in probs]
    fx = [[torch.empty_like(a) for a in s] for s in sig]
    fy = [[torch.empty_like(a) for a in s] for s in sig]
    batch.solve(sig, fx, fy)
    torch.cuda.synchronize()
    for k, (nest, s) in enumerate(probs):
        gx, gy = run_gpu(plans[k], s)
        for l in range(nest.levels):
            assert np.array_equal(fx[k][l].double().cpu().numpy(), gx[l])
            assert np.array_equal(fy[k][l].double().cpu().numpy(), gy[l])
