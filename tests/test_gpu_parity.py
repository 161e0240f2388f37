"""GPU parity: the CUDA path (through the C ABI) against the CPU FP64 oracle.

Element-by-element comparisons on seeded inputs, at sizes the oracle finishes
in seconds (several FFT tiles, ragged column counts N+1, every pair case and
refinement ratios up to 8), and on sampled targets at the full benchmark
sizes.  Bound: relative L-infinity per level (tests/_gpu.py: tol).
"""
import numpy as np
import pytest

import oracle
from paper_1603_03142_gb300 import workloads as W
from tests._gpu import rel_linf_levels, run_gpu, sgf, tol

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    return sgf()


def _random_sigma(nest, seed, lo=0.2, hi=1.5):
    rng = np.random.Generator(np.random.PCG64(seed))
    return [rng.uniform(lo, hi, (nest.n, nest.n)) for _ in range(nest.levels)]


NESTS = [
    (16, 1, [(0, 0)]),
    (32, 1, [(0, 0)]),
    (16, 2, [(0, 0), (8, 0)]),           # child on the parent's edges
    (16, 4, [(0, 0), (4, 4), (0, 8), (8, 2)]),  # m = 8 with two-row phase slabs
    (16, 2, [(0, 0), (3, 5)]),
    (16, 3, [(0, 0), (8, 0), (1, 7)]),
    (32, 3, [(0, 0), (5, 9), (4, 12)]),
    (32, 4, [(0, 0), (8, 8), (8, 8), (8, 8)]),   # m = 8
    (64, 2, [(0, 0), (16, 16)]),
]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("case", NESTS, ids=[f"n{n}L{L}" for n, L, _ in NESTS])
def test_nests_full_oracle(lib, prec, case):
    n, L, off = case
    nest = W.Nest(n=n, levels=L, off=off)
    sigma = _random_sigma(nest, 100 + n + L)
    plan = lib.Plan(nest, prec)
    gx, gy = run_gpu(plan, sigma)
    ox, oy = oracle.force(nest, sigma)
    errs = rel_linf_levels(nest, gx, gy, ox, oy)
    assert max(errs) <= tol(prec, n), errs
    for l in range(L):  # covered cells report exactly 0
        cov = nest.covered_mask(l)
        assert np.all(gx[l][cov] == 0.0) and np.all(gy[l][cov] == 0.0)


def test_config1_maclaurin_fp64(lib):
    """64^2 uniform level, Maclaurin disk a = 0.8, FP64: full oracle parity."""
    nest, sigma = W.config1(64)
    plan = lib.Plan(nest, "fp64")
    gx, gy = run_gpu(plan, sigma)
    ox, oy = oracle.force(nest, sigma)
    assert max(rel_linf_levels(nest, gx, gy, ox, oy)) <= tol("fp64", 64)


def _sampled(nest, seed, per_level, rows=()):
    rng = np.random.Generator(np.random.PCG64(seed))
    lv, ii, jj = [], [], []
    for l in range(nest.levels):
        cov = nest.covered_mask(l)
        cand = np.argwhere(~cov)
        pick = cand[rng.choice(len(cand), size=min(per_level, len(cand)), replace=False)]
        for j, i in pick:
            lv.append(l); ii.append(i); jj.append(j)
        for j in rows:
            for i in range(nest.n):
                if not cov[j, i]:
                    lv.append(l); ii.append(i); jj.append(j)
    return np.array(lv), np.array(ii), np.array(jj)


def _sampled_rel(nest, gx, gy, lv, ii, jj, ox, oy):
    worst = 0.0
    for l in range(nest.levels):
        k = lv == l
        if not np.any(k):
            continue
        ax = gx[l][jj[k], ii[k]]
        ay = gy[l][jj[k], ii[k]]
        scale = max(np.abs(ox[k]).max(), np.abs(oy[k]).max())
        worst = max(worst, max(np.abs(ax - ox[k]).max(), np.abs(ay - oy[k]).max()) / scale)
    return worst


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_config2_nest_sampled(lib, prec):
    """3 levels of 256^2 centred at (0.3, 0), Maclaurin + clump + 1% noise."""
    nest, sigma = W.config2()
    plan = lib.Plan(nest, prec)
    gx, gy = run_gpu(plan, sigma)
    lv, ii, jj = _sampled(nest, 5, 300, rows=(128,))
    ox, oy = oracle.force_at(nest, sigma, lv, ii, jj)
    assert _sampled_rel(nest, gx, gy, lv, ii, jj, ox, oy) <= tol(prec, 256)


def test_config3_uniform_4096_sampled(lib):
    """4096^2 lognormal tapered density, FP32, in the benchmark's launch configuration."""
    nest, sigma = W.config3()
    plan = lib.Plan(nest, "fp32")
    gx, gy = run_gpu(plan, sigma)
    rng = np.random.Generator(np.random.PCG64(9))
    ii = np.concatenate([rng.integers(0, 4096, 40), [0, 4095, 2048, 2047, 200, 3900]])
    jj = np.concatenate([rng.integers(0, 4096, 40), [0, 4095, 2048, 2047, 3900, 200]])
    lv = np.zeros_like(ii)
    ox, oy = oracle.force_at(nest, sigma, lv, ii, jj)
    assert _sampled_rel(nest, gx, gy, lv, ii, jj, ox, oy) <= tol("fp32", 4096)


def test_newton_third_law_4096(lib):
    """Net self-force vanishes: sum sigma F = 0 (zero rim, odd x-kernel, commuting slopes)."""
    nest, sigma = W.config3()
    plan = lib.Plan(nest, "fp32")
    gx, gy = run_gpu(plan, sigma)
    s = sigma[0]
    assert abs(np.sum(s * gx[0])) <= 1e-5 * np.sum(np.abs(s * gx[0]))
    assert abs(np.sum(s * gy[0])) <= 1e-5 * np.sum(np.abs(s * gy[0]))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_mirror_symmetry(lib, prec):
    nest = W.Nest(n=64, levels=2, off=[(0, 0), (16, 10)])
    s = _random_sigma(nest, 3)
    s = [0.5 * (a + a[:, ::-1]) for a in s]
    gx, gy = run_gpu(lib.Plan(nest, prec), s)
    for l in range(2):
        assert np.max(np.abs(gx[l] + gx[l][:, ::-1])) <= tol(prec, 64) * np.max(np.abs(gx[l]))
        assert np.max(np.abs(gy[l] - gy[l][:, ::-1])) <= tol(prec, 64) * np.max(np.abs(gy[l]))
