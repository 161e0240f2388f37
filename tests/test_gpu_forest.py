"""GPU parity of forest plans (several patches per level, Sec. 2.1 Omega^l_k;
Examples 3-4 of Sec. 3) against the CPU FP64 oracle.

Element by element on forests the oracle finishes in seconds: root tiles
(Case 1 with lattice offsets), two patches per refined level, a patch
straddling four roots, three levels with m up to 4; the printed Table 3
errors reproduced by the FP64 GPU path; sampled targets at 8 x 256^2; the
potential; batches mixing forests and nests; the schedules; the no-allocation
solve; and a nest against the forest of its levels (the same plan, bit for bit).
"""
import math

import numpy as np
import pytest

import oracle
from oracle import analytic
from paper_1603_03142_gb300 import workloads as W
from tests._golden import error_table
from tests._gpu import run_gpu, sgf, tol
from tests.test_oracle_paper_tables import assert_printed

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    return sgf()


def _random_sigma(geom, seed, lo=0.2, hi=1.5):
    rng = np.random.Generator(np.random.PCG64(seed))
    return [rng.uniform(lo, hi, (geom.n, geom.n)) for _ in range(geom.levels)]


def straddle_forest(n):
    """2 x 2 root tiles and a level-1 patch over their common corner."""
    return W.Forest(n=n, level=[0] * 4 + [1], org=[(0, 0), (n, 0), (0, n), (n, n), (3 * n // 2, 3 * n // 2)],
                    h0=1.0 / n)


def tiles_and_two_children(n):
    """A 2 x 1 row of roots, a level-1 patch inside each, a level-2 patch straddling nothing."""
    return W.Forest(n=n, level=[0, 0, 1, 1, 2], org=[(0, 0), (n, 0), (n // 2, n // 2), (2 * n, n // 2),
                                                     (3 * n // 2, 3 * n // 2)], h0=1.0 / n)


FORESTS = {
    "example3": lambda: W.example3_forest(16),
    "two_patch": lambda: W.two_patch_forest(32),
    "example4": lambda: W.example4_forest(16),
    "straddle": lambda: straddle_forest(16),
    "three_levels": lambda: tiles_and_two_children(16),
}


def _rel(geom, gx, gy, ox, oy):
    out = []
    for p in range(geom.levels):
        keep = ~geom.covered_mask(p)
        scale = max(np.abs(ox[p][keep]).max(), np.abs(oy[p][keep]).max())
        out.append(max(np.abs(gx[p] - ox[p])[keep].max(), np.abs(gy[p] - oy[p])[keep].max()) / scale)
    return out


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16x"])
@pytest.mark.parametrize("name", list(FORESTS))
def test_forest_full_oracle(lib, prec, name):
    f = FORESTS[name]()
    assert oracle.validate(f)
    sigma = _random_sigma(f, 300 + len(name))
    gx, gy = run_gpu(lib.Plan(f, prec), sigma)
    ox, oy = oracle.force(f, sigma)
    errs = _rel(f, gx, gy, ox, oy)
    assert max(errs) <= tol(prec, f.n), errs
    for p in range(f.levels):
        cov = f.covered_mask(p)
        assert np.all(gx[p][cov] == 0.0) and np.all(gy[p][cov] == 0.0)


def test_table3_from_the_gpu(lib):
    """Example 3 at N = 64 (the paper's level-0 cell count across [-1, 1]), FP64."""
    f = W.example3_forest(32)
    sigma = W.two_disk_density(f)
    gx, gy = run_gpu(lib.Plan(f, "fp64"), sigma)
    alpha = math.sqrt(2.0) / 4.0
    ex, ey = [], []
    for p in range(f.patches):
        X, Y = f.centres(p)
        ax = ay = 0.0
        for cx in (-0.5, 0.5):
            a, b = analytic.force_dn_xy(X, Y, 5, alpha, cx=cx)
            ax, ay = ax + a, ay + b
        keep = ~f.covered_mask(p) & (np.abs(X) < 1.0) & (np.abs(Y) < 1.0)
        ex.append(np.abs(gx[p] - ax)[keep])
        ey.append(np.abs(gy[p] - ay)[keep])
    ex, ey = np.concatenate(ex), np.concatenate(ey)
    got = [ex.mean(), np.sqrt((ex ** 2).mean()), ex.max(), ey.mean(), np.sqrt((ey ** 2).mean()), ey.max()]
    assert_printed(got, error_table("table3_example3.txt")[64])


def test_example3_sampled_256(lib):
    """8 patches of 256^2 (the paper's N = 512), FP32, sampled targets on every patch."""
    f = W.example3_forest(256)
    sigma = W.two_disk_density(f)
    gx, gy = run_gpu(lib.Plan(f, "fp32"), sigma)
    rng = np.random.Generator(np.random.PCG64(21))
    pv, iv, jv = [], [], []
    for p in range(f.patches):
        cand = np.argwhere(~f.covered_mask(p))
        for j, i in cand[rng.choice(len(cand), size=60, replace=False)]:
            pv.append(p), iv.append(i), jv.append(j)
    pv, iv, jv = map(np.array, (pv, iv, jv))
    ox, oy = oracle.force_at(f, sigma, pv, iv, jv)
    scale = max(np.abs(ox).max(), np.abs(oy).max())
    ax = np.array([gx[p][j, i] for p, i, j in zip(pv, iv, jv)])
    ay = np.array([gy[p][j, i] for p, i, j in zip(pv, iv, jv)])
    assert max(np.abs(ax - ox).max(), np.abs(ay - oy).max()) <= tol("fp32", 256) * scale


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_forest_potential(lib, prec):
    import torch
    f = W.example4_forest(16)
    sigma = _random_sigma(f, 17)
    plan = lib.Plan(f, prec, potential=True)
    dt = torch.float64 if prec == "fp64" else torch.float32
    phi = plan.solve_potential([torch.from_numpy(s).to(device="cuda", dtype=dt) for s in sigma])
    torch.cuda.synchronize()
    ref = oracle.potential(f, sigma)
    for p in range(f.patches):
        keep = ~f.covered_mask(p)
        got = phi[p].double().cpu().numpy()
        assert np.abs(got - ref[p])[keep].max() <= tol(prec, 16) * np.abs(ref[p][keep]).max()


def test_nest_and_its_forest_are_the_same_plan(lib):
    nest = W.Nest(n=32, levels=3, off=[(0, 0), (5, 9), (4, 12)])
    sigma = _random_sigma(nest, 5)
    a = run_gpu(lib.Plan(nest, "fp32"), sigma)
    b = run_gpu(lib.Plan(W.Forest.from_nest(nest), "fp32"), sigma)
    for l in range(3):
        assert np.array_equal(a[0][l], b[0][l]) and np.array_equal(a[1][l], b[1][l])


def test_batch_mixes_forests_and_nests(lib):
    import torch
    geoms = [W.example3_forest(16), W.Nest(n=16, levels=2, off=[(0, 0), (4, 4)]), straddle_forest(16)]
    sig = [_random_sigma(g, 40 + k) for k, g in enumerate(geoms)]
    plans = [lib.Plan(g, "fp32") for g in geoms]
    batch = lib.Batch(plans)
    ts = [[torch.from_numpy(a).float().cuda() for a in s] for s in sig]
    fx = [[torch.empty_like(a) for a in s] for s in ts]
    fy = [[torch.empty_like(a) for a in s] for s in ts]
    batch.solve(ts, fx, fy)
    torch.cuda.synchronize()
    eps = np.finfo(np.float32).eps
    for k, g in enumerate(geoms):
        gx, gy = run_gpu(plans[k], sig[k])
        for p in range(g.levels):
            scale = max(np.abs(gx[p]).max(), np.abs(gy[p]).max())
            assert np.abs(fx[k][p].double().cpu().numpy() - gx[p]).max() <= 64 * eps * scale
            assert np.abs(fy[k][p].double().cpu().numpy() - gy[p]).max() <= 64 * eps * scale


def test_forest_schedules_and_launches(lib):
    f = W.example4_forest(16)
    sigma = _random_sigma(f, 9)
    plan = lib.Plan(f, "fp64")
    res = {}
    for inv in (0, 1, 2):
        for c3 in (0, 1):
            plan.set_schedule(0, inv, c3)
            res[(inv, c3)] = run_gpu(plan, sigma)
            st = plan.stats()
            # restrictions of the 3 covered patches; row_fwd, col, row_inv1 for the root (+ row_inv
            # for the other 4); k_col_g; k_col_sum (the root's main output has 1 + 8 + 32 inputs)
            assert st["launches_per_solve"] == 3 + 3 + (0 if inv == 1 else 1) + (1 - c3) + 1
    eps = np.finfo(np.float64).eps
    a = res[(0, 0)]
    for key, b in res.items():
        for p in range(f.patches):
            scale = max(np.abs(a[0][p]).max(), np.abs(a[1][p]).max())
            assert max(np.abs(a[0][p] - b[0][p]).max(), np.abs(a[1][p] - b[1][p]).max()) <= 64 * eps * scale, key


def test_noalloc_solve_on_a_forest(lib):
    import torch
    f = straddle_forest(16)
    sigma = _random_sigma(f, 11)
    plan = lib.Plan(f, "fp32")
    ref = run_gpu(plan, sigma)
    ts = [torch.from_numpy(a).float().cuda() for a in sigma]
    fx = [torch.empty_like(a) for a in ts]
    fy = [torch.empty_like(a) for a in ts]
    for _ in range(2):
        plan.solve_noalloc_ptrs([t.data_ptr() for t in ts], [t.data_ptr() for t in fx], [t.data_ptr() for t in fy])
        torch.cuda.synchronize()
        for p in range(f.patches):
            assert np.array_equal(fx[p].double().cpu().numpy(), ref[0][p])
            assert np.array_equal(fy[p].double().cpu().numpy(), ref[1][p])
