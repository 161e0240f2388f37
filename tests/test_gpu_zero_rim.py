"""GPU tests of the SGF_PLAN_ZERO_RIM path (single level, density zero on the
two outer rings): it computes the same discrete sum as the general path (the
slopes become central differences, folded into two merged kernel tables), and
the device check reports inputs that break the guarantee."""
import numpy as np
import pytest

import oracle
from paper_1603_03142_gb300 import workloads as W
from tests._gpu import rel_linf_levels, run_gpu, sgf, tol

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    return sgf()


def rim_free(n, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    s = np.zeros((n, n))
    s[2:-2, 2:-2] = rng.uniform(0.1, 2.0, (n - 4, n - 4))
    return s


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("n", [16, 32, 64, 128])
def test_zero_rim_matches_oracle(lib, prec, n):
    nest = W.Nest(n=n)
    s = rim_free(n, n)
    plan = lib.Plan(nest, prec, zero_rim=True)
    gx, gy = run_gpu(plan, [s])
    plan.check()
    ox, oy = oracle.force(nest, [s])
    assert max(rel_linf_levels(nest, gx, gy, ox, oy)) <= tol(prec, n)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_zero_rim_equals_general_path(lib, prec):
    nest, sigma = W.config3(512, seed=3)   # tapered lognormal: zero beyond r = 0.95
    a = run_gpu(lib.Plan(nest, prec), sigma)
    plan = lib.Plan(nest, prec, zero_rim=True)
    b = run_gpu(plan, sigma)
    plan.check()
    errs = rel_linf_levels(nest, b[0], b[1], a[0], a[1])
    assert max(errs) <= tol(prec, 512)


def test_zero_rim_4096_sampled(lib):
    nest, sigma = W.config3()
    plan = lib.Plan(nest, "fp32", zero_rim=True)
    gx, gy = run_gpu(plan, sigma)
    plan.check()
    rng = np.random.Generator(np.random.PCG64(19))
    ii = np.concatenate([rng.integers(0, 4096, 40), [0, 4095, 2048, 100]])
    jj = np.concatenate([rng.integers(0, 4096, 40), [0, 4095, 2047, 3996]])
    ox, oy = oracle.force_at(nest, sigma, np.zeros_like(ii), ii, jj)
    scale = max(np.abs(ox).max(), np.abs(oy).max())
    err = max(np.abs(gx[0][jj, ii] - ox).max(), np.abs(gy[0][jj, ii] - oy).max())
    assert err <= tol("fp32", 4096) * scale
    s = sigma[0]  # net self-force vanishes
    assert abs(np.sum(s * gx[0])) <= 1e-5 * np.sum(np.abs(s * gx[0]))


@pytest.mark.parametrize("n,row_fwd", [(64, 0), (1024, 1), (1024, 2)])
@pytest.mark.parametrize("where", ["row0", "row_last", "col1", "col_last"])
def test_rim_violation_reported(lib, where, n, row_fwd):
    """Every forward row kernel of the zero-rim plan checks the rim: k_row_fwd_m
    (row_fwd 0), k_row_fwd_m2 (1) and the walking k_row_fwd_x (2)."""
    nest = W.Nest(n=n)
    s = rim_free(n, 5)
    plan = lib.Plan(nest, "fp32", zero_rim=True)
    plan.set_schedule(0, 0, 0, 0, 0, row_fwd)
    run_gpu(plan, [s])
    plan.check()  # clean input: no report
    bad = s.copy()
    if where == "row0":
        bad[0, n // 2 - 2] = 1.0
    elif where == "row_last":
        bad[n - 2, 7] = 1.0
    elif where == "col1":
        bad[n // 2 + 1, 1] = 1.0
    else:
        bad[12, n - 1] = 1.0
    run_gpu(plan, [bad])
    with pytest.raises(lib.SgfError) as e:
        plan.check()
    assert e.value.status == lib.SGF_EINVAL
    run_gpu(plan, [s])
    plan.check()  # the record was cleared
