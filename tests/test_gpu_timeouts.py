"""The bounded device waits and their error path.  Every wait of a kernel on an
mbarrier (the tensor-core MMA commit of SGF_BF16X, the tensor-memory-accelerator
gather of the inverse row pass) gives up after a bound, records a status bit and
lets the kernel end; sgf_plan_check then reports SGF_ETIMEOUT.  Here a test
withholds the producer of those waits for one solve (nothing is issued, so
nothing is in flight) with a short bound: the waits run out, the status says
so, and the next solve of the same plan in the same context is the method's
again (checked against the oracle)."""
import numpy as np
import pytest

import oracle
from paper_1603_03142_gb300 import workloads as W
from tests._gpu import rel_linf_levels, run_gpu, sgf, tol

pytestmark = pytest.mark.gpu

SHORT = 200_000  # SM cycles, about 0.1 ms


@pytest.fixture(scope="module")
def lib():
    return sgf()


def test_tensor_core_commit_withheld(lib):
    rng = np.random.Generator(np.random.PCG64(17))
    nest, sigma = W.random_nest_problem(rng, 64, 2)
    plan = lib.Plan(nest, "bf16x")
    run_gpu(plan, sigma)
    plan.check()  # clean
    plan.inject_timeout(lib.INJECT_TC_COMMIT, SHORT)
    run_gpu(plan, sigma)
    with pytest.raises(lib.SgfError) as e:
        plan.check()
    assert e.value.status == lib.SGF_ETIMEOUT
    plan.check()  # the record was cleared
    gx, gy = run_gpu(plan, sigma)  # the injection applied to one solve only
    plan.check()
    ox, oy = oracle.force(nest, sigma)
    assert max(rel_linf_levels(nest, gx, gy, ox, oy)) <= tol("bf16x", 64)


@pytest.mark.parametrize("n,row_inv0", [(512, 3), (1024, 4), (1024, 5), (2048, 5)])
def test_tma_gather_withheld(lib, n, row_inv0):
    """k_row_inv1t (one row pair per CTA), k_row_inv1x (walking CTAs that
    gather their next row pair behind the transforms) and k_row_inv2x (two row
    pairs per gather; three groups per CTA at 1024, two at 2048)."""
    nest = W.Nest(n=n)
    s = np.zeros((n, n))
    s[2:-2, 2:-2] = np.random.Generator(np.random.PCG64(4)).uniform(0.1, 1.0, (n - 4, n - 4))
    plan = lib.Plan(nest, "fp32", zero_rim=True)
    plan.set_schedule(2, row_inv0)  # the level-0 inverse rows gathered by the tensor memory accelerator
    ref = run_gpu(plan, [s])
    plan.check()
    plan.inject_timeout(lib.INJECT_TMA_GATHER, SHORT)
    run_gpu(plan, [s])
    with pytest.raises(lib.SgfError) as e:
        plan.check()
    assert e.value.status == lib.SGF_ETIMEOUT
    gx, gy = run_gpu(plan, [s])
    plan.check()
    assert np.array_equal(gx[0], ref[0][0]) and np.array_equal(gy[0], ref[1][0])
    rx, ry = oracle.force_row(nest, [s], n // 2)
    scale = max(np.abs(rx).max(), np.abs(ry).max())
    assert max(np.abs(gx[0][n // 2] - rx).max(), np.abs(gy[0][n // 2] - ry).max()) <= tol("fp32", n) * scale


def test_injection_arguments(lib):
    plan = lib.Plan(W.Nest(n=64), "fp32")
    for which, cyc in ((0x4, SHORT), (lib.INJECT_TC_COMMIT, 0), (lib.INJECT_TMA_GATHER, -5)):
        with pytest.raises(lib.SgfError) as e:
            plan.inject_timeout(which, cyc)
        assert e.value.status == lib.SGF_EINVAL
