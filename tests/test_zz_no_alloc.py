"""sgf_solve_noalloc: the solve for callers that cannot allocate device memory
at solve time (it allocates nothing; its intermediates live in a fixed array
inside the library).  Its output must match sgf_solve's on the same plan, call
after call, and a plan too large for the fixed array is refused with a clear
error.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

from paper_1603_03142_gb300 import workloads as W
from tests._gpu import rel_linf_levels, run_gpu, sgf, tol, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    return sgf()


def _noalloc(plan, sigma):
    dt = torch.float64 if plan.precision == 0 else torch.float32
    sig = [torch.from_numpy(np.ascontiguousarray(s)).to(device="cuda", dtype=dt) for s in sigma]
    fx = [torch.empty_like(s) for s in sig]
    fy = [torch.empty_like(s) for s in sig]
    plan.solve_noalloc_ptrs([s.data_ptr() for s in sig], [t.data_ptr() for t in fx], [t.data_ptr() for t in fy])
    torch.cuda.synchronize()
    return [t.double().cpu().numpy() for t in fx], [t.double().cpu().numpy() for t in fy]


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("shape", [(64, 3), (512, 1)])
def test_noalloc_matches_solve_twice(lib, prec, shape):
    n, L = shape
    rng = np.random.Generator(np.random.PCG64(n + L))
    nest, _ = W.random_nest_problem(rng, n, L)
    plan = lib.Plan(nest, prec)
    for call in range(2):  # two calls in a row: the fixed array keeps the previous call's contents
        sigma = [rng.uniform(0.1, 1.5, (n, n)) for _ in range(L)]
        ref = run_gpu(plan, sigma)
        got = _noalloc(plan, sigma)
        errs = rel_linf_levels(nest, got[0], got[1], ref[0], ref[1])
        assert max(errs) <= tol(prec, n), (call, errs)


def test_noalloc_zero_rim_plan(lib):
    nest = W.Nest(n=256)
    plan = lib.Plan(nest, "fp32", zero_rim=True)
    rng = np.random.Generator(np.random.PCG64(7))
    for _ in range(2):
        s = np.zeros((256, 256))
        s[2:-2, 2:-2] = rng.uniform(0.1, 2.0, (252, 252))
        ref = run_gpu(plan, [s])
        got = _noalloc(plan, [s])
        plan.check()
        assert max(rel_linf_levels(nest, got[0], got[1], ref[0], ref[1])) <= tol("fp32", 256)


def test_noalloc_refuses_plans_beyond_the_limit(lib):
    plan = lib.Plan(W.Nest(n=1024), "fp32")  # 40 MiB of intermediates > 32 MiB
    s = torch.zeros((1024, 1024), device="cuda", dtype=torch.float32)
    fx, fy = torch.empty_like(s), torch.empty_like(s)
    with pytest.raises(lib.SgfError) as e:
        plan.solve_noalloc_ptrs([s.data_ptr()], [fx.data_ptr()], [fy.data_ptr()])
    assert e.value.status == lib.SGF_EUNSUPPORTED
    assert "SGF_NOALLOC_SCRATCH_BYTES" in str(e.value)


def test_noalloc_bf16x_nest(lib):
    """The split-BF16 tensor-core kernels (and the level-0 inverse row schedule
    that replaces the plan's tensor-map gather) through the fixed scratch."""
    n, L = 256, 2
    rng = np.random.Generator(np.random.PCG64(23))
    nest, _ = W.random_nest_problem(rng, n, L)
    plan = lib.Plan(nest, "bf16x")
    for call in range(2):
        sigma = [rng.uniform(0.1, 1.5, (n, n)) for _ in range(L)]
        ref = run_gpu(plan, sigma)
        got = _noalloc(plan, sigma)
        plan.check()
        errs = rel_linf_levels(nest, got[0], got[1], ref[0], ref[1])
        assert max(errs) <= tol("fp32", n), (call, errs)


def test_noalloc_example3_forest(lib):
    """Several level-0 patches: the Case-3 group and chunk-sum launches that
    read the scratch's partial-accumulator region."""
    f = W.example3_forest(32)
    sigma = W.two_disk_density(f)
    plan = lib.Plan(f, "fp32")
    ref = run_gpu(plan, sigma)
    for _ in range(2):
        got = _noalloc(plan, sigma)
        for p in range(f.patches):
            assert np.array_equal(got[0][p], ref[0][p]) and np.array_equal(got[1][p], ref[1][p]), p


_FRESH = r"""
import sys, numpy as np, torch
sys.path.insert(0, sys.argv[1])
from paper_1603_03142_gb300 import sgf, workloads as W
torch.cuda.set_device(0)
nest = W.Nest(n=256, levels=2, off=[(0, 0), (64, 64)])
plan = sgf.Plan(nest, "fp32")  # the scratch address is looked up here
sig = [torch.rand((256, 256), device="cuda") for _ in range(2)]
fx = [torch.empty_like(s) for s in sig]
fy = [torch.empty_like(s) for s in sig]
torch.cuda.synchronize()
free0 = torch.cuda.mem_get_info()[0]
plan.solve_noalloc_ptrs([s.data_ptr() for s in sig], [t.data_ptr() for t in fx], [t.data_ptr() for t in fy])
torch.cuda.synchronize()
free1 = torch.cuda.mem_get_info()[0]
print("FREE", free0, free1)
"""


def test_noalloc_first_call_reserves_no_device_memory(lib):
    """In a fresh process, the first no-allocation solve on the device leaves the
    device's free memory unchanged: the library's array was reserved when the
    plan was made, so the call itself takes nothing."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", _FRESH, root], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    line = [x for x in r.stdout.splitlines() if x.startswith("FREE")][-1]
    free0, free1 = map(int, line.split()[1:])
    assert free0 == free1, (free0, free1)
