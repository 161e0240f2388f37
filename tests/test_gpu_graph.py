"""A solve captured into a CUDA graph: the boundary promises that sgf_solve is
stream-ordered, allocates nothing and can be captured.  The capture comes
before any eager solve of the plan, so every launch it records is that
instance's first in the plan; its replays must equal the eager solve bit for
bit.  Cases: the zero-rim FP32 path at 2048^2 (a column pass that walks its
columns), the split-BF16 tensor-core path (kernels that walk their rows and
columns), and three-level nests in both precisions."""
import numpy as np
import pytest

from paper_1603_03142_gb300 import workloads as W
from tests._gpu import sgf, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    return sgf()


def _zero_rim(n, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    s = np.zeros((n, n), np.float32)
    s[2:-2, 2:-2] = rng.uniform(0.1, 1.0, (n - 4, n - 4))
    return [s]


def _nest_sigma(nest, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    return [rng.uniform(0.1, 1.0, (nest.n, nest.n)).astype(np.float32) for _ in range(nest.levels)]


NEST3 = dict(n=256, levels=3, off=[(0, 0), (64, 64), (64, 64)])
CASES = {
    "zero_rim_fp32_2048": (lambda: W.Nest(n=2048), "fp32", True),
    "zero_rim_bf16x_1024": (lambda: W.Nest(n=1024), "bf16x", True),
    "nest_fp32_256x3": (lambda: W.Nest(**NEST3), "fp32", False),
    "nest_bf16x_256x3": (lambda: W.Nest(**NEST3), "bf16x", False),
}


def _ptrs(ts):
    return [t.data_ptr() for t in ts]


@pytest.mark.parametrize("name", list(CASES))
def test_captured_solve_replays_bitwise(lib, name):
    make, prec, zero_rim = CASES[name]
    nest = make()
    sigma = _zero_rim(nest.n, 5) if zero_rim else _nest_sigma(nest, 5)
    plan = lib.Plan(nest, prec, zero_rim=zero_rim)
    ts = [torch.from_numpy(a).cuda() for a in sigma]
    gx = [torch.empty_like(a) for a in ts]
    gy = [torch.empty_like(a) for a in ts]
    torch.cuda.synchronize()

    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.graph(graph, stream=side):
        plan.solve_ptrs(_ptrs(ts), _ptrs(gx), _ptrs(gy))
    torch.cuda.synchronize()

    ex = [torch.empty_like(a) for a in ts]
    ey = [torch.empty_like(a) for a in ts]
    for _ in range(2):
        for t in gx + gy:
            t.fill_(float("nan"))
        graph.replay()
        torch.cuda.synchronize()
        plan.solve_ptrs(_ptrs(ts), _ptrs(ex), _ptrs(ey))
        torch.cuda.synchronize()
        for l in range(nest.levels):
            assert torch.equal(gx[l], ex[l]) and torch.equal(gy[l], ey[l]), (name, l)
    plan.check()
