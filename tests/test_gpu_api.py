"""GPU tests of the C ABI's behaviour: edge cases, host-buffer and batched
entry points, shared plans, determinism, error paths."""
import numpy as np
import pytest

import oracle
from paper_1603_03142_gb300 import workloads as W
from tests._gpu import rel_linf_levels, run_gpu, sgf, tol, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    return sgf()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_zero_density_gives_zero_force(lib, prec):
    nest = W.Nest(n=32, levels=2, off=[(0, 0), (8, 8)])
    gx, gy = run_gpu(lib.Plan(nest, prec), [np.zeros((32, 32))] * 2)
    assert all(np.all(a == 0.0) for a in gx + gy)


def test_single_cell_sign(lib):
    nest = W.Nest(n=16)
    s = np.zeros((16, 16))
    s[5, 12] = 1.0
    gx, gy = run_gpu(lib.Plan(nest, "fp64"), [s])
    ox, oy = oracle.force(nest, [s])
    assert gx[0][5, 3] > 0.0
    assert max(rel_linf_levels(nest, gx, gy, ox, oy)) <= tol("fp64", 16)


def test_host_buffers_match_device(lib):
    nest = W.Nest(n=64, levels=3, off=[(0, 0), (10, 20), (16, 0)])
    rng = np.random.Generator(np.random.PCG64(2))
    sigma = [rng.uniform(0, 1, (64, 64)).astype(np.float32) for _ in range(3)]
    plan = lib.Plan(nest, "fp32")
    dx, dy = run_gpu(plan, sigma)
    hx, hy = plan.solve_host(sigma)
    for l in range(3):
        assert np.array_equal(hx[l].astype(np.float64), dx[l])
        assert np.array_equal(hy[l].astype(np.float64), dy[l])


def _pinned(a):
    return torch.from_numpy(np.ascontiguousarray(a)).pin_memory()


@pytest.mark.parametrize("mapped", ["all", "sigma", "forces"])
def test_mapped_host_buffers_are_used_in_place(lib, mapped):
    """Page-locked output buffers are written by the kernels in place, pageable
    ones through the staging; sigma is copied either way.  Same bits as the
    device-buffer solve in every mix."""
    nest = W.Nest(n=64, levels=3, off=[(0, 0), (10, 20), (16, 0)])
    rng = np.random.Generator(np.random.PCG64(12))
    sigma = [rng.uniform(0, 1, (64, 64)).astype(np.float32) for _ in range(3)]
    plan = lib.Plan(nest, "fp32")
    dx, dy = run_gpu(plan, sigma)
    before = plan.stats()["workspace_bytes"]
    ps = [_pinned(a) for a in sigma] if mapped in ("all", "sigma") else [np.ascontiguousarray(a) for a in sigma]
    if mapped in ("all", "forces"):
        hx = [_pinned(np.full((64, 64), np.nan, np.float32)) for _ in range(3)]
        hy = [_pinned(np.full((64, 64), np.nan, np.float32)) for _ in range(3)]
    else:
        hx = [np.full((64, 64), np.nan, np.float32) for _ in range(3)]
        hy = [np.full((64, 64), np.nan, np.float32) for _ in range(3)]

    def ptr(a):
        return a.data_ptr() if isinstance(a, torch.Tensor) else a.ctypes.data

    for _ in range(2):
        plan.solve_host_ptrs([ptr(a) for a in ps], [ptr(a) for a in hx], [ptr(a) for a in hy])
        for l in range(3):
            gx = hx[l].numpy() if isinstance(hx[l], torch.Tensor) else hx[l]
            gy = hy[l].numpy() if isinstance(hy[l], torch.Tensor) else hy[l]
            assert np.array_equal(gx.astype(np.float64), dx[l])
            assert np.array_equal(gy.astype(np.float64), dy[l])
    assert plan.stats()["workspace_bytes"] == before + 3 * 3 * 64 * 64 * 4


def test_mapped_host_buffers_zero_rim_4096(lib):
    """The bench's end-to-end call: 4096^2 zero-rim FP32 with page-locked buffers."""
    nest, sigma = W.config3(4096, seed=3)
    sigma = sigma[0].astype(np.float32)
    plan = lib.Plan(nest, "fp32", zero_rim=True)
    ts = torch.from_numpy(sigma).cuda()
    dx, dy = torch.empty_like(ts), torch.empty_like(ts)
    plan.solve_ptrs([ts.data_ptr()], [dx.data_ptr()], [dy.data_ptr()])
    torch.cuda.synchronize()
    ps, hx, hy = _pinned(sigma), _pinned(np.zeros_like(sigma)), _pinned(np.zeros_like(sigma))
    plan.solve_host_ptrs([ps.data_ptr()], [hx.data_ptr()], [hy.data_ptr()])
    assert torch.equal(hx, dx.cpu()) and torch.equal(hy, dy.cpu())


@pytest.mark.parametrize("pinned", [True, False], ids=["pinned", "pageable"])
def test_host_many_matches_device_solves(lib, pinned):
    """sgf_solve_host_many over five 3-level problems (both staging sets used
    twice or more, a distinct density per problem): every problem's forces are
    the device-buffer solve's, bit for bit, and nothing else is written."""
    nest = W.Nest(n=64, levels=3, off=[(0, 0), (10, 20), (16, 0)])
    rng = np.random.Generator(np.random.PCG64(21))
    probs = [[rng.uniform(0, 1, (64, 64)).astype(np.float32) for _ in range(3)] for _ in range(5)]
    plan = lib.Plan(nest, "fp32")
    ref = [run_gpu(plan, s) for s in probs]
    before = plan.stats()["workspace_bytes"]
    wrap = _pinned if pinned else np.ascontiguousarray
    ps = [[wrap(a) for a in s] for s in probs]
    hx = [[wrap(np.full((64, 64), np.nan, np.float32)) for _ in range(3)] for _ in probs]
    hy = [[wrap(np.full((64, 64), np.nan, np.float32)) for _ in range(3)] for _ in probs]

    def ptr(a):
        return a.data_ptr() if isinstance(a, torch.Tensor) else a.ctypes.data

    def arr(a):
        return a.numpy() if isinstance(a, torch.Tensor) else a

    flat = lambda xs: [ptr(a) for s in xs for a in s]  # noqa: E731
    for _ in range(2):
        plan.solve_host_many_ptrs(len(probs), flat(ps), flat(hx), flat(hy))
        for k in range(len(probs)):
            for l in range(3):
                assert np.array_equal(arr(hx[k][l]).astype(np.float64), ref[k][0][l]), (k, l)
                assert np.array_equal(arr(hy[k][l]).astype(np.float64), ref[k][1][l]), (k, l)
    assert plan.stats()["workspace_bytes"] == before + 6 * 3 * 64 * 64 * 4
    plan.solve_host_many_ptrs(0, [], [], [])  # a no-op
    with pytest.raises(lib.SgfError) as e:
        plan.solve_host_many_ptrs(-1, [], [], [])
    assert e.value.status == lib.SGF_EINVAL
    with pytest.raises(lib.SgfError) as e:  # problem 1's level 2 density missing
        plan.solve_host_many_ptrs(2, flat(ps)[:5] + [0], flat(hx)[:6], flat(hy)[:6])
    assert e.value.status == lib.SGF_EINVAL


def test_host_many_zero_rim_4096(lib):
    """The bench's end-to-end call: three 4096^2 zero-rim FP32 problems, page-locked."""
    plan = lib.Plan(W.Nest(n=4096), "fp32", zero_rim=True)
    sig = [W.config3(4096, seed=3 + k)[1][0].astype(np.float32) for k in range(3)]
    ref = []
    for s in sig:
        ts = torch.from_numpy(s).cuda()
        dx, dy = torch.empty_like(ts), torch.empty_like(ts)
        plan.solve_ptrs([ts.data_ptr()], [dx.data_ptr()], [dy.data_ptr()])
        ref.append((dx.cpu(), dy.cpu()))
    ps = [_pinned(s) for s in sig]
    hx = [_pinned(np.zeros_like(s)) for s in sig]
    hy = [_pinned(np.zeros_like(s)) for s in sig]
    plan.solve_host_many_ptrs(3, [a.data_ptr() for a in ps], [a.data_ptr() for a in hx], [a.data_ptr() for a in hy])
    plan.check()
    for k in range(3):
        assert torch.equal(hx[k], ref[k][0]) and torch.equal(hy[k], ref[k][1])


def test_deterministic_and_shared_plan(lib):
    nest, sigma = W.config2(n=64)
    plan = lib.Plan(nest, "fp32")
    a = run_gpu(plan, sigma)
    b = run_gpu(plan, sigma)
    shared = plan.share()
    c = run_gpu(shared, sigma)
    for l in range(3):
        assert np.array_equal(a[0][l], b[0][l]) and np.array_equal(a[1][l], b[1][l])
        assert np.array_equal(a[0][l], c[0][l]) and np.array_equal(a[1][l], c[1][l])
    st = plan.stats()
    assert st["spectra_bytes"] == shared.stats()["spectra_bytes"] > 0


def test_batched_matches_single(lib):
    rng = np.random.Generator(np.random.PCG64(4))
    probs = [W.random_nest_problem(rng, n, L) for n, L in [(32, 1), (64, 3), (16, 2), (64, 2)]]
    plans = [lib.Plan(nest, "fp32") for nest, _ in probs]
    singles = [run_gpu(p, s) for p, (_, s) in zip(plans, probs)]
    sig = [[torch.from_numpy(a).float().cuda() for a in s] for _, s in probs]
    fx = [[torch.empty_like(a) for a in s] for s in sig]
    fy = [[torch.empty_like(a) for a in s] for s in sig]
    lib.solve_batched(plans, sig, fx, fy)
    torch.cuda.synchronize()
    for k in range(len(probs)):
        for l in range(len(sig[k])):
            assert np.array_equal(fx[k][l].double().cpu().numpy(), singles[k][0][l])
            assert np.array_equal(fy[k][l].double().cpu().numpy(), singles[k][1][l])


def test_null_buffers_rejected(lib):
    plan = lib.Plan(W.Nest(n=16), "fp32")
    with pytest.raises(lib.SgfError) as e:
        plan.solve_ptrs([0], [0], [0])
    assert e.value.status == lib.SGF_EINVAL
