"""Plans over a spectra budget (sgf_plan_create's spectra_budget): the kernel
spectra of the shallowest level pairs stay resident, the others are
regenerated in FP64 at every solve through a window (Sec. 2.2: a pair of
levels m = 2^d apart needs m^2 sets).  The forces are those of the same direct
sum (Sec. 2.1): against the oracle on sampled cells, against the plan with all
spectra resident, call after call; the footprint stays within the budget."""
import numpy as np
import pytest

import oracle
from paper_1603_03142_gb300 import workloads as W
from tests._gpu import run_gpu, sgf, tol, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    return sgf()


def _sampled(nest, sigma, per_level, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    lv, ii, jj = [], [], []
    for l in range(nest.levels):
        free = np.argwhere(~nest.covered_mask(l))
        pick = free[rng.choice(len(free), size=min(per_level, len(free)), replace=False)]
        lv.append(np.full(len(pick), l)), jj.append(pick[:, 0]), ii.append(pick[:, 1])
    lv, ii, jj = np.concatenate(lv), np.concatenate(ii), np.concatenate(jj)
    ox, oy = oracle.force_at(nest, sigma, lv, ii, jj)
    return lv, ii, jj, ox, oy


def _rel_sampled(nest, gx, gy, samp):
    lv, ii, jj, ox, oy = samp
    worst = 0.0
    for l in range(nest.levels):
        m = lv == l
        scale = max(np.abs(ox[m]).max(), np.abs(oy[m]).max())
        err = max(np.abs(gx[l][jj[m], ii[m]] - ox[m]).max(), np.abs(gy[l][jj[m], ii[m]] - oy[m]).max())
        worst = max(worst, err / scale)
    return worst


@pytest.mark.parametrize("prec", ["fp32", "fp64", "bf16x"])
def test_budget_plan_matches_resident_plan_and_oracle(lib, prec):
    rng = np.random.Generator(np.random.PCG64(41))
    nest, sigma = W.random_nest_problem(rng, 128, 4)
    full = lib.Plan(nest, prec)
    total = full.stats()["spectra_bytes"]
    budget = total // 5
    plan = lib.Plan(nest, prec, spectra_budget=budget)
    st = plan.stats()
    assert st["spectra_sets_streamed"] > 0 and st["spectra_waves"] >= 2
    fp = plan.footprint()
    assert fp["spectra_bytes"] <= budget
    assert st["spectra_bytes"] + st["spectra_window_bytes"] == fp["spectra_bytes"]
    ref = run_gpu(full, sigma)
    samp = _sampled(nest, sigma, 64, 7)
    eps = np.finfo(np.float64 if prec == "fp64" else np.float32).eps
    for call in range(2):  # the window is refilled at every solve
        got = run_gpu(plan, sigma)
        plan.check()
        for l in range(nest.levels):  # the same sum in another order of the inputs
            scale = max(np.abs(ref[0][l]).max(), np.abs(ref[1][l]).max())
            d = max(np.abs(got[0][l] - ref[0][l]).max(), np.abs(got[1][l] - ref[1][l]).max())
            assert d <= (tol("bf16x", 128) if prec == "bf16x" else 256 * eps) * scale, (call, l, d / scale)
        assert _rel_sampled(nest, got[0], got[1], samp) <= tol(prec, 128), call


def test_budget_1024_five_levels_against_oracle(lib):
    """A serving shape whose resident spectra would take tens of GB: (1024, 5
    levels) under a 6 GiB budget, sampled cells of every level against the oracle."""
    rng = np.random.Generator(np.random.PCG64(5))
    nest, sigma = W.random_nest_problem(rng, 1024, 5)
    est = lib.estimate(nest, "fp32")
    budget = 6 << 30
    assert est["spectra_bytes"] > 4 * budget
    plan = lib.Plan(nest, "fp32", spectra_budget=budget)
    st = plan.stats()
    assert plan.footprint()["spectra_bytes"] <= budget and st["spectra_sets_streamed"] > 0
    gx, gy = run_gpu(plan, sigma)
    plan.check()
    samp = _sampled(nest, sigma, 12, 9)
    assert _rel_sampled(nest, gx, gy, samp) <= tol("fp32", 1024)


def test_budget_plan_refusals(lib):
    rng = np.random.Generator(np.random.PCG64(3))
    nest, sigma = W.random_nest_problem(rng, 64, 3)
    full = lib.Plan(nest, "fp32")
    total = full.stats()["spectra_bytes"]
    with pytest.raises(lib.SgfError) as e:  # below one set of spectra
        lib.Plan(nest, "fp32", spectra_budget=4096)
    assert e.value.status == lib.SGF_ENOMEM
    roomy = lib.Plan(nest, "fp32", spectra_budget=2 * total)  # fits: nothing streamed
    assert roomy.stats()["spectra_sets_streamed"] == 0
    plan = lib.Plan(nest, "fp32", spectra_budget=total // 3)
    assert plan.stats()["spectra_sets_streamed"] > 0
    with pytest.raises(lib.SgfError) as e:
        lib.Batch([plan])
    assert e.value.status == lib.SGF_EUNSUPPORTED
    s = [torch.from_numpy(a).float().cuda() for a in sigma]
    fx, fy = [torch.empty_like(a) for a in s], [torch.empty_like(a) for a in s]
    with pytest.raises(lib.SgfError) as e:
        plan.solve_noalloc_ptrs([a.data_ptr() for a in s], [a.data_ptr() for a in fx], [a.data_ptr() for a in fy])
    assert e.value.status == lib.SGF_EUNSUPPORTED
    shared = plan.share()  # its own window, the same resident sets
    a = run_gpu(plan, sigma)
    b = run_gpu(shared, sigma)
    for l in range(3):
        assert np.array_equal(a[0][l], b[0][l]) and np.array_equal(a[1][l], b[1][l])


def test_server_streams_shapes_over_the_cap(lib):
    """SGF_SERVER_STREAM: a shape whose spectra exceed max_shape_bytes is served by
    plans over a spectra budget instead of rejected, and its result is that of
    the plan with every spectrum resident."""
    from paper_1603_03142_gb300 import serving
    rng = np.random.Generator(np.random.PCG64(11))
    nest, sigma = W.random_nest_problem(rng, 128, 4)
    est = lib.estimate(nest, "fp32")
    cap = est["build_bytes"] + est["spectra_bytes"] // 4
    srv = lib.Server(hbm_budget=8 << 30, max_inflight=2, max_shape_bytes=cap, stream_large=True, autotune=False)
    sig = [serving.pinned((128, 128), np.float32) for _ in range(4)]
    for l in range(4):
        sig[l][:] = sigma[l]
    fx = [serving.pinned((128, 128), np.float32) for _ in range(4)]
    fy = [serving.pinned((128, 128), np.float32) for _ in range(4)]
    assert srv.submit(1, nest, "fp32", sig, fx, fy) == lib.SGF_OK
    done = []
    import time
    t0 = time.time()
    while not done and time.time() - t0 < 120:
        done = srv.progress()
        time.sleep(0.01)
    assert done and done[0]["status"] == lib.SGF_OK
    ref = run_gpu(lib.Plan(nest, "fp32"), sigma)
    eps = np.finfo(np.float32).eps
    for l in range(4):
        scale = max(np.abs(ref[0][l]).max(), np.abs(ref[1][l]).max())
        assert np.abs(fx[l] - ref[0][l]).max() <= 256 * eps * scale
        assert np.abs(fy[l] - ref[1][l]).max() <= 256 * eps * scale
    srv.close()
    srv2 = lib.Server(hbm_budget=8 << 30, max_inflight=2, max_shape_bytes=cap, autotune=False)
    assert srv2.submit(2, nest, "fp32", sig, fx, fy) == lib.SGF_ENOMEM  # without the flag: rejected
    srv2.close()
