"""Tile schedules and the autotuner (sgf_plan_schedule_*, sgf_plan_autotune).

Every schedule evaluates the same expressions in the same order, so the forces
agree across schedules to rounding: the compiler may contract a multiply and an
add into one FMA in one kernel and not in another, which moves the last bits
(bound here: 64 units of roundoff of the field's largest value, far below the
method's parity bounds); the autotuner must pick one of the
candidates, report a time for each, and record its choice for later plans of
the same key (in the process and in the SGF_AUTOTUNE_CACHE table file).
"""
import os
import subprocess
import sys
from pathlib import Path

import numpy as np
import pytest

from paper_1603_03142_gb300 import workloads as W
from tests._gpu import run_gpu, sgf

pytestmark = pytest.mark.gpu
ROOT = Path(__file__).resolve().parent.parent


@pytest.fixture(scope="module")
def lib():
    return sgf()


def _zero_rim_sigma(n, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    s = np.zeros((n, n))
    s[2:-2, 2:-2] = rng.uniform(0.1, 1.0, (n - 4, n - 4))
    return [s]


@pytest.mark.parametrize("prec", ["fp32", "bf16x", "fp64"])
@pytest.mark.parametrize("n", [64, 512, 2048])
def test_schedules_agree_zero_rim(lib, prec, n):
    nest = W.Nest(n=n)
    sigma = _zero_rim_sigma(n, n)
    plan = lib.Plan(nest, prec, zero_rim=True)
    outs = []
    tma = prec == "fp32" and n >= 512  # row_inv0 = 3: the level-0 gather by the tensor memory accelerator
    if not tma:
        with pytest.raises(lib.SgfError) as ei:
            plan.set_schedule(0, 3)
        assert ei.value.status == lib.SGF_EUNSUPPORTED
    mx = prec == "fp32" and n >= 1024  # col_pass = 3: k_col_mx (both halves per thread, register twiddles)
    if not mx:
        with pytest.raises(lib.SgfError) as ei:
            plan.set_schedule(3, 0)
        assert ei.value.status == lib.SGF_EUNSUPPORTED
    # (choice, radix plan): col_pass 3 and row_inv0 4, 5 in both radix plans (register-twiddle kernels)
    invs = [(0, 0), (1, 0), (2, 0)] + ([(3, 0)] if tma else []) + (
        [(4, 0), (4, 1), (5, 0), (5, 1)] if tma and n >= 1024 else [])
    cols = [(0, 0), (1, 0), (2, 0)] + ([(3, 0), (3, 1)] if mx else [])
    fwds = (0, 1, 2) if mx else (0,)  # row_fwd = 1, 2: two row pairs per CTA in the forward rows (2 walking)
    for col, cr in cols:
        for inv, ir in invs:
            for fw in fwds:
                plan.set_schedule(col, inv, 0, cr, ir, fw)
                assert plan.schedule() == {"col_pass": col, "row_inv0": inv, "col_case3": 0, "col_radix": cr,
                                           "inv_radix": ir, "row_fwd": fw}
                outs.append(run_gpu(plan, sigma))
                plan.check()
    with pytest.raises(lib.SgfError) as ei:  # a radix plan without its register-twiddle kernel
        plan.set_schedule(2, 0, 0, 1, 0)
    assert ei.value.status == lib.SGF_EUNSUPPORTED
    eps = np.finfo(np.float64 if prec == "fp64" else np.float32).eps
    scale = max(np.abs(outs[0][0][0]).max(), np.abs(outs[0][1][0]).max())
    for gx, gy in outs[1:]:
        d = max(np.abs(gx[0] - outs[0][0][0]).max(), np.abs(gy[0] - outs[0][1][0]).max())
        assert d <= 64 * eps * scale, d / scale


@pytest.mark.parametrize("prec", ["fp32", "fp64", "bf16x"])
def test_nest_schedules_agree(lib, prec):
    """row_inv0 and col_case3 (grouped Case-3 outputs) on a 3-level nest."""
    rng = np.random.Generator(np.random.PCG64(8))
    nest, sigma = W.random_nest_problem(rng, 128, 3)
    plan = lib.Plan(nest, prec)
    res = {}
    for inv in (0, 1, 2):
        for c3 in (0, 1):
            plan.set_schedule(0, inv, c3)
            res[(inv, c3)] = run_gpu(plan, sigma)
            # restrictions 2, row_fwd, col (+ k_col_g), k_col_sum (level 0 has 21 inputs, more than
            # one chunk), row_inv1 + row_inv or one row_inv
            assert plan.stats()["launches_per_solve"] == 2 + 3 + (0 if inv == 1 else 1) + (1 - c3) + 1
    eps = np.finfo(np.float64 if prec == "fp64" else np.float32).eps
    a = res[(0, 0)]
    for key, b in res.items():
        for l in range(3):
            scale = max(np.abs(a[0][l]).max(), np.abs(a[1][l]).max())
            d = max(np.abs(a[0][l] - b[0][l]).max(), np.abs(a[1][l] - b[1][l]).max())
            assert d <= 64 * eps * scale, (key, l, d / scale)


@pytest.mark.parametrize("levels", [1, 3])
def test_general_forward_two_pairs(lib, levels):
    """row_fwd = 1 on plans without the zero rim (k_row_fwd2: two row pairs and
    the three fields per CTA) and, on the uniform grid, 2 (k_row_fwd3x: the
    register-twiddle engine, walking row pairs) against row_fwd = 0 (k_row_fwd:
    one CTA per row pair and field), on a uniform 1024^2 grid and on a 3-level
    1024^2 nest whose Case-2 phase slabs (m = 2, 4) give items of several slabs;
    same expressions, so the forces agree to rounding.  Refused for BF16X, FP64,
    n < 1024 and (row_fwd 2) several patches."""
    rng = np.random.Generator(np.random.PCG64(40 + levels))
    if levels == 1:
        nest = W.Nest(n=1024)
        sigma = [rng.uniform(0.1, 1.0, (1024, 1024))]
    else:
        nest, sigma = W.random_nest_problem(rng, 1024, levels)
    plan = lib.Plan(nest, "fp32")
    res = []
    fws = (0, 1, 2) if levels == 1 else (0, 1)  # 2: k_row_fwd3x, plans of one patch
    for fw in fws:
        plan.set_schedule(2, 0, 0, 0, 0, fw)
        res.append(run_gpu(plan, sigma))
        plan.check()
    eps = np.finfo(np.float32).eps
    for other in res[1:]:
        for l in range(nest.levels):
            scale = max(np.abs(res[0][0][l]).max(), np.abs(res[0][1][l]).max())
            d = max(np.abs(res[0][0][l] - other[0][l]).max(), np.abs(res[0][1][l] - other[1][l]).max())
            assert d <= 64 * eps * scale, (l, d / scale)
    for p in (lib.Plan(nest, "bf16x"), lib.Plan(W.Nest(n=1024), "fp64"), lib.Plan(W.Nest(n=512), "fp32")):
        with pytest.raises(lib.SgfError) as ei:
            p.set_schedule(0, 0, 0, 0, 0, 1)
        assert ei.value.status == lib.SGF_EUNSUPPORTED
    if levels > 1:  # row_fwd = 2: zero-rim plans and plans of one patch only
        with pytest.raises(lib.SgfError) as ei:
            plan.set_schedule(2, 0, 0, 0, 0, 2)
        assert ei.value.status == lib.SGF_EUNSUPPORTED
    else:  # a shared plan takes the schedule (checked against its own lists), or falls back per pass
        plan.set_schedule(2, 0, 0, 0, 0, 2)
        q = plan.share()
        assert q.schedule()["row_fwd"] == 2
        gq = run_gpu(q, sigma)
        assert np.array_equal(gq[0][0], res[2][0][0]) and np.array_equal(gq[1][0], res[2][1][0])
        assert plan.share("bf16x").schedule()["row_fwd"] == 0


def test_bf16x_4096_refuses_nest_inverse_schedule(lib):
    plan = lib.Plan(W.Nest(n=4096), "bf16x", zero_rim=True)
    for sched in ((0, 1), (2, 0)):
        with pytest.raises(lib.SgfError) as ei:
            plan.set_schedule(*sched)
        assert ei.value.status == lib.SGF_EUNSUPPORTED
    r = plan.autotune(reps=1)
    assert r["ms"]["row_inv0_1"] < 0 and r["chosen"]["row_inv0"] != 1
    assert r["ms"]["col_pass2"] < 0 and r["chosen"]["col_pass"] != 2


def test_batch_follows_schedule(lib):
    rng = np.random.Generator(np.random.PCG64(9))
    probs = [W.random_nest_problem(rng, 64, L) for L in (1, 2, 3)]
    plans = [lib.Plan(nest, "fp32") for nest, _ in probs]
    for p in plans:
        p.set_schedule(0, 1)
    import torch
    batch = lib.Batch(plans)
    sig = [[torch.from_numpy(a).float().cuda() for a in s] for _, s in probs]
    fx = [[torch.empty_like(a) for a in s] for s in sig]
    fy = [[torch.empty_like(a) for a in s] for s in sig]
    batch.solve(sig, fx, fy)
    torch.cuda.synchronize()
    for k, (nest, s) in enumerate(probs):
        plans[k].set_schedule(0, 0)
        gx, gy = run_gpu(plans[k], s)
        for l in range(nest.levels):
            g = fx[k][l].double().cpu().numpy()
            assert np.abs(g - gx[l]).max() <= 64 * np.finfo(np.float32).eps * np.abs(gx[l]).max()


def test_autotune_picks_and_records(lib, tmp_path):
    """In a fresh process (the record is process-wide): tune a 1024^2 zero-rim plan,
    check the reported times and that a new plan of the same key starts from the
    recorded schedule, read back from the table file by another fresh process."""
    table = tmp_path / "tune.txt"
    code = r"""
import sys, json
sys.path.insert(0, %r)
from paper_1603_03142_gb300 import sgf, workloads as W
p = sgf.Plan(W.Nest(n=1024), "fp32", zero_rim=True)
r = p.autotune(reps=3)
q = sgf.Plan(W.Nest(n=1024), "fp32", zero_rim=True)
print(json.dumps({"r": r, "q": q.schedule()}))
""" % str(ROOT)
    env = dict(os.environ, SGF_AUTOTUNE_CACHE=str(table))
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr
    import json
    d = json.loads(out.stdout.strip().splitlines()[-1])
    ms = d["r"]["ms"]
    assert all(ms[k] > 0 for k in ("col_pass0", "col_pass1", "col_pass2", "row_inv0_0", "row_inv0_1", "row_inv0_2"))
    ch = d["r"]["chosen"]
    assert ms["col_pass3"] > 0 and ms["col_pass3_radix1"] > 0  # FP32 zero-rim force plan, n = 1024
    cp = [ms["col_pass0"], ms["col_pass1"], ms["col_pass2"], ms["col_pass3"], ms["col_pass3_radix1"]]
    best = cp.index(min(cp))
    assert (ch["col_pass"], ch["col_radix"]) == ((best, 0) if best < 4 else (3, 1))
    assert ms["row_inv0_3"] > 0  # FP32, n = 1024, one level-0 patch
    assert ms["row_inv0_4"] > 0 and ms["row_inv0_4_radix1"] > 0
    assert ms["row_inv0_5"] > 0 and ms["row_inv0_5_radix1"] > 0
    inv = [ms["row_inv0_0"], ms["row_inv0_1"], ms["row_inv0_2"], ms["row_inv0_3"], ms["row_inv0_4"],
           ms["row_inv0_4_radix1"], ms["row_inv0_5"], ms["row_inv0_5_radix1"]]
    best = inv.index(min(inv))
    assert (ch["row_inv0"], ch["inv_radix"]) == [(0, 0), (1, 0), (2, 0), (3, 0), (4, 0), (4, 1), (5, 0), (5, 1)][best]
    assert ms["row_fwd0"] > 0 and ms["row_fwd1"] > 0 and ms["row_fwd2"] > 0
    fw = [ms["row_fwd0"], ms["row_fwd1"], ms["row_fwd2"]]
    assert ch["row_fwd"] == fw.index(min(fw))
    assert d["q"] == ch
    lines = table.read_text().split("\n")
    assert any("/n1024/p1/zr1/" in ln for ln in lines)
    code2 = r"""
import sys, json
sys.path.insert(0, %r)
from paper_1603_03142_gb300 import sgf, workloads as W
print(json.dumps(sgf.Plan(W.Nest(n=1024), "fp32", zero_rim=True).schedule()))
""" % str(ROOT)
    out2 = subprocess.run([sys.executable, "-c", code2], env=env, capture_output=True, text=True, timeout=600)
    assert out2.returncode == 0, out2.stderr
    assert json.loads(out2.stdout.strip().splitlines()[-1]) == ch


@pytest.mark.parametrize("case", ["zero_rim_4096", "general_1024", "nest_512", "potential_1024"])
def test_tma_gather_matches_lane_gather(lib, case):
    """row_inv0 = 3 (k_row_inv1t), 4 (k_row_inv1x) and 5 (k_row_inv2x) against
    row_inv0 = 0 (k_row_inv1): the same arithmetic on the same bins, only the
    gather and the thread layout differ."""
    rng = np.random.Generator(np.random.PCG64(31))
    kw = {}
    if case == "zero_rim_4096":
        nest, sigma, kw = W.Nest(n=4096), _zero_rim_sigma(4096, 3), {"zero_rim": True}
    elif case == "general_1024":
        nest = W.Nest(n=1024)
        sigma = [rng.uniform(0.1, 1.0, (1024, 1024))]
    elif case == "nest_512":
        nest, sigma = W.random_nest_problem(rng, 512, 2)
    else:
        nest = W.Nest(n=1024)
        sigma = [rng.uniform(0.1, 1.0, (1024, 1024))]
        kw = {"potential": True}
    plan = lib.Plan(nest, "fp32", **kw)

    def run():
        if kw.get("potential"):
            import torch
            phi = plan.solve_potential([torch.from_numpy(s).float().cuda() for s in sigma])
            torch.cuda.synchronize()
            return [t.double().cpu().numpy() for t in phi], []
        return run_gpu(plan, sigma)
    plan.set_schedule(0, 0)
    a = run()
    plan.set_schedule(0, 3)
    b = run()
    plan.check()  # no bounded wait gave up
    eps = np.finfo(np.float32).eps
    for ga, gb in zip(a[0] + a[1], b[0] + b[1]):
        assert np.abs(ga - gb).max() <= 64 * eps * np.abs(ga).max()
    if nest.n >= 1024:  # row_inv0 = 4, 5: k_row_inv1x / k_row_inv2x, walking CTAs, both parity halves per thread
        for inv in (4, 5):
            plan.set_schedule(0, inv)
            c = run()
            plan.check()
            for ga, gc in zip(a[0] + a[1], c[0] + c[1]):
                assert np.abs(ga - gc).max() <= 64 * eps * np.abs(ga).max()


def test_tma_schedule_falls_back_where_it_cannot_apply(lib):
    import torch
    nest = W.Nest(n=512)
    rng = np.random.Generator(np.random.PCG64(32))
    sigma = [rng.uniform(0.1, 1.0, (512, 512))]
    plan = lib.Plan(nest, "fp32")
    plan.set_schedule(0, 0)
    ref = run_gpu(plan, sigma)
    plan.set_schedule(0, 3)
    # the no-allocation solve's intermediates are not the plan's: it runs row_inv0 = 0
    ts = [torch.from_numpy(sigma[0]).float().cuda()]
    fx, fy = [torch.empty_like(ts[0])], [torch.empty_like(ts[0])]
    plan.solve_noalloc_ptrs([ts[0].data_ptr()], [fx[0].data_ptr()], [fy[0].data_ptr()])
    torch.cuda.synchronize()
    assert np.array_equal(fx[0].double().cpu().numpy(), ref[0][0])
    assert np.array_equal(fy[0].double().cpu().numpy(), ref[1][0])
    # batches keep their own launch maps: a plan at row_inv0 = 3 runs k_row_inv1 there
    batch = lib.Batch([plan])
    bx, by = [[torch.empty_like(ts[0])]], [[torch.empty_like(ts[0])]]
    batch.solve([ts], bx, by)
    torch.cuda.synchronize()
    assert np.array_equal(bx[0][0].double().cpu().numpy(), ref[0][0])
    # not available: FP64, BF16X, two level-0 patches
    for p in (lib.Plan(nest, "fp64"), lib.Plan(nest, "bf16x"),
              lib.Plan(W.Forest(n=512, level=[0, 0], org=[(0, 0), (512, 0)]), "fp32")):
        for inv in (3, 4, 5):
            with pytest.raises(lib.SgfError) as ei:
                p.set_schedule(0, inv)
            assert ei.value.status == lib.SGF_EUNSUPPORTED


@pytest.mark.parametrize("n", [512, 1024])
def test_zero_rim_noalloc_matches_solve(lib, n):
    """The no-allocation solve of a zero-rim FP32 plan (scratch intermediates)
    against its ordinary solve: same kernels, same arithmetic, bit-identical forces."""
    import torch
    plan = lib.Plan(W.Nest(n=n), "fp32", zero_rim=True)
    plan.set_schedule(1, 0)
    sig = _zero_rim_sigma(n, 5)
    ref = run_gpu(plan, sig)
    plan.check()
    ts = torch.from_numpy(sig[0]).float().cuda()
    fx, fy = torch.empty_like(ts), torch.empty_like(ts)
    plan.solve_noalloc_ptrs([ts.data_ptr()], [fx.data_ptr()], [fy.data_ptr()])
    torch.cuda.synchronize()
    assert np.array_equal(fx.double().cpu().numpy(), ref[0][0])
    assert np.array_equal(fy.double().cpu().numpy(), ref[1][0])


@pytest.mark.parametrize("case", ["general_1024", "potential_1024", "nest_512", "forest_512"])
def test_general_col_pass_one_cta_matches_cluster(lib, case):
    """col_pass 2 on a general plan (k_col_w: both parity halves in one CTA) against
    col_pass 0 (k_col: a 2-CTA cluster per column), including chunked main outputs
    (the nest's level 0 has 1 + 4 + 16 inputs) and Case-1 offsets (the forest)."""
    import torch
    rng = np.random.Generator(np.random.PCG64(33))
    kw = {}
    if case.startswith("general") or case.startswith("potential"):
        geom = W.Nest(n=1024)
        sigma = [rng.uniform(0.1, 1.0, (1024, 1024))]
        kw = {"potential": case.startswith("potential")}
    elif case == "nest_512":
        geom, sigma = W.random_nest_problem(rng, 512, 3)
    else:
        geom = W.two_patch_forest(512)
        sigma = [rng.uniform(0.1, 1.0, (512, 512)) for _ in range(geom.levels)]
    plan = lib.Plan(geom, "fp32", **kw)

    def run():
        if kw.get("potential"):
            phi = plan.solve_potential([torch.from_numpy(s).float().cuda() for s in sigma])
            torch.cuda.synchronize()
            return [t.double().cpu().numpy() for t in phi]
        gx, gy = run_gpu(plan, sigma)
        return gx + gy
    res = {}
    for c3 in (0, 1):
        for col in (0, 2):
            plan.set_schedule(col, 0, c3)
            res[(col, c3)] = run()
    eps = np.finfo(np.float32).eps
    a = res[(0, 0)]
    for key, b in res.items():
        for ga, gb in zip(a, b):
            assert np.abs(ga - gb).max() <= 64 * eps * np.abs(ga).max(), key
    for p in (lib.Plan(W.Nest(n=256), "fp32"), lib.Plan(W.Nest(n=512), "fp64"), lib.Plan(W.Nest(n=512), "bf16x")):
        with pytest.raises(lib.SgfError) as ei:
            p.set_schedule(2, 0)
        assert ei.value.status == lib.SGF_EUNSUPPORTED


def test_batch_with_one_cta_column_pass(lib):
    """A batch group of plans at col_pass 2 runs k_col_w (batch view) for the column pass."""
    import torch
    rng = np.random.Generator(np.random.PCG64(34))
    probs = [W.random_nest_problem(rng, 512, L) for L in (1, 2, 3)]
    plans = [lib.Plan(nest, "fp32") for nest, _ in probs]
    for p in plans:
        p.set_schedule(2, 0)
    batch = lib.Batch(plans)
    sig = [[torch.from_numpy(a).float().cuda() for a in s] for _, s in probs]
    fx = [[torch.empty_like(a) for a in s] for s in sig]
    fy = [[torch.empty_like(a) for a in s] for s in sig]
    batch.solve(sig, fx, fy)
    torch.cuda.synchronize()
    eps = np.finfo(np.float32).eps
    for k, (nest, s) in enumerate(probs):
        plans[k].set_schedule(0, 0)
        gx, gy = run_gpu(plans[k], s)
        for l in range(nest.levels):
            scale = max(np.abs(gx[l]).max(), np.abs(gy[l]).max())
            assert np.abs(fx[k][l].double().cpu().numpy() - gx[l]).max() <= 64 * eps * scale
            assert np.abs(fy[k][l].double().cpu().numpy() - gy[l]).max() <= 64 * eps * scale
