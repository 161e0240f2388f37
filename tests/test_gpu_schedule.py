"""Tile schedules and the autotuner (sgf_plan_schedule_*, sgf_plan_autotune).

Every schedule performs the same arithmetic in the same order, so the forces
must agree bit for bit across schedules; the autotuner must pick one of the
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
def test_schedules_agree_bitwise_zero_rim(lib, prec, n):
    nest = W.Nest(n=n)
    sigma = _zero_rim_sigma(n, n)
    plan = lib.Plan(nest, prec, zero_rim=True)
    outs = []
    for col in (0, 1):
        for inv in (0, 1):
            plan.set_schedule(col, inv)
            assert plan.schedule() == {"col_pass": col, "row_inv0": inv}
            outs.append(run_gpu(plan, sigma))
            plan.check()
    for gx, gy in outs[1:]:
        assert np.array_equal(gx[0], outs[0][0][0]) and np.array_equal(gy[0], outs[0][1][0])


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_row_inv_schedules_agree_on_nests(lib, prec):
    rng = np.random.Generator(np.random.PCG64(8))
    nest, sigma = W.random_nest_problem(rng, 128, 3)
    plan = lib.Plan(nest, prec)
    plan.set_schedule(0, 0)
    a = run_gpu(plan, sigma)
    plan.set_schedule(0, 1)
    b = run_gpu(plan, sigma)
    assert plan.stats()["launches_per_solve"] == 2 + 3
    for l in range(3):
        assert np.array_equal(a[0][l], b[0][l]) and np.array_equal(a[1][l], b[1][l])


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
            assert np.array_equal(fx[k][l].double().cpu().numpy(), gx[l])


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
    assert all(ms[k] > 0 for k in ("col_pass0", "col_pass1", "row_inv0_0", "row_inv0_1"))
    ch = d["r"]["chosen"]
    assert ch["col_pass"] == (1 if ms["col_pass1"] < ms["col_pass0"] else 0)
    assert ch["row_inv0"] == (1 if ms["row_inv0_1"] < ms["row_inv0_0"] else 0)
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
