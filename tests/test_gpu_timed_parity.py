"""Oracle parity of the configurations the benchmark times, schedule by schedule.

The benchmark autotunes its 4096^2 plans and then times one kernel schedule
(on the zero-rim FP32 path the column pass with both parity halves in one CTA
and the level-0 inverse rows gathered by the tensor memory accelerator).  Here
every schedule of every path, at every compiled transform size, is compared
with the FP64 oracle (the direct sum of Sec. 2.1):
  - n <= 128: every cell;
  - n >= 256: the full row j = n/2 and the full column i = n/2, seeded rows
    with seeded columns (1024 targets at n = 4096), and the cells of largest
    |Fx| and |Fy| of the GPU result.
Rows and columns come from oracle.force_row / force_col (the same direct sum
with the cell integrals shared along the row); the argmax cells from
oracle.force_at.  Relative L-infinity per component family as in the other
parity tests: max |F - F_oracle| over the sampled cells / max |F_oracle|."""
import numpy as np
import pytest

import oracle
from paper_1603_03142_gb300 import workloads as W
from tests._gpu import run_gpu, sgf, tol

pytestmark = pytest.mark.gpu

NS = [16, 32, 64, 128, 256, 512, 1024, 2048, 4096]


@pytest.fixture(scope="module")
def lib():
    return sgf()


class Sample:
    """Oracle forces at the sampled cells of a single-level workload."""

    def __init__(self, n, seed=0):
        self.n = n
        self.nest, self.sigma = W.config3(n, seed=seed)
        # the taper leaves the two outer rings empty from n = 64 on; below, clear
        # them so the zero-rim plans' guarantee holds (the general plans see the same density)
        s0 = self.sigma[0].copy()
        s0[:2, :] = s0[-2:, :] = s0[:, :2] = s0[:, -2:] = 0.0
        self.sigma = [s0]
        if n <= 128:
            fx, fy = oracle.force(self.nest, self.sigma)
            jj, ii = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
            self.ii, self.jj = ii.ravel(), jj.ravel()
            self.ox, self.oy = fx[0].ravel(), fy[0].ravel()
            return
        prep = oracle.prepare(self.nest, self.sigma)
        ii, jj, ox, oy = [], [], [], []
        rx, ry = oracle.force_row(self.nest, None, n // 2, prepared=prep)  # full centre row
        ii.append(np.arange(n)), jj.append(np.full(n, n // 2)), ox.append(rx), oy.append(ry)
        cx, cy = oracle.force_col(self.nest, self.sigma, n // 2)          # full centre column
        ii.append(np.full(n, n // 2)), jj.append(np.arange(n)), ox.append(cx), oy.append(cy)
        rng = np.random.Generator(np.random.PCG64(1000 + n))
        rows = rng.choice(n, size=8 if n == 4096 else 4, replace=False)
        per = 128 if n == 4096 else 64
        for jt in rows:                                                    # seeded rows x seeded columns
            cols = rng.choice(n, size=per, replace=False)
            sx, sy = oracle.force_row(self.nest, None, int(jt), cols, prepared=prep)
            ii.append(cols), jj.append(np.full(per, jt)), ox.append(sx), oy.append(sy)
        self.prep = prep
        self.ii, self.jj = np.concatenate(ii), np.concatenate(jj)
        self.ox, self.oy = np.concatenate(ox), np.concatenate(oy)

    def rel_err(self, gx, gy):
        """Relative L-inf over the sample, plus the argmax-|F| cells of the GPU result."""
        ii, jj, ox, oy = self.ii, self.jj, self.ox, self.oy
        if self.n > 128:
            extra = [np.unravel_index(np.argmax(np.abs(g)), g.shape) for g in (gx, gy)]
            ej = np.array([e[0] for e in extra])
            ei = np.array([e[1] for e in extra])
            ex, ey = oracle.force_at(self.nest, None, np.zeros(2, int), ei, ej, prepared=self.prep)
            ii, jj = np.concatenate([ii, ei]), np.concatenate([jj, ej])
            ox, oy = np.concatenate([ox, ex]), np.concatenate([oy, ey])
        scale = max(np.abs(ox).max(), np.abs(oy).max())
        err = max(np.abs(gx[jj, ii] - ox).max(), np.abs(gy[jj, ii] - oy).max())
        return err / scale


_samples = {}


def sample(n):
    if n not in _samples:
        _samples[n] = Sample(n)
    return _samples[n]


def schedules(n, prec, zero_rim):
    """Every (col_pass, row_inv0) the plan accepts (sgf.h: schedule rules); the
    register-twiddle kernels (col_pass 3, row_inv0 4 and 5) also in radix plan 1."""
    cols = ((0, 1, 2, 3) if prec == "fp32" and n >= 1024 else (0, 1, 2)) if zero_rim else (0, 2)
    invs = (0, 1, 2, 3, 4, 5)
    out = []
    for c in cols:
        for i in invs:
            if c == 2 and not zero_rim and (prec != "fp32" or n < 512):
                continue
            if i == 3 and (prec != "fp32" or n < 512):
                continue
            if i in (4, 5) and (prec != "fp32" or n < 1024):
                continue
            if prec == "bf16x" and n == 4096 and (c == 2 or i == 1):
                continue
            out.append((c, i, 0, 0, 0))
            if c == 3:
                out.append((c, i, 1, 0, 0))
            if i in (4, 5):
                out.append((c, i, 0, 1, 0))
            if prec == "fp32" and n >= 1024 and (c in (2, 3) or not zero_rim):
                out.append((c, i, 0, 0, 1))  # two row pairs per CTA in the forward rows
            if prec == "fp32" and n >= 1024 and i in (3, 5) and (c in (2, 3) or not zero_rim):
                out.append((c, i, 0, 0, 2))  # the walking register-twiddle forward rows
    return out


def _check_all(lib, n, prec, zero_rim):
    s = sample(n)
    plan = lib.Plan(s.nest, prec, zero_rim=zero_rim)
    bound = tol(prec, n)
    worst = {}
    for c, i, cr, ir, fw in schedules(n, prec, zero_rim):
        plan.set_schedule(c, i, 0, cr, ir, fw)
        gx, gy = run_gpu(plan, s.sigma)
        plan.check()
        worst[(c, i, cr, ir, fw)] = s.rel_err(gx[0], gy[0])
    bad = {k: v for k, v in worst.items() if not v <= bound}
    assert not bad, (bad, bound)
    return worst


@pytest.mark.parametrize("n", NS)
@pytest.mark.parametrize("zero_rim", [True, False], ids=["zero_rim", "general"])
def test_fp32_every_schedule_against_oracle(lib, n, zero_rim):
    _check_all(lib, n, "fp32", zero_rim)


@pytest.mark.parametrize("n", [128, 256, 512, 1024, 2048, 4096])
@pytest.mark.parametrize("zero_rim", [True, False], ids=["zero_rim", "general"])
def test_bf16x_every_schedule_against_oracle(lib, n, zero_rim):
    _check_all(lib, n, "bf16x", zero_rim)


@pytest.mark.parametrize("zero_rim", [True, False], ids=["zero_rim", "general"])
@pytest.mark.parametrize("prec", ["fp32", "bf16x"])
def test_4096_autotuned_plan_against_oracle(lib, prec, zero_rim):
    """The benchmark's own sequence: a fresh plan, autotuned, then solved."""
    s = sample(4096)
    plan = lib.Plan(s.nest, prec, zero_rim=zero_rim)
    plan.autotune(reps=3)
    gx, gy = run_gpu(plan, s.sigma)
    plan.check()
    assert s.rel_err(gx[0], gy[0]) <= tol(prec, 4096)


@pytest.mark.parametrize("col_pass,row_inv0,row_fwd", [(2, 3, 0), (3, 3, 1), (3, 4, 1), (3, 5, 1), (3, 5, 2)])
def test_4096_timed_schedule_explicitly(lib, col_pass, row_inv0, row_fwd):
    """Zero-rim FP32 with the level-0 inverse rows gathered by the tensor memory
    accelerator (k_row_inv1t, k_row_inv1x, k_row_inv2x) behind either walking column pass
    (k_col_mw, k_col_mx), the candidates the benchmark's autotuner chooses
    from, solved twice (the second solve runs on the first one's leftover
    intermediates)."""
    s = sample(4096)
    plan = lib.Plan(s.nest, "fp32", zero_rim=True)
    plan.set_schedule(col_pass, row_inv0, 0, 0, 0, row_fwd)
    for _ in range(2):
        gx, gy = run_gpu(plan, s.sigma)
        plan.check()
        assert s.rel_err(gx[0], gy[0]) <= tol("fp32", 4096)


@pytest.mark.parametrize("n", [16, 64, 256, 1024, 2048])
def test_fp64_every_schedule_against_oracle(lib, n):
    for zr in (True, False):
        _check_all(lib, n, "fp64", zr)
