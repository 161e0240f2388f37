"""GPU parity of the potential (SGF_PLAN_POTENTIAL: kernel -1/r of Sec. 2, G = 1,
the linear density of Eq. eqnSigma) against the CPU FP64 oracle.

Element by element on seeded nests the oracle finishes in seconds (every pair
case, refinement ratios up to 8); on sampled targets at 256^2 x 3 levels and
at 4096^2 in FP32 and split-BF16; the Maclaurin disk's closed form; the scaling
of the potential with the cell size; the schedules; and the refusals of the
force-only entry points.  Bound: relative L-infinity per level (tests/_gpu.py).
"""
import math

import numpy as np
import pytest

import oracle
from paper_1603_03142_gb300 import workloads as W
from tests._gpu import sgf, tol

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    return sgf()


def run_phi(plan, sigma):
    import torch
    dt = torch.float64 if plan.precision == 0 else torch.float32
    sig = [torch.from_numpy(np.ascontiguousarray(s)).to(device="cuda", dtype=dt) for s in sigma]
    phi = plan.solve_potential(sig)
    torch.cuda.synchronize()
    return [t.double().cpu().numpy() for t in phi]


def _random_sigma(nest, seed, lo=0.2, hi=1.5):
    rng = np.random.Generator(np.random.PCG64(seed))
    return [rng.uniform(lo, hi, (nest.n, nest.n)) for _ in range(nest.levels)]


def _rel(nest, got, ref):
    out = []
    for l in range(nest.levels):
        keep = ~nest.covered_mask(l)
        out.append(np.abs(got[l] - ref[l])[keep].max() / np.abs(ref[l][keep]).max())
    return out


NESTS = [
    (16, 1, [(0, 0)]),
    (32, 1, [(0, 0)]),
    (16, 2, [(0, 0), (8, 0)]),
    (16, 4, [(0, 0), (4, 4), (0, 8), (8, 2)]),   # m = 8
    (32, 3, [(0, 0), (5, 9), (4, 12)]),
    (64, 2, [(0, 0), (16, 16)]),
    (128, 1, [(0, 0)]),
]


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16x"])
@pytest.mark.parametrize("case", NESTS, ids=[f"n{n}L{L}" for n, L, _ in NESTS])
def test_potential_full_oracle(lib, prec, case):
    n, L, off = case
    nest = W.Nest(n=n, levels=L, off=off)
    sigma = _random_sigma(nest, 200 + n + L)
    phi = run_phi(lib.Plan(nest, prec, potential=True), sigma)
    ref = oracle.potential(nest, sigma)
    errs = _rel(nest, phi, ref)
    assert max(errs) <= tol(prec, n), errs
    for l in range(L):
        assert np.all(phi[l][nest.covered_mask(l)] == 0.0)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_config2_nest_sampled(lib, prec):
    """3 levels of 256^2 centred at (0.3, 0), Maclaurin + clump + 1% noise."""
    nest, sigma = W.config2()
    phi = run_phi(lib.Plan(nest, prec, potential=True), sigma)
    rng = np.random.Generator(np.random.PCG64(12))
    lv, ii, jj = [], [], []
    for l in range(nest.levels):
        cand = np.argwhere(~nest.covered_mask(l))
        for j, i in cand[rng.choice(len(cand), size=200, replace=False)]:
            lv.append(l), ii.append(i), jj.append(j)
    lv, ii, jj = map(np.array, (lv, ii, jj))
    ref = oracle.potential_at(nest, sigma, lv, ii, jj)
    for l in range(nest.levels):
        k = lv == l
        got = phi[l][jj[k], ii[k]]
        assert np.abs(got - ref[k]).max() <= tol(prec, 256) * np.abs(ref[k]).max()


@pytest.mark.parametrize("prec", ["fp32", "bf16x"])
def test_uniform_4096_sampled(lib, prec):
    """4096^2 lognormal tapered density, one level: sampled targets incl. corners and centre."""
    nest, sigma = W.config3()
    phi = run_phi(lib.Plan(nest, prec, potential=True), sigma)[0]
    rng = np.random.Generator(np.random.PCG64(13))
    ii = np.concatenate([rng.integers(0, 4096, 24), [0, 4095, 2048, 2047, 200, 3900]])
    jj = np.concatenate([rng.integers(0, 4096, 24), [0, 4095, 2048, 2047, 3900, 200]])
    ref = oracle.potential_at(nest, sigma, np.zeros_like(ii), ii, jj)
    assert np.abs(phi[jj, ii] - ref).max() <= tol(prec, 4096) * np.abs(ref).max()


def test_maclaurin_closed_form(lib):
    """Inside the disk sigma0 sqrt(1 - r^2/a^2): Phi = -(pi^2 sigma0 / (4a)) (2a^2 - r^2)."""
    a, n = 0.8, 256
    nest, sigma = W.config1(n)
    phi = run_phi(lib.Plan(nest, "fp32", potential=True), sigma)[0]
    x = nest.x0 + (np.arange(n) + 0.5) * nest.h0
    X, Y = np.meshgrid(x, x)
    R = np.hypot(X, Y)
    inside = R < 0.7 * a
    exact = -(math.pi ** 2) / (4 * a) * (2 * a * a - R[inside] ** 2)
    assert np.abs(phi[inside] - exact).max() <= 2e-5 * np.abs(exact).max()


def test_scales_with_cell_size(lib):
    """Same sigma on a nest twice as large: the potential doubles (the force would not change)."""
    off = [(0, 0), (8, 8), (4, 12)]
    n1 = W.Nest(n=32, levels=3, off=off, x0=-1.0, y0=-1.0, h0=1.0 / 16)
    n2 = W.Nest(n=32, levels=3, off=off, x0=-2.0, y0=-2.0, h0=1.0 / 8)
    sigma = _random_sigma(n1, 7)
    p1 = run_phi(lib.Plan(n1, "fp64", potential=True), sigma)
    p2 = run_phi(lib.Plan(n2, "fp64", potential=True), sigma)
    for l in range(3):
        assert np.abs(p2[l] - 2.0 * p1[l]).max() <= 1e-13 * np.abs(p2[l]).max()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_schedules_and_launches(lib, prec):
    rng = np.random.Generator(np.random.PCG64(8))
    nest, sigma = W.random_nest_problem(rng, 128, 3)
    plan = lib.Plan(nest, prec, potential=True)
    res = {}
    for inv in (0, 1):
        for c3 in (0, 1):
            plan.set_schedule(0, inv, c3)
            res[(inv, c3)] = run_phi(plan, sigma)
            assert plan.stats()["launches_per_solve"] == 2 + 3 + (0 if inv == 1 else 1) + (1 - c3) + 1
    with pytest.raises(lib.SgfError) as ei:
        plan.set_schedule(0, 2)  # both components per CTA: the potential has one
    assert ei.value.status == lib.SGF_EUNSUPPORTED
    eps = np.finfo(np.float64 if prec == "fp64" else np.float32).eps
    a = res[(0, 0)]
    for key, b in res.items():
        for l in range(3):
            assert np.abs(a[l] - b[l]).max() <= 64 * eps * np.abs(a[l]).max(), (key, l)
    r = plan.autotune(reps=1)
    assert r["ms"]["row_inv0_2"] < 0 and r["chosen"]["row_inv0"] != 2
    ref = oracle.potential(nest, sigma)
    assert max(_rel(nest, run_phi(plan, sigma), ref)) <= tol(prec, 128)


def test_force_entry_points_refuse_potential_plans(lib):
    import torch
    nest = W.Nest(n=32, levels=1, off=[(0, 0)])
    pp = lib.Plan(nest, "fp32", potential=True)
    fp = lib.Plan(nest, "fp32")
    s = [torch.ones((32, 32), device="cuda")]
    with pytest.raises(lib.SgfError) as ei:
        pp.solve(s)
    assert ei.value.status == lib.SGF_EINVAL
    with pytest.raises(lib.SgfError) as ei:
        fp.solve_potential(s)
    assert ei.value.status == lib.SGF_EINVAL
    with pytest.raises(lib.SgfError) as ei:
        lib.Batch([pp])
    assert ei.value.status == lib.SGF_EUNSUPPORTED
    zr = lib.Plan(nest, "fp32", zero_rim=True, potential=True)  # the zero-rim potential: col_pass 2 (3 from n = 1024)
    assert zr.schedule()["col_pass"] == 2
    for col in (0, 3):
        with pytest.raises(lib.SgfError) as ei:
            zr.set_schedule(col, 0)
        assert ei.value.status == lib.SGF_EUNSUPPORTED
    # a shared plan keeps the potential spectra, and gives the same numbers
    q = pp.share()
    a = pp.solve_potential(s)[0]
    b = q.solve_potential(s)[0]
    torch.cuda.synchronize()
    assert torch.equal(a, b)


def _zero_rim_sigma(n, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    s = np.zeros((n, n))
    s[2:-2, 2:-2] = rng.uniform(0.1, 1.0, (n - 4, n - 4))
    return [s]


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16x"])
@pytest.mark.parametrize("n", [64, 512])
def test_zero_rim_potential_oracle(lib, prec, n):
    """SGF_PLAN_ZERO_RIM | SGF_PLAN_POTENTIAL (one merged real table over sigma)
    against the oracle on a density that is zero on the two outer rings."""
    nest = W.Nest(n=n)
    sigma = _zero_rim_sigma(n, 40 + n)
    plan = lib.Plan(nest, prec, potential=True, zero_rim=True)
    phi = run_phi(plan, sigma)
    plan.check()
    if n <= 64:
        ref = oracle.potential(nest, sigma)[0]
        assert np.abs(phi[0] - ref).max() <= tol(prec, n) * np.abs(ref).max()
    else:
        rng = np.random.Generator(np.random.PCG64(41))
        ii, jj = rng.integers(0, n, 40), rng.integers(0, n, 40)
        ref = oracle.potential_at(nest, sigma, np.zeros_like(ii), ii, jj)
        assert np.abs(phi[0][jj, ii] - ref).max() <= tol(prec, n) * np.abs(ref).max()


@pytest.mark.parametrize("n", [1024, 2048])
def test_zero_rim_potential_register_twiddle_column(lib, n):
    """col_pass 3 on a zero-rim potential plan (k_col_mx with one component, in
    both radix plans, behind both walking forward row kernels) against col_pass 2
    (k_col_mw): same expressions, so the potentials agree to rounding; and
    against the oracle on sampled cells."""
    nest = W.Nest(n=n)
    sigma = _zero_rim_sigma(n, 50 + n)
    plan = lib.Plan(nest, "fp32", potential=True, zero_rim=True)
    plan.set_schedule(2, 0)
    ref_gpu = run_phi(plan, sigma)[0]
    eps = np.finfo(np.float32).eps
    scale = np.abs(ref_gpu).max()
    for radix in (0, 1):
        for fw in (0, 2):
            plan.set_schedule(3, 5, 0, radix, 0, fw)
            phi = run_phi(plan, sigma)[0]
            plan.check()
            assert np.abs(phi - ref_gpu).max() <= 64 * eps * scale, (radix, fw)
    rng = np.random.Generator(np.random.PCG64(51))
    ii, jj = rng.integers(0, n, 24), rng.integers(0, n, 24)
    ref = oracle.potential_at(nest, sigma, np.zeros_like(ii), ii, jj)
    assert np.abs(phi[jj, ii] - ref).max() <= tol("fp32", n) * np.abs(ref).max()


def test_zero_rim_potential_matches_general_4096(lib):
    """The merged table and the three-table general plan evaluate the same sum."""
    nest, sigma = W.config3()
    a = run_phi(lib.Plan(nest, "fp32", potential=True, zero_rim=True), sigma)[0]
    b = run_phi(lib.Plan(nest, "fp32", potential=True), sigma)[0]
    assert np.abs(a - b).max() <= 1e-5 * np.abs(b).max()


def test_zero_rim_potential_autotune(lib):
    """The tuner keeps the zero-rim potential on its one applicable column schedule."""
    n = 512
    nest = W.Nest(n=n)
    sigma = _zero_rim_sigma(n, 7)
    plan = lib.Plan(nest, "fp32", potential=True, zero_rim=True)
    r = plan.autotune(reps=1)
    assert r["chosen"]["col_pass"] == 2
    assert r["ms"]["col_pass0"] < 0 and r["ms"]["col_pass1"] < 0 and r["ms"]["col_pass2"] > 0
    phi = run_phi(plan, sigma)[0]
    rng = np.random.Generator(np.random.PCG64(42))
    ii, jj = rng.integers(0, n, 30), rng.integers(0, n, 30)
    ref = oracle.potential_at(nest, sigma, np.zeros_like(ii), ii, jj)
    assert np.abs(phi[jj, ii] - ref).max() <= tol("fp32", n) * np.abs(ref).max()
