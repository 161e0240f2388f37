"""Fused batches (sgf_batch_*): many independent nests of uneven N, level count
and path solved with one launch per pass and per N group, replayed as a CUDA
graph.  Every nest's result must equal its own single solve bitwise (the same
kernels do the same arithmetic), call after call, with and without the graph."""
import numpy as np
import pytest

from paper_1603_03142_gb300 import workloads as W
from tests._gpu import run_gpu, sgf, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    return sgf()


def _problems(seed, count):
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(count):
        n = int(rng.choice([16, 32, 64, 128]))
        L = int(rng.integers(1, min(4, n.bit_length() - 3) + 1))
        out.append(W.random_nest_problem(rng, n, L))
    return out


@pytest.mark.parametrize("graph", [True, False])
def test_batch_equals_single_solves(lib, graph):
    probs = _problems(21, 24)
    plans = [lib.Plan(nest, "fp32") for nest, _ in probs]
    # one zero-rim single-level nest in the mix (its own kernel group)
    zr = W.Nest(n=64)
    zs = np.zeros((64, 64))
    zs[2:-2, 2:-2] = np.random.Generator(np.random.PCG64(3)).uniform(0.1, 1.0, (60, 60))
    plans.append(lib.Plan(zr, "fp32", zero_rim=True))
    probs.append((zr, [zs]))
    batch = lib.Batch(plans, graph=graph)
    info = batch.info()
    # per group: row_fwd, col (+ col_g for Case-3 groups, col_sum for chunked outputs), row_inv1 (+ row_inv for the finer
    # levels); one restriction per depth
    assert info["groups"] >= 4 and info["launches_per_solve"] <= 6 * info["groups"] + 3
    for call in range(3):
        sig = [[torch.from_numpy(a * (1.0 + 0.1 * call)).float().cuda() for a in s] for _, s in probs]
        fx = [[torch.empty_like(a) for a in s] for s in sig]
        fy = [[torch.empty_like(a) for a in s] for s in sig]
        batch.solve(sig, fx, fy)
        torch.cuda.synchronize()
        for k, (nest, s) in enumerate(probs):
            gx, gy = run_gpu(plans[k], [a * (1.0 + 0.1 * call) for a in s])
            for l in range(nest.levels):
                assert np.array_equal(fx[k][l].double().cpu().numpy(), gx[l]), (call, k, l)
                assert np.array_equal(fy[k][l].double().cpu().numpy(), gy[l]), (call, k, l)
    plans[-1].check()


def test_batch_rejects_duplicates(lib):
    p = lib.Plan(W.Nest(n=16), "fp32")
    with pytest.raises(lib.SgfError):
        lib.Batch([p, p])


def _c4_subset():
    """The first nest of every (N, levels) of the seeded 256-nest batched workload
    (N in {128, 256, 512, 1024}, 1-4 levels): 16 nests."""
    rng = np.random.Generator(np.random.PCG64(0))  # the draws of W.config4(seed=0), in order
    seen, out = set(), []
    for _ in range(256):
        n = int(rng.choice((128, 256, 512, 1024)))
        L = int(rng.integers(1, 5))
        nest, sigma = W.random_nest_problem(rng, n, L)
        if (n, L) not in seen:
            seen.add((n, L))
            out.append((nest, sigma))
        if len(out) == 16:
            break
    return out


def _sampled_oracle(nest, sigma, per_level, seed):
    import oracle
    rng = np.random.Generator(np.random.PCG64(seed))
    lv, ii, jj = [], [], []
    for l in range(nest.levels):
        free = np.argwhere(~nest.covered_mask(l))
        pick = free[rng.choice(len(free), size=min(per_level, len(free)), replace=False)]
        lv.append(np.full(len(pick), l)), jj.append(pick[:, 0]), ii.append(pick[:, 1])
    lv, ii, jj = np.concatenate(lv), np.concatenate(ii), np.concatenate(jj)
    ox, oy = oracle.force_at(nest, sigma, lv, ii, jj)
    return lv, ii, jj, ox, oy


@pytest.mark.parametrize("col_pass", [0, 2])
def test_c4_sized_batch_against_oracle(lib, col_pass):
    """One fused batch of C4-sized nests (N up to 1024, up to 4 levels), each
    level compared with the direct-sum oracle on sampled uncovered cells; with
    col_pass 2 the groups of N >= 512 run the one-CTA column kernels."""
    from tests._gpu import tol
    probs = _c4_subset()
    assert len(probs) == 16
    plans = [lib.Plan(nest, "fp32") for nest, _ in probs]
    for p, (nest, _) in zip(plans, probs):
        if col_pass == 2 and nest.n >= 512:
            p.set_schedule(2, 0)
    batch = lib.Batch(plans)
    sig = [[torch.from_numpy(a).float().cuda() for a in s] for _, s in probs]
    fx = [[torch.empty_like(a) for a in s] for s in sig]
    fy = [[torch.empty_like(a) for a in s] for s in sig]
    batch.solve(sig, fx, fy)
    torch.cuda.synchronize()
    for k, (nest, s) in enumerate(probs):
        lv, ii, jj, ox, oy = _sampled_oracle(nest, s, 64 if nest.n <= 256 else 16, 100 + k)
        for l in range(nest.levels):
            m = lv == l
            gx = fx[k][l].double().cpu().numpy()[jj[m], ii[m]]
            gy = fy[k][l].double().cpu().numpy()[jj[m], ii[m]]
            scale = max(np.abs(ox[m]).max(), np.abs(oy[m]).max())
            err = max(np.abs(gx - ox[m]).max(), np.abs(gy - oy[m]).max())
            assert err <= tol("fp32", nest.n) * scale, (nest.n, nest.levels, l, err / scale)
