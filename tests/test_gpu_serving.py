"""The request loop (sgf_server_*) on the GPU.

The serving contract: requests admitted while others run share the device
(their copies and kernels overlap on separate streams), and each result is the
same alone and in the mix.  Solves are deterministic (fixed summation order, no
atomics), so "the same" is checked bit for bit; the FP32 parity bound against
the oracle is checked on a subset.  Every third request is SGF_BF16X, so the
mix holds both precisions; FP32 and BF16X requests of one shape share its FP32
spectra.
"""
import numpy as np
import pytest

import oracle
from paper_1603_03142_gb300 import serving
from paper_1603_03142_gb300 import workloads as W
from tests._gpu import rel_linf_levels, sgf, tol

pytestmark = pytest.mark.gpu

SHAPES = [(64, 1), (64, 2), (64, 3), (128, 1), (128, 2), (128, 3), (256, 2), (32, 3)]


def _requests(count, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    reqs = []
    for k in range(count):
        n, L = SHAPES[int(rng.integers(len(SHAPES)))]
        nest, sig = W.random_nest_problem(rng, n, L)
        s = []
        for a in sig:
            p = serving.pinned((n, n), np.float32)
            p[...] = a
            s.append(p)
        reqs.append((nest, s, "bf16x" if k % 3 == 2 else "fp32"))
    return reqs


def _outputs(nest):
    return ([serving.pinned((nest.n, nest.n), np.float32) for _ in range(nest.levels)],
            [serving.pinned((nest.n, nest.n), np.float32) for _ in range(nest.levels)])


def _drain(srv, want, done=None):
    done = [] if done is None else done
    while len(done) < want:
        done += srv.progress()
    return done


def _mixed(reqs, budget, inflight):
    lib = sgf()
    srv = lib.Server(hbm_budget=budget, max_inflight=inflight)
    outs = {}
    for k, (nest, sig, prec) in enumerate(reqs):
        outs[k] = _outputs(nest)
        assert srv.submit(k, nest, prec, sig, *outs[k]) == lib.SGF_OK
    done = _drain(srv, len(reqs))
    assert all(d["status"] == lib.SGF_OK for d in done), done
    stats = srv.stats()
    srv.close()
    return outs, done, stats


def _alone(reqs):
    lib = sgf()
    srv = lib.Server(max_inflight=1)
    outs = {}
    for k, (nest, sig, prec) in enumerate(reqs):
        outs[k] = _outputs(nest)
        assert srv.submit(k, nest, prec, sig, *outs[k]) == lib.SGF_OK
        d = _drain(srv, 1)
        assert d[0]["status"] == lib.SGF_OK
    srv.close()
    return outs


@pytest.fixture(scope="module")
def reqs():
    return _requests(24, 11)


@pytest.fixture(scope="module")
def alone(reqs):
    return _alone(reqs)


def test_alone_vs_mixed_bitwise(reqs, alone):
    mixed, done, stats = _mixed(reqs, budget=8 << 30, inflight=4)
    assert stats["inflight_peak"] > 1, "requests never overlapped"
    assert stats["shapes_built"] == len({(n.n, n.levels) for n, _, _ in reqs})
    for k in range(len(reqs)):
        for l in range(reqs[k][0].levels):
            assert np.array_equal(mixed[k][0][l], alone[k][0][l]), (k, l)
            assert np.array_equal(mixed[k][1][l], alone[k][1][l]), (k, l)


def test_mixed_under_eviction(reqs, alone):
    """A budget that holds about one large shape forces slot evictions and spectra
    rebuilds; the results do not change."""
    lib = sgf()
    big = max(lib.estimate(n, "fp32")["spectra_bytes"] + lib.estimate(n, "fp32")["build_bytes"]
              for n, _, _ in reqs)
    mixed, done, stats = _mixed(reqs, budget=int(1.5 * big), inflight=3)
    assert stats["slots_evicted"] > 0
    assert stats["bytes_peak"] <= stats["hbm_budget"]
    for k in range(len(reqs)):
        for l in range(reqs[k][0].levels):
            assert np.array_equal(mixed[k][0][l], alone[k][0][l]), (k, l)
            assert np.array_equal(mixed[k][1][l], alone[k][1][l]), (k, l)


def test_served_results_match_plan_and_oracle(reqs, alone):
    lib = sgf()
    for k in (0, 1, 2):
        nest, sig, prec = reqs[k]
        plan = lib.Plan(nest, prec)
        fx, fy = plan.solve_host([np.asarray(s) for s in sig])
        plan.close()
        for l in range(nest.levels):
            assert np.array_equal(fx[l], alone[k][0][l]) and np.array_equal(fy[l], alone[k][1][l])
    for k in range(len(reqs)):
        nest, sig, prec = reqs[k]
        if nest.n <= 64:
            ox, oy = oracle.force(nest, [np.asarray(s, dtype=np.float64) for s in sig])
            errs = rel_linf_levels(nest, alone[k][0], alone[k][1], ox, oy)
            assert max(errs) <= tol(prec, nest.n), (k, errs)


def test_poisson_stream_small():
    lib = sgf()
    arr = serving.poisson_arrivals(300.0, 1.0, 5, (64, 128, 256), (1, 3), ("fp32", "bf16x"))
    pools = serving.make_pools({(a.n, a.levels, a.precision) for a in arr}, seed=2)
    srv = lib.Server(hbm_budget=16 << 30, max_inflight=4)
    recs, _ = serving.run_stream(srv, arr, pools, max_seconds=120.0)
    s = serving.summarize(recs, 1.0)
    assert s["completed"] == len(arr) and s["failed"] == 0
    assert 0 < s["p50_ms"] <= s["p99_ms"]
    srv.close()
