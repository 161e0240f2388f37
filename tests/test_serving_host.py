"""Host logic of the request loop (sgf_server_*), with SGF_SERVER_SIMULATE: no
GPU and no CUDA call, every request "runs" for its modelled bytes / rate.

Checks the admission contract of include/sgf.h: arrival order, at most
max_inflight on the device, device memory never above the budget, spectra
reused per shape, least-recently-used idle slots evicted under pressure,
requests that can never fit rejected at submit, and continuous admission
(a request that arrives while others run starts before they all finish).
Also pins the footprint estimate and the driver's summary arithmetic.
"""
import time

import numpy as np
import pytest

from paper_1603_03142_gb300 import serving, sgf
from paper_1603_03142_gb300 import workloads as W


def _arrays(n, L):
    return [np.zeros((n, n), np.float32) for _ in range(L)]


def _drain(srv, want, timeout=10.0):
    done, t0 = [], time.time()
    while len(done) < want:
        done += srv.progress()
        st = srv.stats()
        assert st["bytes_used"] <= st["hbm_budget"]
        assert st["inflight"] <= st["inflight_peak"]
        assert time.time() - t0 < timeout, "simulated requests did not finish"
        time.sleep(1e-4)
    return done


def test_estimate_matches_formula():
    """Spectra of a uniform FP32 level: 6 quarter-stored real tables of (N+1) x (N+8)
    (one 256-byte aligned set); generator: 6 P^2 doubles + 6 (N+1) P double2 + P double2
    (P = 2N)."""
    n = 256
    e = sgf.estimate(W.Nest(n=n, levels=1, off=[(0, 0)]), "fp32")
    assert e["spectra_bytes"] == (6 * (n + 1) * (n + 8) * 4 + 255) // 256 * 256
    P = 2 * n
    assert e["build_bytes"] == 6 * P * P * 8 + 6 * (n + 1) * P * 16 + P * 16
    # forward slabs (3 fields of (N+1) x N complex) and backward (2 fields) dominate the workspace
    inter = (3 + 2) * (n + 1) * n * 8
    assert inter <= e["workspace_bytes"] <= inter + 64 * 1024
    # deeper nests cost more spectra (Case-2/3 phases)
    e2 = sgf.estimate(W.centred_nest(n, 2), "fp32")
    assert e2["spectra_bytes"] > 2 * e["spectra_bytes"]


def test_fifo_inflight_and_reuse():
    srv = sgf.Server(hbm_budget=4 << 30, max_inflight=3, simulate_gbs=80.0)
    shapes = [(256, 2), (256, 3), (512, 2), (256, 2), (256, 3), (512, 2), (256, 2), (128, 2)]
    for i, (n, L) in enumerate(shapes):
        assert srv.submit(i, W.centred_nest(n, L), "fp32", _arrays(n, L), _arrays(n, L), _arrays(n, L)) == 0
    done = _drain(srv, len(shapes))
    st = srv.stats()
    assert st["inflight_peak"] == 3
    assert st["completed"] == len(shapes) and all(d["status"] == 0 for d in done)
    admits = {d["id"]: d["t_admit"] for d in done}
    assert all(admits[i] <= admits[i + 1] for i in range(len(shapes) - 1)), "admission out of arrival order"
    assert st["shapes_built"] == 4  # one spectra build per distinct shape
    assert sum(d["built_shape"] for d in done) == 4
    assert st["bytes_peak"] <= st["hbm_budget"]
    srv.close()


def test_eviction_under_pressure():
    a, b = W.centred_nest(256, 3), W.centred_nest(512, 2)
    ea, eb = sgf.estimate(a, "fp32"), sgf.estimate(b, "fp32")
    io = lambda n, L: 3 * L * n * n * 4
    worst = max(ea["workspace_bytes"] + ea["spectra_bytes"] + ea["build_bytes"] + io(256, 3),
                eb["workspace_bytes"] + eb["spectra_bytes"] + eb["build_bytes"] + io(512, 2))
    budget = worst + (1 << 20)  # room for one shape at a time
    srv = sgf.Server(hbm_budget=budget, max_inflight=2, simulate_gbs=200.0)
    order = [a, b, a, b, a]
    for i, nest in enumerate(order):
        n, L = nest.n, nest.levels
        assert srv.submit(i, nest, "fp32", _arrays(n, L), _arrays(n, L), _arrays(n, L)) == 0
    done = _drain(srv, len(order))
    st = srv.stats()
    assert all(d["status"] == 0 for d in done)
    assert st["slots_evicted"] >= 4 and st["shapes_built"] == 5
    assert st["bytes_peak"] <= budget
    assert st["shapes_resident"] == 1
    srv.close()


def test_reject_never_fits():
    nest = W.centred_nest(1024, 3)
    e = sgf.estimate(nest, "fp32")
    srv = sgf.Server(hbm_budget=e["spectra_bytes"] // 2, max_inflight=2, simulate_gbs=100.0)
    st = srv.submit(1, nest, "fp32", _arrays(1024, 3), _arrays(1024, 3), _arrays(1024, 3))
    assert st == sgf.SGF_ENOMEM
    s = srv.stats()
    assert s["rejected"] == 1 and s["submitted"] == 0 and s["queued"] == 0
    # a small request still goes through
    small = W.centred_nest(64, 2)
    assert srv.submit(2, small, "fp32", _arrays(64, 2), _arrays(64, 2), _arrays(64, 2)) == 0
    assert [d["id"] for d in _drain(srv, 1)] == [2]
    srv.close()


def test_bad_requests():
    srv = sgf.Server(hbm_budget=1 << 30, max_inflight=1, simulate_gbs=100.0)
    with pytest.raises(ValueError):
        srv.submit(0, W.centred_nest(64, 2), "fp32", _arrays(64, 1), _arrays(64, 2), _arrays(64, 2))
    with pytest.raises(sgf.SgfError):  # n odd
        srv.submit(0, W.Nest(n=47, levels=1, off=[(0, 0)]), "fp32", _arrays(47, 1), _arrays(47, 1), _arrays(47, 1))
    with pytest.raises(sgf.SgfError):
        sgf.Server(hbm_budget=1 << 30, max_inflight=0, simulate_gbs=1.0)
    with pytest.raises(sgf.SgfError):
        sgf.Server(hbm_budget=0, max_inflight=1, simulate_gbs=1.0)  # a simulation needs a budget
    srv.close()


def test_continuous_admission():
    """A request arriving while a long one runs starts (in a free slot) before it ends."""
    srv = sgf.Server(hbm_budget=8 << 30, max_inflight=2, simulate_gbs=2.0)
    big, small = W.centred_nest(512, 3), W.centred_nest(64, 2)
    assert srv.submit(0, big, "fp32", _arrays(512, 3), _arrays(512, 3), _arrays(512, 3)) == 0
    srv.progress()
    time.sleep(0.01)
    assert srv.submit(1, small, "fp32", _arrays(64, 2), _arrays(64, 2), _arrays(64, 2)) == 0
    done = _drain(srv, 2, timeout=30.0)
    d = {x["id"]: x for x in done}
    assert d[1]["t_admit"] < d[0]["t_done"] and d[1]["t_done"] < d[0]["t_done"]
    assert srv.stats()["inflight_peak"] == 2
    srv.close()


def test_poisson_arrivals_seeded():
    a = serving.poisson_arrivals(200.0, 5.0, 0, (256, 512), (2, 3))
    b = serving.poisson_arrivals(200.0, 5.0, 0, (256, 512), (2, 3))
    assert [(x.t, x.n, x.levels) for x in a] == [(x.t, x.n, x.levels) for x in b]
    assert 800 < len(a) < 1200  # 1000 expected
    gaps = np.diff([0.0] + [x.t for x in a])
    assert abs(np.mean(gaps) - 1 / 200.0) < 0.15 / 200.0
    assert {x.n for x in a} == {256, 512} and {x.levels for x in a} == {2, 3}


def test_percentile_and_summary():
    assert serving.percentile([3.0, 1.0, 2.0, 4.0], 50) == 2.0
    assert serving.percentile(list(range(1, 101)), 99) == 99.0
    assert serving.percentile([5.0], 99) == 5.0
    recs = [serving.Record(i, 64, 2, "fp32", t_arrival=0.1 * i, status=0, t_admit=0.1 * i, t_done=0.1 * i + 0.01 * (i + 1))
            for i in range(10)]
    recs.append(serving.Record(10, 64, 2, "fp32", t_arrival=1.0, status=sgf.SGF_ENOMEM))
    s = serving.summarize(recs, duration=1.1)
    assert s["completed"] == 10 and s["rejected"] == 1
    assert abs(s["p50_ms"] - 50.0) < 1e-9 and abs(s["max_ms"] - 100.0) < 1e-9
    assert s["cells"] == 10 * 64 * 64 * 2


def test_stream_driver_simulated():
    """The open-loop driver against a simulating server: every request completes,
    latency >= 0, and requests that can never fit are counted as rejected."""
    arr = serving.poisson_arrivals(400.0, 0.25, 3, (64, 128), (1, 2))
    pools = serving.make_pools({(a.n, a.levels, a.precision) for a in arr}, seed=1)
    srv = sgf.Server(hbm_budget=2 << 30, max_inflight=3, simulate_gbs=500.0)
    recs, _ = serving.run_stream(srv, arr, pools, max_seconds=30.0)
    assert len(recs) == len(arr) and all(r.status == 0 for r in recs)
    assert all(r.latency >= 0 and r.t_admit >= r.t_arrival - 1e-3 for r in recs)
    s = serving.summarize(recs, 0.25)
    assert s["completed"] == len(arr) and s["p99_ms"] >= s["p50_ms"]
    srv.close()


def test_bf16x_limits():
    """SGF_BF16X takes FP32-sized buffers; nests of n = 4096 are refused (the
    inverse row kernel has no shared memory left for the tensor-core tiles)."""
    e32 = sgf.estimate(W.centred_nest(256, 2), "fp32")
    eb = sgf.estimate(W.centred_nest(256, 2), "bf16x")
    assert e32 == eb
    assert sgf.estimate(W.Nest(n=4096, levels=1, off=[(0, 0)]), "bf16x")["spectra_bytes"] > 0
    with pytest.raises(sgf.SgfError) as ei:
        sgf.estimate(W.centred_nest(4096, 2), "bf16x")
    assert ei.value.status == sgf.SGF_EUNSUPPORTED


def test_fp32_and_bf16x_share_spectra():
    """FP32 and BF16X requests of one shape hold one set of FP32 spectra."""
    srv = sgf.Server(hbm_budget=4 << 30, max_inflight=2, simulate_gbs=100.0)
    nest = W.centred_nest(256, 2)
    for i, prec in enumerate(["fp32", "bf16x", "fp32", "bf16x"]):
        assert srv.submit(i, nest, prec, _arrays(256, 2), _arrays(256, 2), _arrays(256, 2)) == 0
    _drain(srv, 4)
    st = srv.stats()
    assert st["shapes_built"] == 1 and st["shapes_resident"] == 1 and st["slots"] == 2
    srv.close()


def test_max_shape_bytes_rejects_large_shapes():
    big, small = W.centred_nest(1024, 3), W.centred_nest(128, 2)
    eb = sgf.estimate(big, "fp32")
    cap = eb["spectra_bytes"] + eb["build_bytes"] - 1
    srv = sgf.Server(hbm_budget=64 << 30, max_inflight=2, simulate_gbs=100.0, max_shape_bytes=cap)
    assert srv.submit(0, big, "fp32", _arrays(1024, 3), _arrays(1024, 3), _arrays(1024, 3)) == sgf.SGF_ENOMEM
    assert "max_shape_bytes" in sgf.last_error()
    assert srv.submit(1, small, "fp32", _arrays(128, 2), _arrays(128, 2), _arrays(128, 2)) == 0
    assert [d["id"] for d in _drain(srv, 1)] == [1]
    assert srv.stats()["rejected"] == 1
    srv.close()
