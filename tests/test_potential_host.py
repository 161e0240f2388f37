"""Host logic of potential plans (SGF_PLAN_POTENTIAL), no GPU: the spectra
footprint (three tables per set, one Case-1 set per level since the tables
carry the finer cell size), the flag rules, and the refusals of the force-only
entry points that need no device."""
import numpy as np
import pytest

from paper_1603_03142_gb300 import sgf
from paper_1603_03142_gb300 import workloads as W


def _al(b):
    return (b + 255) // 256 * 256


def test_estimate_uniform_half_of_forces():
    n = 256
    nest = W.Nest(n=n, levels=1, off=[(0, 0)])
    ef = sgf.estimate(nest, "fp32")
    ep = sgf.estimate(nest, "fp32", flags=sgf.PLAN_POTENTIAL)
    assert ep["spectra_bytes"] == _al(3 * (n + 1) * (n + 8) * 4)
    assert ef["spectra_bytes"] == _al(6 * (n + 1) * (n + 8) * 4)
    # same intermediates: three forward fields, two backward components
    assert ep["workspace_bytes"] == ef["workspace_bytes"]


@pytest.mark.parametrize("prec,esize", [("fp32", 4), ("fp64", 8)])
def test_estimate_two_level_sets(prec, esize):
    """Two levels: one quarter set per level (the cell size differs), 4 Case-2 and
    4 Case-3 phase sets of three complex tables of (N+1) x 2N."""
    n = 64
    nest = W.centred_nest(n, 2)
    ep = sgf.estimate(nest, prec, flags=sgf.PLAN_POTENTIAL)
    q = _al(3 * (n + 1) * (n + 8) * esize)
    f = _al(3 * (n + 1) * 2 * n * 2 * esize)
    assert ep["spectra_bytes"] == 2 * q + 8 * f


@pytest.mark.parametrize("nest,flags", [(W.Nest(n=64, levels=1, off=[(0, 0)]), 0x4),
                                        (W.centred_nest(64, 2), sgf.PLAN_POTENTIAL | sgf.PLAN_ZERO_RIM)])
def test_flag_rules(nest, flags):
    with pytest.raises(sgf.SgfError) as ei:
        sgf.estimate(nest, "fp32", flags=flags)
    assert ei.value.status == sgf.SGF_EINVAL


def test_zero_rim_potential_one_merged_table():
    n = 256
    e = sgf.estimate(W.Nest(n=n, levels=1, off=[(0, 0)]), "fp32", flags=sgf.PLAN_POTENTIAL | sgf.PLAN_ZERO_RIM)
    assert e["spectra_bytes"] == _al(1 * (n + 1) * (n + 8) * 4)


def test_request_loop_refuses_potential():
    srv = sgf.Server(hbm_budget=1 << 30, max_inflight=1, simulate_gbs=50.0)
    a = [np.zeros((64, 64), np.float32)]
    with pytest.raises(sgf.SgfError) as ei:
        srv.submit(0, W.Nest(n=64, levels=1, off=[(0, 0)]), "fp32", a, a, a, plan_flags=sgf.PLAN_POTENTIAL)
    assert ei.value.status == sgf.SGF_EUNSUPPORTED and "POTENTIAL" in str(ei.value)
    srv.close()
