"""Host logic of forest plans (several patches per level), no GPU: the
descriptor rules agree with the oracle's, a nest and the forest of its levels
give the same plan, and the spectra footprint counts one set per distinct
(case, ratio, phase, lattice offset) of the patch pairs."""
import numpy as np
import pytest

import oracle
from paper_1603_03142_gb300 import sgf
from paper_1603_03142_gb300 import workloads as W


def _al(b):
    return (b + 255) // 256 * 256


def _sets(f):
    """Distinct spectra sets of the patch pairs (Sec. 2.2 Cases 1-3): Case 1 of a
    patch with itself is one shared set; other same-level pairs differ by their
    lattice offset; Cases 2 and 3 by ratio, phase and offset."""
    quarter, full = set(), set()
    for t in range(f.patches):
        for s in range(f.patches):
            ls, lt = f.level[s], f.level[t]
            if s == t:
                quarter.add(1)
            elif ls == lt:
                full.add(("offset", f.org[s][0] - f.org[t][0], f.org[s][1] - f.org[t][1]))
            elif ls > lt:
                m = 1 << (ls - lt)
                A = (f.org[s][0] - m * f.org[t][0], f.org[s][1] - m * f.org[t][1])
                full.update(("c2", m, px, py, A) for px in range(m) for py in range(m))
            else:
                m = 1 << (lt - ls)
                A = (f.org[t][0] - m * f.org[s][0], f.org[t][1] - m * f.org[s][1])
                full.update(("c3", m, px, py, A) for px in range(m) for py in range(m))
    return len(quarter), len(full)


@pytest.mark.parametrize("make", [W.example3_forest, W.example4_forest, W.two_patch_forest])
def test_spectra_bytes_count_distinct_pairs(make):
    n = 16
    f = make(n)
    nq, nf = _sets(f)
    e = sgf.estimate(f, "fp32")
    assert e["spectra_bytes"] == nq * _al(6 * (n + 1) * (n + 8) * 4) + nf * _al(6 * (n + 1) * 2 * n * 8)


@pytest.mark.parametrize("case", [(16, 3, [(0, 0), (3, 5), (4, 2)]), (64, 2, [(0, 0), (16, 16)])])
def test_nest_and_its_forest_estimate_alike(case):
    n, L, off = case
    nest = W.Nest(n=n, levels=L, off=off)
    for flags in (0, sgf.PLAN_POTENTIAL):
        assert sgf.estimate(nest, "fp32", flags) == sgf.estimate(W.Forest.from_nest(nest), "fp32", flags)


FORESTS = [
    ([0, 1], [(0, 0), (4, 6)], True),
    ([0, 1], [(0, 0), (3, 4)], False),           # odd corner
    ([0, 0], [(0, 0), (8, 0)], False),           # overlapping roots
    ([0, 0], [(0, 0), (16, 0)], True),           # touching roots
    ([0, 1], [(0, 0), (20, 0)], False),          # child partly outside the root
    ([0, 0, 1], [(0, 0), (16, 0), (24, 8)], True),   # child straddling two roots
    ([0, 0, 1], [(0, 0), (32, 0), (24, 8)], False),  # straddling a gap
    ([1, 0], [(0, 0), (0, 0)], False),           # finer patch first
    ([0, 2], [(0, 0), (0, 0)], False),           # skipped level
    ([0, 1, 1], [(0, 0), (0, 0), (16, 16)], True),
    ([0, 1, 1], [(0, 0), (0, 0), (8, 8)], False),  # overlapping level-1 patches
]


@pytest.mark.parametrize("level,org,valid", FORESTS)
def test_rules_agree_with_the_oracle(level, org, valid):
    f = W.Forest(n=16, level=level, org=org)
    assert oracle.validate(f) == valid
    if valid:
        sgf.estimate(f, "fp32")
    else:
        with pytest.raises(sgf.SgfError) as ei:
            sgf.estimate(f, "fp32")
        assert ei.value.status == sgf.SGF_EINVAL


def test_flags_on_forests():
    f = W.two_patch_forest(16)
    with pytest.raises(sgf.SgfError) as ei:
        sgf.estimate(f, "fp32", flags=sgf.PLAN_ZERO_RIM)
    assert ei.value.status == sgf.SGF_EINVAL
    ep = sgf.estimate(f, "fp32", flags=sgf.PLAN_POTENTIAL)
    assert ep["spectra_bytes"] < sgf.estimate(f, "fp32")["spectra_bytes"]
    with pytest.raises(sgf.SgfError) as ei:
        sgf.estimate(W.Forest(n=4096, level=[0, 0], org=[(0, 0), (4096, 0)]), "bf16x")
    assert ei.value.status == sgf.SGF_EUNSUPPORTED
