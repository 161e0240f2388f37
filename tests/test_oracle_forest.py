"""Pins of the oracle on forests: several patches per level (Sec. 2.1, Omega^l_k).

- Table 3 of Sec. 3 (Example 3, two disks on two levels with two level-1
  patches): the printed L1, L2, L-infinity errors to four digits.
- A one-patch-per-level nest written as a forest gives bit-identical forces
  and potential (the forest code reduces to the pinned nest code).
- A linear density is integrated exactly by any covering, so splitting the
  root into tiles, or refining any part of it (including a patch that
  straddles several tiles), leaves the force at every common cell centre
  unchanged to rounding.
- Second-order convergence on the three-level two-disk forest (Example 4's
  finest patches), against the closed-form D_5 forces.
- The validity rules (ordering, alignment, overlap, nesting).
"""
import math

import numpy as np
import pytest

import oracle
from oracle import analytic
from paper_1603_03142_gb300 import workloads as W
from tests._golden import error_table
from tests.test_oracle_paper_tables import assert_printed

ALPHA = math.sqrt(2.0) / 4.0


def two_disk_errors(forest, inside_only=True):
    sig = W.two_disk_density(forest)
    fx, fy = oracle.force(forest, sig)
    ex, ey = [], []
    for p in range(forest.patches):
        X, Y = forest.centres(p)
        ax = ay = 0.0
        for cx in (-0.5, 0.5):
            a, b = analytic.force_dn_xy(X, Y, 5, ALPHA, cx=cx)
            ax, ay = ax + a, ay + b
        keep = ~forest.covered_mask(p)
        if inside_only:
            keep &= (np.abs(X) < 1.0) & (np.abs(Y) < 1.0)
        ex.append(np.abs(fx[p] - ax)[keep])
        ey.append(np.abs(fy[p] - ay)[keep])
    ex, ey = np.concatenate(ex), np.concatenate(ey)
    return np.array([ex.mean(), np.sqrt((ex ** 2).mean()), ex.max(), ey.mean(), np.sqrt((ey ** 2).mean()), ey.max()])


@pytest.mark.parametrize("N", [32, 64])
def test_table3_example3(N):
    f = W.example3_forest(N // 2)
    assert oracle.validate(f)
    assert_printed(two_disk_errors(f), error_table("table3_example3.txt")[N])


@pytest.mark.parametrize("case", [(16, 3, [(0, 0), (3, 5), (4, 2)]), (32, 2, [(0, 0), (16, 0)]),
                                  (16, 4, [(0, 0), (4, 4), (0, 8), (8, 2)])])
def test_nest_as_forest_is_bit_identical(case):
    n, L, off = case
    nest = W.Nest(n=n, levels=L, off=off)
    forest = W.Forest.from_nest(nest)
    rng = np.random.Generator(np.random.PCG64(n + L))
    sigma = [rng.uniform(0.1, 1.0, (n, n)) for _ in range(L)]
    fx, fy = oracle.force(nest, sigma)
    gx, gy = oracle.force(forest, sigma)
    pa, pb = oracle.potential(nest, sigma), oracle.potential(forest, sigma)
    for l in range(L):
        assert np.array_equal(fx[l], gx[l]) and np.array_equal(fy[l], gy[l])
        assert np.array_equal(pa[l], pb[l])
        assert np.array_equal(nest.covered_mask(l), forest.covered_mask(l))


def _linear(forest, p):
    X, Y = forest.centres(p)
    return 0.7 + 0.3 * X - 0.2 * Y


def test_linear_density_any_covering():
    n = 16
    # one root of 2n cells over [-1, 1]^2, and the same root as 2 x 2 tiles of n
    nest = W.Nest(n=2 * n, levels=1, x0=-1.0, y0=-1.0, h0=1.0 / n)
    tiles = W.Forest(n=n, level=[0] * 4, org=[(0, 0), (n, 0), (0, n), (n, n)], h0=1.0 / n)
    # the tiles plus a level-1 patch straddling all four (its corner at the centre minus n/4 tiles cells)
    refined = W.Forest(n=n, level=[0] * 4 + [1], org=tiles.org + [(3 * n // 2, 3 * n // 2)], h0=1.0 / n)
    assert oracle.validate(tiles) and oracle.validate(refined)
    for p in range(4):
        assert refined.covered_mask(p).sum() == (n // 4) ** 2  # a quarter of the child over each tile
    sn = [_linear(nest, 0)]
    fxn, fyn = oracle.force(nest, sn)
    ft = oracle.force(tiles, [_linear(tiles, p) for p in range(4)])
    fr = oracle.force(refined, [_linear(refined, p) for p in range(5)])
    scale = np.abs(fxn[0]).max()
    for p in range(4):
        ox, oy = tiles.org[p]
        sx = fxn[0][oy:oy + n, ox:ox + n]
        sy = fyn[0][oy:oy + n, ox:ox + n]
        assert np.abs(ft[0][p] - sx).max() <= 1e-12 * scale
        assert np.abs(ft[1][p] - sy).max() <= 1e-12 * scale
        keep = ~refined.covered_mask(p)
        assert np.abs(fr[0][p] - sx)[keep].max() <= 1e-12 * scale
        assert np.abs(fr[1][p] - sy)[keep].max() <= 1e-12 * scale
        assert np.all(fr[0][p][~keep] == 0.0)
    # the child's cell centres (its corner at (-1/4, -1/4), cell 1/(2n)) are the first n x n
    # centres of the fine level of a two-level nest with the same corner: again the exact
    # force of the linear density on [-1, 1]^2
    nest2 = W.Nest(n=2 * n, levels=2, x0=-1.0, y0=-1.0, h0=1.0 / n, off=[(0, 0), (3 * n // 4, 3 * n // 4)])
    assert np.allclose(nest2.origin(1), refined.origin(4))
    fx2, fy2 = oracle.force(nest2, [_linear(nest2, 0), _linear(nest2, 1)])
    assert np.abs(fr[0][4] - fx2[1][:n, :n]).max() <= 1e-12 * scale
    assert np.abs(fr[1][4] - fy2[1][:n, :n]).max() <= 1e-12 * scale


def test_example4_forest_second_order():
    """Three levels, two patches on each refined level (Example 4's level-2 patches)."""
    errs = [two_disk_errors(W.example4_forest(n)) for n in (16, 32)]
    order = np.log2(errs[0] / errs[1])
    assert np.all(order[[0, 1, 3, 4]] > 1.8), order
    assert np.all(order[[2, 5]] > 1.6), order


@pytest.mark.parametrize("level,org,why", [
    ([0, 1], [(0, 0), (3, 4)], "odd corner"),
    ([0, 0], [(0, 0), (8, 0)], "overlapping roots"),
    ([0, 1], [(0, 0), (20, 0)], "child outside the root"),
    ([1, 0], [(0, 0), (0, 0)], "finer patch first"),
    ([0, 2], [(0, 0), (0, 0)], "skipped level"),
])
def test_invalid_forests(level, org, why):
    assert not oracle.validate(W.Forest(n=16, level=level, org=org)), why


def test_touching_patches_are_valid():
    f = W.two_patch_forest(16)
    assert oracle.validate(f)
    assert f.covered_mask(0).sum() == 2 * 8 * 8
