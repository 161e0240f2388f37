"""oracle.force_row / force_col: the direct sum of oracle.force_at evaluated for
many targets of one row (or column) of a single-level grid, with the cell
integrals shared across the row's targets.  Pinned to force_at, which the paper's
Tables 1-3 and 5, the quadrature pins and the invariants pin in their turn."""
import numpy as np
import pytest

import oracle
from paper_1603_03142_gb300 import workloads as W


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("n", [32, 24])
def test_force_row_equals_direct_targets(n):
    nest = W.Nest(n=n)
    rng = np.random.Generator(np.random.PCG64(n))
    sigma = [rng.uniform(0.1, 2.0, (n, n))]
    for jt in (0, 5, n - 1):
        ii = np.arange(n)
        rx, ry = oracle.force_row(nest, sigma, jt)
        dx, dy = oracle.force_at(nest, sigma, np.zeros(n, int), ii, np.full(n, jt))
        scale = max(np.abs(dx).max(), np.abs(dy).max())
        assert max(np.abs(rx - dx).max(), np.abs(ry - dy).max()) <= 1e-13 * scale, jt


def test_force_row_subset_and_order():
    nest = W.Nest(n=32)
    rng = np.random.Generator(np.random.PCG64(3))
    sigma = [rng.uniform(0.1, 2.0, (32, 32))]
    ii = np.array([31, 0, 7, 7, 16])
    rx, ry = oracle.force_row(nest, sigma, 9, ii)
    fx, fy = oracle.force_row(nest, sigma, 9)
    assert np.array_equal(rx, fx[ii]) and np.array_equal(ry, fy[ii])


def test_force_col_equals_direct_targets():
    n = 32
    nest = W.Nest(n=n)
    rng = np.random.Generator(np.random.PCG64(5))
    sigma = [rng.uniform(0.1, 2.0, (n, n))]
    for it in (0, 13, n - 1):
        jj = np.arange(n)
        cx, cy = oracle.force_col(nest, sigma, it)
        dx, dy = oracle.force_at(nest, sigma, np.zeros(n, int), np.full(n, it), jj)
        scale = max(np.abs(dx).max(), np.abs(dy).max())
        assert max(np.abs(cx - dx).max(), np.abs(cy - dy).max()) <= 1e-13 * scale, it


def test_force_row_on_the_tapered_lognormal_grid():
    nest, sigma = W.config3(64, seed=2)  # zero beyond r = 0.95: empty cells skipped
    rx, ry = oracle.force_row(nest, sigma, 32)
    dx, dy = oracle.force_at(nest, sigma, np.zeros(64, int), np.arange(64), np.full(64, 32))
    assert _rel(rx, dx) <= 1e-13 and _rel(ry, dy) <= 1e-13


def test_force_row_refuses_nests():
    rng = np.random.Generator(np.random.PCG64(1))
    nest, sigma = W.random_nest_problem(rng, 32, 2)
    with pytest.raises(ValueError):
        oracle.force_row(nest, sigma, 0)
    with pytest.raises(ValueError):
        oracle.force_row(W.Nest(n=32), [np.ones((32, 32))], 32)
