"""Invariants and special cases the mathematics fixes for the oracle.

- Newton's third law on one level: with sigma zero on the two outer rings the
  x-kernel is odd and the slope operators commute with the even kernels, so
  sum_t sigma_t F(t) vanishes up to round-off.
- Mirror symmetry: sigma even in x about the grid centre makes Fx odd and Fy even.
- Sign: a single positive cell at larger x pulls a target towards +x (G = 1,
  attractive force, Sec. 2.1 sign of -dPhi/dx).
- The density reconstruction (Eq. eqnSigma with the slope reading) is exact for
  linear densities on every level, including patch edges and cells next to a
  covered region, and zero on covered cells.
- D_1 (Maclaurin) disk: the error against the Appendix closed form falls under
  refinement (first derivative of sigma is singular at the rim, so the order is
  below 2, as Sec. 4 notes for D_2).
"""
import numpy as np
import pytest

import oracle
from oracle import analytic
from paper_1603_03142_gb300 import workloads as W


def test_newton_third_law_uniform():
    n = 24
    nest = W.Nest(n=n)
    rng = np.random.Generator(np.random.PCG64(3))
    s = np.zeros((n, n))
    s[2:-2, 2:-2] = rng.uniform(0.1, 2.0, (n - 4, n - 4))
    fx, fy = oracle.force(nest, [s])
    scale = np.sum(np.abs(s * fx[0]))
    assert abs(np.sum(s * fx[0])) < 1e-12 * scale
    assert abs(np.sum(s * fy[0])) < 1e-12 * np.sum(np.abs(s * fy[0]))


def test_mirror_symmetry():
    n = 20
    nest = W.Nest(n=n, levels=2, off=[(0, 0), (5, 3)])
    # level-1 patch spans cells 5..14 of level 0: symmetric about the level-0 centre
    rng = np.random.Generator(np.random.PCG64(4))
    s0 = rng.uniform(0.5, 1.5, (n, n))
    s0 = 0.5 * (s0 + s0[:, ::-1])
    s1 = rng.uniform(0.5, 1.5, (n, n))
    s1 = 0.5 * (s1 + s1[:, ::-1])
    fx, fy = oracle.force(nest, [s0, s1])
    for l in range(2):
        assert np.max(np.abs(fx[l] + fx[l][:, ::-1])) < 1e-12 * np.max(np.abs(fx[l]))
        assert np.max(np.abs(fy[l] - fy[l][:, ::-1])) < 1e-12 * np.max(np.abs(fy[l]))


def test_sign_of_force():
    n = 8
    nest = W.Nest(n=n)
    s = np.zeros((n, n))
    s[3, 6] = 1.0  # mass at larger x than the target (3, 3), same row
    fx, fy = oracle.force_at(nest, [s], [0], [3], [3])
    assert fx[0] > 0.0 and abs(fy[0]) < 1e-14
    s = np.zeros((n, n))
    s[6, 3] = 1.0  # mass at larger y
    fx, fy = oracle.force_at(nest, [s], [0], [3], [3])
    assert fy[0] > 0.0 and abs(fx[0]) < 1e-14


@pytest.mark.parametrize("levels,off", [(1, [(0, 0)]), (2, [(0, 0), (4, 2)]), (3, [(0, 0), (0, 8), (8, 0)])])
def test_linear_density_reconstruction_is_exact(levels, off):
    n = 16
    nest = W.Nest(n=n, levels=levels, off=off)
    a, b, c = 0.7, -1.3, 2.1
    sigma = []
    for l in range(levels):
        X, Y = nest.centres(l)
        sigma.append(a + b * X + c * Y)
    sig, dsx, dsy = oracle.prepare(nest, sigma)
    for l in range(levels):
        cov = nest.covered_mask(l)
        assert np.all(sig[l][cov] == 0) and np.all(dsx[l][cov] == 0) and np.all(dsy[l][cov] == 0)
        np.testing.assert_allclose(dsx[l][~cov], b, rtol=1e-12)
        np.testing.assert_allclose(dsy[l][~cov], c, rtol=1e-12)
        np.testing.assert_allclose(sig[l][~cov], sigma[l][~cov], rtol=1e-14)


def test_restriction_feeds_coarse_slopes():
    """A coarse cell beside the fine patch differences against the mean of the fine children."""
    n = 8
    nest = W.Nest(n=n, levels=2, off=[(0, 0), (2, 2)])
    s0 = np.zeros((n, n))
    s1 = np.zeros((n, n))
    s1[0:2, 0:2] = 4.0  # children of coarse cell (2, 2)
    sig, dsx, dsy = oracle.prepare(nest, [s0, s1])
    h0 = nest.h(0)
    # coarse cell (i=1, j=2) is uncovered; its right neighbour (2, 2) is covered with mean 4
    assert dsx[0][2, 1] == pytest.approx((4.0 - 0.0) / (2 * h0))
    assert dsy[0][1, 2] == pytest.approx((4.0 - 0.0) / (2 * h0))


def test_maclaurin_disk_converges():
    errs = []
    for n in (32, 64, 128):
        nest, sig = W.config1(n)
        fx, fy = oracle.force(nest, sig)
        X, Y = nest.centres(0)
        ax, ay = analytic.force_dn_xy(X, Y, 1, 0.8)
        errs.append(np.mean(np.abs(fx[0] - ax)) + np.mean(np.abs(fy[0] - ay)))
    order = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(order > 1.2), order
    assert errs[-1] < 0.01
