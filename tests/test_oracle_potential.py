"""Pins of the oracle's potential (G = 1) of the linear-density cells (Sec. 2.1):

  Phi(t) = - sum_c Int_c [sig_c + dx_c (xb - x_c) + dy_c (yb - y_c)] / r.

Checked against: brute-force quadrature of each cell integral (scipy dblquad;
the cell that contains the target in polar coordinates), the closed-form
potential of the Maclaurin disk with second-order convergence, the oracle's
own force as the negative gradient (an independent code path of the same
density), and symmetry.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1603_03142_gb300 import workloads as W

integrate = pytest.importorskip("scipy.integrate")


CELLS = [(0.3, 1.1, 0.2, 0.9), (-2.5, -1.5, 0.5, 1.5), (1.0, 2.0, -3.0, -2.0), (-0.5, 0.5, 2.0, 3.0),
         (0.0, 1.0, 0.0, 1.0)]


@pytest.mark.parametrize("cell", CELLS)
def test_cell_integrals_vs_quadrature(cell):
    a, b, c, d = cell
    got = oracle.cell_integrals_potential(a, b, c, d)
    opts = dict(epsabs=1e-13, epsrel=1e-12)
    ref = [integrate.dblquad(f, a, b, c, d, **opts)[0] for f in (
        lambda v, u: 1.0 / math.hypot(u, v),
        lambda v, u: u / math.hypot(u, v),
        lambda v, u: v / math.hypot(u, v))]
    np.testing.assert_allclose(got, ref, rtol=1e-9, atol=1e-11)


def _rect_polar(A, B):
    """Int over [0,A]x[0,B] of 1/r by polar quadrature: Int R(theta) dtheta."""
    t0 = math.atan2(B, A)
    f1 = integrate.quad(lambda t: A / math.cos(t), 0.0, t0, epsabs=1e-14, epsrel=1e-13)[0]
    f2 = integrate.quad(lambda t: B / math.sin(t), t0, math.pi / 2, epsabs=1e-14, epsrel=1e-13)[0]
    return f1 + f2


@pytest.mark.parametrize("cell", [(-0.5, 0.5, -0.5, 0.5), (-0.2, 0.8, -0.7, 0.3)])
def test_cell_containing_target_polar(cell):
    """The self cell: 1/r is integrable; split at the target into four rectangles
    with a corner there.  u/r and v/r: quadrature is smooth enough."""
    a, b, c, d = cell
    ref0 = _rect_polar(b, d) + _rect_polar(-a, d) + _rect_polar(b, -c) + _rect_polar(-a, -c)
    got = oracle.cell_integrals_potential(a, b, c, d)
    assert abs(got[0] - ref0) <= 1e-11 * abs(ref0)
    refx = integrate.dblquad(lambda v, u: u / math.hypot(u, v) if (u or v) else 0.0, a, b, c, d,
                             epsabs=1e-12, epsrel=1e-11)[0]
    assert abs(got[1] - refx) <= 1e-9


def test_unit_square_closed_form():
    """Int over [-1/2,1/2]^2 of 1/r = 4 asinh(1) (= 8 a asinh(1) for half-width a)."""
    assert abs(oracle.cell_integrals_potential(-0.5, 0.5, -0.5, 0.5)[0] - 4.0 * math.asinh(1.0)) < 1e-14


def _maclaurin_phi(r, a, s0=1.0):
    """Potential inside the generalized Maclaurin disk s0 sqrt(1 - r^2/a^2), G = 1."""
    return -(math.pi ** 2) * s0 / (4.0 * a) * (2.0 * a * a - r * r)


def test_maclaurin_second_order():
    a = 0.8
    errs = []
    for n in (32, 64, 128):
        nest, sigma = W.config1(n)
        phi = oracle.potential(nest, sigma)[0]
        h = nest.h0
        x = nest.x0 + (np.arange(n) + 0.5) * h
        X, Y = np.meshgrid(x, x)
        R = np.hypot(X, Y)
        inside = R < 0.7 * a
        exact = _maclaurin_phi(R[inside], a)
        errs.append(np.abs(phi[inside] - exact).max() / np.abs(exact).max())
    # the density's slope is singular at the rim, so single doublings of N
    # oscillate about order 2; the order over two doublings is clean
    assert errs[-1] < 1e-4, errs
    order = 0.5 * math.log2(errs[0] / errs[2])
    assert order > 1.8, (errs, order)


def test_negative_gradient_is_the_force():
    """Central difference of Phi against the oracle's force of the same nest and
    density: the mismatch is the O(h^2) error of the difference quotient."""
    rel = []
    for n in (32, 64):
        nest = W.Nest(n=n, levels=1, off=[(0, 0)])
        x = nest.x0 + (np.arange(n) + 0.5) * nest.h0
        X, Y = np.meshgrid(x, x)
        sig = [np.exp(-((X - 0.1) ** 2 + (Y + 0.05) ** 2) / (2 * 0.25 ** 2))]
        phi = oracle.potential(nest, sig)[0]
        fx, fy = oracle.force(nest, sig)
        h = nest.h0
        gx = -(phi[:, 2:] - phi[:, :-2]) / (2 * h)
        gy = -(phi[2:, :] - phi[:-2, :]) / (2 * h)
        inner = (slice(n // 4, 3 * n // 4), slice(n // 4, 3 * n // 4))
        sx = fx[0][:, 1:-1][inner]
        sy = fy[0][1:-1, :][inner]
        scale = max(np.abs(fx[0]).max(), np.abs(fy[0]).max())
        rel.append(max(np.abs(gx[inner] - sx).max(), np.abs(gy[inner] - sy).max()) / scale)
    assert rel[0] < 2e-2 and rel[1] < rel[0] / 3.0, rel


def test_sign_symmetry_and_nest_covered_cells():
    nest = W.Nest(n=32, levels=2, off=[(0, 0), (8, 8)])
    rng = np.random.Generator(np.random.PCG64(4))
    s0 = rng.uniform(0.2, 1.0, (32, 32))
    sig = [0.5 * (s0 + s0[:, ::-1]), np.full((32, 32), 0.7)]
    phi = oracle.potential(nest, sig)
    cov = nest.covered_mask(0)
    assert np.all(phi[0][cov] == 0.0)
    assert np.all(phi[0][~cov] < 0.0) and np.all(phi[1] < 0.0)
    # the level-1 patch is centred and uniform, so the mirror x -> -x is a symmetry
    np.testing.assert_allclose(phi[0], phi[0][:, ::-1], rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(phi[1], phi[1][:, ::-1], rtol=1e-11, atol=1e-12)
