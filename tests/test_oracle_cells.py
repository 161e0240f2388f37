"""Pin the oracle's exact cell integrals and direct sum to brute-force quadrature.

Each cell integral of Sec. 2.1 is checked against scipy's adaptive 2-D
quadrature of the integrand itself (u/r^3, v/r^3, u^2/r^3, v^2/r^3, uv/r^3),
on cells placed as in Case 1 (same level), Case 2 (fine source, coarse target:
the target can sit on a cell's edge line) and Case 3 (coarse source, fine
target) with refinement ratios 2 and 4.  The cell that contains the target is
checked in polar coordinates about the target.  Then the whole force sum on
8x8 grids (one and two levels) is checked against a cell-by-cell quadrature of
the linear density of Eq. (eqnSigma).
"""
import numpy as np
import pytest
from scipy import integrate

import oracle
from paper_1603_03142_gb300 import workloads as W

INTEGRANDS = [
    lambda v, u: u / np.hypot(u, v) ** 3,
    lambda v, u: v / np.hypot(u, v) ** 3,
    lambda v, u: u * u / np.hypot(u, v) ** 3,
    lambda v, u: v * v / np.hypot(u, v) ** 3,
    lambda v, u: u * v / np.hypot(u, v) ** 3,
]


def quad_cell(a, b, c, d):
    return np.array([integrate.dblquad(f, a, b, c, d, epsabs=1e-13, epsrel=1e-12)[0] for f in INTEGRANDS])


# (a, b, c, d) relative to the target; units of the finer cell size
CELLS = [
    # Case 1 neighbours and a far cell (edges at half-integers)
    (0.5, 1.5, -0.5, 0.5), (-1.5, -0.5, 0.5, 1.5), (2.5, 3.5, -4.5, -3.5), (-7.5, -6.5, 6.5, 7.5),
    # Case 2, m = 2 and 4: fine cells with edges on the integer lattice; the
    # coarse target centre sits on an edge line (u = 0 or v = 0 corners)
    (0.0, 1.0, 1.0, 2.0), (-1.0, 0.0, -3.0, -2.0), (2.0, 3.0, 0.0, 1.0), (-5.0, -4.0, 0.0, 1.0),
    (0.0, 1.0, -6.0, -5.0),
    # Case 3, m = 2 and 4: coarse cells two or four fine cells wide
    (0.5, 2.5, -1.5, 0.5), (-3.5, -1.5, 1.5, 3.5), (1.5, 5.5, -2.5, 1.5), (-8.5, -4.5, 3.5, 7.5),
]


@pytest.mark.parametrize("cell", CELLS)
def test_cell_integrals_match_quadrature(cell):
    got = oracle.cell_integrals(*cell)
    ref = quad_cell(*cell)
    np.testing.assert_allclose(got, ref, rtol=1e-10, atol=1e-12)


def _self_cell_u2(half):
    # int over [-half, half]^2 of u^2/r^3 = int_0^{2pi} cos^2(t) R(t) dt, R(t) = half/max(|cos|,|sin|)
    f = lambda t: np.cos(t) ** 2 * half / max(abs(np.cos(t)), abs(np.sin(t)))
    pts = [k * np.pi / 4 for k in range(1, 8)]
    return integrate.quad(f, 0.0, 2 * np.pi, points=pts, epsabs=1e-14, epsrel=1e-13, limit=200)[0]


@pytest.mark.parametrize("half", [0.5, 1.0, 0.125])
def test_self_cell(half):
    got = oracle.cell_integrals(-half, half, -half, half)
    ref = _self_cell_u2(half)
    assert abs(got[0]) < 1e-15 and abs(got[1]) < 1e-15 and abs(got[4]) < 1e-15
    assert got[2] == pytest.approx(ref, rel=1e-12)
    assert got[3] == pytest.approx(ref, rel=1e-12)


def test_printed_slope_kernels_are_not_the_slope_integrals():
    """Reading of Sec. 2.1: the printed K^{x,x} = x K^{x,0} - y ln(x + r) double-differences to
    the integral of -1/r (the potential kernel), and the printed K^{x,y} = y K^{x,0} - r to neither
    slope integral; the oracle uses antiderivatives that differentiate back to u^2/r^3 and uv/r^3."""
    def k0(x, y):
        return -np.log(y + np.hypot(x, y))

    def printed_xx(x, y):
        return x * k0(x, y) - y * np.log(x + np.hypot(x, y))

    def printed_xy(x, y):
        return y * k0(x, y) - np.hypot(x, y)

    def dd(f, a, b, c, d):
        return f(b, d) - f(a, d) - f(b, c) + f(a, c)

    a, b, c, d = 1.5, 2.5, 0.5, 1.5
    ref = quad_cell(a, b, c, d)
    inv_r = integrate.dblquad(lambda v, u: -1.0 / np.hypot(u, v), a, b, c, d, epsabs=1e-13)[0]
    assert abs(dd(printed_xx, a, b, c, d) - inv_r) < 1e-10
    assert abs(dd(printed_xx, a, b, c, d) - ref[2]) > 1e-2
    assert abs(dd(printed_xy, a, b, c, d) - ref[4]) > 1e-2
    assert abs(dd(printed_xy, a, b, c, d) - ref[2]) > 1e-2


def _brute_force(nest, sigma, level, i, j):
    """F at one target by quadrature of the linear density cell by cell."""
    sig, dsx, dsy = oracle.prepare(nest, sigma)
    X0, Y0 = nest.origin(level)
    ht = nest.h(level)
    xt, yt = X0 + (i + 0.5) * ht, Y0 + (j + 0.5) * ht
    fx = fy = 0.0
    for s in range(nest.levels):
        Xs, Ys = nest.origin(s)
        h = nest.h(s)
        for jj in range(nest.n):
            for ii in range(nest.n):
                s0, sx, sy = sig[s][jj, ii], dsx[s][jj, ii], dsy[s][jj, ii]
                if s0 == 0.0 and sx == 0.0 and sy == 0.0:
                    continue
                a, c = Xs + ii * h - xt, Ys + jj * h - yt
                uc, vc = a + 0.5 * h, c + 0.5 * h
                if abs(uc) < 1e-14 and abs(vc) < 1e-14:
                    # the target's own cell: odd parts vanish, u^2/r^3 and v^2/r^3 are integrable
                    q = _self_cell_u2(0.5 * h)
                    fx += sx * q
                    fy += sy * q
                    continue
                dens = lambda v, u: s0 + sx * (u - uc) + sy * (v - vc)
                fx += integrate.dblquad(lambda v, u: u / np.hypot(u, v) ** 3 * dens(v, u),
                                        a, a + h, c, c + h, epsabs=1e-12, epsrel=1e-11)[0]
                fy += integrate.dblquad(lambda v, u: v / np.hypot(u, v) ** 3 * dens(v, u),
                                        a, a + h, c, c + h, epsabs=1e-12, epsrel=1e-11)[0]
    return fx, fy


def _smooth_random(nest, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for l in range(nest.levels):
        X, Y = nest.centres(l)
        a, b, c = rng.uniform(0.5, 1.5, 3)
        out.append(a + b * X - 0.7 * c * Y + 0.3 * X * Y + rng.uniform(-0.05, 0.05, X.shape))
    return out


@pytest.mark.parametrize("case", [
    (1, [(0, 0)], 0, 3, 5),
    (2, [(0, 0), (2, 4)], 0, 1, 5),   # coarse target beside the fine patch (Case 2 and Case 1)
    (2, [(0, 0), (2, 4)], 1, 0, 7),   # fine target at the patch corner (Case 3 and Case 1)
])
def test_direct_sum_matches_quadrature(case):
    levels, off, tl, ti, tj = case
    nest = W.Nest(n=8, levels=levels, off=off)
    sigma = _smooth_random(nest, 7 + tl)
    fx, fy = oracle.force_at(nest, sigma, [tl], [ti], [tj])
    bx, by = _brute_force(nest, sigma, tl, ti, tj)
    assert fx[0] == pytest.approx(bx, rel=1e-9, abs=1e-11)
    assert fy[0] == pytest.approx(by, rel=1e-9, abs=1e-11)
