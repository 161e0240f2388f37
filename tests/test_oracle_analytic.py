"""Pin the Appendix potential-density pairs used as closed-form references.

- D_1 from the recurrence equals the printed Maclaurin potential and force.
- D_n forces agree with an independent Hankel-transform quadrature
  F_R(R) = -2 pi int_0^inf k J_1(kR) S(k) dk,  S(k) = sigma0 alpha^2 2^nu Gamma(nu+1)
  J_{nu+1}(k alpha)/(k alpha)^{nu+1}, nu = n - 1/2 (Sonine's integral), inside and outside.
- The analytic derivative agrees with a finite difference of the potential.
- Reading: the printed b_{n+1,0} (division by 2k+1) differs from c_{n+1,0} for
  n >= 3 and then the rim force diverges; with 2k+2, b_{n,0} = c_{n,0}.
"""
import numpy as np
import pytest

from oracle import analytic as A

mp = pytest.importorskip("mpmath")


def hankel_radial_force(R, n, alpha):
    nu = n - 0.5
    mp.mp.dps = 16

    def f(k):
        return k * mp.besselj(1, k * R) * alpha ** 2 * 2 ** nu * mp.gamma(nu + 1) * \
            mp.besselj(nu + 1, k * alpha) / (k * alpha) ** (nu + 1)
    return float(-2 * mp.pi * mp.quadosc(f, [0, mp.inf], omega=max(R, alpha)))


def test_d1_is_maclaurin():
    R = np.linspace(0.01, 2.0, 57)
    np.testing.assert_allclose(A.radial_force_dn(R, 1, 0.8), A.maclaurin_force_closed(R, 0.8),
                               rtol=1e-13, atol=1e-14)
    # inside potential: -(pi^2 sigma0 / 4 alpha)(2 alpha^2 - R^2)
    Ri = np.linspace(0.0, 0.8, 9)
    np.testing.assert_allclose(A.potential_dn(Ri, 1, 0.8), -(np.pi ** 2 / 3.2) * (1.28 - Ri ** 2), rtol=1e-14)


@pytest.mark.parametrize("n", [2, 5])
@pytest.mark.parametrize("R", [0.3, 1.2])
def test_hankel_quadrature(n, R):
    assert A.radial_force_dn(np.array([R]), n, 0.85)[0] == pytest.approx(hankel_radial_force(R, n, 0.85), rel=1e-9)


@pytest.mark.parametrize("n", [1, 2, 3, 5])
def test_derivative_of_potential(n):
    # R stays within the sqrt(2)-radius of the paper's domains: further out the
    # outside-disk series cancels to ~(alpha/R)^(2n+1) and both sides lose digits
    R = np.array([0.2, 0.6, 0.84, 0.87, 1.3, 1.45])
    h = 1e-4
    P = lambda x: A.potential_dn(x, n, 0.85)
    # fourth-order central difference: truncation ~h^4, round-off ~eps |Phi| / h
    num = -(P(R - 2 * h) - 8 * P(R - h) + 8 * P(R + h) - P(R + 2 * h)) / (12 * h)
    np.testing.assert_allclose(A.radial_force_dn(R, n, 0.85), num, rtol=1e-8, atol=1e-9)


def test_printed_b0_reading():
    for n in range(1, 8):
        b, c = A.coefficients(n)
        assert b[0] == c[0]
    assert A.coefficients(2, printed_b0=True)[0][0] == A.coefficients(2)[0][0]
    assert A.coefficients(3, printed_b0=True)[0][0] != A.coefficients(3)[0][0]
