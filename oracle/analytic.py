"""Closed-form potential-density pairs of the finite disks D_n (Appendix).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Surface density  Sigma_n(R) = sigma0 (1 - R^2/alpha^2)^(n - 1/2)  for R < alpha.
The mid-plane potential follows the Appendix's representation, Eq. (eqnPhiDn)
outside the disk and the polynomial form inside, with coefficients b_{n,k},
c_{n,k} from the Appendix recurrence.  Exact rational arithmetic
(``fractions.Fraction``) is used for the coefficients.

Reading (the printed recurrence is at odds with itself): the printed b_{n+1,0}
divides b_{n,k} by (2k+1) inside the sum, while c_{n+1,0} divides by (2k+2).
The two disagree for n >= 3, and only b_{n+1,0} = c_{n+1,0} keeps the force
finite at the rim (the 1/sqrt(1 - xi^2) terms of dPhi/dR cancel only when
b_{n,0} = c_{n,0}).  This module therefore uses (2k+2) for both; the test
suite pins the result against an independent Hankel-transform quadrature.

Force:  F_R = -dPhi/dR (attractive: negative for positive sigma0), G = 1,
F_x = F_R x/R, F_y = F_R y/R.
"""
from __future__ import annotations

from fractions import Fraction
from functools import lru_cache
from math import prod

import numpy as np


def H(k: int, m: int) -> Fraction:
    """H(k, m) = (-1)^(k-m) prod_{j=m}^{k} (2j+1)/(2j+2)  (Appendix)."""
    out = Fraction(1)
    for j in range(m, k + 1):
        out *= Fraction(2 * j + 1, 2 * j + 2)
    return out if (k - m) % 2 == 0 else -out


@lru_cache(maxsize=None)
def coefficients(n: int, printed_b0: bool = False):
    """(b_{n,0..n}, c_{n,0..n-1}) as tuples of Fractions.

    ``printed_b0=True`` reproduces the recurrence exactly as printed (used only by
    the test that shows the printed form breaks rim finiteness for n >= 3)."""
    if n < 1:
        raise ValueError("n >= 1")
    b = [Fraction(1), Fraction(2)]  # b_{1,0}, b_{1,1}
    c = [Fraction(1)]               # c_{1,0}
    for nn in range(1, n):
        # common leading factor (b_{n,n}/(2n+2) + c_{n,n-1})
        lead = b[nn] / (2 * nn + 2) + c[nn - 1]
        nb = [Fraction(0)] * (nn + 2)
        nc = [Fraction(0)] * (nn + 1)
        for k in range(1, nn + 2):
            nb[k] = b[k - 1] / (2 * k)
        # c_{n+1,m}, m = 1..n
        nc[nn] = lead * H(nn, nn) / (2 * nn + 1)
        for m in range(1, nn):
            acc = lead * H(nn, m) / (2 * m + 1)
            for k in range(m, nn):
                acc += (b[k] / (2 * k + 2) + c[k] + c[k - 1]) * H(k, m) / (2 * m + 1)
            nc[m] = acc
        # c_{n+1,0}
        acc = lead * H(nn, 0)
        for k in range(1, nn):
            acc += (b[k] / (2 * k + 2) + c[k] + c[k - 1]) * H(k, 0)
        acc += b[0] / 4 + c[0] / 2
        nc[0] = acc
        if printed_b0:
            accb = lead * H(nn, 0)
            for k in range(1, nn):
                accb += (b[k] / (2 * k + 1) + c[k] + c[k - 1]) * H(k, 0)
            accb += b[0] / 4 + c[0] / 2
            nb[0] = accb
        else:
            nb[0] = nc[0]
        b, c = nb, nc
    return tuple(b), tuple(c)


def _odd_product(n: int) -> int:
    return prod(2 * j + 1 for j in range(n))


def sigma_dn(r, n: int, alpha: float, sigma0: float = 1.0):
    r = np.asarray(r, dtype=np.float64)
    inside = r < alpha
    out = np.zeros_like(r)
    out[inside] = sigma0 * (1.0 - (r[inside] / alpha) ** 2) ** (n - 0.5)
    return out


def potential_dn(R, n: int, alpha: float, sigma0: float = 1.0, printed_b0: bool = False):
    """Mid-plane potential Phi_{D_n}(R) (G = 1)."""
    R = np.asarray(R, dtype=np.float64)
    b, c = coefficients(n, printed_b0)
    bf = [float(x) for x in b]
    cf = [float(x) for x in c]
    pref = _odd_product(n) / alpha ** (2 * n - 1)
    out = np.empty_like(R)
    ins = R <= alpha
    # inside: -(pi^2 sigma0/4) pref sum_k b_k R^(2n-2k) (alpha^2 - R^2)^k
    Ri = R[ins]
    s = sum(bk * Ri ** (2 * n - 2 * k) * (alpha ** 2 - Ri ** 2) ** k for k, bk in enumerate(bf))
    out[ins] = -(np.pi ** 2 * sigma0 / 4.0) * pref * s
    Ro = R[~ins]
    xi = alpha / Ro
    t = xi ** 2 - 1.0
    Bv = sum(bk * t ** k for k, bk in enumerate(bf))
    Cv = sum(ck * t ** k for k, ck in enumerate(cf))
    G = Bv * np.arcsin(xi) + xi * Cv * np.sqrt(1.0 - xi ** 2)
    out[~ins] = -(np.pi * sigma0 / 2.0) * pref * Ro ** (2 * n) * G
    return out


def radial_force_dn(R, n: int, alpha: float, sigma0: float = 1.0):
    """F_R = -dPhi_{D_n}/dR, differentiated analytically (G = 1)."""
    R = np.asarray(R, dtype=np.float64)
    b, c = coefficients(n)
    bf = [float(x) for x in b]
    cf = [float(x) for x in c] + [0.0]
    pref = _odd_product(n) / alpha ** (2 * n - 1)
    out = np.empty_like(R)
    ins = R <= alpha
    # inside: Phi = Cin * p(R^2), p(q) = sum_k b_k q^(n-k) (alpha^2 - q)^k
    Ri = R[ins]
    q = Ri ** 2
    a2 = alpha ** 2
    dp = np.zeros_like(q)
    for k, bk in enumerate(bf):
        # d/dq [q^(n-k) (a2 - q)^k]
        term = np.zeros_like(q)
        if n - k > 0:
            term += (n - k) * q ** (n - k - 1) * (a2 - q) ** k
        if k > 0:
            term -= k * q ** (n - k) * (a2 - q) ** (k - 1)
        dp += bk * term
    out[ins] = (np.pi ** 2 / 4.0) * sigma0 * pref * dp * 2.0 * Ri  # F = -dPhi/dR
    # outside: Phi = Cout R^(2n) G(xi), xi = alpha/R, Cout = -(pi sigma0/2) pref
    Ro = R[~ins]
    xi = alpha / Ro
    t = xi ** 2 - 1.0
    sq = np.sqrt(np.maximum(1.0 - xi ** 2, 0.0))
    Bv = sum(bk * t ** k for k, bk in enumerate(bf))
    dB = sum(bk * k * t ** (k - 1) * 2.0 * xi for k, bk in enumerate(bf) if k > 0)
    Cv = sum(ck * t ** k for k, ck in enumerate(cf))
    dC = sum(ck * k * t ** (k - 1) * 2.0 * xi for k, ck in enumerate(cf) if k > 0)
    # (B - xi^2 C)/sqrt(1 - xi^2): with b_0 = c_0 the numerator is t * S(t) and t/sq = -sq
    S = sum((bf[k] - cf[k] - cf[k - 1]) * t ** (k - 1) for k in range(1, len(bf)))
    sing = (bf[0] - cf[0]) / np.where(sq > 0, sq, np.inf) - sq * S
    G = Bv * np.arcsin(xi) + xi * Cv * sq
    dG = dB * np.arcsin(xi) + sing + Cv * sq + xi * dC * sq
    dPhi = -(np.pi * sigma0 / 2.0) * pref * Ro ** (2 * n - 1) * (2 * n * G - xi * dG)
    out[~ins] = -dPhi
    return out


def force_dn_xy(x, y, n: int, alpha: float, sigma0: float = 1.0, cx: float = 0.0, cy: float = 0.0):
    """(F_x, F_y) of a D_n disk centred at (cx, cy)."""
    dx = np.asarray(x, dtype=np.float64) - cx
    dy = np.asarray(y, dtype=np.float64) - cy
    R = np.hypot(dx, dy)
    FR = radial_force_dn(np.maximum(R, 1e-300), n, alpha, sigma0)
    with np.errstate(invalid="ignore", divide="ignore"):
        fx = np.where(R > 0, FR * dx / R, 0.0)
        fy = np.where(R > 0, FR * dy / R, 0.0)
    return fx, fy


def maclaurin_force_closed(R, alpha: float, sigma0: float = 1.0):
    """D_1 radial force from the printed Maclaurin potential (Appendix):
    inside  F_R = -pi^2 sigma0 R / (2 alpha);
    outside F_R = -(pi sigma0/alpha) [R asin(alpha/R) - alpha sqrt(R^2 - alpha^2)/R]."""
    R = np.asarray(R, dtype=np.float64)
    out = np.empty_like(R)
    ins = R <= alpha
    out[ins] = -np.pi ** 2 * sigma0 * R[ins] / (2.0 * alpha)
    Ro = R[~ins]
    out[~ins] = -(np.pi * sigma0 / alpha) * (Ro * np.arcsin(alpha / Ro)
                                              - alpha * np.sqrt(Ro ** 2 - alpha ** 2) / Ro)
    return out
