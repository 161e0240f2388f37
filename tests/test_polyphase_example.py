"""The worked example of Sec. 2.2 (m = 2, b of length 8, c of length 4).

Pins the oracle's generalized convolutions (Eqs. eqnbmnn, eqnbnmn) to the
printed expansions of a_0..a_5 (Case 2') and a_0..a_13 (Case 3'), and checks
the polyphase identities the paper states for them: the z-transform of a equals
the sum over phases of products of phase z-transforms (Case 2'), and each output
phase is one product (Case 3').  The CUDA path evaluates Cases 2 and 3 through
exactly this phase split, in two dimensions.
"""
import numpy as np

import oracle
from tests._golden import polyphase_example


def test_printed_expansions():
    rng = np.random.Generator(np.random.PCG64(11))
    b = rng.integers(-9, 10, 8).astype(float)
    c = rng.integers(-9, 10, 4).astype(float)
    ex = polyphase_example()
    a2 = oracle.genconv_case2(b, c, 2, 6)
    a3 = oracle.genconv_case3(b, c, 2, 14)
    for (case, k), pairs in ex.items():
        want = sum(b[i] * c[j] for i, j in pairs)
        got = a2[k] if case == "case2" else a3[k]
        assert got == want, (case, k)
    assert len([k for k in ex if k[0] == "case2"]) == 6
    assert len([k for k in ex if k[0] == "case3"]) == 14


def _poly(coeffs_by_power):
    deg = max(coeffs_by_power) if coeffs_by_power else 0
    p = np.zeros(deg + 1)
    for e, v in coeffs_by_power.items():
        p[e] += v
    return p


def test_polyphase_identities():
    rng = np.random.Generator(np.random.PCG64(12))
    b = rng.integers(-9, 10, 8).astype(float)
    c = rng.integers(-9, 10, 4).astype(float)
    # Case 2': a(z^2) = (b0 + b2 z^2 + b4 z^4 + b6 z^6)(c0 + c2 z^2) + (b1 z + ... + b7 z^7)(c1 z + c3 z^3)
    a2 = oracle.genconv_case2(b, c, 2, 6)
    lhs = _poly({2 * k: a2[k] for k in range(6)})
    even = np.polymul(_poly({k: b[k] for k in (0, 2, 4, 6)})[::-1], _poly({0: c[0], 2: c[2]})[::-1])[::-1]
    odd = np.polymul(_poly({k: b[k] for k in (1, 3, 5, 7)})[::-1], _poly({1: c[1], 3: c[3]})[::-1])[::-1]
    rhs = np.zeros(max(len(even), len(odd)))
    rhs[:len(even)] += even
    rhs[:len(odd)] += odd
    # products also hold odd powers of z; they cancel in the sum only at even powers the paper
    # compares, so compare the even-power coefficients
    assert np.array_equal(lhs[::2], rhs[:len(lhs)][::2])
    # Case 3': each output phase k of a is one product b(z;2,k) c(z^2;1,0)
    a3 = oracle.genconv_case3(b, c, 2, 14)
    cz2 = _poly({2 * j: c[j] for j in range(4)})
    for k in (0, 1):
        prod = np.polymul(_poly({e: b[e] for e in range(k, 8, 2)})[::-1], cz2[::-1])[::-1]
        want = _poly({n: a3[n] for n in range(k, 14, 2)})
        m = max(len(prod), len(want))
        pp = np.pad(prod, (0, m - len(prod)))
        ww = np.pad(want, (0, m - len(want)))
        assert np.array_equal(pp, ww)
