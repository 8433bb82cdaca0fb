"""Exact-arithmetic checks of the per-piece integral identities the kernels
rely on (CPU, rational arithmetic; no GPU):

- the integral over [0, 1] of a product of K linear factors, each given by
  its end values (l_i, r_i), equals the mean of the product's Bernstein
  coefficients of degree K (the uniform and histogram piece integral);
- for K = 4 it also equals the form built from the factors in two pairs,
  (b0 c0 + b2 c2)/5 + ((b0 + b2) c1 + b1 (c0 + c2))/20 + (b0 c2 + b2 c0 +
  b1 c1)/30 with b0 = l0 l1, b2 = r0 r1, b1 = l0 r1 + r0 l1 and c0, c1, c2
  likewise (the row walk's piece integral).
"""
import itertools
import random
from fractions import Fraction as Fr
from math import comb


def exact_integral(L, R):
    """Expand prod (l_i + (r_i - l_i) t) and integrate term by term."""
    poly = [Fr(1)]
    for l, r in zip(L, R):
        nxt = [Fr(0)] * (len(poly) + 1)
        for k, c in enumerate(poly):
            nxt[k] += c * l
            nxt[k + 1] += c * (r - l)
        poly = nxt
    return sum(c / (k + 1) for k, c in enumerate(poly))


def bernstein_mean(L, R):
    """Mean of the degree-K Bernstein coefficients: coefficient j is the
    average over the subsets of j factors of (their right values) x (the
    others' left values)."""
    K = len(L)
    total = Fr(0)
    for j in range(K + 1):
        s = Fr(0)
        for S in itertools.combinations(range(K), j):
            p = Fr(1)
            for i in range(K):
                p *= R[i] if i in S else L[i]
            s += p
        total += s / comb(K, j)
    return total / (K + 1)


def pairs_form(L, R):
    b0, b2, b1 = L[0] * L[1], R[0] * R[1], L[0] * R[1] + R[0] * L[1]
    c0, c2, c1 = L[2] * L[3], R[2] * R[3], L[2] * R[3] + R[2] * L[3]
    return (Fr(1, 5) * (b0 * c0 + b2 * c2) + Fr(1, 20) * ((b0 + b2) * c1 + b1 * (c0 + c2))
            + Fr(1, 30) * (b0 * c2 + b2 * c0 + b1 * c1))


def _values(rng, K):
    return ([Fr(rng.randint(0, 64), 64) for _ in range(K)],
            [Fr(rng.randint(0, 64), 64) for _ in range(K)])


def test_bernstein_mean_is_the_integral():
    rng = random.Random(5)
    for K in range(1, 5):
        for _ in range(60):
            L, R = _values(rng, K)
            assert bernstein_mean(L, R) == exact_integral(L, R)


def test_pairs_form_is_the_integral():
    rng = random.Random(7)
    for _ in range(300):
        L, R = _values(rng, 4)
        assert pairs_form(L, R) == exact_integral(L, R)


def test_special_cases():
    one = [Fr(1)] * 4
    assert pairs_form(one, one) == 1                       # constant factors
    z = [Fr(0)] * 4
    assert pairs_form(z, z) == 0
    # a factor vanishing at both ends vanishes on the piece
    L = [Fr(0), Fr(1), Fr(1), Fr(1)]
    assert pairs_form(L, L) == 0
    # four identical ramps 0 -> 1: the integral of t^4 is 1/5
    assert pairs_form(z, one) == Fr(1, 5)
    assert pairs_form(one, z) == Fr(1, 5)
