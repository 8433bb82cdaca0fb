"""Pins of the oracle's independent-Gaussian model (the parametric model the
paper compares with, Sec. Comparison of Parametric Vs. Nonparametric Models):
the two-vertex closed form, exchangeability, brute-force Monte Carlo with
numpy's normal sampler, the negation identity, point masses and steps, and
the fit."""
import math

import numpy as np
import pytest

import helpers as H_


def _phi_cdf(z):
    return 0.5 * math.erfc(-z / math.sqrt(2.0))


def test_gauss_two_vertex_closed_form(orc):
    """X1 < X2 for independent normals: Phi((m2 - m1) / sqrt(s1^2 + s2^2))."""
    rng = np.random.default_rng(1)
    for _ in range(20):
        m = rng.normal(0, 1, 2)
        s = rng.uniform(0.05, 2.0, 2)
        p = np.array([[[m[0], m[1]]], [[s[0], s[1]]]])
        pmin, pmax, _, st = orc.gauss(p)
        ref = _phi_cdf((m[1] - m[0]) / math.hypot(s[0], s[1]))
        assert st[0, 0] == 0
        assert abs(pmin[0, 0] - ref) < 1e-12
        assert abs(pmax[0, 0] - (1 - ref)) < 1e-12


def test_gauss_exchangeable(orc):
    p = np.zeros((2, 4, 5))
    p[0], p[1] = 0.3, 0.8
    pmin, pmax, sad, _ = orc.gauss(p)
    k = np.full((4, 5), 4)
    k[0, :] -= 1
    k[-1, :] -= 1
    k[:, 0] -= 1
    k[:, -1] -= 1
    np.testing.assert_allclose(pmin, 1.0 / (k + 1), atol=1e-12)
    np.testing.assert_allclose(pmax, 1.0 / (k + 1), atol=1e-12)
    ref = np.zeros((4, 5))
    ref[1:-1, 1:-1] = 1.0 / 15
    np.testing.assert_allclose(sad, ref, atol=1e-12)
    line = np.zeros((2, 1, 6))
    line[1] = 1.0
    _, _, sad, _ = orc.gauss(line)
    np.testing.assert_allclose(sad[0], [0, 1 / 3, 1 / 3, 1 / 3, 1 / 3, 0], atol=1e-12)


def test_gauss_bruteforce_monte_carlo(orc):
    rng = np.random.default_rng(2)
    H, W = 4, 5
    m = rng.normal(0, 0.6, (H, W))
    s = rng.uniform(0.2, 1.0, (H, W))
    s[1, 2] = 0.02                          # a sharp neighbour / centre
    p = np.stack([m, s])
    pmin, pmax, sad, _ = orc.gauss(p)
    n = 600_000
    cmin = np.zeros((H, W))
    cmax = np.zeros((H, W))
    csad = np.zeros((H, W))
    for _ in range(6):
        X = m + s * rng.standard_normal((n // 6, H, W))
        a, b = H_.neighbour_events(X)
        cmin += a
        cmax += b
        csad += H_.saddle_events(X)
    for P, c in ((pmin, cmin / n), (pmax, cmax / n), (sad, csad / n)):
        sd = np.sqrt(np.maximum(P * (1 - P), 1e-12) / n)
        assert (np.abs(P - c) <= 5 * sd + 1e-6).all()


def test_gauss_negation_identity(orc):
    rng = np.random.default_rng(3)
    p = np.stack([rng.normal(0, 1, (6, 7)), rng.uniform(0.1, 1.5, (6, 7))])
    n = p.copy()
    n[0] = -n[0]
    pmin, pmax, sad, _ = orc.gauss(p)
    nmin, nmax, nsad, _ = orc.gauss(n)
    np.testing.assert_allclose(pmax, nmin, atol=1e-12)
    np.testing.assert_allclose(pmin, nmax, atol=1e-12)
    np.testing.assert_allclose(sad, nsad, atol=1e-12)


def test_gauss_point_masses_and_steps(orc):
    # a point-mass centre: product of the strict tails at its value
    p = np.zeros((2, 3, 3))
    p[0] = np.array([[0, 0.5, 0], [1.0, 0.2, -0.3], [0, 0.9, 0]])
    p[1] = 1.0
    p[1, 1, 1] = 0.0
    pmin, pmax, _, st = orc.gauss(p)
    tails = [(0.5, 1.0), (1.0, 1.0), (-0.3, 1.0), (0.9, 1.0)]
    ref_min = np.prod([1 - _phi_cdf((0.2 - mm) / ss) for mm, ss in tails])
    ref_max = np.prod([_phi_cdf((0.2 - mm) / ss) for mm, ss in tails])
    assert st[1, 1] == orc.ST_DEGENERATE
    assert abs(pmin[1, 1] - ref_min) < 1e-13 and abs(pmax[1, 1] - ref_max) < 1e-13
    # a point-mass neighbour is the limit of a sharp one
    q = np.array([[[0.0, 0.4]], [[1.0, 0.0]]])
    r = np.array([[[0.0, 0.4]], [[1.0, 1e-7]]])
    a, b, _, _ = orc.gauss(q)
    c, d, _, _ = orc.gauss(r)
    assert abs(a[0, 0] - _phi_cdf(0.4)) < 1e-12
    assert abs(a[0, 0] - c[0, 0]) < 1e-6 and abs(b[0, 0] - d[0, 0]) < 1e-6
    # invalid and non-finite parameters
    bad = np.array([[[0.0, 0.0, np.nan]], [[1.0, -1.0, 1.0]]])
    a, b, s, st = orc.gauss(bad)
    assert st[0, 1] & orc.ST_BAD_PARAMS and st[0, 2] & orc.ST_NONFINITE
    assert np.isnan(a).all() and np.isnan(b).all()


def test_gauss_fit_matches_numpy(orc):
    rng = np.random.default_rng(4)
    ens = rng.normal(0, 1, (20, 5, 6)).astype(np.float32)
    ens[:, 0, 0] = 2.5
    p, st = orc.fit(ens, orc.GAUSSIAN)
    np.testing.assert_allclose(p[0], ens.astype(np.float64).mean(0), rtol=0, atol=1e-12)
    sd = ens.astype(np.float64).std(0, ddof=1)
    np.testing.assert_allclose(p[1], sd, rtol=1e-12, atol=1e-14)
    assert st[0, 0] == orc.ST_DEGENERATE and p[1, 0, 0] == 0.0
