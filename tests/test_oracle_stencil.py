"""Pins of the oracle's larger neighbourhoods (the extension named in the
paper's Sec. Conclusion: six- and eight-neighbour stencils of a triangulated
2D grid, and the six axis neighbours of a 3D grid): exact closed forms
(tests/golden/stencil_closed_forms.json, re-derived by symbolic
integration), exchangeability, brute-force Monte Carlo with independent
samplers, the negation identity, disjoint supports, the boundary modes, and
reduction to the four-neighbour oracle where the extra neighbours are absent.
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import helpers as H_

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden", "stencil_closed_forms.json")
MODEL_ID = {"uniform": 0, "epanechnikov": 1, "histogram": 2}

# (dz, dy, dx) of each stencil, in the library's neighbour order
OFFSETS = {
    0: [(0, 0, 1), (0, -1, 0), (0, 0, -1), (0, 1, 0)],
    1: [(0, 0, 1), (0, -1, 0), (0, 0, -1), (0, 1, 0), (0, -1, 1), (0, 1, -1)],
    2: [(0, 0, 1), (0, -1, 0), (0, 0, -1), (0, 1, 0), (0, -1, 1), (0, -1, -1), (0, 1, -1),
        (0, 1, 1)],
    3: [(0, 0, 1), (0, -1, 0), (0, 0, -1), (0, 1, 0), (-1, 0, 0), (1, 0, 0)],
}


def _golden():
    with open(GOLDEN) as f:
        return json.load(f)["cases"]


def _as3d(p):
    return p[:, None] if p.ndim == 3 else p


def in_grid_count(D, H, W, stencil):
    k = np.zeros((D, H, W), int)
    z, y, x = np.meshgrid(np.arange(D), np.arange(H), np.arange(W), indexing="ij")
    for dz, dy, dx in OFFSETS[stencil]:
        k += ((z + dz >= 0) & (z + dz < D) & (y + dy >= 0) & (y + dy < H) & (x + dx >= 0)
              & (x + dx < W))
    return k


@pytest.mark.parametrize("case", _golden(), ids=lambda c: c["name"])
def test_stencil_golden(orc, case):
    p = np.array(case["params"], float)
    z, y, x = case["vertex"]
    pmin, pmax, st = orc.prob_stencil(p, MODEL_ID[case["model"]], case["stencil"])
    pmin, pmax, st = (a.reshape((-1,) + a.shape[-2:]) for a in (pmin, pmax, st))
    assert st[z, y, x] == 0
    assert abs(pmin[z, y, x] - float(Fraction(case["p_min"]))) < 1e-14
    assert abs(pmax[z, y, x] - float(Fraction(case["p_max"]))) < 1e-14


@pytest.mark.parametrize("case", _golden(), ids=lambda c: c["name"])
def test_stencil_golden_by_symbolic_integration(case):
    sp = pytest.importorskip("sympy")
    xs = sp.symbols("x")
    p = _as3d(np.array(case["params"], float))
    D, Hh, Ww = p.shape[1:]
    z0, y0, x0 = case["vertex"]

    def dist(z, y, x):
        a, b = (sp.nsimplify(v) for v in p[:, z, y, x])
        if case["model"] == "uniform":
            return a, b, 1 / (b - a), (b - xs) / (b - a)
        u = (xs - a) / b
        return a - b, a + b, sp.Rational(3, 4) / b * (1 - u ** 2), (1 - u) ** 2 * (2 + u) / 4

    lo1, hi1, pdf1, _ = dist(z0, y0, x0)
    nbrs = [dist(z0 + dz, y0 + dy, x0 + dx) for dz, dy, dx in OFFSETS[case["stencil"]]
            if 0 <= z0 + dz < D and 0 <= y0 + dy < Hh and 0 <= x0 + dx < Ww]
    pts = sorted({lo1, hi1} | {q for n in nbrs for q in n[:2] if lo1 < q < hi1})
    tmin = tmax = 0
    for s, t in zip(pts[:-1], pts[1:]):
        mid = (s + t) / 2
        fmin = fmax = pdf1
        for lo, hi, _, G in nbrs:
            g = 1 if mid < lo else (0 if mid > hi else G)
            fmin *= g
            fmax *= 1 - g
        tmin += sp.integrate(sp.expand(fmin), (xs, s, t))
        tmax += sp.integrate(sp.expand(fmax), (xs, s, t))
    assert sp.nsimplify(tmin) == sp.Rational(case["p_min"])
    assert sp.nsimplify(tmax) == sp.Rational(case["p_max"])


@pytest.mark.parametrize("stencil,shape", [(1, (1, 4, 5)), (2, (1, 4, 5)), (3, (3, 4, 5))])
@pytest.mark.parametrize("model", [0, 1, 2])
def test_stencil_exchangeable(orc, model, stencil, shape):
    """Identically distributed independent variables: 1/(k+1) with k the
    in-grid stencil neighbours."""
    rng = np.random.default_rng(17 + stencil)
    one = H_.random_params(model, 1, 1, rng, bins=5)
    p = np.broadcast_to(one[:, :, :, None], (one.shape[0],) + shape).copy()
    pmin, pmax, _ = orc.prob_stencil(p, model, stencil, bins=5)
    k = in_grid_count(*shape, stencil)
    np.testing.assert_allclose(pmin, 1.0 / (k + 1), atol=1e-13)
    np.testing.assert_allclose(pmax, 1.0 / (k + 1), atol=1e-13)


def _events(X, stencil):
    """Counts per vertex of 'below every in-grid stencil neighbour' and
    'above every one', for samples X (n, D, H, W)."""
    n, D, H, W = X.shape
    lt = np.ones(X.shape, bool)
    gt = np.ones(X.shape, bool)
    for dz, dy, dx in OFFSETS[stencil]:
        sl_c, sl_n = [slice(None)], [slice(None)]
        for d, L in ((dz, D), (dy, H), (dx, W)):
            sl_c.append(slice(max(0, -d), L - max(0, d)))
            sl_n.append(slice(max(0, d), L + min(0, d)))
        c, m = X[tuple(sl_c)], X[tuple(sl_n)]
        lt[tuple(sl_c)] &= c < m
        gt[tuple(sl_c)] &= c > m
    return lt.sum(0), gt.sum(0)


@pytest.mark.parametrize("stencil,shape", [(1, (1, 4, 4)), (2, (1, 4, 4)), (3, (3, 3, 4))])
@pytest.mark.parametrize("model", [0, 1, 2])
def test_stencil_bruteforce_monte_carlo(orc, model, stencil, shape):
    rng = np.random.default_rng(31 + 3 * model + stencil)
    D, H, W = shape
    p2 = H_.random_params(model, D * H, W, rng, bins=3)       # vertex-wise independent
    p = p2.reshape((p2.shape[0], D, H, W))
    pmin, pmax, _ = orc.prob_stencil(p, model, stencil, bins=3)
    n, done = 400_000, 0
    cmin = np.zeros(shape)
    cmax = np.zeros(shape)
    while done < n:
        m = min(100_000, n - done)
        X = H_.sample_field(p2, model, rng, m).reshape((m, D, H, W))
        a, b = _events(X, stencil)
        cmin += a
        cmax += b
        done += m
    for P, c in ((pmin, cmin / n), (pmax, cmax / n)):
        sd = np.sqrt(np.maximum(P * (1 - P), 1e-12) / n)
        assert (np.abs(P - c) <= 5 * sd + 1e-6).all()


@pytest.mark.parametrize("stencil", [1, 2, 3])
@pytest.mark.parametrize("model", [0, 1, 2])
def test_stencil_negation_identity(orc, model, stencil):
    rng = np.random.default_rng(41 + stencil)
    D = 3 if stencil == 3 else 1
    p2 = H_.random_params(model, D * 6, 7, rng, bins=4)
    p = p2.reshape((p2.shape[0], D, 6, 7))
    n = H_.negate_params(p2, model).reshape(p.shape)
    pmin, pmax, _ = orc.prob_stencil(p, model, stencil, bins=4)
    nmin, nmax, _ = orc.prob_stencil(n, model, stencil, bins=4)
    np.testing.assert_allclose(pmax, nmin, atol=1e-12)
    np.testing.assert_allclose(pmin, nmax, atol=1e-12)


@pytest.mark.parametrize("model", [0, 1, 2])
def test_stencil_reduces_to_four_neighbours(orc, model):
    """The 3D stencil on one slice and the 4-stencil are the paper's
    four-neighbour oracle; the 6- and 8-stencils differ from it."""
    rng = np.random.default_rng(53)
    p = H_.random_params(model, 7, 9, rng, bins=4)
    ref = orc.prob(p, model, bins=4)
    for st in (0, 3):
        got = orc.prob_stencil(p[:, None] if st == 3 else p, model, st, bins=4)
        np.testing.assert_array_equal(got[0].reshape(7, 9), ref[0])
        np.testing.assert_array_equal(got[1].reshape(7, 9), ref[1])
    for st in (1, 2):
        got = orc.prob_stencil(p, model, st, bins=4)
        assert np.abs(got[0] - ref[0]).max() > 1e-3
        # more neighbours can only lower both probabilities
        assert (got[0] <= ref[0] + 1e-12).all() and (got[1] <= ref[1] + 1e-12).all()


def test_stencil_disjoint_and_boundary_modes(orc):
    a = np.full((3, 3), 2.0)
    b = np.full((3, 3), 3.0)
    a[1, 1], b[1, 1] = 0.0, 1.0
    pmin, pmax, _ = orc.prob_stencil(np.stack([a, b]), 0, 2)
    assert pmin[1, 1] == 1.0 and pmax[1, 1] == 0.0
    rng = np.random.default_rng(3)
    p = H_.random_params(0, 4 * 5, 6, rng).reshape(2, 4, 5, 6)
    z0, z1, _ = orc.prob_stencil(p, 0, 3, boundary=1)
    i0, i1, _ = orc.prob_stencil(p, 0, 3, boundary=0)
    full = in_grid_count(4, 5, 6, 3) == 6
    assert (z0[~full] == 0).all() and (z1[~full] == 0).all()
    np.testing.assert_array_equal(z0[full], i0[full])
    np.testing.assert_array_equal(z1[full], i1[full])


def test_stencil_rejects_bad_arguments(orc):
    p = np.zeros((2, 2, 3, 3))
    with pytest.raises(ValueError):
        orc.prob_stencil(p, 0, 2)        # a 2D stencil on more than one slice
    with pytest.raises(ValueError):
        orc.prob_stencil(p, 0, 4)        # no such stencil
