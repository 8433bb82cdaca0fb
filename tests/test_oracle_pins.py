"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Every oracle function used as a parity reference is checked here against
something other than itself: exact closed forms of the paper's worked
orderings (tests/golden), exact symbolic integration, exchangeability,
disjoint supports, the negation identity, probability bounds, the paper's
second histogram route, brute-force Monte Carlo with independent samplers,
Gaussian closed forms and quadrature, a library Philox implementation, and
central finite differences for the gradient.
"""
import json
import math
import os
import subprocess
import sys
from fractions import Fraction

import numpy as np
import pytest

import helpers as H_

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden", "closed_forms.json")
MODEL_ID = {"uniform": 0, "epanechnikov": 1, "histogram": 2}


def _golden():
    with open(GOLDEN) as f:
        return json.load(f)["cases"]


# --------------------------------------------------------------------------
# exact closed forms


@pytest.mark.parametrize("case", _golden(), ids=lambda c: c["name"])
def test_golden_closed_forms(orc, case):
    p = np.array(case["params"], float)
    y, x = case["vertex"]
    pmin, pmax, st = orc.prob(p, MODEL_ID[case["model"]])
    assert st[y, x] == 0
    if "p_min" in case:
        assert abs(pmin[y, x] - float(Fraction(case["p_min"]))) < 1e-14
    if "p_max" in case:
        assert abs(pmax[y, x] - float(Fraction(case["p_max"]))) < 1e-14
    if "p_saddle" in case:
        sad, _ = orc.saddle(p, MODEL_ID[case["model"]])
        assert abs(sad[y, x] - float(Fraction(case["p_saddle"]))) < 1e-14


@pytest.mark.parametrize("case", _golden(), ids=lambda c: c["name"])
def test_golden_values_by_symbolic_integration(case):
    """Re-derive each golden value by exact integration of the definition."""
    sp = pytest.importorskip("sympy")
    x = sp.symbols("x")
    p = np.array(case["params"], float)
    y0, x0 = case["vertex"]
    Hh, Ww = p.shape[1:]

    def dist(y, xx):
        a, b = (sp.nsimplify(v) for v in p[:, y, xx])
        if case["model"] == "uniform":
            lo, hi = a, b
            pdf = 1 / (b - a)
            G = (b - x) / (b - a)
        else:
            m, w = a, b
            lo, hi = m - w, m + w
            u = (x - m) / w
            pdf = sp.Rational(3, 4) / w * (1 - u ** 2)
            G = (1 - u) ** 2 * (2 + u) / 4
        return lo, hi, pdf, G

    lo1, hi1, pdf1, _ = dist(y0, x0)
    nbrs = [dist(y0 + dy, x0 + dx) for dy, dx in ((0, 1), (-1, 0), (0, -1), (1, 0))
            if 0 <= y0 + dy < Hh and 0 <= x0 + dx < Ww]
    pts = sorted({lo1, hi1} | {q for n in nbrs for q in n[:2] if lo1 < q < hi1})
    tot_min = tot_max = tot_sad = 0
    for s, t in zip(pts[:-1], pts[1:]):
        mid = (s + t) / 2
        fmin = fmax = pdf1
        gs = []
        for lo, hi, _, G in nbrs:
            g = 1 if mid < lo else (0 if mid > hi else G)
            gs.append(g)
            fmin *= g
            fmax *= 1 - g
        tot_min += sp.integrate(sp.expand(fmin), (x, s, t))
        tot_max += sp.integrate(sp.expand(fmax), (x, s, t))
        if len(gs) == 4:   # e, n, w, s: t1 = G F G F, t2 = F G F G
            t1 = pdf1 * gs[0] * (1 - gs[1]) * gs[2] * (1 - gs[3])
            t2 = pdf1 * (1 - gs[0]) * gs[1] * (1 - gs[2]) * gs[3]
            tot_sad += sp.integrate(sp.expand(t1 + t2), (x, s, t))
    if "p_min" in case:
        assert sp.nsimplify(tot_min) == sp.Rational(case["p_min"])
    if "p_max" in case:
        assert sp.nsimplify(tot_max) == sp.Rational(case["p_max"])
    if "p_saddle" in case:
        assert sp.nsimplify(tot_sad) == sp.Rational(case["p_saddle"])


# --------------------------------------------------------------------------
# invariants


@pytest.mark.parametrize("model", [0, 1, 2])
def test_exchangeable_gives_one_over_k_plus_one(orc, model):
    rng = np.random.default_rng(7)
    one = H_.random_params(model, 1, 1, rng, bins=5)
    p = np.broadcast_to(one, (one.shape[0], 4, 5)).copy()
    pmin, pmax, _ = orc.prob(p, model, bins=5)
    k = np.full((4, 5), 4)
    k[0, :] -= 1
    k[-1, :] -= 1
    k[:, 0] -= 1
    k[:, -1] -= 1
    np.testing.assert_allclose(pmin, 1.0 / (k + 1), atol=1e-13)
    np.testing.assert_allclose(pmax, 1.0 / (k + 1), atol=1e-13)


def test_disjoint_supports(orc):
    a = np.full((3, 3), 2.0)
    b = np.full((3, 3), 3.0)
    a[1, 1], b[1, 1] = 0.0, 1.0           # centre entirely below
    pmin, pmax, _ = orc.prob(np.stack([a, b]), 0)
    assert pmin[1, 1] == 1.0 and pmax[1, 1] == 0.0
    a[1, 1], b[1, 1] = 4.0, 5.0           # entirely above: b_min < a_1
    pmin, pmax, _ = orc.prob(np.stack([a, b]), 0)
    assert pmin[1, 1] == 0.0 and pmax[1, 1] == 1.0


@pytest.mark.parametrize("model", [0, 1, 2])
def test_negation_identity(orc, model):
    """P_max(X) = P_min(-X) (Sec. Local Maximum Probability)."""
    rng = np.random.default_rng(11 + model)
    p = H_.random_params(model, 6, 7, rng, bins=6)
    pmin, pmax, _ = orc.prob(p, model, bins=6)
    nmin, nmax, _ = orc.prob(H_.negate_params(p, model), model, bins=6)
    np.testing.assert_allclose(pmax, nmin, atol=1e-13)
    np.testing.assert_allclose(pmin, nmax, atol=1e-13)


@pytest.mark.parametrize("model", [0, 1, 2])
def test_bounds(orc, model):
    """0 <= P, P_min + P_max <= 1, and the Frechet/association bounds
    prod_n Pr[X1<X_n] <= P_min <= min_n Pr[X1<X_n]."""
    rng = np.random.default_rng(21 + model)
    p = H_.random_params(model, 5, 5, rng, bins=4)
    pmin, pmax, _ = orc.prob(p, model, bins=4)
    assert (pmin >= -1e-15).all() and (pmax >= -1e-15).all()
    assert (pmin + pmax <= 1 + 1e-12).all()
    for y in range(1, 4):
        for x in range(1, 4):
            pair = []
            for dy, dx in ((0, 1), (-1, 0), (0, -1), (1, 0)):
                q = np.stack([p[:, y, x], p[:, y + dy, x + dx]], axis=-1)[:, None, :]
                pair.append(orc.prob(q, model, bins=4)[0][0, 0])
            assert pmin[y, x] <= min(pair) + 1e-12
            assert pmin[y, x] >= np.prod(pair) - 1e-12


def test_histogram_merge_equals_paper_h5_route(orc):
    """Eq. localMinProbHistogram (sum over bin combinations) vs the merged
    piecewise integral, for B = 1..4."""
    rng = np.random.default_rng(5)
    for B in (1, 2, 3, 4):
        p = H_.random_params(2, 4, 4, rng, bins=B)
        idx = np.arange(16)
        a_min, a_max, _ = orc.prob_at(p, 2, idx, bins=B)
        b_min, b_max = orc.prob_hist_h5_at(p, B, idx)
        np.testing.assert_allclose(a_min, b_min, atol=1e-13)
        np.testing.assert_allclose(a_max, b_max, atol=1e-13)


def test_one_bin_histogram_is_uniform(orc):
    rng = np.random.default_rng(6)
    pu = H_.random_params(0, 5, 6, rng)
    ph = np.concatenate([pu, np.ones((1, 5, 6))])
    u = orc.prob(pu, 0)
    h = orc.prob(ph, 2, bins=1)
    np.testing.assert_allclose(u[0], h[0], atol=1e-14)
    np.testing.assert_allclose(u[1], h[1], atol=1e-14)


# --------------------------------------------------------------------------
# brute-force Monte Carlo with independent samplers


@pytest.mark.parametrize("model", [0, 1, 2])
def test_bruteforce_monte_carlo(orc, model):
    rng = np.random.default_rng(31 + model)
    p = H_.random_params(model, 4, 5, rng, bins=4)
    n = 2_000_000
    mc_min, mc_max = H_.mc_probabilities(p, model, n, seed=100 + model)
    pmin, pmax, _ = orc.prob(p, model, bins=4)
    for ref, mc in ((pmin, mc_min), (pmax, mc_max)):
        sig = np.sqrt(np.maximum(ref * (1 - ref), 1e-12) / n)
        z = np.abs(mc - ref) / sig
        assert z.max() < 5.5, (z.max(), ref, mc)


# --------------------------------------------------------------------------
# point masses, statuses, boundary mode


def test_point_masses(orc):
    # centre point mass at 0.3 among uniform neighbours: prod_n Pr[X_n > 0.3]
    a = np.array([[0.0, 0.3, 0.1]])
    b = np.array([[1.0, 0.3, 0.5]])
    pmin, pmax, st = orc.prob(np.stack([a, b]), 0)
    assert st[0, 1] & orc.ST_DEGENERATE
    assert abs(pmin[0, 1] - 0.7 * 0.5) < 1e-15
    assert abs(pmax[0, 1] - 0.3 * 0.5) < 1e-15
    # continuous centre next to a point-mass neighbour: Pr[X1 < c]
    a = np.array([[0.0, 0.25]])
    b = np.array([[1.0, 0.25]])
    pmin, pmax, _ = orc.prob(np.stack([a, b]), 0)
    assert abs(pmin[0, 0] - 0.25) < 1e-15 and abs(pmax[0, 0] - 0.75) < 1e-15
    # two equal point masses: strict comparison -> 0 for both
    pmin, pmax, _ = orc.prob(np.stack([np.full((1, 2), 2.0)] * 2), 0)
    assert (pmin == 0).all() and (pmax == 0).all()


def test_bad_and_nonfinite_params(orc):
    p = np.stack([np.zeros((3, 3)), np.ones((3, 3))])
    p[0, 1, 1] = 2.0                                      # a > b at the centre
    pmin, _, st = orc.prob(p, 0)
    assert st[1, 1] & orc.ST_BAD_PARAMS and np.isnan(pmin[1, 1])
    assert np.isnan(pmin[0, 1]) and not np.isnan(pmin[0, 0])   # neighbours see it
    p = np.stack([np.zeros((3, 3)), np.ones((3, 3))])
    p[1, 2, 2] = np.nan
    pmin, _, st = orc.prob(p, 0)
    assert st[2, 2] & orc.ST_NONFINITE and np.isnan(pmin[2, 1])


def test_boundary_zero_mode(orc):
    rng = np.random.default_rng(3)
    p = H_.random_params(0, 4, 5, rng)
    pmin, pmax, _ = orc.prob(p, 0, boundary=1)
    ref_min, ref_max, _ = orc.prob(p, 0, boundary=0)
    inner = (slice(1, -1), slice(1, -1))
    assert (pmin[0] == 0).all() and (pmin[:, -1] == 0).all()
    np.testing.assert_array_equal(pmin[inner], ref_min[inner])
    np.testing.assert_array_equal(pmax[inner], ref_max[inner])


# --------------------------------------------------------------------------
# fitting


def test_fit_matches_numpy(orc):
    rng = np.random.default_rng(9)
    ens = rng.normal(size=(13, 6, 7)).astype(np.float32)
    ens[:, 2, 3] = 1.5                        # degenerate vertex
    u, st = orc.fit(ens, 0)
    np.testing.assert_array_equal(u[0], ens.min(0))
    np.testing.assert_array_equal(u[1], ens.max(0))
    assert st[2, 3] == orc.ST_DEGENERATE and st.sum() == orc.ST_DEGENERATE
    e, _ = orc.fit(ens, 1)
    e64 = ens.astype(np.float64)
    ref_w = math.sqrt(5) * e64.std(0, ddof=1)
    ref_w[2, 3] = 0.0
    np.testing.assert_allclose(e[0], e64.mean(0), rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(e[1], ref_w, rtol=1e-12, atol=1e-15)
    B = 8
    h, _ = orc.fit(ens, 2, bins=B)
    lo, hi = ens.min(0), ens.max(0)
    with np.errstate(invalid="ignore", divide="ignore"):
        q = (ens - lo) * (np.float32(B) / (hi - lo))       # float32 numpy ops
    idx = np.clip(np.nan_to_num(np.floor(q), nan=0.0).astype(np.int64), 0, B - 1)
    idx[:, 2, 3] = 0
    for j in range(B):
        np.testing.assert_array_equal(h[2 + j], (idx == j).sum(0) / 13.0)


def test_fit_mvn_matches_numpy_cov(orc):
    rng = np.random.default_rng(10)
    ens = rng.normal(size=(9, 4, 5)).astype(np.float32)
    prm, _ = orc.fit(ens, 3)
    offs = ((0, 0), (0, 1), (-1, 0), (0, -1), (1, 0))
    for y in range(4):
        for x in range(5):
            present = [0 <= y + dy < 4 and 0 <= x + dx < 5 for dy, dx in offs]
            cols = [ens[:, y + dy, x + dx].astype(np.float64) if pr else np.zeros(9)
                    for (dy, dx), pr in zip(offs, present)]
            C = np.cov(np.stack(cols))
            r = 5
            for a in range(5):
                assert abs(prm[a, y, x] - (cols[a].mean() if present[a] else 0)) < 1e-12
                for b in range(a + 1):
                    ref = C[a, b] if (present[a] and present[b]) else 0.0
                    assert abs(prm[r, y, x] - ref) < 1e-12
                    r += 1


def test_fit_nonfinite(orc):
    ens = np.zeros((4, 3, 3), np.float32)
    ens[:, 1, 1] = np.arange(4)
    ens[2, 0, 0] = np.inf
    ens[1, 2, 2] = np.nan
    for model in (0, 1, 2):
        prm, st = orc.fit(ens, model, bins=4)
        assert st[0, 0] & orc.ST_NONFINITE and st[2, 2] & orc.ST_NONFINITE
        assert np.isnan(prm[:, 0, 0]).all() and not np.isnan(prm[:, 1, 1]).any()


# --------------------------------------------------------------------------
# multivariate Gaussian Monte Carlo


def test_philox_matches_library_implementation(orc):
    """The oracle's Philox4x32-10 against triton's (run in its CPU
    interpreter, a separate implementation of the same published generator)."""
    pytest.importorskip("triton")
    code = r"""
import os, sys, json
os.environ["TRITON_INTERPRET"] = "1"
import torch, triton, triton.language as tl
@triton.jit
def k(out, seed, c0, c1, c2, c3):
    a, b, c, d = tl.philox(seed, c0, c1, c2, c3)
    tl.store(out + 0, a); tl.store(out + 1, b); tl.store(out + 2, c); tl.store(out + 3, d)
res = []
for seed, c in json.loads(sys.argv[1]):
    o = torch.zeros(4, dtype=torch.int32)
    k[(1,)](o, seed, *c)
    res.append([v & 0xffffffff for v in o.tolist()])
print(json.dumps(res))
"""
    cases = [(0, [0, 0, 0, 0]), (0x5EED, [7, 123456, 3, 1]),
             (0x0123456789ABCDEF, [2147483647, 1, 2, 0]), (42, [9999, 262143, 0, 1]),
             (0xFFFFFFFFFFFFFFFF, [0x7ABCDEF0, 0x76543210, 0x7FFFFFFF, 1])]
    env = dict(os.environ, TRITON_INTERPRET="1")
    try:
        out = subprocess.run([sys.executable, "-c", code, json.dumps(cases)], env=env,
                             capture_output=True, text=True, timeout=600, check=True)
    except subprocess.CalledProcessError as e:  # pragma: no cover
        pytest.skip("triton interpreter unavailable: " + e.stderr[-300:])
    ref = json.loads(out.stdout.strip().splitlines()[-1])
    for (seed, c), r in zip(cases, ref):
        key = [seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF]
        assert orc.philox4x32_10(c, key).tolist() == r


def _phi(x):
    return 0.5 * (1 + math.erf(x / math.sqrt(2)))


def test_mvn_two_vertex_closed_form(orc):
    mu = np.array([[0.3, 0.5]])
    s11, s22, s12 = 0.5, 0.8, 0.3
    prm = H_.mvn_params(1, 2, mu, lambda y, x, pr: np.array(
        [[s11, s12, 0, 0, 0], [s12, s22, 0, 0, 0], [0] * 5, [0] * 5, [0] * 5]) if x == 0
        else np.array([[s22, 0, 0, s12, 0], [0] * 5, [0] * 5, [s12, 0, 0, s11, 0], [0] * 5]))
    S = 400_000
    hmin, hmax, _, st = orc.mvn_mc_at(prm, [0, 1], S, seed=0x5EED)
    p = _phi((0.5 - 0.3) / math.sqrt(s11 + s22 - 2 * s12))
    sig = math.sqrt(p * (1 - p) / S)
    assert abs(hmin[0] / S - p) < 5 * sig
    assert abs(hmax[1] / S - p) < 5 * sig
    assert abs(hmax[0] / S - (1 - p)) < 5 * sig


def test_mvn_diagonal_matches_quadrature(orc):
    scipy_integrate = pytest.importorskip("scipy.integrate")
    rng = np.random.default_rng(12)
    mu = rng.normal(0, 0.5, (3, 3))
    var = rng.uniform(0.2, 1.0, (3, 3))
    offs = ((0, 0), (0, 1), (-1, 0), (0, -1), (1, 0))
    prm = H_.mvn_params(3, 3, mu, lambda y, x, pr: np.diag(
        [var[y + dy, x + dx] if p_ else 0 for (dy, dx), p_ in zip(offs, pr)]))
    S = 400_000
    hmin, hmax, _, _ = orc.mvn_mc_at(prm, [4], S, seed=99)
    sd = np.sqrt(var)

    def integrand(t, want_max):
        v = math.exp(-0.5 * ((t - mu[1, 1]) / sd[1, 1]) ** 2) / (sd[1, 1] * math.sqrt(2 * math.pi))
        for dy, dx in offs[1:]:
            c = _phi((t - mu[1 + dy, 1 + dx]) / sd[1 + dy, 1 + dx])
            v *= c if want_max else 1 - c
        return v
    for hits, wm in ((hmin[0], False), (hmax[0], True)):
        p = scipy_integrate.quad(integrand, -20, 20, args=(wm,), epsabs=1e-13, limit=200)[0]
        assert abs(hits / S - p) < 5 * math.sqrt(p * (1 - p) / S) + 1e-9


def test_mvn_exchangeable_is_one_over_k_plus_one(orc):
    mu = np.full((3, 4), 0.7)
    rho, s2 = 0.6, 0.9

    def cov(y, x, pr):
        return s2 * ((1 - rho) * np.eye(5) + rho * np.ones((5, 5)))
    prm = H_.mvn_params(3, 4, mu, cov)
    S = 200_000
    idx = np.array([5, 0, 1])   # interior, corner, edge
    hmin, hmax, _, st = orc.mvn_mc_at(prm, idx, S, seed=3)
    for h, k in zip(hmin, (4, 2, 3)):
        p = 1 / (k + 1)
        assert abs(h / S - p) < 5 * math.sqrt(p * (1 - p) / S)
    for h, k in zip(hmax, (4, 2, 3)):
        p = 1 / (k + 1)
        assert abs(h / S - p) < 5 * math.sqrt(p * (1 - p) / S)


def test_mvn_degenerate_and_jitter(orc):
    mu = np.array([[0.0, 1.0, 2.0]])
    prm = H_.mvn_params(1, 3, mu, lambda y, x, pr: np.zeros((5, 5)))
    hmin, hmax, _, st = orc.mvn_mc_at(prm, [0, 1, 2], 100, seed=1)
    assert hmin.tolist() == [100, 0, 0] and hmax.tolist() == [0, 0, 100]
    assert (st == orc.ST_DEGENERATE).all()
    # rank-deficient covariance: identical neighbours -> jitter path
    prm = H_.mvn_params(1, 3, mu, lambda y, x, pr: np.ones((5, 5)))
    _, _, _, st = orc.mvn_mc_at(prm, [1], 100, seed=1)
    assert st[0] & orc.ST_CHOL_JITTER


# --------------------------------------------------------------------------
# gradients


def _loss(orc, p, model, W, cptype, bins):
    pmin, pmax, _ = orc.prob(p, model, bins=bins)
    return float(((pmin if cptype == 1 else pmax) * W).sum())


@pytest.mark.parametrize("model", [0, 1, 2])
@pytest.mark.parametrize("cptype", [1, 2])
def test_gradient_matches_central_differences(orc, model, cptype):
    rng = np.random.default_rng(40 + 3 * model + cptype)
    bins = 4
    p = H_.random_params(model, 4, 5, rng, bins=bins)
    W = rng.uniform(0, 1, (4, 5))
    g = orc.grad(p, model, W, cptype=cptype, bins=bins)
    nq = g.shape[0]
    off = 2 if model == 2 else 0
    h = 1e-6
    worst = 0.0
    for q in range(nq):
        for y in range(4):
            for x in range(5):
                pp = p.copy()
                pm = p.copy()
                pp[off + q, y, x] += h
                pm[off + q, y, x] -= h
                fd = (_loss(orc, pp, model, W, cptype, bins) -
                      _loss(orc, pm, model, W, cptype, bins)) / (2 * h)
                worst = max(worst, abs(fd - g[q, y, x]) / (1 + abs(fd)))
    assert worst < 2e-6


def _fd_check(orc, p, model, W, cptype, bins, boundary, skip=(), h=1e-6):
    """Central differences of the loss against orc.grad at every parameter
    (q, y, x) not in `skip`; returns the worst relative difference and the
    gradient."""
    g = orc.grad(p, model, W, cptype=cptype, bins=bins, boundary=boundary)
    off = 2 if model == 2 else 0
    worst = 0.0

    def loss(pp):
        pmin, pmax, _ = orc.prob(pp, model, bins=bins, boundary=boundary)
        return float(((pmin if cptype == 1 else pmax) * W).sum())
    for q in range(g.shape[0]):
        for y in range(p.shape[1]):
            for x in range(p.shape[2]):
                if (q, y, x) in skip:
                    continue
                pp = p.copy()
                pm = p.copy()
                pp[off + q, y, x] += h
                pm[off + q, y, x] -= h
                fd = (loss(pp) - loss(pm)) / (2 * h)
                worst = max(worst, abs(fd - g[q, y, x]) / (1 + abs(fd)))
    return worst, g


@pytest.mark.parametrize("model", [0, 1, 2])
@pytest.mark.parametrize("cptype", [1, 2])
def test_gradient_boundary_zero_mode_matches_central_differences(orc, model, cptype):
    """Boundary mode 1 writes P = 0 at every vertex with fewer than four
    neighbours, so those vertices drop out of the loss; a vertex on the
    boundary still has gradient through its interior neighbours.  A skip
    keyed on the wrong vertex (u's neighbour count instead of v's) changes
    the gradient of every boundary vertex and fails here."""
    rng = np.random.default_rng(140 + 3 * model + cptype)
    bins = 4
    p = H_.random_params(model, 5, 6, rng, bins=bins)
    W = rng.uniform(0.5, 1, (5, 6))
    worst, g = _fd_check(orc, p, model, W, cptype, bins, boundary=1)
    assert worst < 2e-6
    # the corner has no interior neighbour on a 5 x 6 grid: zero gradient
    assert np.all(g[:, 0, 0] == 0.0) and np.all(g[:, -1, -1] == 0.0)
    # edge vertices next to interior ones do have gradients
    edge = np.concatenate([g[:, 0, 1:-1], g[:, -1, 1:-1], g[:, 1:-1, 0], g[:, 1:-1, -1]], 1)
    assert np.abs(edge).max() > 1e-3
    # and they differ from mode 0 (the edge vertices' own P is dropped)
    g0 = orc.grad(p, model, W, cptype=cptype, bins=bins, boundary=0)
    assert np.abs(g0[:, 0, :] - g[:, 0, :]).max() > 1e-3


def _point_mass_grid(model, rng, bins):
    """A 6 x 7 grid with point masses at an interior vertex, an edge
    vertex, a corner and two adjacent interior vertices (so that a point
    mass is both a centre and a neighbour of a point mass)."""
    p = H_.random_params(model, 6, 7, rng, bins=bins)
    sites = ((2, 3), (0, 4), (0, 0), (4, 1), (4, 2))
    for (y, x) in sites:
        if model == 1:
            p[1, y, x] = 0.0
        else:
            p[1, y, x] = p[0, y, x]
    return p, sites


@pytest.mark.parametrize("model", [0, 1, 2])
@pytest.mark.parametrize("cptype", [1, 2])
def test_gradient_point_masses_match_central_differences(orc, model, cptype):
    """Point masses (all members equal) as centres and as neighbours.
    Histogram: P is linear in every vertex's masses, point masses
    included, so central differences are exact to rounding for every mass
    (a wrong sign in the point-mass neighbour factor [x < c] / [x > c]
    fails here).  Uniform / Epanechnikov: every parameter of the other
    vertices is checked by central differences; the point mass's own
    support parameters are not differentiable there (a > b and w < 0 are
    invalid, so only one side exists) and the reading is that their
    derivative is 0, which is asserted exactly."""
    rng = np.random.default_rng(150 + 3 * model + cptype)
    bins = 4
    p, sites = _point_mass_grid(model, rng, bins)
    W = rng.uniform(0.5, 1, (6, 7))
    nq = bins if model == 2 else 2
    skip = () if model == 2 else {(q, y, x) for (y, x) in sites for q in range(nq)}
    worst, g = _fd_check(orc, p, model, W, cptype, bins, boundary=0, skip=skip)
    assert worst < 2e-6
    if model != 2:
        for (y, x) in sites:
            assert np.all(g[:, y, x] == 0.0)
    else:
        # a point-mass centre's mass derivative is the product of the
        # neighbours' strict tails at its position; it is not zero here
        assert np.abs(g[:, 2, 3]).max() > 1e-3


def test_gradient_point_mass_histogram_closed_form(orc):
    """Hand-built 1 x 3 histogram line: a point mass c = 0.5 of total mass
    T between two one-bin histograms U[0, 1] (mass s) and U[0.25, 1.25]
    (mass r).  P_min(centre) = T * s * (1 - 0.5) * r * (1.25 - 0.5) / 1, so
    dP/dT = 0.375 s r, dP/ds = 0.375 T r, dP/dr = 0.375 T s; with weight 1 on
    the centre only."""
    T, s, r = 0.7, 1.3, 0.9
    p = np.array([[[0.0, 0.5, 0.25]], [[1.0, 0.5, 1.25]], [[s, T, r]]])
    W = np.array([[0.0, 1.0, 0.0]])
    g = orc.grad(p, 2, W, cptype=1, bins=1)
    assert abs(orc.prob(p, 2, bins=1)[0][0, 1] - 0.375 * T * s * r) < 1e-15
    np.testing.assert_allclose(g[0, 0], [0.375 * T * r, 0.375 * s * r, 0.375 * T * s],
                               rtol=0, atol=1e-15)
    # maximum: Pr[X_l < c] = 0.5 s, Pr[X_r < c] = 0.25 r
    g = orc.grad(p, 2, W, cptype=2, bins=1)
    np.testing.assert_allclose(g[0, 0], [0.125 * T * r, 0.125 * s * r, 0.125 * T * s],
                               rtol=0, atol=1e-15)


def test_gradient_identities(orc):
    """Translation and scale invariance of each P_v (all five participants
    shifted/scaled together) and Euler's identity for histogram masses."""
    rng = np.random.default_rng(77)
    for model in (0, 1):
        p = H_.random_params(model, 3, 3, rng)
        onehot = np.zeros((3, 3))
        onehot[1, 1] = 1.0
        for cptype in (1, 2):
            g = orc.grad(p, model, onehot, cptype=cptype)
            if model == 0:
                assert abs((g[0] + g[1]).sum()) < 1e-12
                assert abs((p[0] * g[0] + p[1] * g[1]).sum()) < 1e-12
            else:
                assert abs(g[0].sum()) < 1e-12
                assert abs((p[0] * g[0] + p[1] * g[1]).sum()) < 1e-12
    p = H_.random_params(2, 3, 3, rng, bins=5)
    onehot = np.zeros((3, 3))
    onehot[1, 1] = 1.0
    for cptype in (1, 2):
        g = orc.grad(p, 2, onehot, cptype=cptype, bins=5)
        P = orc.prob(p, 2, bins=5)[cptype - 1][1, 1]
        for (y, x) in ((1, 1), (0, 1), (1, 0), (1, 2), (2, 1)):
            assert abs((p[2:, y, x] * g[:, y, x]).sum() - P) < 1e-13


# --------------------------------------------------------------------------
# saddle probability (Eq. saddleProb)


@pytest.mark.parametrize("model", [0, 1, 2])
def test_saddle_exchangeable(orc, model):
    """i.i.d. variables: t1 needs X_n, X_s < X_1 < X_e, X_w, one ordering in
    5!/(2!2!) = 30, so P = 2/30 = 1/15 inside; on a line 2 * 1/3! = 1/3;
    0 on the boundary of a 2D grid."""
    rng = np.random.default_rng(70)
    one = H_.random_params(model, 1, 1, rng, bins=5)
    p = np.broadcast_to(one, (one.shape[0], 4, 5)).copy()
    sad, _ = orc.saddle(p, model, bins=5)
    ref = np.zeros((4, 5))
    ref[1:-1, 1:-1] = 1.0 / 15
    np.testing.assert_allclose(sad, ref, atol=1e-13)
    line = np.broadcast_to(one, (one.shape[0], 1, 6)).copy()
    sad, _ = orc.saddle(line, model, bins=5)
    np.testing.assert_allclose(sad[0], [0, 1 / 3, 1 / 3, 1 / 3, 1 / 3, 0], atol=1e-13)
    col = np.broadcast_to(one, (one.shape[0], 6, 1)).copy()
    sad, _ = orc.saddle(col, model, bins=5)
    np.testing.assert_allclose(sad[:, 0], [0, 1 / 3, 1 / 3, 1 / 3, 1 / 3, 0], atol=1e-13)


@pytest.mark.parametrize("model", [0, 1, 2])
def test_saddle_invariances(orc, model):
    """X -> -X swaps t1 and t2; transposing the grid swaps the roles of the
    axes (e <-> s, n <-> w), which also swaps t1 and t2: both leave P."""
    rng = np.random.default_rng(71 + model)
    p = H_.random_params(model, 6, 7, rng, bins=5)
    sad, _ = orc.saddle(p, model, bins=5)
    neg, _ = orc.saddle(H_.negate_params(p, model), model, bins=5)
    tr, _ = orc.saddle(np.ascontiguousarray(p.transpose(0, 2, 1)), model, bins=5)
    np.testing.assert_allclose(neg, sad, atol=1e-13)
    np.testing.assert_allclose(tr.T, sad, atol=1e-13)


@pytest.mark.parametrize("model", [0, 1, 2])
def test_saddle_bruteforce_monte_carlo(orc, model):
    rng = np.random.default_rng(81 + model)
    p = H_.random_params(model, 4, 5, rng, bins=4, spread=0.6)
    n = 2_000_000
    mc = H_.mc_saddle(p, model, n, seed=500 + model)
    sad, _ = orc.saddle(p, model, bins=4)
    sig = np.sqrt(np.maximum(sad * (1 - sad), 1e-12) / n)
    assert (np.abs(mc - sad) / sig).max() < 5.5


def test_saddle_mvn_diagonal_quadrature(orc):
    scipy_integrate = pytest.importorskip("scipy.integrate")
    rng = np.random.default_rng(13)
    mu = rng.normal(0, 0.3, (3, 3))
    var = rng.uniform(0.2, 1.0, (3, 3))
    offs = ((0, 0), (0, 1), (-1, 0), (0, -1), (1, 0))
    prm = H_.mvn_params(3, 3, mu, lambda y, x, pr: np.diag(
        [var[y + dy, x + dx] if p_ else 0 for (dy, dx), p_ in zip(offs, pr)]))
    S = 400_000
    _, _, _, _, hs = orc.mvn_mc_at(prm, [4], S, seed=5, with_saddle=True)
    sd = np.sqrt(var)

    def integrand(t):
        v = math.exp(-0.5 * ((t - mu[1, 1]) / sd[1, 1]) ** 2) / (sd[1, 1] * math.sqrt(2 * math.pi))
        c = [_phi((t - mu[1 + dy, 1 + dx]) / sd[1 + dy, 1 + dx]) for dy, dx in offs[1:]]
        g = [1 - q for q in c]
        return v * (g[0] * c[1] * g[2] * c[3] + c[0] * g[1] * c[2] * g[3])
    p = scipy_integrate.quad(integrand, -20, 20, epsabs=1e-13, limit=200)[0]
    assert abs(hs[0] / S - p) < 5 * math.sqrt(p * (1 - p) / S)


# --------------------------------------------------------------------------
# semianalytical histogram estimator (Sec. Semianalytical Solution)


def test_semianalytical_converges_to_closed_form(orc):
    rng = np.random.default_rng(91)
    B = 6
    p = H_.random_params(2, 5, 6, rng, bins=B)
    idx = np.arange(30)
    c = 100_000
    smin, smax, ssad, sdmin, sdmax = orc.semi_at(p, B, idx, c, seed=17)
    rmin, rmax, _ = orc.prob_at(p, 2, idx, bins=B)
    rsad, _ = orc.saddle(p, 2, bins=B, idx=idx)
    zmin = np.abs(smin - rmin) / np.maximum(sdmin, 1e-12)
    zmax = np.abs(smax - rmax) / np.maximum(sdmax, 1e-12)
    assert zmin.max() < 5.5 and zmax.max() < 5.5
    # the saddle estimate: the per-sample terms lie in [0, 1]
    assert np.abs(ssad - rsad).max() < 5.5 * 0.5 / np.sqrt(c)
    # the error shrinks like 1/sqrt(c)
    s2, _, _, _, _ = orc.semi_at(p, B, idx, c // 100, seed=17)
    assert np.abs(s2 - rmin).mean() > 3 * np.abs(smin - rmin).mean()


def test_semianalytical_point_mass_centre_is_exact(orc):
    rng = np.random.default_rng(92)
    B = 4
    p = H_.random_params(2, 3, 3, rng, bins=B)
    p[1, 1, 1] = p[0, 1, 1]           # centre is a point mass
    smin, smax, ssad, sdmin, _ = orc.semi_at(p, B, [4], 7, seed=1)
    rmin, rmax, _ = orc.prob_at(p, 2, [4], bins=B)
    rsad, _ = orc.saddle(p, 2, bins=B, idx=[4])
    assert abs(smin[0] - rmin[0]) < 1e-14 and abs(smax[0] - rmax[0]) < 1e-14
    assert abs(ssad[0] - rsad[0]) < 1e-14 and sdmin[0] == 0.0
