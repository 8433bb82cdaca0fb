"""GPU independent-Gaussian model (the parametric model of the paper's model
comparison, Sec. Comparison of Parametric Vs. Nonparametric Models) against
the oracle's adaptive quadrature: |dP| <= 1e-5 on the GPU's FP32 parameters
for minimum, maximum and saddle; and the multivariate-Gaussian Monte Carlo
with a diagonal covariance (independent Gaussians sampled) within its
sampling error of the quadrature."""
import numpy as np
import pytest
import torch

import helpers as H_

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def ucp():
    from paper_2407_18015_gb300 import build
    build.build()
    from paper_2407_18015_gb300 import ucp as u
    return u


@pytest.fixture(scope="module")
def ctx(ucp):
    c = ucp.Context(0)
    yield c
    c.close()


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _cmp(g, r, what):
    a = g.cpu().numpy().astype(np.float64)
    assert (np.isnan(a) == np.isnan(r)).all(), what
    ok = ~np.isnan(r)
    d = np.abs(a[ok] - r[ok])
    assert d.max() <= TOL, f"{what}: {d.max():.3e}"


@pytest.mark.parametrize("shape", [(64, 64), (37, 45), (1, 40)])
def test_gauss_from_members(ucp, ctx, orc, shape):
    from paper_2407_18015_gb300 import synth
    H, W = shape
    ens_np = synth.ensemble_bimodal(H, W, 20, seed=21, lam_scale=0.5)
    ens = _dev(ens_np)
    desc = ucp.make_desc("gaussian")
    params = ctx.fit(ens, desc)
    pmin, pmax, st = ctx.probability(ens, desc)
    sad, sst = ctx.saddle(ens, desc)
    torch.cuda.synchronize()
    gp = params.double().cpu().numpy()
    op, _ = orc.fit(ens_np, orc.GAUSSIAN)
    np.testing.assert_allclose(gp[0], op[0], rtol=0, atol=4e-6)
    np.testing.assert_allclose(gp[1], op[1], rtol=2e-6, atol=1e-7)
    rmin, rmax, rsad, rst = orc.gauss(gp)
    _cmp(pmin, rmin, "min")
    _cmp(pmax, rmax, "max")
    _cmp(sad, rsad, "saddle")
    np.testing.assert_array_equal(st.cpu().numpy(), rst)


def test_gauss_from_params_edge_cases(ucp, ctx, orc):
    rng = np.random.default_rng(22)
    H, W = 11, 17
    m = rng.normal(0, 0.7, (H, W))
    s = rng.uniform(0.05, 1.2, (H, W))
    s[2, 3] = 0.0                    # point-mass centre
    s[5, 6] = 0.0                    # point-mass neighbour of (5,5), (4,6), ...
    s[7, 8] = 1e-4                   # a very sharp one
    s[8, 1] = 30.0                   # a very wide one
    m[9, 9] = np.nan
    s[1, 12] = -0.3
    p = np.stack([m, s]).astype(np.float32)
    for boundary in (0, 1):
        desc = ucp.make_desc("gaussian", boundary=boundary)
        pmin, pmax, st = ctx.probability_from_params(_dev(p), desc)
        sad, _ = ctx.saddle_from_params(_dev(p), desc)
        torch.cuda.synchronize()
        rmin, rmax, rsad, rst = orc.gauss(p.astype(np.float64), boundary=boundary)
        _cmp(pmin, rmin, f"min b{boundary}")
        _cmp(pmax, rmax, f"max b{boundary}")
        _cmp(sad, rsad, f"saddle b{boundary}")
        np.testing.assert_array_equal(st.cpu().numpy(), rst)


def test_gauss_matches_independent_gaussian_monte_carlo(ucp, ctx, orc):
    """The multivariate-Gaussian Monte Carlo with the covariance reduced to
    its diagonal samples independent Gaussians: its estimate must agree
    with the quadrature within the binomial error."""
    from paper_2407_18015_gb300 import synth
    ens = _dev(synth.ensemble_bimodal(48, 48, 20, seed=23, lam_scale=0.5))
    gdesc = ucp.make_desc("gaussian")
    gmin, gmax, _ = ctx.probability(ens, gdesc)
    S = 20000
    mdesc = ucp.make_desc("mvn", mc_samples=S, seed=77)
    mp = ctx.fit(ens, mdesc)
    diag = {5, 7, 10, 14, 19}        # (i, i) entries of the packed lower triangle
    for q in range(5, 20):
        if q not in diag:
            mp[q].zero_()
    mmin, mmax, _ = ctx.probability_from_params(mp, mdesc)
    torch.cuda.synchronize()
    for g, mc in ((gmin, mmin), (gmax, mmax)):
        P = g.double().cpu().numpy()
        E = mc.double().cpu().numpy()
        z = (E - P) / np.sqrt(np.maximum(P * (1 - P), 1e-9) / S)
        assert np.abs(z).max() < 6.0
        assert abs(z.mean()) < 0.1


def test_gauss_unsupported(ucp, ctx):
    p = torch.zeros((2, 8, 8), device="cuda")
    w = torch.zeros((8, 8), device="cuda")
    with pytest.raises(ucp.UcpError) as e:
        ucp.ucp_backward(ctx.handle, p, ucp.make_desc("gaussian"), 1, w, p)
    assert e.value.status == ucp.UCP_ERR_UNSUPPORTED
    with pytest.raises(ucp.UcpError) as e:
        ctx.probability_from_params(p, ucp.make_desc("gaussian", stencil=2))
    assert e.value.status == ucp.UCP_ERR_UNSUPPORTED
