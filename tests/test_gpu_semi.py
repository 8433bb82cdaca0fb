"""GPU semianalytical histogram estimator (Sec. Semianalytical Solution)
against the oracle's estimator at identical streams (the bin of every
sample is decided in binary32 on both sides, so only the rounding of the
sample position and of the neighbours' tails differs: |dP| <= 1e-5), and
against the closed form within its sampling error."""
import numpy as np
import pytest
import torch

import helpers as H_

pytestmark = pytest.mark.gpu


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


@pytest.mark.parametrize("B", [4, 8, 16])
def test_semi_identical_streams(ucp, ctx, orc, B):
    rng = np.random.default_rng(50 + B)
    p = H_.random_params(2, 21, 34, rng, bins=B)
    p[1, 3, 3] = p[0, 3, 3]              # a point-mass centre (exact)
    p[2:, 5, 5] *= 1.3                   # masses not summing to 1
    p[0, 9, 9] = np.nan
    p32 = p.astype(np.float32)
    S = 1000
    desc = ucp.make_desc("histogram_semi", bins=B, mc_samples=S, seed=0xABC, field_id=3)
    pmin, pmax, st = ctx.probability_from_params(_dev(p32), desc)
    sad, _ = ctx.saddle_from_params(_dev(p32), desc)
    torch.cuda.synchronize()
    idx = np.arange(21 * 34)
    rmin, rmax, rsad, _, _ = orc.semi_at(p32.astype(np.float64), B, idx, S, 0xABC, field=3)
    for g, r in ((pmin, rmin), (pmax, rmax), (sad, rsad)):
        a = g.cpu().numpy().ravel().astype(np.float64)
        assert (np.isnan(a) == np.isnan(r)).all()
        ok = ~np.isnan(r)
        assert np.abs(a[ok] - r[ok]).max() <= 1e-5
    ref_st = orc.prob(p32.astype(np.float64), 2, bins=B)[2]
    np.testing.assert_array_equal(st.cpu().numpy(), ref_st)


def test_semi_from_members_converges_to_closed_form(ucp, ctx, orc):
    from paper_2407_18015_gb300 import synth
    ens = synth.ensemble_bimodal(64, 96, 20, seed=9, lam_scale=0.5)
    S = 20000
    desc = ucp.make_desc("histogram_semi", bins=8, mc_samples=S, seed=5)
    pmin, pmax, _ = ctx.probability(_dev(ens), desc)
    torch.cuda.synchronize()
    prm, _ = orc.fit(ens, 2, bins=8)
    rmin, rmax, _ = orc.prob(prm, 2, bins=8)
    idx = np.arange(64 * 96)
    _, _, _, sdmin, sdmax = orc.semi_at(prm, 8, idx, S, 5)
    zmin = np.abs(pmin.cpu().numpy().ravel() - rmin.ravel()) / np.maximum(sdmin, 1e-9)
    zmax = np.abs(pmax.cpu().numpy().ravel() - rmax.ravel()) / np.maximum(sdmax, 1e-9)
    assert np.percentile(zmin, 99) < 4.0 and np.percentile(zmax, 99) < 4.0
    assert np.abs(pmin.cpu().numpy() - rmin).max() < 0.02


def test_semi_rejected_where_unsupported(ucp, ctx):
    desc = ucp.make_desc("histogram_semi", bins=8)
    p = torch.zeros((10, 4, 5), device="cuda")
    with pytest.raises(ucp.UcpError) as e:
        ctx.backward(p, desc, 1, torch.zeros((4, 5), device="cuda"))
    assert e.value.status == ucp.UCP_ERR_UNSUPPORTED
    with pytest.raises(ucp.UcpError) as e:
        ctx.probability_from_params(p, ucp.make_desc("histogram_semi", bins=8, mc_samples=0))
    assert e.value.status == ucp.UCP_ERR_ARG
