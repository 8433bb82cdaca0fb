"""GPU saddle probability (Eq. saddleProb) against the oracle: closed-form
models within 1e-5 on the same FP32 parameters; the Monte Carlo model at
identical Philox streams within the near-tie bound."""
import numpy as np
import pytest
import torch

import helpers as H_

pytestmark = pytest.mark.gpu

MODELS = [("uniform", 0, 0), ("epanechnikov", 1, 0), ("histogram", 2, 8)]


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


def _cmp(g, ref):
    a = g.cpu().numpy().astype(np.float64)
    assert (np.isnan(a) == np.isnan(ref)).all()
    ok = ~np.isnan(ref)
    if ok.any():
        assert np.abs(a[ok] - ref[ok]).max() <= 1e-5


@pytest.mark.parametrize("model,mid,bins", MODELS)
@pytest.mark.parametrize("shape", [(1, 1), (1, 7), (9, 1), (2, 3), (19, 37), (33, 65)])
def test_saddle_from_members(ucp, ctx, orc, model, mid, bins, shape):
    from paper_2407_18015_gb300 import synth
    Hh, Ww = shape
    ens = _dev(synth.ensemble_bimodal(Hh, Ww, 9, seed=700 + Hh + 3 * Ww, lam_scale=0.3))
    desc = ucp.make_desc(model, bins=bins or 8)
    out, st = ctx.saddle(ens, desc)
    params = ctx.fit(ens, desc)
    torch.cuda.synchronize()
    ref, rst = orc.saddle(params.double().cpu().numpy(), mid, bins=desc.bins)
    _cmp(out, ref)
    np.testing.assert_array_equal(st.cpu().numpy(), rst)


@pytest.mark.parametrize("model,mid,bins", MODELS)
def test_saddle_from_params_edge_cases(ucp, ctx, orc, model, mid, bins):
    rng = np.random.default_rng(31 + mid)
    p = H_.random_params(mid, 14, 15, rng, bins=bins or 8)
    if mid == 1:
        p[1, 4, 4] = 0.0
    else:
        p[1, 4, 4] = p[0, 4, 4]
    p[:, 7, 7] = p[:, 7, 8]
    p[0, 10, 3] = np.nan
    p32 = p.astype(np.float32)
    desc = ucp.make_desc(model, bins=bins or 8)
    out, st = ctx.saddle_from_params(_dev(p32), desc)
    torch.cuda.synchronize()
    ref, rst = orc.saddle(p32.astype(np.float64), mid, bins=desc.bins)
    _cmp(out, ref)
    np.testing.assert_array_equal(st.cpu().numpy(), rst)


def test_saddle_full_size_sampled(ucp, ctx, orc):
    from paper_2407_18015_gb300 import synth
    ens = _dev(synth.ensemble_bimodal(1024, 1024, 20, seed=2))
    rng = np.random.default_rng(1)
    idx = rng.integers(0, 1024 * 1024, 2000)
    for model, mid, bins in MODELS:
        desc = ucp.make_desc(model, bins=bins or 8)
        out, _ = ctx.saddle(ens, desc)
        params = ctx.fit(ens, desc)
        torch.cuda.synchronize()
        ref, _ = orc.saddle(params.double().cpu().numpy(), mid, bins=desc.bins, idx=idx)
        a = out.cpu().numpy().ravel()[idx]
        assert np.abs(a - ref).max() <= 1e-5


def test_saddle_mvn_identical_streams(ucp, ctx, orc):
    from paper_2407_18015_gb300 import synth
    for shape in ((24, 31), (1, 40)):
        ens_np = synth.ensemble_correlated(shape[0], shape[1], 40, seed=17) if shape[0] > 1 \
            else synth.ensemble_iid(1, 40, 40, seed=17)
        prm, _ = orc.fit(ens_np, orc.MVN)
        p32 = prm.astype(np.float32)
        S = 10_000
        desc = ucp.make_desc("mvn", mc_samples=S, seed=77)
        out, st = ctx.saddle_from_params(_dev(p32), desc)
        torch.cuda.synchronize()
        idx = np.arange(shape[0] * shape[1])
        _, _, ties, ost, hs = orc.mvn_mc_at(p32.astype(np.float64), idx, S, 77, with_saddle=True)
        a = out.cpu().numpy().ravel().astype(np.float64)
        assert (np.abs(a - hs / S) <= 1e-6 + ties / S).all()
        np.testing.assert_array_equal(st.cpu().numpy().ravel(), ost)
