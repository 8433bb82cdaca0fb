"""GPU parity of the larger neighbour sets (six- and eight-neighbour 2D
stencils, six axis neighbours of a 3D grid; the extension named in the
paper's Sec. Conclusion) against the FP64 oracle, through the C ABI.

Tolerance: |P_gpu - P_oracle| <= 1e-5 per vertex on the GPU's own FP32
parameters (widened to FP64 for the oracle), as for the four-neighbour path.
"""
import numpy as np
import pytest
import torch

import helpers as H_

pytestmark = pytest.mark.gpu

TOL = 1e-5
MODELS = [("uniform", 0), ("epanechnikov", 0), ("histogram", 8)]
STENCILS = [(1, 1), (2, 1), (3, 5)]          # (stencil, slices D)


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


def _compare(p_gpu, p_ref, tol=TOL, what=""):
    a = p_gpu.cpu().numpy().astype(np.float64).reshape(p_ref.shape)
    nan_a, nan_b = np.isnan(a), np.isnan(p_ref)
    assert (nan_a == nan_b).all(), f"{what}: NaN pattern differs"
    d = np.abs(a[~nan_a] - p_ref[~nan_b])
    if d.size:
        assert d.max() <= tol, f"{what}: max |diff| {d.max():.3e} at {np.argmax(d)}"
    return float(d.max()) if d.size else 0.0


def _ensemble(D, H, W, N, seed):
    from paper_2407_18015_gb300 import synth
    e = synth.ensemble_bimodal(D * H, W, N, seed=seed, lam_scale=0.5)
    return e.reshape(N, D, H, W) if D > 1 else e


@pytest.mark.parametrize("stencil,D", STENCILS)
@pytest.mark.parametrize("model,bins", MODELS)
def test_stencil_from_members(ucp, ctx, orc, model, bins, stencil, D):
    H, W = (13, 21) if D > 1 else (37, 45)
    ens_np = _ensemble(D, H, W, 20, seed=60 + stencil)
    ens = _dev(ens_np)
    desc = ucp.make_desc(model, bins=bins or 8, stencil=stencil, depth=D)
    params = ctx.fit(ens, desc)
    pmin, pmax, st = ctx.probability(ens, desc)
    torch.cuda.synchronize()
    gp = params.double().cpu().numpy()
    rmin, rmax, rst = orc.prob_stencil(gp, desc.model, stencil, bins=desc.bins)
    _compare(pmin, rmin, what=f"{model} stencil {stencil} min")
    _compare(pmax, rmax, what=f"{model} stencil {stencil} max")
    np.testing.assert_array_equal(st.cpu().numpy().reshape(rst.shape), rst)
    if model != "epanechnikov":
        # the per-vertex fit is the four-neighbour one: bit-exact
        op, _ = orc.fit(ens_np.reshape(20, D * H, W), desc.model, bins=desc.bins)
        np.testing.assert_array_equal(gp.reshape(op.shape)[:2], op[:2])


@pytest.mark.parametrize("stencil,D", STENCILS)
@pytest.mark.parametrize("model,bins", MODELS)
def test_stencil_from_params_edge_cases(ucp, ctx, orc, model, bins, stencil, D):
    mid = {"uniform": 0, "epanechnikov": 1, "histogram": 2}[model]
    rng = np.random.default_rng(70 + stencil)
    H, W = (6, 9) if D > 1 else (11, 17)
    p = H_.random_params(mid, D * H, W, rng, bins=bins or 4).astype(np.float32)
    flat = p.reshape(p.shape[0], -1)
    V = flat.shape[1]
    # point masses (centre and neighbour), a NaN, invalid parameters
    for v in (3, 4, V // 2):
        if mid == 1:
            flat[1, v] = 0.0
        else:
            flat[1, v] = flat[0, v]
    flat[0, V - 5] = np.nan
    if mid == 1:
        flat[1, V - 9] = -0.5
    else:
        flat[0, V - 9] = flat[1, V - 9] + 1.0
    if mid == 2:
        flat[2:, 7] *= 1.7                  # masses not summing to one
    pp = p.reshape((p.shape[0], D, H, W)) if D > 1 else p
    for boundary in (0, 1):
        desc = ucp.make_desc(model, bins=bins or 4, stencil=stencil, depth=D, boundary=boundary)
        pmin, pmax, st = ctx.probability_from_params(_dev(pp), desc)
        torch.cuda.synchronize()
        rmin, rmax, rst = orc.prob_stencil(pp.astype(np.float64), mid, stencil,
                                           bins=bins or 4, boundary=boundary)
        _compare(pmin, rmin, what=f"{model} st{stencil} b{boundary} min")
        _compare(pmax, rmax, what=f"{model} st{stencil} b{boundary} max")
        np.testing.assert_array_equal(st.cpu().numpy().reshape(rst.shape), rst)


@pytest.mark.parametrize("stencil,shape", [(2, (1, 1024, 1024)), (3, (64, 128, 128))])
def test_stencil_full_size_sampled(ucp, ctx, orc, stencil, shape):
    """The benchmark's sizes: all three models, 2000 sampled vertices each."""
    D, H, W = shape
    ens_np = _ensemble(D, H, W, 20, seed=80 + stencil)
    ens = _dev(ens_np)
    rng = np.random.default_rng(81)
    idx = np.concatenate([[0, D * H * W - 1, W - 1],
                          rng.integers(0, D * H * W, 2000)]).astype(np.int64)
    for model, bins in MODELS:
        desc = ucp.make_desc(model, bins=bins or 8, stencil=stencil, depth=D)
        params = ctx.fit(ens, desc)
        pmin, pmax, _ = ctx.probability(ens, desc)
        torch.cuda.synchronize()
        gp = params.double().cpu().numpy()
        rmin, rmax, _ = orc.prob_stencil(gp, desc.model, stencil, bins=desc.bins, idx=idx)
        _compare(pmin.reshape(-1)[torch.from_numpy(idx).cuda()], rmin, what=f"{model} min")
        _compare(pmax.reshape(-1)[torch.from_numpy(idx).cuda()], rmax, what=f"{model} max")
        del params, pmin, pmax
    del ens


def test_stencil_unsupported_and_invalid(ucp, ctx):
    ens = _dev(_ensemble(1, 8, 8, 10, seed=90))
    out = torch.empty((8, 8), device="cuda")
    for kw, status in ((dict(model="mvn", stencil=2), ucp.UCP_ERR_UNSUPPORTED),
                       (dict(model="histogram_semi", stencil=1), ucp.UCP_ERR_UNSUPPORTED),
                       (dict(model="uniform", stencil=5), ucp.UCP_ERR_ARG)):
        with pytest.raises(ucp.UcpError) as e:
            ucp.ucp_probability(ctx.handle, ens, ucp.make_desc(**kw), 3, out, out)
        assert e.value.status == status
    with pytest.raises(ucp.UcpError) as e:
        ucp.ucp_saddle(ctx.handle, ens, ucp.make_desc("uniform", stencil=2), out)
    assert e.value.status == ucp.UCP_ERR_UNSUPPORTED
    p = ctx.fit(ens, ucp.make_desc("uniform"))
    with pytest.raises(ucp.UcpError) as e:
        ucp.ucp_backward(ctx.handle, p, ucp.make_desc("uniform", stencil=1), 1, out, p)
    assert e.value.status == ucp.UCP_ERR_UNSUPPORTED
    # depth > 1 needs the 3D stencil
    e4 = ens.reshape(10, 2, 4, 8)
    with pytest.raises(ucp.UcpError) as e:
        ucp.ucp_probability(ctx.handle, e4, ucp.make_desc("uniform", stencil=2, depth=2), 3,
                            out, out)
    assert e.value.status == ucp.UCP_ERR_ARG
