"""GPU adjoint (ucp_backward) against the oracle gradient and against FP64
central finite differences of the oracle, through the C ABI; and the
torch.autograd.Function wrapper.

Tolerance: |g_gpu - g_ref| <= 1e-4 |g_ref| + 2e-5 max(1, max|g_ref|): the
partials are sums of FP32 products of values in [0, 1] scaled by inverse
support widths, so their relative error is a few 1e-6; the absolute floor
covers entries that cancel to ~0.
"""
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


def _close(g, ref, what):
    g = g.astype(np.float64)
    scale = max(1.0, np.abs(ref).max())
    err = np.abs(g - ref)
    lim = 1e-4 * np.abs(ref) + 2e-5 * scale
    bad = err > lim
    assert not bad.any(), (what, np.argwhere(bad)[:4].tolist(), g[bad][:4], ref[bad][:4])


@pytest.mark.parametrize("model,mid,bins", MODELS)
@pytest.mark.parametrize("cptype", [1, 2])
@pytest.mark.parametrize("boundary", [0, 1])
def test_backward_matches_oracle(ucp, ctx, orc, model, mid, bins, cptype, boundary):
    rng = np.random.default_rng(100 + 10 * mid + cptype + 3 * boundary)
    p = H_.random_params(mid, 13, 17, rng, bins=bins or 8).astype(np.float32)
    W = rng.uniform(0, 1, (13, 17)).astype(np.float32)
    desc = ucp.make_desc(model, bins=bins or 8, boundary=boundary)
    g = ctx.backward(_dev(p), desc, cptype, _dev(W))
    torch.cuda.synchronize()
    ref = orc.grad(p.astype(np.float64), mid, W.astype(np.float64), cptype=cptype,
                   bins=bins or 8, boundary=boundary)
    _close(g.cpu().numpy(), ref, f"{model} cp{cptype} b{boundary}")


@pytest.mark.parametrize("model,mid,bins", MODELS + [("histogram", 2, 16)])
@pytest.mark.parametrize("cptype", [1, 2])
def test_backward_multi_tile_ragged(ucp, ctx, orc, model, mid, bins, cptype):
    """A grid of 3 x 3 adjoint tiles (8 x 32), ragged in both directions:
    partials handed between tiles through the rings (north / south and west
    / east) and the fix-up pass, against the oracle."""
    rng = np.random.default_rng(700 + 10 * mid + cptype + bins)
    Hh, Ww = 21, 75
    p = H_.random_params(mid, Hh, Ww, rng, bins=bins or 8).astype(np.float32)
    W = rng.uniform(0, 1, (Hh, Ww)).astype(np.float32)
    desc = ucp.make_desc(model, bins=bins or 8)
    g = ctx.backward(_dev(p), desc, cptype, _dev(W))
    torch.cuda.synchronize()
    ref = orc.grad(p.astype(np.float64), mid, W.astype(np.float64), cptype=cptype,
                   bins=bins or 8)
    _close(g.cpu().numpy(), ref, f"{model} B{bins} cp{cptype} 21x75")


@pytest.mark.parametrize("model,mid,bins", MODELS)
def test_backward_point_masses(ucp, ctx, orc, model, mid, bins):
    rng = np.random.default_rng(7)
    p = H_.random_params(mid, 7, 9, rng, bins=bins or 8)
    # point masses at a few vertices
    for (y, x) in ((2, 3), (4, 4), (0, 0)):
        if mid == 1:
            p[1, y, x] = 0.0
        else:
            p[1, y, x] = p[0, y, x]
    p = p.astype(np.float32)
    W = rng.uniform(0, 1, (7, 9)).astype(np.float32)
    for cptype in (1, 2):
        desc = ucp.make_desc(model, bins=bins or 8)
        g = ctx.backward(_dev(p), desc, cptype, _dev(W))
        torch.cuda.synchronize()
        ref = orc.grad(p.astype(np.float64), mid, W.astype(np.float64), cptype=cptype,
                       bins=bins or 8)
        _close(g.cpu().numpy(), ref, f"{model} point masses cp{cptype}")


def _crop_grad(orc, p, W, mid, bins, y0, x0, n=32, margin=2):
    Hh, Ww = W.shape
    ya, yb = max(0, y0 - margin), min(Hh, y0 + n + margin)
    xa, xb = max(0, x0 - margin), min(Ww, x0 + n + margin)
    pc = p[:, ya:yb, xa:xb].astype(np.float64)
    Wc = W[ya:yb, xa:xb].astype(np.float64)
    # the boundary of the extended crop is not the grid boundary: only the
    # inner n x n block is exact; grid-boundary rows/cols are genuine
    g = orc.grad(pc, mid, Wc, cptype=1, bins=bins)
    return g[:, y0 - ya:y0 - ya + n, x0 - xa:x0 - xa + n], (pc, Wc, ya, xa)


@pytest.mark.parametrize("model,mid,bins", [("histogram", 2, 16), ("epanechnikov", 1, 0)])
def test_backward_2048_crops_and_fd(ucp, ctx, orc, model, mid, bins):
    """2048 x 2048 x 50 bimodal ensemble, forward P_min and the adjoint of
    sum(P_min * W), W ~ U[0,1]; four 32 x 32 crops (one at a grid corner)
    against the oracle gradient and FP64 central differences."""
    from paper_2407_18015_gb300 import synth
    ens = _dev(synth.ensemble_bimodal(2048, 2048, 50, seed=4))
    W = synth.weight_field(2048, 2048, seed=44)
    desc = ucp.make_desc(model, bins=bins or 8)
    params = ctx.fit(ens, desc)
    g = ctx.backward(params, desc, 1, _dev(W))
    torch.cuda.synchronize()
    p = params.cpu().numpy()
    gg = g.cpu().numpy()
    rng = np.random.default_rng(44)
    corners = [(0, 0)] + [tuple(rng.integers(2, 2048 - 34, 2)) for _ in range(3)]
    off = 2 if mid == 2 else 0
    for (y0, x0) in corners:
        ref, (pc, Wc, ya, xa) = _crop_grad(orc, p, W, mid, bins or 8, y0, x0)
        got = gg[:, y0:y0 + 32, x0:x0 + 32]
        _close(got, ref, f"crop {y0},{x0}")
        # finite differences of the oracle on a few parameters
        for _ in range(6):
            q = int(rng.integers(0, ref.shape[0]))
            yy, xx = (int(v) for v in rng.integers(0, 32, 2))
            h = 1e-6
            pp, pm = pc.copy(), pc.copy()
            pp[off + q, y0 - ya + yy, x0 - xa + xx] += h
            if mid != 2:
                pm[off + q, y0 - ya + yy, x0 - xa + xx] -= h
            lp = (orc.prob(pp, mid, bins=bins or 8)[0] * Wc).sum()
            lm = (orc.prob(pm, mid, bins=bins or 8)[0] * Wc).sum()
            # P is linear in each mass (a zero mass cannot be decreased):
            # one-sided there, central otherwise
            fd = (lp - lm) / (h if mid == 2 else 2 * h)
            gv = got[q, yy, xx]
            assert abs(gv - fd) <= 1e-4 * abs(fd) + 5e-4 * max(1.0, abs(fd)), (q, yy, xx, gv, fd)


def test_autograd_function(ucp, ctx):
    rng = np.random.default_rng(3)
    for model, mid, bins in MODELS:
        p = _dev(H_.random_params(mid, 11, 12, rng, bins=bins or 8).astype(np.float32))
        W = _dev(rng.uniform(0, 1, (11, 12)).astype(np.float32))
        x = p.clone().requires_grad_(True)
        P = ucp.UcpProbability.apply(x, model, bins or 8, ucp.UCP_MAX, 0)
        (P * W).sum().backward()
        desc = ucp.make_desc(model, bins=bins or 8)
        g = ctx.backward(p, desc, ucp.UCP_MAX, W)
        torch.cuda.synchronize()
        if mid == 2:
            assert (x.grad[:2] == 0).all()
            assert torch.equal(x.grad[2:], g)
        else:
            assert torch.equal(x.grad, g)
