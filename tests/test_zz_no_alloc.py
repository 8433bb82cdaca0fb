"""The allocation-free adjoint (ucp_backward_static) against the context
adjoint (ucp_backward), through the C ABI, on two calls in a row.

ucp_backward_static serves callers that must not allocate device memory once
running; its scratch is a fixed device array inside the library, shared by
all calls on a device.  This file is collected last so that a run stopping
at the first failure has run every other test first; it also passes alone in
a fresh process.
"""
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


@pytest.mark.parametrize("model,mid,bins", [("uniform", 0, 0), ("epanechnikov", 1, 0),
                                            ("histogram", 2, 16)])
def test_static_adjoint_matches_context_adjoint(ucp, model, mid, bins):
    torch.cuda.set_device(0)
    ctx = ucp.Context(0)
    rng = np.random.default_rng(71 + mid)
    desc = ucp.make_desc(model, bins=bins or 8)
    # two calls in a row with different inputs and shapes: the shared scratch
    # keeps the previous call's contents, which must not leak into the next
    for (Hh, Ww, cptype) in ((37, 53, ucp.UCP_MIN), (29, 64, ucp.UCP_MAX)):
        p = torch.from_numpy(H_.random_params(mid, Hh, Ww, rng, bins=bins or 8)
                             .astype(np.float32)).cuda()
        W = torch.from_numpy(rng.uniform(0, 1, (Hh, Ww)).astype(np.float32)).cuda()
        ref = ctx.backward(p, desc, cptype, W)
        got = torch.full_like(ref, float("nan"))
        ucp.ucp_backward_static(p, desc, cptype, W, got)
        torch.cuda.synchronize()
        a, b = got.cpu().numpy().astype(np.float64), ref.cpu().numpy().astype(np.float64)
        scale = max(1.0, np.abs(b).max())
        assert np.all(np.abs(a - b) <= 1e-4 * np.abs(b) + 2e-5 * scale)
    ctx.close()


def test_static_adjoint_rejects_oversize(ucp):
    """Shapes whose scratch exceeds the fixed array are refused before any
    launch: 160 floats per 8 x 32 tile for uniform / Epanechnikov; for
    histograms of at most 16 bins 80 * B floats per tile plus 1280 * B."""
    cap = ucp.ucp_backward_static_capacity()
    assert cap == 4 << 20
    cases = [("histogram", 16, 8 * 60, 32 * 60),       # 3600 tiles: ring alone too large
             ("uniform", 8, 8 * 160, 32 * 168)]         # 26880 tiles: 4.3 M floats of rings
    for model, bins, Hh, Ww in cases:
        desc = ucp.make_desc(model, bins=bins)
        P = 2 + bins if model == "histogram" else 2
        Q = bins if model == "histogram" else 2
        tiles = ((Hh + 7) // 8) * ((Ww + 31) // 32)
        assert (tiles * 80 * bins + 1280 * bins if model == "histogram" else tiles * 160) > cap
        p = torch.zeros((P, Hh, Ww), device="cuda")
        W = torch.zeros((Hh, Ww), device="cuda")
        g = torch.zeros((Q, Hh, Ww), device="cuda")
        with pytest.raises(ucp.UcpError) as e:
            ucp.ucp_backward_static(p, desc, ucp.UCP_MIN, W, g)
        assert e.value.status == ucp.UCP_ERR_SHAPE


def test_static_adjoint_checks_shapes_before_launch(ucp):
    """A short gradient, weight or parameter array is rejected by the
    binding before anything is launched (it would be written or read out
    of bounds on the device)."""
    desc = ucp.make_desc("histogram", bins=8)
    p = torch.zeros((10, 12, 13), device="cuda")
    W = torch.zeros((12, 13), device="cuda")
    g = torch.zeros((8, 12, 13), device="cuda")
    ctx = ucp.Context(0)
    for args in ((p, W, g[:4]), (p, W[:6], g), (p[:9], W, g), (p, W.double(), g)):
        with pytest.raises((ValueError, TypeError)):
            ucp.ucp_backward_static(args[0], desc, ucp.UCP_MIN, args[1], args[2])
        with pytest.raises((ValueError, TypeError)):
            ucp.ucp_backward(ctx.handle, args[0], desc, ucp.UCP_MIN, args[1], args[2])
    ctx.close()
    torch.cuda.synchronize()
    assert bool((g == 0).all())


def test_static_adjoint_status_matches_context_adjoint(ucp):
    """The same invalid descriptions give the same status through both
    adjoint entry points (shared argument checks)."""
    ctx = ucp.Context(0)
    p = torch.zeros((2, 4, 5), device="cuda")
    W = torch.zeros((4, 5), device="cuda")
    for kw in (dict(model="uniform", depth=-1), dict(model="uniform", stencil=7),
               dict(model="uniform", stencil=1), dict(model="gaussian"),
               dict(model="mvn"), dict(model="uniform", boundary=5)):
        desc = ucp.make_desc(**kw)
        st = []
        for call in (lambda: ucp.ucp_backward_static(p, desc, 1, W, p),
                     lambda: ucp.ucp_backward(ctx.handle, p, desc, 1, W, p)):
            with pytest.raises(ucp.UcpError) as e:
                call()
            st.append(e.value.status)
        assert st[0] == st[1], (kw, st)
    ctx.close()
