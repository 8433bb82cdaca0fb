"""The tile kernels' member staging into a shared-memory box: by the tensor
memory accelerator (widths that are a multiple of 4 on a 16-byte aligned
base) and by 4-byte asynchronous copies (any other members: a base one
float off 16 bytes, or a width that is not a multiple of 4).  Against the
oracle and against each other: identical parameters and probabilities,
across narrow grids, grids smaller than a box, several boxes per tile (N up
to 100), non-finite members, all models, minimum / maximum and saddle."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

TOL = 1e-5
MODELS = [("uniform", 0), ("epanechnikov", 0), ("histogram", 8), ("gaussian", 0),
          ("histogram_semi", 8)]


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


def _aligned_and_offset(ens_np):
    """The same members twice on the device: 16-byte aligned, and one float
    past a 16-byte boundary."""
    a = torch.from_numpy(np.ascontiguousarray(ens_np)).cuda()
    buf = torch.empty(ens_np.size + 4, dtype=torch.float32, device="cuda")
    b = buf[1:1 + ens_np.size].view(ens_np.shape)
    b.copy_(a)
    assert a.data_ptr() % 16 == 0 and b.data_ptr() % 16 == 4
    return a, b


def _members(shape, N, seed):
    from paper_2407_18015_gb300 import synth
    H, W = shape
    return synth.ensemble_bimodal(H, W, N, seed=seed, lam_scale=0.3)


def _run_both(ucp, ctx, ens_np, model, bins, **kw):
    a, b = _aligned_and_offset(ens_np)
    d = ucp.make_desc(model, bins=bins or 8, mc_samples=64, seed=9, **kw)
    ra = ctx.probability(a, d)
    rb = ctx.probability(b, d)
    sa, _ = ctx.saddle(a, d)
    sb, _ = ctx.saddle(b, d)
    torch.cuda.synchronize()
    return d, a, ra, rb, sa, sb


@pytest.mark.parametrize("model,bins", MODELS)
@pytest.mark.parametrize("shape,N", [((1, 4), 7), ((3, 8), 20), ((5, 12), 1), ((17, 36), 50),
                                     ((33, 64), 100), ((100, 4), 13), ((16, 32), 14),
                                     ((19, 40), 27)])
def test_tma_matches_per_thread_staging(ucp, ctx, model, bins, shape, N):
    ens_np = _members(shape, N, seed=7 * shape[0] + shape[1] + N)
    d, _, ra, rb, sa, sb = _run_both(ucp, ctx, ens_np, model, bins)
    for x, y in zip(ra, rb):
        np.testing.assert_array_equal(x.cpu().numpy(), y.cpu().numpy())
    np.testing.assert_array_equal(sa.cpu().numpy(), sb.cpu().numpy())


@pytest.mark.parametrize("model,bins", MODELS[:4])
@pytest.mark.parametrize("shape,N", [((17, 36), 50), ((33, 64), 100), ((3, 8), 20)])
def test_tma_against_oracle(ucp, ctx, orc, model, bins, shape, N):
    ens_np = _members(shape, N, seed=3 * shape[0] + N)
    d, a, ra, _, sa, _ = _run_both(ucp, ctx, ens_np, model, bins)
    params = ctx.fit(a, d)
    torch.cuda.synchronize()
    gp = params.double().cpu().numpy()
    if model == "gaussian":
        rmin, rmax, rsad, _ = orc.gauss(gp)
    else:
        rmin, rmax, _ = orc.prob(gp, d.model, bins=d.bins)
        rsad, _ = orc.saddle(gp, d.model, bins=d.bins)
    for g, r in ((ra[0], rmin), (ra[1], rmax), (sa, rsad)):
        assert np.abs(g.cpu().numpy() - r).max() <= TOL
    if model in ("uniform", "histogram"):
        op, _ = orc.fit(ens_np, d.model, bins=d.bins)
        np.testing.assert_array_equal(gp[:2], op[:2])


@pytest.mark.parametrize("model,bins", MODELS)
def test_tma_nonfinite_and_degenerate_members(ucp, ctx, model, bins):
    ens_np = np.random.default_rng(11).normal(size=(30, 9, 12)).astype(np.float32)
    ens_np[2, 4, 4] = np.nan
    ens_np[17, 0, 11] = np.inf
    ens_np[:, 7, 2] = 0.25
    _, _, ra, rb, sa, sb = _run_both(ucp, ctx, ens_np, model, bins)
    for x, y in zip(ra, rb):
        np.testing.assert_array_equal(x.cpu().numpy(), y.cpu().numpy())
    np.testing.assert_array_equal(sa.cpu().numpy(), sb.cpu().numpy())
    st = ra[2].cpu().numpy()
    assert st[4, 4] & ucp.UCP_V_NONFINITE and st[0, 11] & ucp.UCP_V_NONFINITE
    assert not (st & ucp.UCP_V_TIMEOUT).any()


def test_tma_boundary_zero(ucp, ctx):
    ens_np = _members((20, 44), 25, seed=5)
    for model, bins in MODELS[:3]:
        _, _, ra, rb, _, _ = _run_both(ucp, ctx, ens_np, model, bins, boundary=1)
        for x, y in zip(ra, rb):
            np.testing.assert_array_equal(x.cpu().numpy(), y.cpu().numpy())


def test_large_grid_64bit_offsets(ucp, ctx, orc):
    """A 12288 x 12288 grid with 3 members (453 M member floats; member and
    output offsets beyond 2^31): uniform and histogram-4 minimum / maximum on
    sampled vertices against the oracle on the GPU's parameters."""
    H = W = 12288
    N = 3
    g = torch.Generator(device="cuda").manual_seed(3)
    ens = torch.randn((N, H, W), device="cuda", generator=g)
    rng = np.random.default_rng(12)
    idx = np.concatenate([[0, W - 1, (H - 1) * W, H * W - 1],
                          rng.integers(0, H * W, 400)]).astype(np.int64)
    for model, bins in (("uniform", 0), ("histogram", 4)):
        d = ucp.make_desc(model, bins=bins or 8)
        pmin, pmax, _ = ctx.probability(ens, d)
        params = ctx.fit(ens, d)
        torch.cuda.synchronize()
        for i in idx:
            y, x = int(i // W), int(i % W)
            y0, y1, x0, x1 = max(y - 1, 0), min(y + 2, H), max(x - 1, 0), min(x + 2, W)
            # the in-grid neighbourhood: its edges are the grid's edges
            grid = params[:, y0:y1, x0:x1].double().cpu().numpy()
            c = (y - y0) * (x1 - x0) + (x - x0)
            a, b, _ = orc.prob_at(grid, d.model, [c], bins=d.bins)
            assert abs(pmin[y, x].item() - a[0]) <= 1e-5
            assert abs(pmax[y, x].item() - b[0]) <= 1e-5
        del pmin, pmax, params


@pytest.mark.parametrize("model,bins", MODELS + [("histogram", 16), ("histogram", 13)])
@pytest.mark.parametrize("shape,N", [((17, 37), 20), ((9, 2), 7), ((33, 63), 50),
                                     ((8, 130), 100), ((40, 101), 300)])
def test_async_staging_odd_widths(ucp, ctx, orc, model, bins, shape, N):
    """Members of a width the tensor memory accelerator cannot address,
    staged by asynchronous copies, against the same members padded to the
    next multiple of 4 columns (staged by the accelerator): bit for bit on
    every column whose neighbourhood the padding leaves alone (all but the
    last), for minimum, maximum, status and saddle; the last column against
    the oracle."""
    H, W = shape
    if N > 100 and model in ("gaussian", "histogram_semi"):
        pytest.skip("covered at smaller N")
    ens_np = _members(shape, N, seed=H * 13 + W + N)
    Wp = (W + 3) // 4 * 4
    pad = np.zeros((N, H, Wp), np.float32)
    pad[:, :, :W] = ens_np
    pad[:, :, W:] = ens_np[:, :, W - 1:W]
    odd = torch.from_numpy(np.ascontiguousarray(ens_np)).cuda()
    al = torch.from_numpy(pad).cuda()
    d = ucp.make_desc(model, bins=bins or 8, mc_samples=64, seed=9)
    ro = ctx.probability(odd, d)
    so, _ = ctx.saddle(odd, d)
    if model == "histogram_semi":
        # its samples are keyed by the vertex index y * W + x, which the
        # padding changes: against the same estimator from the fitted
        # parameters instead
        params = ctx.fit(odd, d)
        rp = ctx.probability_from_params(params, d)
        torch.cuda.synchronize()
        for x, y in zip(ro[:2], rp[:2]):
            np.testing.assert_allclose(x.cpu().numpy(), y.cpu().numpy(), rtol=0, atol=1e-6)
        return
    ra = ctx.probability(al, d)
    sa, _ = ctx.saddle(al, d)
    torch.cuda.synchronize()
    for x, y in zip(ro, ra):
        np.testing.assert_array_equal(x.cpu().numpy()[:, :W - 1], y.cpu().numpy()[:, :W - 1])
    np.testing.assert_array_equal(so.cpu().numpy()[:, :W - 1], sa.cpu().numpy()[:, :W - 1])
    if model == "gaussian":
        return
    params = ctx.fit(odd, d)
    torch.cuda.synchronize()
    gp = params.double().cpu().numpy()
    rmin, rmax, _ = orc.prob(gp, d.model, bins=d.bins)
    assert np.abs(ro[0].cpu().numpy() - rmin).max() <= TOL
    assert np.abs(ro[1].cpu().numpy() - rmax).max() <= TOL
