"""GPU parity of the closed-form models (uniform, Epanechnikov, histogram)
against the FP64 oracle, through the C ABI.

Tolerance: |P_gpu - P_oracle| <= 1e-5 per vertex when both sides use the same
parameters (the GPU's FP32 parameters, widened to FP64 for the oracle).
Uniform and histogram fits are bit-exact (min/max; integer bin counts), so
their end-to-end comparison uses the oracle's own fit.  The Epanechnikov fit
differs from the FP64 fit by FP32 rounding: the parameters are compared with
a relative tolerance and the probabilities from the GPU parameters.
"""
import numpy as np
import pytest
import torch

import helpers as H_

pytestmark = pytest.mark.gpu

TOL = 1e-5
MODELS = [("uniform", 0), ("epanechnikov", 0), ("histogram", 8)]


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
    a = p_gpu.cpu().numpy().astype(np.float64)
    nan_a, nan_b = np.isnan(a), np.isnan(p_ref)
    assert (nan_a == nan_b).all(), f"{what}: NaN pattern differs"
    d = np.abs(a[~nan_a] - p_ref[~nan_b])
    if d.size:
        assert d.max() <= tol, f"{what}: max |diff| {d.max():.3e} at {np.argmax(d)}"
    return float(d.max()) if d.size else 0.0


def _run_field(ucp, ctx, orc, ens_np, model, bins, boundary=0):
    ens = _dev(ens_np)
    desc = ucp.make_desc(model, bins=bins or 8, boundary=boundary)
    params, fst = ctx.fit(ens, desc, with_status=True)
    pmin, pmax, st = ctx.probability(ens, desc)
    torch.cuda.synchronize()
    gp = params.double().cpu().numpy()
    rmin, rmax, rst = orc.prob(gp, desc.model, bins=desc.bins, boundary=boundary)
    e1 = _compare(pmin, rmin, what=f"{model} min")
    e2 = _compare(pmax, rmax, what=f"{model} max")
    np.testing.assert_array_equal(st.cpu().numpy(), rst)
    return ens, desc, params, fst, max(e1, e2)


@pytest.mark.parametrize("model,bins", MODELS)
def test_small_ensemble_parity(ucp, ctx, orc, model, bins):
    """64 x 64 x 20: smooth sinusoid base + i.i.d. N(0, 0.2^2) noise."""
    from paper_2407_18015_gb300 import synth
    ens_np = synth.ensemble_iid(64, 64, 20, seed=1)
    _, desc, params, fst, err = _run_field(ucp, ctx, orc, ens_np, model, bins)
    oparams, ost = orc.fit(ens_np, desc.model, bins=desc.bins)
    gp = params.double().cpu().numpy()
    np.testing.assert_array_equal(fst.cpu().numpy(), ost)
    if model == "uniform":
        np.testing.assert_array_equal(gp, oparams)
    elif model == "histogram":
        np.testing.assert_array_equal(gp[:2], oparams[:2])
        np.testing.assert_array_equal(np.rint(gp[2:] * 20), np.rint(oparams[2:] * 20))
    else:
        np.testing.assert_allclose(gp[0], oparams[0], rtol=0, atol=4e-6)
        np.testing.assert_allclose(gp[1], oparams[1], rtol=2e-6, atol=1e-7)


@pytest.mark.parametrize("model,bins", MODELS)
@pytest.mark.parametrize("shape", [(1, 1), (1, 3), (2, 2), (3, 1), (1, 100), (100, 1),
                                   (17, 33), (37, 70), (16, 32), (33, 65)])
def test_shapes_ragged_tiles(ucp, ctx, orc, model, bins, shape):
    """Grids smaller than a tile, 1D grids, and sizes that leave ragged tiles."""
    from paper_2407_18015_gb300 import synth
    Hh, Ww = shape
    ens_np = synth.ensemble_bimodal(Hh, Ww, 7, seed=100 + Hh * 131 + Ww, lam_scale=0.3)
    _run_field(ucp, ctx, orc, ens_np, model, bins)


@pytest.mark.parametrize("model,bins", MODELS)
def test_boundary_zero_mode(ucp, ctx, orc, model, bins):
    from paper_2407_18015_gb300 import synth
    ens_np = synth.ensemble_iid(20, 45, 11, seed=4)
    _run_field(ucp, ctx, orc, ens_np, model, bins, boundary=1)


@pytest.mark.parametrize("model,bins", MODELS)
def test_from_params_random_and_edge_cases(ucp, ctx, orc, model, bins):
    """Parameters given directly: random overlapping supports with point
    masses, invalid and non-finite entries planted in."""
    rng = np.random.default_rng(17 + bins)
    Hh, Ww = 23, 41
    mid = {"uniform": 0, "epanechnikov": 1, "histogram": 2}[model]
    p = H_.random_params(mid, Hh, Ww, rng, bins=bins or 8)
    p[:, 3, 4] = p[:, 3, 5]                          # identical neighbours
    if mid == 0:
        p[1, 5, 5] = p[0, 5, 5]                      # point mass
        p[0, 5, 6] = p[1, 5, 6] = p[0, 5, 5]         # equal point masses
        p[0, 9, 9], p[1, 9, 9] = 1.0, 0.5            # a > b
    elif mid == 1:
        p[1, 5, 5] = 0.0
        p[:, 5, 6] = p[:, 5, 5]
        p[1, 9, 9] = -0.1                            # w < 0
    else:
        p[1, 5, 5] = p[0, 5, 5]
        p[2, 9, 9] = -0.1                            # negative mass
        p[2:, 11, 11] *= 1.7                         # masses not summing to 1
    p[0, 15, 20] = np.nan
    p32 = p.astype(np.float32)
    desc = ucp.make_desc(model, bins=bins or 8)
    pmin, pmax, st = ctx.probability_from_params(_dev(p32), desc)
    torch.cuda.synchronize()
    rmin, rmax, rst = orc.prob(p32.astype(np.float64), mid, bins=desc.bins)
    _compare(pmin, rmin, what="min")
    _compare(pmax, rmax, what="max")
    np.testing.assert_array_equal(st.cpu().numpy(), rst)


@pytest.mark.parametrize("model,bins", MODELS)
def test_negation_identity_on_gpu(ucp, ctx, model, bins):
    from paper_2407_18015_gb300 import synth
    ens_np = synth.ensemble_bimodal(96, 130, 12, seed=8, lam_scale=0.5)
    desc = ucp.make_desc(model, bins=bins or 8)
    pmin, pmax, _ = ctx.probability(_dev(ens_np), desc)
    nmin, nmax, _ = ctx.probability(_dev(-ens_np), desc)
    torch.cuda.synchronize()
    tol = 1e-5 if model != "epanechnikov" else 3e-5   # the fit itself is re-rounded
    assert (pmax - nmin).abs().max().item() <= tol
    assert (pmin - nmax).abs().max().item() <= tol


@pytest.mark.parametrize("model,bins", MODELS)
def test_full_size_1024_sampled(ucp, ctx, orc, model, bins):
    """1024 x 1024 x 20 bimodal ensemble (the benchmark workload), in the
    benchmark's launch configuration: sampled vertices against the oracle,
    bounds everywhere."""
    from paper_2407_18015_gb300 import synth
    ens_np = synth.ensemble_bimodal(1024, 1024, 20, seed=2)
    ens = _dev(ens_np)
    desc = ucp.make_desc(model, bins=bins or 8)
    params = ctx.fit(ens, desc)
    pmin, pmax, st = ctx.probability(ens, desc)
    torch.cuda.synchronize()
    assert (pmin >= 0).all() and (pmax >= 0).all()
    assert ((pmin + pmax) <= 1 + 1e-5).all()
    assert (st == 0).all()
    rng = np.random.default_rng(5)
    idx = np.concatenate([rng.integers(0, 1024 * 1024, 3000),
                          np.arange(0, 1024), np.arange(0, 1024 * 1024, 1024),
                          [1024 * 1024 - 1]])
    gp = params.double().cpu().numpy()
    rmin, rmax, _ = orc.prob_at(gp, desc.model, idx, bins=desc.bins)
    a = pmin.cpu().numpy().ravel()[idx]
    b = pmax.cpu().numpy().ravel()[idx]
    assert np.abs(a - rmin).max() <= TOL
    assert np.abs(b - rmax).max() <= TOL


def test_error_bound_params(ucp, ctx, orc):
    """Uniform model [d' - eb/2, d' + eb/2] of a decompressed field."""
    rng = np.random.default_rng(2)
    d = rng.normal(size=(40, 50)).astype(np.float32)
    eb = 0.3
    params = torch.empty((2, 40, 50), dtype=torch.float32, device="cuda")
    ucp.ucp_params_from_error_bound(ctx.handle, _dev(d), eb, params)
    torch.cuda.synchronize()
    h = np.float32(0.5) * np.float32(eb)
    np.testing.assert_array_equal(params[0].cpu().numpy(), d - h)
    np.testing.assert_array_equal(params[1].cpu().numpy(), d + h)
    pmin, pmax, _ = ctx.probability_from_params(params, ucp.make_desc("uniform"))
    torch.cuda.synchronize()
    rmin, rmax, _ = orc.prob(params.double().cpu().numpy(), 0)
    _compare(pmin, rmin)
    _compare(pmax, rmax)


@pytest.mark.parametrize("model,bins", MODELS)
def test_host_entry_point_matches_device(ucp, ctx, model, bins):
    from paper_2407_18015_gb300 import synth
    ens_np = synth.ensemble_bimodal(300, 257, 9, seed=12, lam_scale=0.5)
    desc = ucp.make_desc(model, bins=bins or 8)
    pmin, pmax, st = ctx.probability(_dev(ens_np), desc)
    hmin = np.empty((300, 257), np.float32)
    hmax = np.empty((300, 257), np.float32)
    hst = np.empty((300, 257), np.uint8)
    ens_pinned = torch.from_numpy(ens_np).pin_memory()
    ucp.ucp_probability_host(ctx.handle, ens_pinned, desc, 3, hmin, hmax, hst)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(hmin, pmin.cpu().numpy())
    np.testing.assert_array_equal(hmax, pmax.cpu().numpy())
    np.testing.assert_array_equal(hst, st.cpu().numpy())


def test_nonfinite_members(ucp, ctx, orc):
    ens_np = np.random.default_rng(1).normal(size=(6, 9, 10)).astype(np.float32)
    ens_np[2, 4, 4] = np.nan
    ens_np[0, 0, 9] = np.inf
    ens_np[:, 7, 2] = 0.25                      # degenerate vertex
    for model, bins in MODELS:
        _run_field(ucp, ctx, orc, ens_np, model, bins)


def test_api_errors(ucp, ctx):
    ens = torch.zeros((3, 4, 5), device="cuda")
    d = ucp.make_desc("histogram", bins=0)
    with pytest.raises(ucp.UcpError) as e:
        ctx.probability(ens, d)
    assert e.value.status == ucp.UCP_ERR_ARG
    with pytest.raises(ucp.UcpError) as e:
        ctx.backward(torch.zeros((20, 4, 5), device="cuda"), ucp.make_desc("mvn"), 1,
                     torch.zeros((4, 5), device="cuda"))
    assert e.value.status == ucp.UCP_ERR_UNSUPPORTED


@pytest.mark.parametrize("bins", [1, 2, 3, 5, 8, 9, 16])
def test_histogram_bin_counts(ucp, ctx, orc, bins):
    """Histogram walks across bin counts -- the per-bin row tables (up to 8
    bins) and the segment walker (more) -- from members, and from parameters
    with a point-mass centre and neighbour, supports far below, far above and
    far away from their neighbours, and identical neighbours: minimum, maximum
    and saddle against the oracle."""
    from paper_2407_18015_gb300 import synth
    ens_np = synth.ensemble_bimodal(37, 70, 20, seed=900 + bins, lam_scale=0.3)
    _run_field(ucp, ctx, orc, ens_np, "histogram", bins)
    rng = np.random.default_rng(50 + bins)
    p = H_.random_params(2, 19, 37, rng, bins=bins)
    p[1, 5, 5] = p[0, 5, 5]                          # point-mass centre
    p[1, 5, 8] = p[0, 5, 8] = p[0, 5, 9]             # point mass at a neighbour's edge
    p[:2, 8, 8] -= 5.0                               # far below its neighbours
    p[:2, 10, 10] += 5.0                             # far above
    p[:2, 12, 12] += 1.0e6                           # far away
    p[:, 14, 14] = p[:, 14, 15]                      # identical neighbours
    p32 = p.astype(np.float32)
    desc = ucp.make_desc("histogram", bins=bins)
    pmin, pmax, st = ctx.probability_from_params(_dev(p32), desc)
    sad, _ = ctx.saddle_from_params(_dev(p32), desc)
    torch.cuda.synchronize()
    p64 = p32.astype(np.float64)
    rmin, rmax, rst = orc.prob(p64, 2, bins=bins)
    rsad, _ = orc.saddle(p64, 2, bins=bins)
    _compare(pmin, rmin, what="min")
    _compare(pmax, rmax, what="max")
    _compare(sad, rsad, what="saddle")
    np.testing.assert_array_equal(st.cpu().numpy(), rst)


@pytest.mark.parametrize("shape,N", [((300, 257), 9), ((700, 1024), 20), ((5, 12), 3)])
def test_host_models_match_device(ucp, ctx, shape, N):
    """ucp_probability_host_models: every model of one ensemble from host
    arrays (pinned and pageable), the members copied once in row strips, gives
    exactly the per-model device results; also with a model whose outputs are
    not wanted (NULL) and without status arrays."""
    from paper_2407_18015_gb300 import synth
    H, W = shape
    ens_np = synth.ensemble_bimodal(H, W, N, seed=31 + H, lam_scale=0.5)
    descs = [ucp.make_desc(m, bins=b or 8) for m, b in MODELS] + \
        [ucp.make_desc("histogram", bins=16), ucp.make_desc("mvn", mc_samples=64, seed=7)]
    ref = [ctx.probability(_dev(ens_np), d) for d in descs]
    torch.cuda.synchronize()
    n = len(descs)
    for pinned in (True, False):
        ens_h = torch.from_numpy(ens_np).pin_memory() if pinned else ens_np
        hmin = [np.full((H, W), -1, np.float32) for _ in range(n)]
        hmax = [np.full((H, W), -1, np.float32) for _ in range(n)]
        hst = [np.zeros((H, W), np.uint8) for _ in range(n)]
        ucp.ucp_probability_host_models(ctx.handle, ens_h, descs, 3, hmin, hmax, hst)
        for m in range(n):
            np.testing.assert_array_equal(hmin[m], ref[m][0].cpu().numpy())
            np.testing.assert_array_equal(hmax[m], ref[m][1].cpu().numpy())
            np.testing.assert_array_equal(hst[m], ref[m][2].cpu().numpy())
    # minimum only, the second model's output unwanted, no status
    hmin = [np.full((H, W), -1, np.float32) if m != 1 else None for m in range(n)]
    ucp.ucp_probability_host_models(ctx.handle, ens_np, descs, ucp.UCP_MIN, hmin, [None] * n)
    for m in range(n):
        if m != 1:
            np.testing.assert_array_equal(hmin[m], ref[m][0].cpu().numpy())


@pytest.mark.parametrize("shape,N", [((300, 257), 9), ((1024, 1024), 20), ((65, 1023), 30)])
def test_host_models_pinned_outputs(ucp, ctx, shape, N):
    """ucp_probability_host_models with pinned output arrays: the fused
    kernel writes the caller's mapped arrays directly (no read-back copies).
    The same bits as the device-array call, with and without status arrays,
    minimum only, and with one pageable output (the read-back path)."""
    from paper_2407_18015_gb300 import synth
    H, W = shape
    ens_np = synth.ensemble_bimodal(H, W, N, seed=7 + W, lam_scale=0.5)
    descs = [ucp.make_desc("histogram", bins=8), ucp.make_desc("uniform"),
             ucp.make_desc("epanechnikov")]
    ref = [ctx.probability(_dev(ens_np), d) for d in descs]
    torch.cuda.synchronize()
    ens_h = torch.from_numpy(ens_np).pin_memory()
    pinned = lambda dt: torch.full((H, W), -1, dtype=dt).pin_memory()
    for with_status in (True, False):
        hmin = [pinned(torch.float32) for _ in descs]
        hmax = [pinned(torch.float32) for _ in descs]
        hst = [pinned(torch.uint8) for _ in descs] if with_status else None
        ucp.ucp_probability_host_models(ctx.handle, ens_h, descs, 3, hmin, hmax, hst)
        for m in range(3):
            assert torch.equal(hmin[m], ref[m][0].cpu())
            assert torch.equal(hmax[m], ref[m][1].cpu())
            if with_status:
                assert torch.equal(hst[m], ref[m][2].cpu())
    hmin = [pinned(torch.float32) for _ in descs]
    ucp.ucp_probability_host_models(ctx.handle, ens_h, descs, ucp.UCP_MIN, hmin, [None] * 3)
    for m in range(3):
        assert torch.equal(hmin[m], ref[m][0].cpu())
    hmin = [pinned(torch.float32) for _ in descs]
    hmax = [pinned(torch.float32) for _ in descs]
    hmax[1] = np.full((H, W), -1, np.float32)  # pageable: every output read back
    ucp.ucp_probability_host_models(ctx.handle, ens_h, descs, 3, hmin, hmax)
    for m in range(3):
        assert torch.equal(hmin[m], ref[m][0].cpu())
        np.testing.assert_array_equal(np.asarray(hmax[m]), ref[m][1].cpu().numpy())


def test_host_models_rejects(ucp, ctx):
    ens = np.zeros((3, 8, 8), np.float32)
    out = [np.zeros((8, 8), np.float32)]
    with pytest.raises(ucp.UcpError):
        ucp.ucp_probability_host_models(ctx.handle, ens, [], 3, [], [])
    with pytest.raises(ucp.UcpError):
        ucp.ucp_probability_host_models(ctx.handle, ens, [ucp.make_desc("uniform")], 4, out, out)
    d = ucp.make_desc("uniform", stencil=ucp.UCP_STENCIL_8)
    with pytest.raises(ucp.UcpError):
        ucp.ucp_probability_host_models(ctx.handle, ens, [d], 1, out, out)


def test_models_concurrent_match_single(ucp, ctx):
    """ucp_probability_models (the models' kernels concurrent on the context's
    streams, forked from and joined into the current stream) gives exactly
    the per-model ucp_probability results, with unwanted outputs left
    untouched and on a non-default stream."""
    from paper_2407_18015_gb300 import synth
    ens_np = synth.ensemble_bimodal(333, 260, 20, seed=77, lam_scale=0.5)
    ens = _dev(ens_np)
    descs = [ucp.make_desc(m, bins=b or 8) for m, b in MODELS] + \
        [ucp.make_desc("histogram", bins=16), ucp.make_desc("mvn", mc_samples=64, seed=3),
         ucp.make_desc("gaussian")]
    ref = [ctx.probability(ens, d) for d in descs]
    n = len(descs)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        omin = [torch.full((333, 260), -1.0, device="cuda") for _ in range(n)]
        omax = [torch.full((333, 260), -1.0, device="cuda") if m != 2 else None for m in range(n)]
        ost = [torch.zeros((333, 260), dtype=torch.uint8, device="cuda") for _ in range(n)]
        ucp.ucp_probability_models(ctx.handle, ens, descs, 3, omin, omax, ost)
        got = [(a.clone(), None if b is None else b.clone(), c.clone())
               for a, b, c in zip(omin, omax, ost)]
    torch.cuda.synchronize()
    for m in range(n):
        assert torch.equal(got[m][0], ref[m][0])
        if m != 2:
            assert torch.equal(got[m][1], ref[m][1])
        assert torch.equal(got[m][2], ref[m][2])
    with pytest.raises(ucp.UcpError):
        ucp.ucp_probability_models(ctx.handle, ens, [ucp.make_desc("uniform",
                                                                   stencil=ucp.UCP_STENCIL_6)],
                                   1, omin[:1], omax[:1])


@pytest.mark.parametrize("N", [1, 2, 20, 31, 32, 33, 50, 64, 65, 300])
@pytest.mark.parametrize("bins", [1, 8, 9, 16, 17])
def test_histogram_fit_matches_oracle(ucp, ctx, orc, N, bins):
    """The histogram statistics pass alone (ucp_fit) across member counts on
    both sides of the register path's bounds (32 and 64 members, 16 bins)
    and of the 8-bit counters (255): range bit for bit, the same bin count
    for every bin (mass * N), the same status, with non-finite members and
    point masses."""
    rng = np.random.default_rng(1000 * N + bins)
    H, W = 13, 45
    ens_np = rng.normal(size=(N, H, W)).astype(np.float32)
    ens_np[:, 2, 3] = 0.75                       # point mass
    ens_np[N // 2, 4, 4] = np.nan                # non-finite members
    ens_np[N - 1, 5, 40] = np.inf
    ens_np[0, 6, 7] = -np.inf
    desc = ucp.make_desc("histogram", bins=bins)
    params, fst = ctx.fit(_dev(ens_np), desc, with_status=True)
    torch.cuda.synchronize()
    gp = params.double().cpu().numpy()
    op, ost = orc.fit(ens_np, desc.model, bins=bins)
    np.testing.assert_array_equal(fst.cpu().numpy(), ost)
    np.testing.assert_array_equal(gp[:2], op[:2])
    np.testing.assert_array_equal(np.isnan(gp[2:]), np.isnan(op[2:]))
    np.testing.assert_array_equal(np.nan_to_num(np.rint(gp[2:] * N)),
                                  np.nan_to_num(np.rint(op[2:] * N)))
