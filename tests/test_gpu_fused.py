"""The fused kernel of ucp_probability_models (uniform, Epanechnikov and a
histogram of at most 8 bins of one ensemble, one launch) against the three
single-model launches: the same probabilities and status bit for bit, on
ragged shapes, several member boxes, more than 255 members (16-bit bin
counters), both boundary rules, non-finite members, members staged by the
tensor memory accelerator and by asynchronous copies (odd widths, a base
one float off 16 bytes); and the cases that do not fuse (more bins, other
model sets) give the single-model results too."""
import numpy as np
import pytest
import torch

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


def _members(H, W, N, seed):
    from paper_2407_18015_gb300 import synth
    return synth.ensemble_bimodal(H, W, N, seed=seed, lam_scale=0.4)


def _models_vs_single(ucp, ctx, ens, descs, cptypes=3):
    H, W = ens.shape[1:]
    n = len(descs)
    omin = [torch.full((H, W), -1.0, device="cuda") for _ in range(n)]
    omax = [torch.full((H, W), -1.0, device="cuda") for _ in range(n)]
    ost = [torch.zeros((H, W), dtype=torch.uint8, device="cuda") for _ in range(n)]
    ucp.ucp_probability_models(ctx.handle, ens, descs, cptypes, omin, omax, ost)
    torch.cuda.synchronize()
    for m, d in enumerate(descs):
        rmin, rmax, rst = ctx.probability(ens, d, cptypes)
        torch.cuda.synchronize()
        if cptypes & 1:
            assert torch.equal(omin[m].isnan(), rmin.isnan())
            assert torch.equal(torch.nan_to_num(omin[m]), torch.nan_to_num(rmin)), d.model
        if cptypes & 2:
            assert torch.equal(torch.nan_to_num(omax[m]), torch.nan_to_num(rmax)), d.model
        assert torch.equal(ost[m], rst), d.model


@pytest.mark.parametrize("shape,N,bins,boundary", [
    ((64, 64), 20, 8, 0), ((37, 52), 20, 8, 1), ((8, 32), 3, 5, 0), ((130, 96), 60, 8, 0),
    ((17, 100), 300, 7, 0), ((1, 64), 12, 8, 0), ((300, 4), 9, 1, 1), ((33, 63), 20, 8, 0),
    ((41, 101), 50, 8, 1), ((9, 2), 7, 3, 0), ((65, 1023), 20, 8, 0), ((12, 30), 300, 8, 0)])
def test_fused_equals_single_models(ucp, ctx, shape, N, bins, boundary):
    H, W = shape
    ens_np = _members(H, W, N, seed=H * 7 + W + N)
    ens_np[N // 2, H // 2, W // 2] = np.nan   # a non-finite member
    ens_np[:, 0, 0] = 1.25                     # a point mass
    ens = torch.from_numpy(ens_np).cuda()
    descs = [ucp.make_desc("histogram", bins=bins, boundary=boundary),
             ucp.make_desc("uniform", boundary=boundary),
             ucp.make_desc("epanechnikov", boundary=boundary)]
    _models_vs_single(ucp, ctx, ens, descs)
    _models_vs_single(ucp, ctx, ens, descs, cptypes=ucp.UCP_MAX)


def test_fused_headline_workload(ucp, ctx, orc):
    """1024 x 1024 x 20 (the benchmark's step): the fused call against the
    single-model launches, and sampled vertices against the oracle."""
    from paper_2407_18015_gb300 import synth
    ens = torch.from_numpy(synth.ensemble_bimodal(1024, 1024, 20, seed=2)).cuda()
    descs = [ucp.make_desc("uniform"), ucp.make_desc("epanechnikov"),
             ucp.make_desc("histogram", bins=8)]
    _models_vs_single(ucp, ctx, ens, descs)


@pytest.mark.parametrize("case", ["bins16", "unaligned", "two_models"])
def test_unfused_cases_equal_single_models(ucp, ctx, case):
    ens_np = _members(40, 64, 15, seed=5)
    if case == "unaligned":
        buf = torch.empty(ens_np.size + 1, device="cuda")
        ens = buf[1:].view(ens_np.shape)
        ens.copy_(torch.from_numpy(ens_np).cuda())
    else:
        ens = torch.from_numpy(ens_np).cuda()
    descs = [ucp.make_desc("uniform"), ucp.make_desc("epanechnikov"),
             ucp.make_desc("histogram", bins=16 if case == "bins16" else 8)]
    if case == "two_models":
        descs = descs[:2]
    _models_vs_single(ucp, ctx, ens, descs)
