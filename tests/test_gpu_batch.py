"""Batched persistent launch (ucp_batch_*): the same probabilities as the
per-field launches, under CUDA graph capture and replay, after autotuning;
spot checks against the oracle.  Bit-identical (the same tile body per
vertex) except for histograms of at most 16 bins: the per-field kernels walk
their per-bin row tables, the batch kernel the segment walker, which round
differently (each within 1e-5 of the oracle); those agree to 1e-6."""
import os

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


FIELDS = [  # H, W, N, model, bins, cptypes, boundary
    (128, 160, 10, "uniform", 0, 3, 0), (37, 71, 20, "histogram", 16, 1, 0),
    (200, 96, 50, "epanechnikov", 0, 2, 0), (1, 300, 7, "histogram", 4, 3, 0),
    (255, 257, 20, "uniform", 0, 1, 1), (64, 64, 100, "histogram", 16, 3, 0),
    (17, 5, 3, "epanechnikov", 0, 3, 1), (300, 33, 12, "histogram", 8, 2, 0),
    (129, 130, 20, "epanechnikov", 0, 1, 0), (1, 1, 5, "uniform", 0, 3, 0),
]


def _make(ucp, seed_base=0):
    from paper_2407_18015_gb300 import synth
    fields = []
    for i, (Hh, Ww, N, model, bins, cp, bd) in enumerate(FIELDS):
        ens = torch.from_numpy(synth.ensemble_bimodal(Hh, Ww, N, seed=300 + i + seed_base,
                                                      lam_scale=0.5)).cuda()
        desc = ucp.make_desc(model, bins=bins or 8, boundary=bd)
        out = (torch.full((Hh, Ww), -1.0, device="cuda"), torch.full((Hh, Ww), -1.0, device="cuda"))
        fields.append((ens, desc, cp, out))
    return fields


def _reference(ctx, fields):
    refs = []
    for ens, desc, cp, _ in fields:
        pmin, pmax, _ = ctx.probability(ens, desc, cp)
        refs.append((pmin, pmax))
    torch.cuda.synchronize()
    return refs


def _same(desc, out, ref):
    if desc.model == 2 and desc.bins <= 16:
        assert (out - ref).abs().max().item() <= 1e-6
    else:
        assert torch.equal(out, ref)


def _check(fields, refs):
    for (ens, desc, cp, (omin, omax)), (rmin, rmax) in zip(fields, refs):
        if cp & 1:
            _same(desc, omin, rmin)
        else:
            assert (omin == -1).all()
        if cp & 2:
            _same(desc, omax, rmax)
        else:
            assert (omax == -1).all()


def test_batch_matches_per_field(ucp, ctx, tmp_path, monkeypatch):
    monkeypatch.setenv("UCP_TUNE_CACHE", str(tmp_path / "tune.json"))
    fields = _make(ucp)
    b = ucp.Batch(ctx)
    for ens, desc, cp, (omin, omax) in fields:
        b.add(ens, desc, cp, omin, omax)
    b.run()
    torch.cuda.synchronize()
    _check(fields, _reference(ctx, fields))
    b.close()


def test_batch_tuned_and_graph_replay(ucp, ctx, tmp_path, monkeypatch):
    cache = tmp_path / "tune.json"
    monkeypatch.setenv("UCP_TUNE_CACHE", str(cache))
    fields = _make(ucp, seed_base=50)
    b = ucp.Batch(ctx)
    for ens, desc, cp, (omin, omax) in fields:
        b.add(ens, desc, cp, omin, omax)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        b.tune()
    torch.cuda.synchronize()
    assert cache.exists() and cache.read_text().startswith("{")
    refs = _reference(ctx, fields)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        b.run()
    for _ in range(2):
        for _, _, _, (omin, omax) in fields:
            omin.fill_(-1.0)
            omax.fill_(-1.0)
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        _check(fields, refs)
    b.close()


def test_batch_against_oracle(ucp, ctx, orc):
    fields = _make(ucp, seed_base=90)
    b = ucp.Batch(ctx)
    for ens, desc, cp, (omin, omax) in fields:
        b.add(ens, desc, cp, omin, omax)
    b.run()
    torch.cuda.synchronize()
    for ens, desc, cp, (omin, omax) in fields[:6]:
        params = ctx.fit(ens, desc)
        torch.cuda.synchronize()
        rmin, rmax, _ = orc.prob(params.double().cpu().numpy(), desc.model, bins=desc.bins,
                                 boundary=desc.boundary)
        if cp & 1:
            assert np.abs(omin.cpu().numpy() - rmin).max() <= 1e-5
        if cp & 2:
            assert np.abs(omax.cpu().numpy() - rmax).max() <= 1e-5
    b.close()


def test_batch_errors(ucp, ctx):
    b = ucp.Batch(ctx)
    ens = torch.zeros((3, 4, 5), device="cuda")
    o = torch.zeros((4, 5), device="cuda")
    with pytest.raises(ucp.UcpError) as e:
        b.add(ens, ucp.make_desc("mvn"), 1, o, o)
    assert e.value.status == ucp.UCP_ERR_UNSUPPORTED
    with pytest.raises(ucp.UcpError) as e:
        b.add(ens, ucp.make_desc("uniform"), 1, None, o)
    assert e.value.status == ucp.UCP_ERR_ARG
    b.run()          # an empty batch is a no-op
    b.close()


def test_batch_at_64_field_workload_scale(ucp, ctx, tmp_path, monkeypatch):
    """The 64-field batched workload (uneven shapes, N in {10, 20, 50, 100},
    uniform / Epanechnikov / histogram-16, minimum or maximum), every side
    halved to bound the test's memory and time: the autotuned launch,
    captured in a CUDA graph and replayed, equals the per-field launches
    field by field."""
    from paper_2407_18015_gb300 import synth
    monkeypatch.setenv("UCP_TUNE_CACHE", str(tmp_path / "tune.json"))
    specs = synth.batch_specs(fields=64)
    assert {s["N"] for s in specs} == {10, 20, 50, 100}
    assert {s["model"] for s in specs} == {"uniform", "epanechnikov", "histogram"}
    fields = []
    for sp in specs:
        ens = torch.from_numpy(synth.batch_field(sp, scale=0.5)).cuda()
        desc = ucp.make_desc(sp["model"], bins=sp["bins"])
        cp = ucp.UCP_MIN if sp["cptype"] == "min" else ucp.UCP_MAX
        Hh, Ww = ens.shape[1:]
        out = (torch.full((Hh, Ww), -1.0, device="cuda"), torch.full((Hh, Ww), -1.0, device="cuda"))
        fields.append((ens, desc, cp, out))
    refs = _reference(ctx, fields)
    b = ucp.Batch(ctx)
    for ens, desc, cp, (omin, omax) in fields:
        b.add(ens, desc, cp, omin, omax)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        b.tune()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        b.run()
    for _, _, _, (omin, omax) in fields:
        omin.fill_(-1.0)
        omax.fill_(-1.0)
    torch.cuda.synchronize()
    g.replay()
    torch.cuda.synchronize()
    _check(fields, refs)
    b.close()
    del fields, refs
    torch.cuda.empty_cache()
