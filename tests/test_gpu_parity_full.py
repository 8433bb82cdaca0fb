"""Per-model parity of the fused fit + integration kernels against the FP64
oracle at the benchmark's sizes, in the launch configuration the benchmark
times, with the largest |P_gpu - P_oracle| of every model printed (one JSON
line per workload and model, printed past pytest's output capture).

The oracle runs on the GPU's own FP32 parameters (ucp_fit, widened to
FP64), so the comparison isolates the integration; the bound is the
closed-form tolerance, 1e-5 per vertex.

- 64 x 64 x 20, i.i.d. noise around a sinusoid base: every vertex, minimum,
  maximum and saddle;
- 1024 x 1024 x 20, bimodal mixture ensemble: 20,000 seeded vertices plus
  the four corners and the first row and column, minimum, maximum and saddle;
- 2048 x 2048 x 50, the same recipe: 5,000 seeded vertices plus the four
  corners, the first row and the last column, minimum and maximum (the
  forward pass of the forward + adjoint workload: 16-row tiles and several
  member boxes for Epanechnikov, the segment walker for 16 bins).
"""
import json

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

TOL = 1e-5
MODELS = (("uniform", 0), ("epanechnikov", 0), ("histogram", 8), ("histogram", 16))


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


def _sample(H, W, n, seed, last_col=False):
    """n seeded vertices, the four corners, the first row and the first
    (or last) column, as sorted unique linear indices."""
    if n is None:
        return None
    rng = np.random.default_rng(seed)
    col = W - 1 if last_col else 0
    idx = np.concatenate([rng.choice(H * W, n, replace=False),
                          [0, W - 1, (H - 1) * W, H * W - 1],
                          np.arange(W), np.arange(H) * W + col])
    return np.unique(idx)


def _err(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    assert (np.isnan(a) == np.isnan(b)).all()
    ok = ~np.isnan(a)
    return float(np.abs(a[ok] - b[ok]).max()) if ok.any() else 0.0


def _report(capsys, line):
    with capsys.disabled():
        print("\nparity " + json.dumps(line), flush=True)


WORKLOADS = {
    "64x64x20": (lambda s: s.ensemble_iid(64, 64, 20, seed=1), None, True),
    "1024x1024x20": (lambda s: s.ensemble_bimodal(1024, 1024, 20, seed=2), 20000, True),
    "2048x2048x50": (lambda s: s.ensemble_bimodal(2048, 2048, 50, seed=4), 5000, False),
}


@pytest.mark.parametrize("workload", list(WORKLOADS))
def test_per_model_error_against_oracle(ucp, ctx, orc, capsys, workload):
    from paper_2407_18015_gb300 import synth
    make, nsamp, with_saddle = WORKLOADS[workload]
    ens_np = make(synth)
    N, H, W = ens_np.shape
    ens = torch.from_numpy(ens_np).cuda()
    idx = _sample(H, W, nsamp, seed=2024 + H, last_col=(H == 2048))
    for model, bins in MODELS:
        desc = ucp.make_desc(model, bins=bins or 8)
        params = ctx.fit(ens, desc)
        pmin, pmax, st = ctx.probability(ens, desc)
        sad = ctx.saddle(ens, desc)[0] if with_saddle else None
        torch.cuda.synchronize()
        # everywhere: probabilities, no vertex flagged
        assert bool((pmin >= 0).all()) and bool((pmax >= 0).all())
        assert bool(((pmin + pmax) <= 1 + 1e-5).all())
        gp = params.double().cpu().numpy()
        gmin, gmax = pmin.cpu().numpy().ravel(), pmax.cpu().numpy().ravel()
        if idx is None:
            rmin, rmax, rst = orc.prob(gp, desc.model, bins=desc.bins)
            sel = slice(None)
            np.testing.assert_array_equal(st.cpu().numpy(), rst)
        else:
            rmin, rmax, rst = orc.prob_at(gp, desc.model, idx, bins=desc.bins)
            sel = idx
            np.testing.assert_array_equal(st.cpu().numpy().ravel()[idx], rst)
        line = {"workload": workload, "model": model + (f"-{bins}" if bins else ""),
                "vertices_compared": int(H * W if idx is None else idx.size),
                "max_abs_err_min": _err(gmin[sel], rmin),
                "max_abs_err_max": _err(gmax[sel], rmax)}
        if sad is not None:
            rs, _ = orc.saddle(gp, desc.model, bins=desc.bins, idx=idx)
            line["max_abs_err_saddle"] = _err(sad.cpu().numpy().ravel()[sel], rs)
        _report(capsys, line)
        for k, v in line.items():
            if k.startswith("max_abs_err"):
                assert v <= TOL, (workload, model, bins, k, v)
        del params, pmin, pmax, st, sad
    del ens
    torch.cuda.empty_cache()


@pytest.mark.parametrize("model,bins", [("histogram", 16), ("epanechnikov", 0)])
def test_full_size_2048_min_only_launch(ucp, ctx, orc, model, bins):
    """The forward + adjoint workload's own forward call (P_min alone, fused
    fit): the same values as the two-type launch, and within the tolerance
    of the oracle on the sampled vertices."""
    from paper_2407_18015_gb300 import synth
    ens = torch.from_numpy(synth.ensemble_bimodal(2048, 2048, 50, seed=4)).cuda()
    desc = ucp.make_desc(model, bins=bins or 8)
    only = torch.empty((2048, 2048), device="cuda")
    ucp.ucp_probability(ctx.handle, ens, desc, ucp.UCP_MIN, only, None)
    pmin, _, _ = ctx.probability(ens, desc)
    params = ctx.fit(ens, desc)
    torch.cuda.synchronize()
    assert torch.equal(only, pmin)
    idx = _sample(2048, 2048, 3000, seed=77, last_col=True)
    rmin, _, _ = orc.prob_at(params.double().cpu().numpy(), desc.model, idx, bins=desc.bins)
    assert _err(only.cpu().numpy().ravel()[idx], rmin) <= TOL
