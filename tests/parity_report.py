"""Parity report (test infrastructure, run by hand on a GPU machine):

    python tests/parity_report.py

For each closed-form model, the largest |P_gpu - P_oracle| of the minimum,
maximum and saddle probabilities, the oracle evaluated on the GPU's own FP32
parameters (the integration alone):

- 64 x 64 x 20 (i.i.d. noise around a sinusoid base): every vertex;
- 1024 x 1024 x 20 (bimodal mixture ensemble): 20,000 seeded vertices;
- 2048 x 2048 x 50 (the same recipe): 5,000 seeded vertices, P_min and P_max.

One JSON line per workload and model.  The pass/fail bounds live in the
GPU tests; this prints the figures stated next to the measured numbers.
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

MODELS = (("uniform", 0), ("epanechnikov", 0), ("histogram", 8), ("histogram", 16))


def _err(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    ok = ~(np.isnan(a) | np.isnan(b))
    return float(np.abs(a[ok] - b[ok]).max()) if ok.any() else 0.0


def main():
    import torch

    import oracle
    from paper_2407_18015_gb300 import build, synth, ucp

    build.build()
    oracle.build()
    ctx = ucp.Context(0)
    dev = torch.device("cuda", 0)
    work = (("64x64x20 all vertices", synth.ensemble_iid(64, 64, 20, seed=1), None, True),
            ("1024x1024x20 20000 vertices", synth.ensemble_bimodal(1024, 1024, 20, seed=2),
             20000, True),
            ("2048x2048x50 5000 vertices", synth.ensemble_bimodal(2048, 2048, 50, seed=4),
             5000, False))
    rng = np.random.default_rng(2024)
    for name, ens_np, nsamp, with_saddle in work:
        ens = torch.from_numpy(ens_np).to(dev)
        _, H, W = ens_np.shape
        idx = None if nsamp is None else np.sort(rng.choice(H * W, nsamp, replace=False))
        for model, bins in MODELS:
            desc = ucp.make_desc(model, bins=bins or 8)
            params = ctx.fit(ens, desc)
            pmin, pmax, _ = ctx.probability(ens, desc)
            sad = ctx.saddle(ens, desc)[0] if with_saddle else None
            torch.cuda.synchronize()
            gp = params.double().cpu().numpy()
            gmin, gmax = pmin.cpu().numpy().ravel(), pmax.cpu().numpy().ravel()
            if idx is None:
                rmin, rmax, _ = oracle.prob(gp, desc.model, bins=desc.bins)
                rmin, rmax = rmin.ravel(), rmax.ravel()
                sel = slice(None)
            else:
                rmin, rmax, _ = oracle.prob_at(gp, desc.model, idx, bins=desc.bins)
                sel = idx
            out = {"workload": name, "model": model + (f"-{bins}" if bins else ""),
                   "max_err_min": _err(gmin[sel], rmin), "max_err_max": _err(gmax[sel], rmax)}
            if sad is not None:
                rs, _ = oracle.saddle(gp, desc.model, bins=desc.bins, idx=idx)
                out["max_err_saddle"] = _err(sad.cpu().numpy().ravel()[sel], np.ravel(rs))
            print(json.dumps(out), flush=True)
        del ens
    ctx.close()


if __name__ == "__main__":
    main()
