"""Benchmark: critical-point probability fields on GB300.

Headline workload (one step): a 1024 x 1024 grid with N = 20 float32 members
(seeded bimodal mixture around a smooth sinusoid base), probability of local
minimum and maximum under the uniform, Epanechnikov and 8-bin histogram
models, one ucp_probability_models call: one fused kernel stages the members
once and integrates all three models.  value = grid vertices per second with
all three models evaluated (whole job over all ranks).  per_model times each
model's own kernel (ucp_probability) on the same workload.

Also measured in the same run (key "rows"): the multivariate-Gaussian Monte
Carlo workload (512^2 x 40, 10,000 Philox samples per vertex), the forward +
adjoint workload (2048^2 x 50, histogram-16 and Epanechnikov), and the batched
persistent launch (64 uneven fields) against per-field launches.

--impl reference times the FP64 CPU oracle on the host cores instead (the
reference arm; a bounded sample of the same workload per step).

Multi-GPU (torchrun): every rank runs an independent replica of the workload
(weak scaling); the only collectives are the host-side barrier and the
max-over-ranks of the timed region.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

H2, W2, N2, SEED2, BINS2 = 1024, 1024, 20, 2, 8
MODELS2 = (("uniform", 0), ("epanechnikov", 0), ("histogram", BINS2))
L2_FLUSH_BYTES = 512 << 20          # > 126 MB L2
SM_COUNT, FP32_LANES, SM_MAX_MHZ = 152, 128, 2070.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-rows", action="store_true", help="headline workload only")
    ap.add_argument("--rows", default="mvn,fwdbwd,batch,saddle,gmm,stencil,sizes")
    ap.add_argument("--batch-fields", type=int, default=64, help="fields of the batch row")
    ap.add_argument("--batch-max", type=int, default=2048, help="largest field side of the batch row")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured",
                "sm_max_mhz": float(d.get("sm_max_mhz", SM_MAX_MHZ))}
    except Exception:
        return {"hbm_gbs": 6800.0, "source": "fallback", "sm_max_mhz": SM_MAX_MHZ}


def fp32_peak_tflops(mhz):
    """FP32 pipe: 152 SMs x 128 lanes x 2 flops (FMA) per clock."""
    return SM_COUNT * FP32_LANES * 2 * mhz * 1e6 / 1e12


def issue_peak_tops(mhz):
    """Instruction issue: 152 SMs x 4 schedulers x 32 lanes, one operation
    per lane per clock."""
    return SM_COUNT * FP32_LANES * mhz * 1e6 / 1e12


# ---------------------------------------------------------------------------
# clocks during the timed region


class ClockSampler:
    def __init__(self, index, path):
        self.path = path
        self.proc = None
        try:
            self.f = open(path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(index),
                 "--query-gpu=timestamp,index,clocks.sm,clocks.max.sm,power.draw,"
                 "clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
                 "clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self, t0=None, t1=None):
        """Median SM clock and the throttle reasons seen between wall-clock
        times t0 and t1 (the timed region)."""
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        import datetime
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                if t0 is not None and not (t0 - 0.15 <= ts <= t1 + 0.15):
                    continue
                sm.append(float(parts[2]))
                mx.append(float(parts[3]))
            except ValueError:
                continue
            for n, v in zip(names, parts[6:10]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# algorithmic work of the kernels


def hist_piece_counts(params, bins):
    """Pieces of the exact histogram integration per vertex: the centre's
    B+1 bin edges plus every neighbour bin edge strictly inside the centre's
    support (torch, on the device)."""
    import torch
    lo, hi = params[0], params[1]
    Hh, Ww = lo.shape
    cnt = torch.full_like(lo, float(bins))  # B pieces from the centre's own edges
    j = torch.arange(bins + 1, device=lo.device, dtype=torch.float32).view(-1, 1, 1)
    for dy, dx in ((0, 1), (-1, 0), (0, -1), (1, 0)):
        ys = slice(max(0, -dy), Hh - max(0, dy))
        xs = slice(max(0, -dx), Ww - max(0, dx))
        yn = slice(ys.start + dy, ys.stop + dy)
        xn = slice(xs.start + dx, xs.stop + dx)
        nlo, nhi = lo[yn, xn], hi[yn, xn]
        edges = nlo + j * (nhi - nlo) / bins
        inside = (edges > lo[ys, xs]) & (edges < hi[ys, xs])
        cnt[ys, xs] += inside.sum(0).float()
    return cnt


# Algorithmic work per unit (the scope table's figures): a histogram piece
# costs 3 Gauss-Legendre nodes x ~25 flops per type, an Epanechnikov vertex
# 5 pieces x 8 nodes x ~35 flops per type; the uniform model is counted in
# bytes (4N read + 4 per output type written).  Histogram pieces are counted
# exactly from the data (hist_piece_counts).
HIST_FLOPS_PER_PIECE_TYPE = 3 * 25
EPAN_FLOPS_PER_VERTEX_TYPE = 5 * 8 * 35
# Monte Carlo: per sample two Philox4x32-10 blocks (~200 integer operations),
# three Box-Muller transforms, 14 FMA for L z and 4 comparisons, ~250 lane
# operations, against the issue rate (one operation per lane per clock).
MVN_OPS_PER_SAMPLE = 250
# Histogram adjoint of P_min: on every merged piece the centre's product
# integral and one leave-one-out product integral per neighbour, each counted
# as a forward piece integral.
ADJ_HIST_FLOPS_PER_PIECE = 5 * HIST_FLOPS_PER_PIECE_TYPE
# Epanechnikov adjoint of P_min: at every Gauss-Legendre node of every piece
# the forward's factors and product, plus the derivative factor of each of
# the four neighbours (its density, times (x - m)/w for the width), the two
# derivatives of the centre's density and the ten derivative accumulations:
# about twice the forward's work per node, counted as two forward vertex
# integrals of one type.
ADJ_EPAN_FLOPS_PER_VERTEX = 2 * EPAN_FLOPS_PER_VERTEX_TYPE


# DRAM bytes (read + write) per launch of the step's kernel (the fused
# three-model kernel) and of each model's own kernel, from the ncu captures
# summarised in profiles/; None once a kernel has changed since its counters
# were taken
TRAFFIC_BYTES = {"fused": 93154816, "uniform": 88159744, "epanechnikov": 84930816,
                 "histogram": 85532160, "hist_adjoint_16": 654388992}
# warp instructions per launch of the same kernels (ncu smsp__inst_executed.sum,
# profiles/instructions_bench_headline_1024x1024x20.md): the issue-rate
# fraction reported beside the FP32 / HBM one; None once a kernel changed
ISSUE_WARP_INSTR = {"fused": 206773693, "uniform": 23585236, "epanechnikov": 62221552,
                    "histogram": 142005566}
ISSUE_SOURCE = "profiles/instructions_bench_headline_1024x1024x20.md"


def issue_block(key, ms, mhz):
    """Issue-rate fraction of a kernel of `ms` per launch: its warp
    instructions per launch against 152 SMs x 4 schedulers x 1 instruction
    per clock."""
    n = ISSUE_WARP_INSTR.get(key)
    if n is None:
        return None
    peak = SM_COUNT * 4 * mhz * 1e6 / 1e9
    ach = n / (ms / 1e3) / 1e9
    return {"warp_instructions": n, "achieved": ach, "peak": peak,
            "unit": "G warp instructions/s", "frac": ach / peak, "source": ISSUE_SOURCE}


TRAFFIC_SOURCE = {"fused": "profiles/instructions_bench_headline_1024x1024x20.md",
                  "uniform": "profiles/instructions_bench_headline_1024x1024x20.md",
                  "epanechnikov": "profiles/instructions_bench_headline_1024x1024x20.md",
                  "histogram": "profiles/instructions_bench_headline_1024x1024x20.md",
                  "hist_adjoint_16": "profiles/adjoint_hist16_2048x2048x50.md"}


def work_of(model, N, HW, params=None, bins=BINS2):
    if model == "uniform":
        return "hbm", (4.0 * N + 8.0) * HW
    if model == "epanechnikov":
        return "alu", 2.0 * EPAN_FLOPS_PER_VERTEX_TYPE * HW
    pieces = float(hist_piece_counts(params, bins).sum().item())
    return "alu", 2.0 * HIST_FLOPS_PER_PIECE_TYPE * pieces


# ---------------------------------------------------------------------------
# reference arm: the FP64 oracle on the host cores


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    from paper_2407_18015_gb300 import synth
    oracle.build()
    ens = synth.ensemble_bimodal(H2, W2, N2, seed=SEED2)
    rows = 96                         # bounded sample per step: 96 x 1024 vertices
    times = []
    for s in range(args.warmup + args.steps):
        y0 = (s * rows) % (H2 - rows)
        crop = np.ascontiguousarray(ens[:, y0:y0 + rows, :])
        t = time.perf_counter()
        for model, bins in MODELS2:
            mid = {"uniform": 0, "epanechnikov": 1, "histogram": 2}[model]
            p, _ = oracle.fit(crop, mid, bins=bins or 8)
            oracle.prob(p, mid, bins=bins or 8)
        if s >= args.warmup:
            times.append(time.perf_counter() - t)
    tot = sum(times)
    verts = rows * W2 * len(times)
    value = verts / tot
    cores = oracle.get_threads()
    line = {
        "impl": "reference", "metric": "critical-point probability vertices/s "
        "(uniform + Epanechnikov + histogram-8, min and max, 1024x1024x20)",
        "value": value, "unit": "vertices/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": "bimodal ensemble 1024x1024, N=20, "
                                        "uniform/Epanechnikov/hist-8, min+max",
                                        "sample_rows_per_step": rows},
        "cpu_baseline": {"value": value, "unit": "vertices/s", "cores": cores, "kind": "oracle",
                         "sample": f"{rows} rows x 1024 of the 1024x1024x20 field per step"},
        "e2e": {"value": value, "unit": "vertices/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# our arm


def cpu_baseline_headline(ens_np):
    """The oracle as it stands on the host cores, on the full headline field
    (fit + both probabilities for the three models)."""
    import oracle
    oracle.build()
    t = time.perf_counter()
    for model, bins in MODELS2:
        mid = {"uniform": 0, "epanechnikov": 1, "histogram": 2}[model]
        p, _ = oracle.fit(ens_np, mid, bins=bins or 8)
        oracle.prob(p, mid, bins=bins or 8)
    dt = time.perf_counter() - t
    return {"value": H2 * W2 / dt, "unit": "vertices/s", "cores": oracle.get_threads(),
            "kind": "oracle", "seconds": dt,
            "sample": "the full 1024x1024x20 field, all three models, min and max, once"}


def oracle_mvn_rate(ens_np, crop=128, samples=10000):
    """The oracle's Monte Carlo (FP64, same Philox stream contract) on a
    crop of the workload: vertices/s and samples/s on the host cores, and
    the full field's time extrapolated from them (labelled as such)."""
    import oracle
    oracle.build()
    sub = np.ascontiguousarray(ens_np[:, :crop, :crop])
    t = time.perf_counter()
    p, _ = oracle.fit(sub, oracle.MVN)
    oracle.mvn_mc_at(p, np.arange(crop * crop), samples, 0x5EED)
    dt = time.perf_counter() - t
    full = ens_np.shape[1] * ens_np.shape[2]
    return {"vertices_per_s": crop * crop / dt, "samples_per_s": crop * crop * samples / dt,
            "cores": oracle.get_threads(), "seconds": dt,
            "full_field_seconds_extrapolated": full / (crop * crop / dt),
            "sample": f"a {crop}x{crop} crop (its own boundary), fit + {samples} samples each; "
                      "the full-field time is extrapolated by vertex count"}


def oracle_fwd_bwd_rate(e4, weight, model, bins, rows=None):
    """The oracle's fit, probability and analytic gradient on the 2048x2048x50
    workload: the full field (rows=None) or a strip of `rows` rows, whose
    rates are extrapolated to the full field by vertex count (labelled)."""
    import oracle
    oracle.build()
    Hh, Ww = weight.shape
    rows = Hh if rows is None else rows
    strip = np.ascontiguousarray(e4[:, :rows, :].cpu().numpy())
    wt = np.ascontiguousarray(weight[:rows, :].cpu().numpy())
    mid = {"uniform": 0, "epanechnikov": 1, "histogram": 2}[model]
    t = time.perf_counter()
    p, _ = oracle.fit(strip, mid, bins=bins or 8)
    oracle.prob(p, mid, bins=bins or 8)
    t1 = time.perf_counter()
    oracle.grad(p, mid, wt, cptype=1, bins=bins or 8)
    t2 = time.perf_counter()
    n = rows * Ww
    out = {"fwd_vertices_per_s": n / (t1 - t), "fwd_bwd_vertices_per_s": n / (t2 - t),
           "cores": oracle.get_threads(), "seconds": t2 - t}
    if rows == Hh:
        out["sample"] = ("the full 2048x2048 field (fit, P_min and P_max, gradient of "
                         "sum W P_min)")
    else:
        out["full_field_seconds_extrapolated"] = (t2 - t) * Hh / rows
        out["sample"] = (f"{rows} of the 2048 rows (fit, P_min and P_max, gradient of sum W "
                         "P_min); full-field rates extrapolated by vertex count")
    return out


class L2Flush:
    """Write a 512 MB buffer, then read another: the L2 (126 MB) ends up
    holding clean lines of unrelated data, so the next step neither hits in L2
    nor pays for write-backs of the flush."""

    def __init__(self, torch, dev):
        self.w = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
        self.r = torch.ones(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
        self.acc = torch.zeros((), dtype=torch.float32, device=dev)

    def __call__(self):
        self.w.fill_(1.0)
        self.acc += self.r.sum()


def timed_steps(torch, step, steps, warmup, flush, per_kernel_events=False):
    """Warm-up, then `steps` steps each bracketed by CUDA events on the current
    stream; the L2 is flushed between steps, outside the events."""
    for _ in range(warmup):
        step(None)
    torch.cuda.synchronize()
    total = 0.0
    kernel_ms = {}
    for _ in range(steps):
        flush()
        ev = [] if per_kernel_events else None
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        step(ev)
        b.record()
        torch.cuda.synchronize()
        total += a.elapsed_time(b)
        if ev:
            for name, e0, e1 in ev:
                kernel_ms.setdefault(name, []).append(e0.elapsed_time(e1))
    return total, kernel_ms


def run_ours(args):
    import torch
    from paper_2407_18015_gb300 import replicas
    rank, world, local = replicas.rank_env()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    replicas.init("nccl", dev)
    from paper_2407_18015_gb300 import build, synth, ucp
    build.build()
    ctx = ucp.Context(local)
    ens_np = synth.ensemble_bimodal(H2, W2, N2, seed=SEED2 + 100 * rank)
    ens = torch.from_numpy(ens_np).to(dev)
    outs = {m: (torch.empty((H2, W2), device=dev), torch.empty((H2, W2), device=dev))
            for m, _ in MODELS2}
    descs = {m: ucp.make_desc(m, bins=b or 8) for m, b in MODELS2}
    flush = L2Flush(torch, dev)

    dlist = [descs[m] for m, _ in MODELS2]
    omin = [outs[m][0] for m, _ in MODELS2]
    omax = [outs[m][1] for m, _ in MODELS2]

    def step(ev):
        # the three models of one ensemble: one fused kernel on this stream
        ucp.ucp_probability_models(ctx.handle, ens, dlist, ucp.UCP_MIN | ucp.UCP_MAX, omin, omax)

    def step_seq(ev):
        # the same launches one after another, with events between them, for
        # each kernel's own duration
        for m, _ in MODELS2:
            if ev is not None:
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
            ucp.ucp_probability(ctx.handle, ens, descs[m], ucp.UCP_MIN | ucp.UCP_MAX,
                                outs[m][0], outs[m][1])
            if ev is not None:
                e1.record()
                ev.append((m, e0, e1))

    # the timed region: barrier + synchronize on both sides.  The raw clock
    # samples go to a CSV (UCP_CLOCKS_DIR, else the temporary directory); the
    # JSON line carries their summary.
    clocks_dir = os.environ.get("UCP_CLOCKS_DIR") or tempfile.gettempdir()
    os.makedirs(clocks_dir, exist_ok=True)
    sampler = ClockSampler(local, os.path.join(clocks_dir, f"ucp_clocks_rank{rank}.csv"))
    time.sleep(1.0)                      # let the sampler start before timing
    replicas.barrier()
    torch.cuda.synchronize()
    t_wall0 = time.time()
    total_ms, _ = timed_steps(torch, step, args.steps, args.warmup, flush)
    torch.cuda.synchronize()
    replicas.barrier()
    t_wall1 = time.time()
    clocks = sampler.stop(t_wall0, t_wall1)
    # per-kernel durations (separate pass, same launches, events between kernels)
    _, kms = timed_steps(torch, step_seq, max(5, args.steps // 2), 1, flush,
                         per_kernel_events=True)
    local_ms = total_ms
    total_ms, _, value = replicas.job_throughput(total_ms, H2 * W2 * args.steps, device=dev)

    peaks = measured_peaks()
    per_model = {}
    shares = {}
    for m, b in MODELS2:
        avg = statistics.mean(kms[m])
        params = ctx.fit(ens, descs[m]) if m == "histogram" else None
        bound, amount = work_of(m, N2, H2 * W2, params, BINS2)
        if bound == "hbm":
            ach, peak, unit = amount / (avg / 1e3) / 1e9, peaks["hbm_gbs"], "GB/s"
        else:
            ach, peak, unit = amount / (avg / 1e3) / 1e12, fp32_peak_tflops(
                peaks["sm_max_mhz"]), "TFLOP/s"
        per_model[m] = {"ms": avg, "vertices_per_s": H2 * W2 / (avg / 1e3),
                        "kernel": "the model's own fused fit + integrate kernel",
                        "roofline": {"bound": bound, "achieved": ach, "peak": peak,
                                     "unit": unit, "frac": ach / peak,
                                     "traffic": TRAFFIC_BYTES[m],
                                     "traffic_source": TRAFFIC_SOURCE[m]},
                        "issue": issue_block(m, avg, peaks["sm_max_mhz"])}
        shares[m] = avg
    # The step is one launch of the fused kernel (uniform + Epanechnikov +
    # histogram, members staged once): its duration is the step's.  Its
    # algorithmic work is the FP32 work of the Epanechnikov and histogram
    # integrations (the uniform model has none), both types.
    t_kernel = local_ms / args.steps
    hist_params = ctx.fit(ens, descs["histogram"])
    fl = (2.0 * EPAN_FLOPS_PER_VERTEX_TYPE * H2 * W2 +
          2.0 * HIST_FLOPS_PER_PIECE_TYPE * float(hist_piece_counts(hist_params, BINS2).sum().item()))
    del hist_params
    pk = fp32_peak_tflops(peaks["sm_max_mhz"])
    ach = fl / (t_kernel / 1e3) / 1e12
    hbm_b = (4.0 * N2 + 6 * 4.0) * H2 * W2
    rf = {"bound": "alu", "achieved": ach, "peak": pk, "unit": "TFLOP/s", "frac": ach / pk,
          "kernel": "tile3_kernel (uniform + Epanechnikov + histogram-8 of one ensemble, "
                    "members staged once by TMA)",
          "traffic": TRAFFIC_BYTES["fused"],
          "traffic_source": TRAFFIC_SOURCE["fused"] + " (ncu dram__bytes_read/write)",
          "work": f"{EPAN_FLOPS_PER_VERTEX_TYPE} flops per vertex and type (Epanechnikov) + "
                  f"{HIST_FLOPS_PER_PIECE_TYPE} per merged histogram piece and type",
          "peak_source": f"152 SMs x 128 FP32 lanes x 2 x {peaks['sm_max_mhz']:.0f} MHz (derived)",
          "hbm_achieved_gbs": hbm_b / (t_kernel / 1e3) / 1e9,
          "hbm_frac": hbm_b / (t_kernel / 1e3) / 1e9 / peaks["hbm_gbs"],
          "share": 1.0,
          "issue": issue_block("fused", t_kernel, peaks["sm_max_mhz"])}

    line = {
        "metric": "critical-point probability vertices/s (uniform + Epanechnikov + "
                  "histogram-8, min and max, 1024x1024x20)",
        "value": value, "unit": "vertices/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "bimodal ensemble 1024x1024, N=20, uniform/Epanechnikov/"
                               "hist-8, min+max, fused fit+integrate",
                   "grid": [H2, W2], "members": N2, "bins": BINS2,
                   "parallelism": f"replicas x{world}",
                   "l2": "flushed between timed steps (512 MB written, then another 512 MB read)"},
        "gpu_launches": args.steps,
        "clocks": clocks,
        "roofline": rf,
        "per_model": per_model,
    }
    if rank == 0:
        line["e2e"] = e2e_headline(torch, ucp, ctx, ens_np, args)
        line["cpu_baseline"] = cpu_baseline_headline(ens_np) if world == 1 else None
        if not args.no_rows:
            line["rows"] = other_rows(torch, ucp, ctx, dev, args, flush, peaks)
        line["summary"] = summarise(line)
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def _g(x):
    return None if x is None else float(f"{x:.3g}")


def summarise(line):
    """A compact digest of the line (ms, vertices/s and roofline fraction per
    kernel and row), placed last so that it survives a truncated tail."""
    iss = lambda b: _g(b["frac"]) if isinstance(b, dict) else None
    out = {"headline": {"ms": _g(line["ms_per_step"]), "vps": _g(line["value"]),
                        "frac": _g(line["roofline"]["frac"]),
                        "issue_frac": iss(line["roofline"].get("issue")),
                        "e2e_vps": _g(line.get("e2e", {}).get("value"))}}
    for m, r in line.get("per_model", {}).items():
        out[m] = {"ms": _g(r["ms"]), "vps": _g(r["vertices_per_s"]),
                  "frac": _g(r["roofline"]["frac"]), "bound": r["roofline"]["bound"],
                  "issue_frac": iss(r.get("issue"))}
    for name, r in (line.get("rows") or {}).items():
        d = {}
        for k in ("ms", "ms_fwd", "ms_adjoint", "ms_fwd_bwd", "ms_batched_graph",
                  "ms_per_field_launches", "speedup", "vertices_per_s", "fwd_vertices_per_s",
                  "fwd_bwd_vertices_per_s", "batched_vertices_per_s"):
            if isinstance(r.get(k), (int, float)):
                d[k] = _g(r[k])
        for k in ("roofline", "fwd_roofline_hbm", "fwd_roofline_fp32", "adjoint_roofline"):
            if isinstance(r.get(k), dict):
                d[k + "_frac"] = _g(r[k]["frac"])
        if isinstance(r.get("oracle"), dict):
            o = r["oracle"]
            d["oracle_vps"] = _g(o.get("fwd_bwd_vertices_per_s", o.get("vertices_per_s")))
        if d:
            out[name] = d
    if isinstance(line.get("cpu_baseline"), dict):
        out["cpu_baseline_vps"] = _g(line["cpu_baseline"]["value"])
    return out


def e2e_headline(torch, ucp, ctx, ens_np, args):
    """Same metric end to end through the C ABI with host buffers: every step
    is one ucp_probability_host_models call on pinned host memory -- the
    members copied to the device once, in row strips overlapped with the
    fused kernel, which writes the six probability fields into the pinned
    output arrays over the host link -- so both transfers are inside the
    timed region (wall clock; the call returns after its streams are
    synchronised)."""
    ens_h = torch.from_numpy(ens_np).pin_memory()
    descs = [ucp.make_desc(m, bins=b or 8) for m, b in MODELS2]
    outs_min = [torch.empty((H2, W2)).pin_memory() for _ in MODELS2]
    outs_max = [torch.empty((H2, W2)).pin_memory() for _ in MODELS2]

    def step():
        ucp.ucp_probability_host_models(ctx.handle, ens_h, descs, 3, outs_min, outs_max)
    for _ in range(max(1, args.warmup)):
        step()
    torch.cuda.synchronize()
    n = max(3, min(args.steps, 50))
    t = time.perf_counter()
    for _ in range(n):
        step()
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t) / n
    return {"value": H2 * W2 / dt, "unit": "vertices/s", "ms_per_step": dt * 1e3,
            "h2d_bytes_per_step": ens_np.nbytes,
            "d2h_bytes_per_step": len(MODELS2) * 2 * H2 * W2 * 4,
            "api": "ucp_probability_host_models on pinned host arrays (members copied once "
                   "per step in row strips overlapped with the fused kernel, which writes the "
                   "six fields into the pinned output arrays)"}


def other_rows(torch, ucp, ctx, dev, args, flush, peaks):
    from paper_2407_18015_gb300 import synth
    want = set(args.rows.split(","))
    rows = {}
    steps = max(3, min(args.steps, 5))
    if "mvn" in want:
        e3 = torch.from_numpy(synth.ensemble_correlated(512, 512, 40, seed=3)).to(dev)
        d = ucp.make_desc("mvn", mc_samples=10000, seed=0x5EED)
        pm = torch.empty((512, 512), device=dev)
        px = torch.empty_like(pm)
        ms, _ = timed_steps(torch, lambda ev: ucp.ucp_probability(ctx.handle, e3, d, 3, pm, px),
                            steps, 2, flush)
        ms /= steps
        samples = 512 * 512 * 10000
        ach = samples * MVN_OPS_PER_SAMPLE / (ms / 1e3) / 1e12
        pk = issue_peak_tops(peaks["sm_max_mhz"])
        rows["mvn_512x512x40_S10000"] = {
            "ms": ms, "vertices_per_s": 512 * 512 / (ms / 1e3),
            "samples_per_s": samples / (ms / 1e3), "min_and_max": True,
            "roofline": {"bound": "alu", "achieved": ach, "peak": pk, "unit": "Tops/s",
                         "frac": ach / pk, "work": f"{MVN_OPS_PER_SAMPLE} lane operations per sample",
                         "peak_source": f"152 SMs x 128 lanes x 1 op x {peaks['sm_max_mhz']:.0f} MHz"},
            "oracle": oracle_mvn_rate(e3.cpu().numpy())}
        del e3
    if "fwdbwd" in want:
        e4 = torch.from_numpy(synth.ensemble_bimodal(2048, 2048, 50, seed=4)).to(dev)
        Wt = torch.from_numpy(synth.weight_field(2048, 2048, seed=44)).to(dev)
        HW4, N4 = 2048 * 2048, 50
        fp32 = fp32_peak_tflops(peaks["sm_max_mhz"])
        fp32_src = f"152 SMs x 128 FP32 lanes x 2 x {peaks['sm_max_mhz']:.0f} MHz (derived)"
        for m, b in (("histogram", 16), ("epanechnikov", 0), ("uniform", 0)):
            d = ucp.make_desc(m, bins=b or 8)
            params = ctx.fit(e4, d)
            pmin = torch.empty((2048, 2048), device=dev)
            Q = b if m == "histogram" else 2
            grad = torch.empty((Q, 2048, 2048), device=dev)

            def fb(ev, d=d, params=params, pmin=pmin, grad=grad):
                ucp.ucp_fit(ctx.handle, e4, d, params)
                ucp.ucp_probability_from_params(ctx.handle, params, d, ucp.UCP_MIN, pmin, None)
                ucp.ucp_backward(ctx.handle, params, d, ucp.UCP_MIN, Wt, grad)

            def fw(ev, d=d, pmin=pmin):
                ucp.ucp_probability(ctx.handle, e4, d, ucp.UCP_MIN, pmin, None)

            def bw(ev, d=d, params=params, grad=grad):
                ucp.ucp_backward(ctx.handle, params, d, ucp.UCP_MIN, Wt, grad)
            ms_fb, _ = timed_steps(torch, fb, steps, 2, flush)
            ms_fw, _ = timed_steps(torch, fw, steps, 2, flush)
            ms_bw, _ = timed_steps(torch, bw, steps, 2, flush)
            ms_fb, ms_fw, ms_bw = ms_fb / steps, ms_fw / steps, ms_bw / steps
            # forward (fused fit + P_min): members read once, one field written
            fwd_bytes = (4.0 * N4 + 4.0) * HW4
            hbm = fwd_bytes / (ms_fw / 1e3) / 1e9
            row = {
                "ms_fwd_bwd": ms_fb, "fwd_bwd_vertices_per_s": HW4 / (ms_fb / 1e3),
                "ms_fwd": ms_fw, "fwd_vertices_per_s": HW4 / (ms_fw / 1e3),
                "ms_adjoint": ms_bw,
                "fwd_roofline_hbm": {"bound": "hbm", "achieved": hbm, "peak": peaks["hbm_gbs"],
                                     "unit": "GB/s", "frac": hbm / peaks["hbm_gbs"],
                                     "work": f"{4 * N4 + 4} bytes per vertex (members + P_min)",
                                     "peak_source": "MEASURED_PEAKS.json hbm_gbs"}}
            if m == "histogram":
                pieces = float(hist_piece_counts(params, b).sum().item())
                fl = pieces * HIST_FLOPS_PER_PIECE_TYPE / (ms_fw / 1e3) / 1e12
                row["fwd_roofline_fp32"] = {
                    "bound": "alu", "achieved": fl, "peak": fp32, "unit": "TFLOP/s",
                    "frac": fl / fp32, "work": f"{HIST_FLOPS_PER_PIECE_TYPE} flops per merged "
                    "piece (one type)", "peak_source": fp32_src}
                ach = pieces * ADJ_HIST_FLOPS_PER_PIECE / (ms_bw / 1e3) / 1e12
                row["adjoint_roofline"] = {
                    "bound": "alu", "achieved": ach, "peak": fp32, "unit": "TFLOP/s",
                    "frac": ach / fp32, "work": f"{ADJ_HIST_FLOPS_PER_PIECE} flops per merged piece",
                    "peak_source": fp32_src,
                    "kernel": "hist_adj_tile<16> (+ hist_adj_fixup)",
                    "algorithmic_bytes": (2.0 * b + 3.0) * 4.0 * HW4,
                    "traffic": TRAFFIC_BYTES["hist_adjoint_16"],
                    "traffic_source": TRAFFIC_SOURCE["hist_adjoint_16"] + " (hist_adj_tile alone)"}
                row["oracle"] = oracle_fwd_bwd_rate(e4, Wt, m, b, rows=128)
            elif m == "epanechnikov":
                fl = HW4 * EPAN_FLOPS_PER_VERTEX_TYPE / (ms_fw / 1e3) / 1e12
                row["fwd_roofline_fp32"] = {
                    "bound": "alu", "achieved": fl, "peak": fp32, "unit": "TFLOP/s",
                    "frac": fl / fp32, "work": f"{EPAN_FLOPS_PER_VERTEX_TYPE} flops per vertex "
                    "(one type)", "peak_source": fp32_src}
                ach = HW4 * ADJ_EPAN_FLOPS_PER_VERTEX / (ms_bw / 1e3) / 1e12
                row["adjoint_roofline"] = {
                    "bound": "alu", "achieved": ach, "peak": fp32, "unit": "TFLOP/s",
                    "frac": ach / fp32, "work": f"{ADJ_EPAN_FLOPS_PER_VERTEX} flops per vertex "
                    "(two forward vertex integrals)", "peak_source": fp32_src}
                row["oracle"] = oracle_fwd_bwd_rate(e4, Wt, m, b)
            else:
                # adjoint: params (2 planes) and W read, 2 gradient planes written
                bw_bytes = 4.0 * (2 + 1 + 2) * HW4
                a = bw_bytes / (ms_bw / 1e3) / 1e9
                row["adjoint_roofline"] = {
                    "bound": "hbm", "achieved": a, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "frac": a / peaks["hbm_gbs"], "work": "20 bytes per vertex",
                    "peak_source": "MEASURED_PEAKS.json hbm_gbs"}
            rows[f"fwd_bwd_2048x2048x50_{m}{b or ''}"] = row
            del params, grad
        del e4
    if "batch" in want:
        rows[f"batch_{args.batch_fields}_fields"] = batch_row(torch, ucp, ctx, dev, steps, flush,
                                                              args.batch_fields, args.batch_max,
                                                              peaks)
    if "sizes" in want:
        # the uniform kernel (N=20, both types) over grid sizes: whether its
        # HBM fraction at 1024^2 is a size effect or the kernel's own bound
        out = {}
        for S in (512, 1024, 2048, 4096):
            g = torch.Generator(device=dev).manual_seed(S)
            es = torch.randn((20, S, S), device=dev, generator=g)
            pm = torch.empty((S, S), device=dev)
            px = torch.empty_like(pm)
            d = ucp.make_desc("uniform")
            ms, _ = timed_steps(torch, lambda ev: ucp.ucp_probability(ctx.handle, es, d, 3, pm, px),
                                max(steps, 10), 3, flush)
            ms /= max(steps, 10)
            gbs = (4.0 * 20 + 8.0) * S * S / (ms / 1e3) / 1e9
            out[f"{S}x{S}x20"] = {"ms": ms, "algorithmic_GBps": gbs,
                                  "hbm_frac": gbs / peaks["hbm_gbs"]}
            del es, pm, px
        rows["uniform_sizes_n20"] = out
    if "saddle" in want:
        e2 = torch.from_numpy(synth.ensemble_bimodal(H2, W2, N2, seed=SEED2)).to(dev)
        out = torch.empty((H2, W2), device=dev)
        r = {}
        for m, b in MODELS2:
            d = ucp.make_desc(m, bins=b or 8)
            ms, _ = timed_steps(torch, lambda ev, d=d: ucp.ucp_saddle(ctx.handle, e2, d, out),
                                steps, 2, flush)
            r[m] = {"ms": ms / steps, "vertices_per_s": H2 * W2 / (ms / steps / 1e3)}
        d = ucp.make_desc("histogram_semi", bins=BINS2, mc_samples=1000)
        pm, px = torch.empty((H2, W2), device=dev), torch.empty((H2, W2), device=dev)
        ms, _ = timed_steps(torch, lambda ev: ucp.ucp_probability(ctx.handle, e2, d, 3, pm, px),
                            steps, 2, flush)
        rows["saddle_1024x1024x20"] = r
        rows["semianalytical_hist8_c1000_1024x1024x20"] = {
            "ms": ms / steps, "vertices_per_s": H2 * W2 / (ms / steps / 1e3), "min_and_max": True}
        del e2
    if "gmm" in want:
        rows["gmm_outliers_64x64x50_max"] = gmm_row(torch, ucp, ctx, dev, steps, flush)
    if "stencil" in want:
        rows.update(stencil_rows(torch, ucp, ctx, dev, steps, flush))
    return rows


def stencil_rows(torch, ucp, ctx, dev, steps, flush):
    """Larger neighbour sets, fused fit + probability (min and max): the 6-
    and 8-neighbour 2D stencils on the 1024x1024x20 workload and the 3D
    axis stencil on a 64x128x128 grid (20 members, the same generator)."""
    from paper_2407_18015_gb300 import synth
    out = {}
    for name, stencil, (D, H, W) in (("stencil6_1024x1024x20", ucp.UCP_STENCIL_6, (1, H2, W2)),
                                     ("stencil8_1024x1024x20", ucp.UCP_STENCIL_8, (1, H2, W2)),
                                     ("stencil3d6_64x128x128x20", ucp.UCP_STENCIL_3D6,
                                      (64, 128, 128))):
        e = synth.ensemble_bimodal(D * H, W, N2, seed=SEED2)
        ens = torch.from_numpy(e.reshape((N2, D, H, W)) if D > 1 else e).to(dev)
        grid = (D, H, W) if D > 1 else (H, W)
        pm, px = torch.empty(grid, device=dev), torch.empty(grid, device=dev)
        r = {}
        for m, b in MODELS2:
            d = ucp.make_desc(m, bins=b or 8, stencil=stencil, depth=D)
            ms, _ = timed_steps(torch, lambda ev, d=d: ucp.ucp_probability(
                ctx.handle, ens, d, 3, pm, px), steps, 2, flush)
            r[m] = {"ms": ms / steps, "vertices_per_s": D * H * W / (ms / steps / 1e3)}
        out[name] = r
        del ens
    return out


def gmm_row(torch, ucp, ctx, dev, steps, flush):
    """The model comparison of the paper on the outlier ensemble: local
    maximum probability per model, the time of each, and the probability
    near the true and the outlier peaks."""
    from paper_2407_18015_gb300 import synth
    ens_np, tp, op = synth.ensemble_gmm_outliers()
    ens = torch.from_numpy(ens_np).to(dev)
    H, W = ens_np.shape[1:]
    out = {}
    diag_mvn = None
    for model, bins, S in (("uniform", 0, 0), ("epanechnikov", 0, 0), ("histogram", 5, 0),
                           ("histogram_semi", 5, 1000), ("mvn", 0, 2000), ("gaussian", 0, 0),
                           ("gaussian_mc", 0, 1000)):
        pm = torch.empty((H, W), device=dev)
        if model == "gaussian_mc":
            # independent Gaussians by Monte Carlo: the multivariate model with
            # its covariance reduced to the diagonal
            d = ucp.make_desc("mvn", mc_samples=S)
            diag_mvn = ctx.fit(ens, d)
            for q in range(5, 20):
                if q not in (5, 7, 10, 14, 19):
                    diag_mvn[q].zero_()
            ms, _ = timed_steps(torch, lambda ev, d=d, pm=pm: ucp.ucp_probability_from_params(
                ctx.handle, diag_mvn, d, ucp.UCP_MAX, None, pm), steps, 2, flush)
        else:
            d = ucp.make_desc(model, bins=bins or 8, mc_samples=S or 1000)
            ms, _ = timed_steps(torch, lambda ev, d=d, pm=pm: ucp.ucp_probability(
                ctx.handle, ens, d, ucp.UCP_MAX, None, pm), steps, 2, flush)
        P = pm.cpu().numpy()

        def near(pts):
            return [float(P[y - 2:y + 3, x - 2:x + 3].max()) for (y, x) in pts]
        out[model + (str(bins) if bins else "") + (str(S) if model == "gaussian_mc" else "")] = {
            "ms": ms / steps, "p_max_near_true_peaks": near(tp),
            "p_max_near_outlier_peaks": near(op)}
    return out


def batch_ideal_seconds(torch, ucp, ctx, fields, peaks):
    """The batch's roofline time: per field the larger of its HBM time
    (members read once, one probability field written) and its FP32 time
    (the per-unit flop figures of the tile kernels: Epanechnikov per vertex,
    histogram per merged piece; uniform has none), summed over the fields."""
    fp32 = fp32_peak_tflops(peaks["sm_max_mhz"]) * 1e12
    hbm = peaks["hbm_gbs"] * 1e9
    total = 0.0
    for ens, desc, cp, o in fields:
        N, Hh, Ww = ens.shape
        byt = (4.0 * N + 4.0) * Hh * Ww
        if desc.model == ucp.UCP_EPANECHNIKOV:
            fl = EPAN_FLOPS_PER_VERTEX_TYPE * Hh * Ww
        elif desc.model == ucp.UCP_HISTOGRAM:
            params = ctx.fit(ens, desc)
            fl = HIST_FLOPS_PER_PIECE_TYPE * float(hist_piece_counts(params, desc.bins).sum().item())
            del params
        else:
            fl = 0.0
        total += max(byt / hbm, fl / fp32)
    return total


def batch_row(torch, ucp, ctx, dev, steps, flush, nfields=64, largest=2048, peaks=None):
    """nfields (64) fields of uneven sizes (128^2..largest^2, largest 2048),
    N in {10,20,50,100}, mixed models and types: per-field launches vs one
    autotuned persistent launch replayed from a CUDA graph."""
    from paper_2407_18015_gb300 import synth
    specs = synth.batch_specs(fields=nfields, hi=largest)
    fields = []
    verts = 0
    for sp in specs:
        ens = torch.from_numpy(synth.batch_field(sp)).to(dev)
        desc = ucp.make_desc(sp["model"], bins=sp["bins"])
        cp = ucp.UCP_MIN if sp["cptype"] == "min" else ucp.UCP_MAX
        o = torch.empty((sp["H"], sp["W"]), device=dev)
        fields.append((ens, desc, cp, o))
        verts += sp["H"] * sp["W"]

    def per_field(ev):
        for ens, desc, cp, o in fields:
            ucp.ucp_probability(ctx.handle, ens, desc, cp, o if cp == 1 else None,
                                o if cp == 2 else None)
    ms_pf, _ = timed_steps(torch, per_field, steps, 2, flush)
    b = ucp.Batch(ctx)
    for ens, desc, cp, o in fields:
        b.add(ens, desc, cp, o if cp == 1 else None, o if cp == 2 else None)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        b.tune()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        b.run()
    ms_b, _ = timed_steps(torch, lambda ev: g.replay(), steps, 2, flush)
    b.close()
    ms_pf /= steps
    ms_b /= steps
    out = {"fields": len(fields), "vertices": verts, "ms_per_field_launches": ms_pf,
           "ms_batched_graph": ms_b, "speedup": ms_pf / ms_b,
           "batched_vertices_per_s": verts / (ms_b / 1e3),
           "per_field_vertices_per_s": verts / (ms_pf / 1e3)}
    if peaks is not None:
        ideal = batch_ideal_seconds(torch, ucp, ctx, fields, peaks)
        out["roofline"] = {
            "bound": "mixed", "achieved_ms": ms_b, "roofline_ms": ideal * 1e3,
            "frac": ideal * 1e3 / ms_b,
            "work": "per field max(HBM time of (4N+4) bytes per vertex, FP32 time of the tile "
                    "kernels' flop figures), summed",
            "peak_source": "MEASURED_PEAKS.json hbm_gbs; FP32 152 x 128 x 2 x max SM clock"}
    return out


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
