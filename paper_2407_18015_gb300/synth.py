"""Seeded synthetic ensembles for critical-point probability workloads.

This module only draws random numbers and lays them out as ens[N][H][W]
float32; it holds none of the probability arithmetic, so the CUDA path, the
CPU oracle and the benchmark can all consume it.  Only numpy is used.

Recipes (the paper's real data -- Ackley + noise, E3SM/MGARD climate, Red
Sea -- are not available, so these stand in for them with the same shapes:
smooth multi-scale base fields, tens of members, unimodal/bimodal noise):

  sinusoid_base     sum of 6 plane waves, amplitudes U[0.5, 2], wavelengths
                    U[8, 32] cells (times ``lam_scale``), directions and
                    phases U[0, 2*pi)
  ensemble_iid      base + i.i.d. N(0, sigma^2) noise per member
                    (64x64, N=20, sigma=0.2: the small parity workload)
  ensemble_bimodal  base + s_k * g/2 + N(0, sd^2), s_k = +-1 with p = 1/2 per
                    member and vertex, mode gap g ramping 0 -> 1.5 along x and
                    sd ramping 0.1 -> 0.4 along y (1024^2 x 20, 2048^2 x 50,
                    and every field of the batched workload)
  ensemble_correlated  base + white N(0,1) per member smoothed by a Gaussian
                    kernel of sigma = 3 cells (reflect padding), rescaled to
                    std 0.2 (512^2 x 40: the multivariate-Gaussian workload)
  batch_specs       64 fields: H, W log-uniform integers in [128, 2048],
                    N in {10, 20, 50, 100}, model in {uniform, Epanechnikov,
                    histogram-16}, type in {min, max}
  ensemble_gmm_outliers  50 members with two sharp Gaussian peaks on the NW-SE
                    diagonal, the last 10 rotated by 90 degrees (outliers), as
                    in the paper's model-comparison ensemble
"""
import math

import numpy as np

MODELS_BATCH = ("uniform", "epanechnikov", "histogram")


def sinusoid_base(H, W, rng, waves=6, lam_scale=1.0):
    y = np.arange(H, dtype=np.float64)[:, None]
    x = np.arange(W, dtype=np.float64)[None, :]
    amp = rng.uniform(0.5, 2.0, waves)
    lam = rng.uniform(8.0, 32.0, waves) * lam_scale
    th = rng.uniform(0.0, 2 * math.pi, waves)
    ph = rng.uniform(0.0, 2 * math.pi, waves)
    f = np.zeros((H, W), np.float64)
    for j in range(waves):
        f += amp[j] * np.sin(2 * math.pi * (x * math.cos(th[j]) + y * math.sin(th[j])) / lam[j]
                             + ph[j])
    return f


def ensemble_iid(H=64, W=64, N=20, seed=1, sigma=0.2):
    rng = np.random.default_rng(seed)
    base = sinusoid_base(H, W, rng).astype(np.float32)
    noise = rng.standard_normal((N, H, W), dtype=np.float32) * np.float32(sigma)
    return (base[None] + noise).astype(np.float32)


def ensemble_bimodal(H=1024, W=1024, N=20, seed=2, gap=(0.0, 1.5), sd=(0.1, 0.4),
                     lam_scale=4.0):
    rng = np.random.default_rng(seed)
    base = sinusoid_base(H, W, rng, lam_scale=lam_scale).astype(np.float32)
    g = np.linspace(gap[0], gap[1], W, dtype=np.float32)[None, :]
    s = np.linspace(sd[0], sd[1], H, dtype=np.float32)[:, None]
    out = np.empty((N, H, W), np.float32)
    half_gap = np.float32(0.5) * g
    for k in range(N):
        sign = rng.integers(0, 2, (H, W), dtype=np.int8).astype(np.float32) * 2 - 1
        z = rng.standard_normal((H, W), dtype=np.float32)
        out[k] = base + sign * half_gap + z * s
    return out


def _gauss_kernel(sigma):
    r = int(math.ceil(4 * sigma))
    t = np.arange(-r, r + 1, dtype=np.float64)
    k = np.exp(-0.5 * (t / sigma) ** 2)
    return k / k.sum()


def _smooth_reflect(a, sigma):
    """Separable Gaussian smoothing of a 2D array with reflect padding."""
    k = _gauss_kernel(sigma)
    r = (len(k) - 1) // 2
    p = np.pad(a, ((r, r), (0, 0)), mode="symmetric")
    a = sum(k[i] * p[i:i + a.shape[0], :] for i in range(len(k)))
    p = np.pad(a, ((0, 0), (r, r)), mode="symmetric")
    return sum(k[i] * p[:, i:i + a.shape[1]] for i in range(len(k)))


def ensemble_correlated(H=512, W=512, N=40, seed=3, length=3.0, sd=0.2):
    rng = np.random.default_rng(seed)
    base = sinusoid_base(H, W, rng)
    out = np.empty((N, H, W), np.float32)
    for k in range(N):
        z = _smooth_reflect(rng.standard_normal((H, W)), length)
        z *= sd / z.std()
        out[k] = (base + z).astype(np.float32)
    return out


def weight_field(H, W, seed=44):
    return np.random.default_rng(seed).uniform(0.0, 1.0, (H, W)).astype(np.float32)


def batch_specs(fields=64, seed=5, lo=128, hi=2048):
    """Field shapes/models of the batched workload (no member data)."""
    rng = np.random.default_rng(seed)
    specs = []
    for f in range(fields):
        H = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        W = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        N = int(rng.choice([10, 20, 50, 100]))
        model = MODELS_BATCH[int(rng.integers(0, 3))]
        cptype = ("min", "max")[int(rng.integers(0, 2))]
        specs.append(dict(field=f, H=H, W=W, N=N, model=model, bins=16, cptype=cptype,
                          seed=1000 + f))
    return specs


def batch_field(spec, scale=1.0):
    """Members of one batched field (optionally shrunk by ``scale`` per axis)."""
    H = max(1, int(round(spec["H"] * scale)))
    W = max(1, int(round(spec["W"] * scale)))
    return ensemble_bimodal(H, W, spec["N"], seed=spec["seed"])


def ensemble_gmm_outliers(H=64, W=64, N=50, outliers=10, seed=6, amp=1.0, width=0.025,
                          noise=0.01, jitter=0.0):
    """Two-peak Gaussian-mixture ensemble with rotated outlier members (the
    structure of the paper's model-comparison ensemble): the first N -
    outliers members have their two peaks on the NW-SE diagonal at (0.3, 0.3)
    and (0.7, 0.7) of the unit square (row y grows southwards); the last
    `outliers` members are the same field rotated by 90 degrees (peaks on the
    NE-SW diagonal).  Peak positions are jittered per member by N(0, jitter^2),
    and i.i.d. N(0, noise^2) is added.  Returns (ens, true_peaks, outlier_peaks)
    with the peaks as (y, x) grid indices."""
    rng = np.random.default_rng(seed)
    yy = (np.arange(H, dtype=np.float64)[:, None] + 0.5) / H
    xx = (np.arange(W, dtype=np.float64)[None, :] + 0.5) / W
    true_c = [(0.3, 0.3), (0.7, 0.7)]
    out_c = [(0.3, 0.7), (0.7, 0.3)]
    ens = np.empty((N, H, W), np.float32)
    for k in range(N):
        cs = out_c if k >= N - outliers else true_c
        f = np.zeros((H, W))
        for (cy, cx) in cs:
            cy += rng.normal(0, jitter)
            cx += rng.normal(0, jitter)
            f += amp * np.exp(-((yy - cy) ** 2 + (xx - cx) ** 2) / (2 * width ** 2))
        f += rng.normal(0, noise, (H, W))
        ens[k] = f.astype(np.float32)

    def idx(cs):
        return [(int(cy * H), int(cx * W)) for (cy, cx) in cs]
    return ens, idx(true_c), idx(out_c)
