"""Test-side helpers: independent samplers and parameter transforms.

Nothing here calls the CUDA library or the oracle; the samplers draw each
vertex's variable from its model directly (numpy), so brute-force Monte Carlo
built on them is a route to the probabilities that shares nothing with the
oracle's piecewise integration.
"""
import math

import numpy as np

UNIFORM, EPANECHNIKOV, HISTOGRAM, MVN = 0, 1, 2, 3


def negate_params(params, model):
    """Parameters of -X for every vertex (the paper's negation identity)."""
    p = np.array(params, dtype=np.float64, copy=True)
    if model == UNIFORM:
        return np.stack([-p[1], -p[0]])
    if model == EPANECHNIKOV:
        return np.stack([-p[0], p[1]])
    if model == HISTOGRAM:
        return np.concatenate([np.stack([-p[1], -p[0]]), p[2:][::-1]])
    raise ValueError(model)


def sample_field(params, model, rng, n):
    """n independent draws of the whole field: (n, H, W) float64."""
    p = np.asarray(params, dtype=np.float64)
    H, W = p.shape[1:]
    if model == UNIFORM:
        u = rng.random((n, H, W))
        return p[0] + u * (p[1] - p[0])
    if model == EPANECHNIKOV:
        # inverse CDF of (2 + 3u - u^3)/4 on [-1, 1]: u = 2 cos((acos(1-2q) + 4 pi)/3)
        q = rng.random((n, H, W))
        u = 2.0 * np.cos((np.arccos(1.0 - 2.0 * q) + 4.0 * math.pi) / 3.0)
        return p[0] + p[1] * u
    if model == HISTOGRAM:
        B = p.shape[0] - 2
        w = p[2:] / p[2:].sum(axis=0, keepdims=True)
        cdf = np.cumsum(w, axis=0)
        q = rng.random((n, H, W))
        j = (q[:, None] > cdf[None]).sum(axis=1)
        j = np.minimum(j, B - 1)
        h = (p[1] - p[0]) / B
        return p[0] + (j + rng.random((n, H, W))) * h
    raise ValueError(model)


def neighbour_events(X):
    """For samples X (n, H, W): per-vertex counts of 'strictly below every
    in-grid axis neighbour' and 'strictly above every in-grid neighbour'."""
    n, H, W = X.shape
    lt = np.ones((n, H, W), bool)
    gt = np.ones((n, H, W), bool)
    for dy, dx in ((0, 1), (-1, 0), (0, -1), (1, 0)):
        ys = slice(max(0, -dy), H - max(0, dy))
        xs = slice(max(0, -dx), W - max(0, dx))
        yn = slice(ys.start + dy, ys.stop + dy)
        xn = slice(xs.start + dx, xs.stop + dx)
        lt[:, ys, xs] &= X[:, ys, xs] < X[:, yn, xn]
        gt[:, ys, xs] &= X[:, ys, xs] > X[:, yn, xn]
    return lt.sum(axis=0), gt.sum(axis=0)


def mc_probabilities(params, model, n, seed, batch=250_000):
    rng = np.random.default_rng(seed)
    H, W = np.asarray(params).shape[1:]
    cmin = np.zeros((H, W), np.int64)
    cmax = np.zeros((H, W), np.int64)
    done = 0
    while done < n:
        m = min(batch, n - done)
        a, b = neighbour_events(sample_field(params, model, rng, m))
        cmin += a
        cmax += b
        done += m
    return cmin / n, cmax / n


def random_params(model, H, W, rng, bins=4, spread=1.0):
    """Random, overlapping, non-degenerate parameters on an H x W grid."""
    if model == UNIFORM:
        c = rng.normal(0.0, 0.5 * spread, (H, W))
        hw = rng.uniform(0.2, 1.0, (H, W)) * spread
        return np.stack([c - hw, c + hw])
    if model == EPANECHNIKOV:
        return np.stack([rng.normal(0.0, 0.5 * spread, (H, W)),
                         rng.uniform(0.2, 1.0, (H, W)) * spread])
    if model == HISTOGRAM:
        c = rng.normal(0.0, 0.5 * spread, (H, W))
        hw = rng.uniform(0.2, 1.0, (H, W)) * spread
        w = rng.uniform(0.0, 1.0, (bins, H, W))
        w /= w.sum(axis=0, keepdims=True)
        return np.concatenate([np.stack([c - hw, c + hw]), w])
    raise ValueError(model)


def mvn_params(H, W, mu, cov_fn):
    """Parameter planes [20][H][W] in the library's MVN layout: means of
    (v, e, n, w, s) then their covariance, packed lower triangle row by row;
    absent neighbours get zeros.  cov_fn(y, x, present) -> 5x5 matrix."""
    out = np.zeros((20, H, W))
    offs = ((0, 0), (0, 1), (-1, 0), (0, -1), (1, 0))
    for y in range(H):
        for x in range(W):
            present = [0 <= y + dy < H and 0 <= x + dx < W for dy, dx in offs]
            C = cov_fn(y, x, present)
            for a in range(5):
                if present[a]:
                    out[a, y, x] = mu[y + offs[a][0], x + offs[a][1]]
            r = 5
            for a in range(5):
                for b in range(a + 1):
                    out[r, y, x] = C[a, b] if (present[a] and present[b]) else 0.0
                    r += 1
    return out


def saddle_events(X):
    """Per-vertex counts of the alternating pattern (t1: below e and w, above
    n and s; t2: the reverse) at vertices with all four neighbours, and of
    the two-neighbour pattern on a 1 x W or H x 1 grid (next = e or s,
    previous = w or n)."""
    n, H, W = X.shape
    out = np.zeros((H, W), np.int64)
    if H == 1 or W == 1:
        v = X.reshape(n, -1)
        c, nxt, prv = v[:, 1:-1], v[:, 2:], v[:, :-2]
        hits = ((c < nxt) & (c > prv)) | ((c > nxt) & (c < prv))
        out.reshape(-1)[1:-1] = hits.sum(0)
        return out
    c = X[:, 1:-1, 1:-1]
    e, w = X[:, 1:-1, 2:], X[:, 1:-1, :-2]
    nn, s = X[:, :-2, 1:-1], X[:, 2:, 1:-1]
    t1 = (c < e) & (c > nn) & (c < w) & (c > s)
    t2 = (c > e) & (c < nn) & (c > w) & (c < s)
    out[1:-1, 1:-1] = (t1 | t2).sum(0)
    return out


def mc_saddle(params, model, n, seed, batch=250_000):
    rng = np.random.default_rng(seed)
    H, W = np.asarray(params).shape[1:]
    cnt = np.zeros((H, W), np.int64)
    done = 0
    while done < n:
        m = min(batch, n - done)
        cnt += saddle_events(sample_field(params, model, rng, m))
        done += m
    return cnt / n
