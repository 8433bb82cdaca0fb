"""The bench's algorithmic-work count for the histogram roofline (CPU, no
GPU): hist_piece_counts gives, per vertex, the centre's B bins plus every bin
edge of an in-grid axis neighbour strictly inside the centre's support -- the
pieces of the exact integration.  Checked against a brute-force count."""
import os
import sys

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def brute_pieces(lo, hi, B):
    H, W = lo.shape
    out = np.zeros((H, W))
    for y in range(H):
        for x in range(W):
            c = B
            for dy, dx in ((0, 1), (-1, 0), (0, -1), (1, 0)):
                yy, xx = y + dy, x + dx
                if not (0 <= yy < H and 0 <= xx < W):
                    continue
                for j in range(B + 1):
                    e = np.float32(lo[yy, xx]) + np.float32(j) * (np.float32(hi[yy, xx]) - np.float32(lo[yy, xx])) / np.float32(B)
                    if lo[y, x] < e < hi[y, x]:
                        c += 1
            out[y, x] = c
    return out


def test_piece_counts_match_brute_force():
    import bench
    rng = np.random.default_rng(3)
    for B in (1, 4, 8):
        c = rng.normal(0, 0.5, (7, 9)).astype(np.float32)
        hw = rng.uniform(0.1, 1.0, (7, 9)).astype(np.float32)
        lo, hi = c - hw, c + hw
        lo[2, 3] = hi[2, 3]                 # a point mass
        lo[4, 4], hi[4, 4] = lo[4, 5], hi[4, 5]   # identical neighbours
        params = torch.from_numpy(np.stack([lo, hi]))
        got = bench.hist_piece_counts(params, B).numpy()
        np.testing.assert_array_equal(got, brute_pieces(lo, hi, B))
