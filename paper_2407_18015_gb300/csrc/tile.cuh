// tile.cuh -- one tile of the closed-form path: the statistics pass into a
// shared-memory parameter tile with a one-vertex halo, then the exact
// integration of every vertex of the tile (device.cuh).  Shared by the
// single-field kernel (closed.cu) and the persistent batch kernel (batch.cu).
#pragma once

#include <cuda.h>

#include "device.cuh"
#include "launch.h"

namespace ucp {

__device__ __forceinline__ float qnan() { return __int_as_float(0x7fc00000); }

// shared-memory floats of one tile of height TYv: the parameter rows of the
// (TYv + 2) x 34 halo tile and, for the histogram, the tail-table rows and the
// scratch of the walk ordering (buckets, then two 16-bit arrays of TYv x 32)
__host__ __device__ constexpr long long tile_floats(int model, int B, int TYv) {
  const long long halo = (long long)(TYv + 2) * 34;
  return model == kSemi   ? (2 + 2LL * B) * halo
         : model == kHist ? hist_rows(B) * halo + kSortBuckets + TYv * 32
                          : 2 * halo;
}

// Shared-memory floats of the parameter tile of a histogram tile that walks
// per-bin rows: lo, hi, then the total mass T and the status (rows 2 and 3,
// written once the rows are built); while the rows are built from masses
// held in the tile (rows 2 .. 1 + B), those take their place, else (masses
// from bin counts in registers) a table of the values count / N follows,
// then, for more than 8 bins, the counters' increments per bin
// (ROWS_INC_TABLE floats: 16 bins x two 64-bit words).  The rows themselves
// (hist_r4_rows x hist_r4_stride float4) come on top.
constexpr int ROWS_MASS_TABLE = 256;
constexpr int ROWS_INC_TABLE = 64;
__host__ __device__ constexpr long long hist_rows_tile_floats(int B, int TYv, bool masses) {
  const long long halo = (long long)(TYv + 2) * 34;
  return masses ? (2 + B > 4 ? 2 + B : 4) * halo
                : 4 * halo + ROWS_MASS_TABLE + (B > 8 ? ROWS_INC_TABLE : 0);
}

// resident CTAs per SM each model's register budget is tuned for.  RB > 0:
// histogram tiles that walk per-bin rows of at most RB bins -- four CTAs
// per SM for 8 bins, two for 16 (their rows' shared memory allows no more).
template <int MODEL, int RB = 0>
struct TileOcc {
  static constexpr int value =
      MODEL == kUniform ? 5
                        : (MODEL == kEpan ? 5
                                          : (MODEL == kHist ? (RB == 8 ? 4 : (RB == 16 ? 2 : 3))
                                                            : (MODEL == kSemi ? 4 : 2)));
};

// floats of the parameter tile: the model's tile, or for per-bin-row
// histogram tiles the smaller one of hist_rows_tile_floats (masses held in
// it only when they are not counted in registers)
template <int MODEL, int TYm, bool ROWS>
__host__ __device__ constexpr long long param_tile_floats(int B, bool masses) {
  return ROWS ? hist_rows_tile_floats(B, TYm, masses) : tile_floats(MODEL, B, TYm);
}

// rows of a histogram tile's per-bin tables (hist_r4_rows float4 per halo
// vertex, rows hist_r4_stride apart), in floats
__host__ __device__ constexpr int r4_floats(int B, int TYv) {
  return 4 * hist_r4_rows(B) * hist_r4_stride((TYv + 2) * 34);
}

// Number of pieces of the histogram walk of a tile vertex (0 for a vertex
// that does not walk): the centre's B bins plus every neighbour edge inside
// the centre's support.
template <int HALO>
__device__ __forceinline__ int hist_pieces(const float *sm, int B, int l, const bool *present,
                                           const int *nl) {
  const float lo1 = sm[l], hi1 = sm[HALO + l];
  const int st = (int)sm[(5 + B) * HALO + l];
  if (st != 0) return 0;
  int c = B;
  const float fb = (float)B;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    if (!present[i]) continue;
    const float lo = sm[nl[i]], hi = sm[HALO + nl[i]];
    if (lo == hi) {
      c += (lo > lo1 && lo < hi1) ? 1 : 0;
      continue;
    }
    const float ih = fb / (hi - lo);
    const float a = fminf(fmaxf((lo1 - lo) * ih, -1.f), fb + 1.f);
    const float b = fminf(fmaxf((hi1 - lo) * ih, -1.f), fb + 1.f);
    const int first = max((int)floorf(a) + 1, 0), last = min((int)ceilf(b) - 1, B);
    c += max(last - first + 1, 0);
  }
  return min(c, 5 * B + 4);
}

// Orders the tile's vertices by decreasing walk length (a counting sort in
// shared memory), so that the lanes of a warp take walks of about the same
// number of pieces; returns the order (tile vertex indices).
template <int TY, int HALO>
__device__ __forceinline__ const unsigned short *hist_order(const Field &f, float *sm, int ty0,
                                                           int tx0) {
  constexpr int TX = 32, HX = TX + 2, NV = TY * TX;
  static_assert(NV % NTHREADS == 0, "whole warps per pass");
  const int B = f.B, NB = 5 * B + 5;
  int *bucket = reinterpret_cast<int *>(sm + (long long)hist_rows(B) * HALO);
  unsigned short *cnt = reinterpret_cast<unsigned short *>(bucket + kSortBuckets);
  unsigned short *order = cnt + NV;
  const int lane = threadIdx.x & 31;
  for (int q = threadIdx.x; q < NB; q += NTHREADS) bucket[q] = 0;
  __syncthreads();
  for (int v = threadIdx.x; v < NV; v += NTHREADS) {
    const int r = v / TX + 1, c = v % TX + 1;
    const int gy = ty0 + r - 1, gx = tx0 + c - 1;
    int n = 0;
    if (gy < f.y1 && gx < f.W) {
      const int l = r * HX + c;
      bool present[4];
      int nl[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int yy = gy + kDy[i], xx = gx + kDx[i];
        present[i] = (yy >= 0 && yy < f.H && xx >= 0 && xx < f.W);
        nl[i] = l + kDy[i] * HX + kDx[i];
      }
      n = hist_pieces<HALO>(sm, B, l, present, nl);
    }
    cnt[v] = (unsigned short)n;
    const unsigned peers = __match_any_sync(0xffffffffu, n);
    if (lane == __ffs(peers) - 1) atomicAdd(&bucket[n], __popc(peers));
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    // exclusive offsets in decreasing length order: lane takes `per`
    // consecutive buckets from the top
    const int per = (NB + 31) / 32;
    int sum = 0;
    for (int j = 0; j < per; ++j) {
      const int b = NB - 1 - (lane * per + j);
      if (b >= 0) sum += bucket[b];
    }
    int inc = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += t;
    }
    int run = inc - sum;
    for (int j = 0; j < per; ++j) {
      const int b = NB - 1 - (lane * per + j);
      if (b >= 0) {
        const int k = bucket[b];
        bucket[b] = run;
        run += k;
      }
    }
  }
  __syncthreads();
  for (int v = threadIdx.x; v < NV; v += NTHREADS) {
    const int n = cnt[v];
    const unsigned peers = __match_any_sync(0xffffffffu, n);
    const int leader = __ffs(peers) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(&bucket[n], __popc(peers));
    base = __shfl_sync(0xffffffffu, base, leader);
    order[base + __popc(peers & ((1u << lane) - 1u))] = (unsigned short)v;
  }
  __syncthreads();
  return order;
}

// Statistics of V consecutive vertices of one row (V = 1, or 4 with one
// 16-byte load per member), written to the shared parameter tile at l.
template <int V>
__device__ __forceinline__ void load_v(const float *p, float (&v)[V]) {
  if constexpr (V == 4) {
    const float4 t = __ldg(reinterpret_cast<const float4 *>(p));
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
  } else {
    v[0] = __ldg(p);
  }
}

template <int MODEL, int V, int HALO>
__device__ __forceinline__ void stage_members(const Field &f, float *sm, int l, long long gi) {
  const long long plane = f.plane;
  const float *p = f.ens + gi;
  const int N = f.N;
  float mn[V], mx[V];
  bool nf[V];
  if constexpr (MODEL == kEpan || MODEL == kGauss) {
    // one pass, shifted by the first member (see members_epan)
    float x0[V];
    Kahan s1[V], s2[V];
    load_v<V>(p, x0);
#pragma unroll
    for (int q = 0; q < V; ++q) { mn[q] = mx[q] = x0[q]; nf[q] = false; }
#pragma unroll 4
    for (int k = 0; k < N; ++k) {
      float v[V];
      load_v<V>(p + (long long)k * plane, v);
#pragma unroll
      for (int q = 0; q < V; ++q) {
        nf[q] |= !isfinite(v[q]);
        mn[q] = fminf(mn[q], v[q]);
        mx[q] = fmaxf(mx[q], v[q]);
        const float d = v[q] - x0[q];
        s1[q].add(d);
        s2[q].add(d * d);
      }
    }
#pragma unroll
    for (int q = 0; q < V; ++q) {
      float m, w;
      if (mn[q] == mx[q]) {
        m = mn[q];
        w = 0.f;
      } else {
        const float S1 = s1[q].get(), S2 = s2[q].get();
        const float md = S1 / (float)N;
        m = x0[q] + md;
        const float scale = MODEL == kGauss ? 1.f : f.epan_scale;
        w = scale * sqrtf(fmaxf(S2 - S1 * md, 0.f) / (float)(N - 1));
      }
      sm[l + q] = nf[q] ? qnan() : m;
      sm[HALO + l + q] = nf[q] ? qnan() : w;
    }
  } else {
    {
      float v[V];
      load_v<V>(p, v);
#pragma unroll
      for (int q = 0; q < V; ++q) { mn[q] = mx[q] = v[q]; nf[q] = false; }
    }
#pragma unroll 8
    for (int k = 0; k < N; ++k) {
      float v[V];
      load_v<V>(p + (long long)k * plane, v);
#pragma unroll
      for (int q = 0; q < V; ++q) {
        nf[q] |= !isfinite(v[q]);
        mn[q] = fminf(mn[q], v[q]);
        mx[q] = fmaxf(mx[q], v[q]);
      }
    }
#pragma unroll
    for (int q = 0; q < V; ++q) {
      sm[l + q] = nf[q] ? qnan() : mn[q];
      sm[HALO + l + q] = nf[q] ? qnan() : mx[q];
    }
    if constexpr (hist_params(MODEL)) {
      const int B = f.B;
      float sc[V];
      bool bin[V];
#pragma unroll
      for (int q = 0; q < V; ++q) {
        float *wq = sm + 2 * HALO + l + q;
        for (int b = 0; b < B; ++b) wq[b * HALO] = nf[q] ? qnan() : 0.f;
        bin[q] = !nf[q] && mn[q] != mx[q];
        if (!nf[q] && !bin[q]) wq[0] = 1.f;
        sc[q] = bin[q] ? __fdiv_rn((float)B, __fsub_rn(mx[q], mn[q])) : 0.f;
      }
      bool any = false;
#pragma unroll
      for (int q = 0; q < V; ++q) any |= bin[q];
      if (any) {
#pragma unroll 4
        for (int k = 0; k < N; ++k) {
          float v[V];
          load_v<V>(p + (long long)k * plane, v);
#pragma unroll
          for (int q = 0; q < V; ++q)
            if (bin[q]) sm[(2 + hist_bin(v[q], mn[q], sc[q], B)) * HALO + l + q] += 1.f;
        }
#pragma unroll
        for (int q = 0; q < V; ++q)
          if (bin[q])
            for (int b = 0; b < B; ++b) {
              float *w = sm + (2 + b) * HALO + l + q;
              *w = __fdiv_rn(*w, (float)N);
            }
      }
    }
  }
}

template <int MODEL, bool FROM_MEMBERS, int HALO>
__device__ __forceinline__ void stage_vertex(const Field &f, float *sm, int l, long long gi) {
  const long long plane = f.plane;
  if (!FROM_MEMBERS) {
    const int P = hist_params(MODEL) ? 2 + f.B : 2;
    for (int q = 0; q < P; ++q) sm[q * HALO + l] = __ldg(f.params + q * plane + gi);
    return;
  }
  const float *p = f.ens + gi;
  if (MODEL == kUniform) {
    float mn, mx;
    bool nf;
    members_minmax(p, plane, f.N, mn, mx, nf);
    sm[l] = nf ? qnan() : mn;
    sm[HALO + l] = nf ? qnan() : mx;
  } else if (MODEL == kEpan || MODEL == kGauss) {
    float m, w, mn, mx;
    bool nf;
    members_epan(p, plane, f.N, MODEL == kGauss ? 1.f : f.epan_scale, m, w, mn, mx, nf);
    sm[l] = nf ? qnan() : m;
    sm[HALO + l] = nf ? qnan() : w;
  } else {
    float mn, mx;
    bool nf;
    members_minmax(p, plane, f.N, mn, mx, nf);
    const int B = f.B;
    float *wq = sm + 2 * HALO + l;
    if (nf) {
      sm[l] = sm[HALO + l] = qnan();
      for (int q = 0; q < B; ++q) wq[q * HALO] = qnan();
      return;
    }
    sm[l] = mn;
    sm[HALO + l] = mx;
    for (int q = 0; q < B; ++q) wq[q * HALO] = 0.f;
    if (mn == mx) {
      wq[0] = 1.f;
      return;
    }
    const float s = __fdiv_rn((float)B, __fsub_rn(mx, mn));
    for (int k = 0; k < f.N; ++k) {
      const int j = hist_bin(__ldg(p + (long long)k * plane), mn, s, B);
      wq[j * HALO] += 1.f;
    }
    for (int q = 0; q < B; ++q) wq[q * HALO] = __fdiv_rn(wq[q * HALO], (float)f.N);
  }
}

// Tail table S_0..S_{B+1} in place of the masses of staged vertex l, its total
// mass and its status (rows 2..3+B, 4+B, 5+B; see hist_rows)
template <int HALO>
__device__ __forceinline__ void hist_tail_table(float *sm, int l, int B) {
  const float a = sm[l], b = sm[HALO + l];
  uint8_t st = (!isfinite(a) || !isfinite(b)) ? V_NONFINITE
                                             : (a > b ? V_BAD : (a == b ? V_DEGENERATE : 0));
  float t = 0.f;
  for (int q = 0; q < B; ++q) {
    const float w = sm[(2 + q) * HALO + l];
    if (!isfinite(w)) st |= V_NONFINITE;
    else if (w < 0.f) st |= V_BAD;
    t += w;
  }
  const bool point = a == b;
  float c = 0.f;
  for (int q = 0; q < B; ++q) {
    float *r = sm + (2 + q) * HALO + l;
    const float w = *r;
    *r = point ? 0.f : t - c;
    c += w;
  }
  sm[(2 + B) * HALO + l] = 0.f;
  sm[(3 + B) * HALO + l] = 0.f;
  sm[(4 + B) * HALO + l] = t;
  sm[(5 + B) * HALO + l] = (float)st;
}

// Per-bin rows of one vertex (see hist_r4_rows) from its lo, hi and masses
// m_0..m_{B-1} (all FP32): R[k * RS] for k = 0..B.  T = m_0 + ... + m_{B-1}
// in bin order; the tails S_k = T - (m_0 + ... + m_{k-1}).
template <int RS, typename Mass>
__device__ __forceinline__ void hist_rows_build(float4 *R, float a, float b, float t, int B,
                                                Mass mass) {
  const float4 beyond = make_float4(0.f, t, 0.f, kFar);
  if (a == b) {
    for (int k = 0; k < hist_r4_rows(B); ++k) R[k * RS] = beyond;
    return;
  }
  // for a power of two B the product with 1/B is the quotient exactly
  const float w = b - a;
  const float h = (B & (B - 1)) == 0 ? w * (1.f / (float)B) : w / (float)B, ih = frcp(h);
  float c = 0.f, sk = t;
  for (int k = 0; k < B; ++k) {
    c += mass(k);
    const float sn = k + 1 < B ? t - c : 0.f;
    R[k * RS] = make_float4(sk, t - sk, (sk - sn) * ih, k + 1 < B ? (float)(k + 1) * h : w);
    sk = sn;
  }
  R[B * RS] = beyond;
}

// Per-bin rows of staged vertex l from the masses in its parameter tile
// (rows 2 .. 1 + B); afterwards the tile holds lo, hi, the total mass (row 2)
// and the status bits (row 3), as check_params<kHist, HALO, true> reads them.
template <int HALO, int RS>
__device__ __forceinline__ void hist_row_table(float *sm, float4 *R, int l, int B) {
  const float a = sm[l], b = sm[HALO + l];
  uint8_t st = (!isfinite(a) || !isfinite(b)) ? V_NONFINITE
                                             : (a > b ? V_BAD : (a == b ? V_DEGENERATE : 0));
  float t = 0.f;
  for (int q = 0; q < B; ++q) {
    const float w = sm[(2 + q) * HALO + l];
    if (!isfinite(w)) st |= V_NONFINITE;
    else if (w < 0.f) st |= V_BAD;
    t += w;
  }
  hist_rows_build<RS>(R + l, a, b, t, B, [&](int k) { return sm[(2 + k) * HALO + l]; });
  sm[2 * HALO + l] = t;
  sm[3 * HALO + l] = (float)st;
}

// The same from bin counts kept in registers (fitted mass count / N of bin k
// from cnt_mass(k)), for a vertex fitted from its members: lo = mn, hi = mx;
// nf marks non-finite members (all parameters NaN), mn == mx a point mass
// (mass 1 in bin 0).  The same masses, total, rows and status as the
// parameter tile and hist_row_table give.
template <int HALO, int RS, int RB, typename Mass>
__device__ __forceinline__ void hist_row_table_counts(float *sm, float4 *R, int l, int B, bool nf,
                                                      float mn, float mx, Mass cnt_mass) {
  // at most RB bins: every loop unrolled to RB with the bins past B idle
  float m[RB];
  float t = 0.f;
#pragma unroll
  for (int q = 0; q < RB; ++q) {
    m[q] = 0.f;
    if (q < B) {
      m[q] = nf ? qnan() : (mn == mx ? (q == 0 ? 1.f : 0.f) : cnt_mass(q));
      t += m[q];
    }
  }
  const uint8_t st = nf ? V_NONFINITE : (mn == mx ? V_DEGENERATE : 0);
  R += l;
  const float a = nf ? qnan() : mn, b = nf ? qnan() : mx;
  const float4 beyond = make_float4(0.f, t, 0.f, kFar);
  if (a == b) {
#pragma unroll
    for (int k = 0; k <= RB; ++k)
      if (k <= B) R[k * RS] = beyond;
  } else {
    // as hist_rows_build
    const float w = b - a;
    const float h = (B & (B - 1)) == 0 ? w * (1.f / (float)B) : w / (float)B, ih = frcp(h);
    float c = 0.f, sk = t;
#pragma unroll
    for (int k = 0; k < RB; ++k) {
      if (k < B) {
        c += m[k];
        const float sn = k + 1 < B ? t - c : 0.f;
        R[k * RS] = make_float4(sk, t - sk, (sk - sn) * ih, k + 1 < B ? (float)(k + 1) * h : w);
        sk = sn;
      }
    }
    R[B * RS] = beyond;
  }
  sm[2 * HALO + l] = t;
  sm[3 * HALO + l] = (float)st;
}

// The parameters of one vertex in registers (mirrored: -X, bins
// reversed): support [a, b] and masses m[0..B-1], read with every load in
// flight at once.
template <int RB>
struct HistParamRegs {
  float a, b, m[RB];
  __device__ __forceinline__ void load(const Field &f, long long gi, int B, bool mirrored) {
    const long long plane = f.plane;
    const float a0 = __ldg(f.params + gi), b0 = __ldg(f.params + plane + gi);
    a = mirrored ? -b0 : a0;
    b = mirrored ? -a0 : b0;
#pragma unroll
    for (int q = 0; q < RB; ++q)
      m[q] = q < B ? __ldg(f.params + (long long)(2 + (mirrored ? B - 1 - q : q)) * plane + gi)
                   : 0.f;
  }
};

// Per-bin rows, lo, hi, total and status of one staged vertex from its
// parameters in registers; the same rows and status as hist_row_table
// builds from a parameter tile.
template <int HALO, int RS, int RB>
__device__ __forceinline__ void hist_rows_build_regs(const HistParamRegs<RB> &P, float *sm,
                                                     float4 *R, int l, int B) {
  const float a = P.a, b = P.b;
  uint8_t st = (!isfinite(a) || !isfinite(b)) ? V_NONFINITE
                                             : (a > b ? V_BAD : (a == b ? V_DEGENERATE : 0));
  float t = 0.f;
#pragma unroll
  for (int q = 0; q < RB; ++q) {
    if (q < B) {
      if (!isfinite(P.m[q])) st |= V_NONFINITE;
      else if (P.m[q] < 0.f) st |= V_BAD;
      t += P.m[q];
    }
  }
  R += l;
  const float4 beyond = make_float4(0.f, t, 0.f, kFar);
  if (a == b) {
#pragma unroll
    for (int k = 0; k <= RB; ++k)
      if (k <= B) R[k * RS] = beyond;
  } else {
    // as hist_rows_build
    const float w = b - a;
    const float h = (B & (B - 1)) == 0 ? w * (1.f / (float)B) : w / (float)B, ih = frcp(h);
    float c = 0.f, sk = t;
#pragma unroll
    for (int k = 0; k < RB; ++k) {
      if (k < B) {
        c += P.m[k];
        const float sn = k + 1 < B ? t - c : 0.f;
        R[k * RS] = make_float4(sk, t - sk, (sk - sn) * ih, k + 1 < B ? (float)(k + 1) * h : w);
        sk = sn;
      }
    }
    R[B * RS] = beyond;
  }
  sm[l] = a;
  sm[HALO + l] = b;
  sm[2 * HALO + l] = t;
  sm[3 * HALO + l] = (float)st;
}

// Per-bin rows of every in-grid halo vertex of the tile at (ty0, tx0) from
// the parameters.  BATCH: each thread first reads the parameters of all the
// halo vertices it owns (l = tid, tid + NTHREADS, ...), every load in
// flight at once, then builds their rows -- for kernels at two CTAs per SM,
// whose CTA otherwise waits for two rounds of reads (2048 x 2048 x 50, 16
// bins: forward from parameters 1.11 -> 1.06 ms, adjoint 2.85 -> 2.83 ms);
// else one vertex after another (the 8-bin forward at four CTAs per SM:
// 0.53 ms, against 0.57 batched).
template <int HALO, int RS, int RB, int HX, bool BATCH>
__device__ __forceinline__ void hist_rows_from_params_tile(const Field &f, float *sm, float4 *R,
                                                           int ty0, int tx0, int ylim, int B,
                                                           bool mirrored) {
  if constexpr (!BATCH) {
    for (int l = threadIdx.x; l < HALO; l += NTHREADS) {
      const int r = l / HX, c = l - r * HX;
      const int gy = ty0 + r - 1, gx = tx0 + c - 1;
      if (gy < 0 || gy >= ylim || gx < 0 || gx >= f.W) continue;
      HistParamRegs<RB> P;
      P.load(f, (long long)gy * f.W + gx, B, mirrored);
      hist_rows_build_regs<HALO, RS, RB>(P, sm, R, l, B);
    }
    return;
  }
  constexpr int PER = (HALO + NTHREADS - 1) / NTHREADS;
  HistParamRegs<RB> P[PER];
  bool in[PER];
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    const int l = threadIdx.x + p * NTHREADS;
    const int r = l / HX, c = l - r * HX;
    const int gy = ty0 + r - 1, gx = tx0 + c - 1;
    in[p] = l < HALO && gy >= 0 && gy < ylim && gx >= 0 && gx < f.W;
    if (in[p]) P[p].load(f, (long long)gy * f.W + gx, B, mirrored);
  }
#pragma unroll
  for (int p = 0; p < PER; ++p)
    if (in[p]) hist_rows_build_regs<HALO, RS, RB>(P[p], sm, R, threadIdx.x + p * NTHREADS, B);
}

// ---------------------------------------------------------------------------
// Member staging with the tensor memory accelerator: one bulk tensor copy
// brings a box of nc members x (TYv + 2) rows x 40 columns (x from tx0 - 4, a
// 16-byte boundary; y from ty0 - 1; out-of-range elements read as 0) into
// shared memory, completing on an mbarrier.  Every thread then reduces the
// members of the halo vertices it owns (l = tid, tid + 256, ...).  Larger
// ensembles take several boxes in turn.

constexpr int kBoxW = 40;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_inval(uint64_t *bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void proxy_async_fence() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y,
                                            int z, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}
// one 16-byte asynchronous copy global -> shared (both addresses 16-byte
// aligned; no register round trip, not cached in L1), and the wait for all
// of this thread's copies in flight
__device__ __forceinline__ void cp_async16(void *dst, uintptr_t src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;" ::: "memory");
}

// Members [k0, k0 + min(nc, N - k0)) of the box of the tile at (ty0, tx0),
// rows below ylim, by 16-byte asynchronous copies of the aligned blocks
// that hold each (member, row) segment (see `load` in stage_members_tma for
// the layout: column c of member m, row r at m PLANE + r kBoxW + c + d, d =
// (address / 4) mod 4); the copies have landed for the whole CTA on return.
template <int HY>
__device__ __forceinline__ void box_copy_async(const Field &f, float *box, int k0, int nc,
                                               int ty0, int tx0, int ylim) {
  constexpr int PLANE = HY * kBoxW;
  const int N = f.N;
  constexpr int SLOTS = NTHREADS / 5, DM = SLOTS / HY, DR = SLOTS % HY;
  const int nseg = min(nc, N - k0) * HY;
  if (threadIdx.x < SLOTS * 5) {
    const int q = threadIdx.x % 5;
    int sg = threadIdx.x / 5;
    const int m = sg / HY;
    int r = sg - m * HY;
    // smem columns (before the shift d) that staged vertices read
    const int lo0 = max(tx0 - 1, 0) - tx0 + 4, hi0 = min(tx0 + 33, f.W) - tx0 + 4;
    const uintptr_t rstep = (uintptr_t)f.W * 4u, pstep = (uintptr_t)f.plane * 4u;
    uintptr_t a = reinterpret_cast<uintptr_t>(f.ens) +
                  (uintptr_t)(((long long)(k0 + m) * f.plane +
                               (long long)(ty0 - 1 + r) * f.W + (tx0 - 4)) * 4);
    float *dst = box + m * PLANE + r * kBoxW + 8 * q;
    for (; sg < nseg; sg += SLOTS) {
      const int gy = ty0 - 1 + r;
      if ((unsigned)gy < (unsigned)ylim) {
        const int d = (int)(a >> 2) & 3;
        const int lo = lo0 + d, hi = hi0 + d, j = 8 * q;
        const uintptr_t cb = (a & ~(uintptr_t)15) + 32u * q;
        if (j + 4 > lo && j < hi) cp_async16(dst, cb);
        if (j + 8 > lo && j + 4 < hi) cp_async16(dst + 4, cb + 16);
      }
      r += DR;
      a += DM * pstep + DR * rstep;
      dst += DM * PLANE + DR * kBoxW;
      if (r >= HY) {
        r -= HY;
        a += pstep - HY * rstep;
        dst += PLANE - HY * kBoxW;
      }
    }
  }
  cp_async_wait_all();
  __syncthreads();
}

// wait for the completion of phase `parity`; gives up after a bounded number
// of polls (each poll itself returns after a bounded time)
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity) {
  for (int i = 0; i < (1 << 20); ++i) {
    uint32_t done;
    // each poll may suspend the thread for up to about a microsecond (the
    // time hint, in ns) until the phase completes, so the waiting warp
    // takes few issue slots
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity), "n"(1000)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Statistics of the members of every in-grid halo vertex into the shared
// parameter tile, as stage_members computes them (same arithmetic in the same
// member order).  Returns false if a wait gave up (the tile is then invalid).
// ROWS: histogram per-bin rows into R4 in place of the tail tables (R4 may
// overlap the box: the rows are written after the barrier that ends the last
// read of the box).
template <int MODEL, int TYv, int RB, bool ASYNC>
__device__ __forceinline__ bool stage_members_tma(const Field &f, float *sm, float *box,
                                                  uint64_t *bar, const CUtensorMap *tmap,
                                                  int ty0, int tx0, float4 *R4) {
  constexpr int HY = TYv + 2, HX = 34, HALO = HY * HX;
  constexpr int PER = (HALO + NTHREADS - 1) / NTHREADS;
  constexpr int PLANE = HY * kBoxW;
  const int N = f.N, nc = f.tma_nc;
  const unsigned box_bytes = (unsigned)(PLANE * nc * sizeof(float));
  const int ylim = min(f.H, f.y1 + 1);
  // box filled by the tensor memory accelerator, or (ASYNC) by asynchronous
  // copies with the element shifts described at `load` below (eb, pl, w4
  // all 0 for the accelerator: no shift)
  constexpr bool tma = !ASYNC;
  const int eb = ASYNC ? (int)(reinterpret_cast<uintptr_t>(f.ens) >> 2) & 3 : 0;
  const int pl = ASYNC ? (int)(f.plane & 3) : 0, w4 = ASYNC ? f.W & 3 : 0;
  int off[PER], lv[PER], rq[PER];
  bool in[PER];
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    const int l = threadIdx.x + p * NTHREADS;
    const int r = l / HX, c = l - r * HX;
    const int gy = ty0 + r - 1, gx = tx0 + c - 1;
    lv[p] = l;
    in[p] = l < HALO && gy >= 0 && gy < ylim && gx >= 0 && gx < f.W;
    off[p] = r * kBoxW + c + 3;
    rq[p] = ((gy & 3) * w4) & 3;
  }
  // the shift of member k0 (the box's first) at owned vertex p
  auto shift0 = [&](int p, int k0) { return (eb + (k0 & 3) * pl + rq[p]) & 3; };
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    mbar_init_fence();
  }
  if constexpr (MODEL == kHist && RB > 0) {
    // the masses count / N of up to 255 members (see the per-bin rows
    // below), and for more than 8 bins each bin's increment of the two
    // words of 8-bit counters: bin j adds 1 << 8 (j mod 8) to word j / 8
    // (one 16-byte read instead of a shift and two selects per member;
    // with one word the shift is cheaper: 162.5 vs 169 us at 1024 x 1024 x
    // 20, 8 bins, against 1397 -> 1367 us at 2048 x 2048 x 50, 16 bins)
    if (N <= 255) {
      for (int c = threadIdx.x; c <= N; c += NTHREADS)
        sm[4 * HALO + c] = __fdiv_rn((float)c, (float)N);
      if constexpr (RB > 8) {
        ulonglong2 *itab = reinterpret_cast<ulonglong2 *>(sm + 4 * HALO + ROWS_MASS_TABLE);
        for (int j = threadIdx.x; j < RB; j += NTHREADS)
          itab[j] = make_ulonglong2(j < 8 ? 1ull << (j << 3) : 0ull,
                                    j < 8 ? 0ull : 1ull << ((j - 8) << 3));
      }
    }
  }
  __syncthreads();
  unsigned phase = 0;
  bool ok = true;
  // load members [k0, k0 + nc) into the box; uniform result
  // One warp polls the mbarrier while the copy is in flight; the others
  // wait at the CTA barrier, which takes no issue slots from the warps of
  // other CTAs.  Once the phase is complete every thread tests it once
  // more (it returns at once), so each thread acquires the copied data
  // itself.
  //
  // Members the tensor memory accelerator cannot address (W not a multiple
  // of 4, or a base that is not 16-byte aligned: f.vec4 false, ASYNC) are copied
  // into the same box by 16-byte asynchronous copies of the aligned blocks
  // that hold each (member, row) segment: the element of column c (x =
  // tx0 - 4 + c) then lands at c + d, d = (its address / 4) mod 4, at most
  // 3, so the columns the staged vertices read (3 .. 36) stay inside the
  // 40-float row.  Five threads share a segment, two blocks each; only the
  // blocks that hold a column a staged in-grid vertex reads are copied, so
  // every block read holds an element of the members (no read leaves the
  // allocation).  d = (eb + m pl + gy w4) mod 4 for member m and row gy (eb
  // the base's offset in floats mod 4, pl = H W mod 4, w4 = W mod 4): the
  // readers add it, per row, and per member when pl != 0.
  auto load = [&](int k0) -> bool {
    if constexpr (ASYNC) {
      box_copy_async<HY>(f, box, k0, nc, ty0, tx0, ylim);
      return true;
    }
    if (threadIdx.x == 0) {
      proxy_async_fence();
      mbar_expect_tx(bar, box_bytes);
      tma_load_3d(box, tmap, tx0 - 4, ty0 - 1, k0, bar);
    }
    bool r = true;
    if (threadIdx.x < 32) r = mbar_wait(bar, phase);
    r = __syncthreads_and(r) != 0;
    if (r) (void)mbar_wait(bar, phase);
    phase ^= 1u;
    return r;
  };
  constexpr bool EP = MODEL == kEpan || MODEL == kGauss;
  float mn[PER], mx[PER], x0[PER];
  bool nf[PER];
  Kahan s1[PER], s2[PER];
  for (int k0 = 0; k0 < N && ok; k0 += nc) {
    if (!load(k0)) {
      ok = false;
      break;
    }
    const int kn = min(nc, N - k0);
#pragma unroll
    for (int p = 0; p < PER; ++p) {
      if (!in[p]) continue;
      const int sh = shift0(p, k0);
      const float *col = box + off[p] + sh;
      // member 0 starts the running min / max (and is the shift x0 of the
      // Epanechnikov sums, to which it adds 0); the others go in pairs into
      // NaN-propagating three-input min / max, so that a non-finite member
      // shows in mn / mx (nf below)
      int k = 0;
      if (k0 == 0) {
        x0[p] = mn[p] = mx[p] = col[0];
        k = 1;
      }
      auto add = [&](float v) {
        if constexpr (EP) {
          const float d = v - x0[p];
          s1[p].add(d);
          s2[p].add(d * d);
        }
      };
      auto add2 = [&](float v1, float v2) {
        mn[p] = fmin3_nan(mn[p], v1, v2);
        mx[p] = fmax3_nan(mx[p], v1, v2);
        add(v1);
        add(v2);
      };
      if (pl == 0) {
#pragma unroll 4
        for (; k + 1 < kn; k += 2) add2(col[k * PLANE], col[(k + 1) * PLANE]);
      } else {
        for (; k + 1 < kn; k += 2)
          add2(col[k * PLANE + (((sh + k * pl) & 3) - sh)],
               col[(k + 1) * PLANE + (((sh + (k + 1) * pl) & 3) - sh)]);
      }
      if (k < kn) {
        const float v = col[k * PLANE + (((sh + k * pl) & 3) - sh)];
        mn[p] = fmin_nan(mn[p], v);
        mx[p] = fmax_nan(mx[p], v);
        add(v);
      }
    }
    __syncthreads();
  }
  if (!ok) {
    // the copy that timed out may still land: wait for it (bounded) before
    // the shared memory is left to another CTA
    if (threadIdx.x == 0) mbar_wait(bar, phase ^ 1u);
    __syncthreads();
    return false;
  }
#pragma unroll
  for (int p = 0; p < PER; ++p) nf[p] = !(isfinite(mn[p]) && isfinite(mx[p]));
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    if (!in[p]) continue;
    const int l = lv[p];
    if constexpr (EP) {
      float m, w;
      if (mn[p] == mx[p]) {
        m = mn[p];
        w = 0.f;
      } else {
        const float S1 = s1[p].get(), S2 = s2[p].get();
        const float md = S1 / (float)N;
        m = x0[p] + md;
        const float scale = MODEL == kGauss ? 1.f : f.epan_scale;
        w = scale * sqrtf(fmaxf(S2 - S1 * md, 0.f) / (float)(N - 1));
      }
      sm[l] = nf[p] ? qnan() : m;
      sm[HALO + l] = nf[p] ? qnan() : w;
    } else {
      sm[l] = nf[p] ? qnan() : mn[p];
      sm[HALO + l] = nf[p] ? qnan() : mx[p];
    }
  }
  if constexpr (MODEL == kHist && RB > 0) {
    // per-bin rows (at most RB bins): the bin counts of every owned vertex
    // stay in registers across the boxes, packed 8-bit counters (eight per
    // 64-bit word) for up to 255 members, 16-bit ones (four per word) for
    // more; the rows are built from them once the last box has been read
    // (they take the box's room).  Masses count / N come from a table of
    // the N + 1 possible values (ROWS_MASS_TABLE floats after the parameter
    // tile, filled at the start of the staging) for up to 255 members.
    constexpr int RS = hist_r4_stride(HALO);
    constexpr int NW8 = RB / 8, NW16 = RB / 4;
    const int B = f.B;
    const bool wide = N > 255;
    const float *mtab = sm + 4 * HALO;
    float sc[PER];
    bool bin[PER];
    bool any = false;
    unsigned long long cw[PER][NW16];
#pragma unroll
    for (int p = 0; p < PER; ++p) {
#pragma unroll
      for (int w = 0; w < NW16; ++w) cw[p][w] = 0ull;
      bin[p] = in[p] && !nf[p] && mn[p] != mx[p];
      sc[p] = bin[p] ? __fdiv_rn((float)B, __fsub_rn(mx[p], mn[p])) : 0.f;
      any |= bin[p];
    }
    const int last = ((N - 1) / nc) * nc;
    for (int k0 = last; k0 >= 0; k0 -= nc) {
      if (k0 != last) {
        if (!load(k0)) {
          if (threadIdx.x == 0) mbar_wait(bar, phase ^ 1u);
          __syncthreads();
          return false;
        }
      }
      const int kn = min(nc, N - k0);
      if (any) {
#pragma unroll
        for (int p = 0; p < PER; ++p) {
          if (!bin[p]) continue;
          const int sh = shift0(p, k0);
          const float *col = box + off[p] + sh;
          const ulonglong2 *itab =
              reinterpret_cast<const ulonglong2 *>(sm + 4 * HALO + ROWS_MASS_TABLE);
          auto count8 = [&](float v) {
            const int j = hist_bin_nonneg(v, mn[p], sc[p], B);
            if constexpr (NW8 == 1) {
              cw[p][0] += 1ull << ((j & 7) << 3);
            } else {
              const ulonglong2 inc = itab[j];
              cw[p][0] += inc.x;
              cw[p][1] += inc.y;
            }
          };
          auto count16 = [&](float v) {
            const int j = hist_bin_nonneg(v, mn[p], sc[p], B);
            const unsigned long long inc = 1ull << ((j & 3) << 4);
#pragma unroll
            for (int w = 0; w < NW16; ++w) cw[p][w] += (j >> 2) == w ? inc : 0ull;
          };
          if (pl != 0) {
            for (int k = 0; k < kn; ++k) {
              const float v = col[k * PLANE + (((sh + k * pl) & 3) - sh)];
              if (!wide) count8(v);
              else count16(v);
            }
          } else if (!wide) {
#pragma unroll 4
            for (int k = 0; k < kn; ++k) count8(col[k * PLANE]);
          } else {
            for (int k = 0; k < kn; ++k) count16(col[k * PLANE]);
          }
        }
      }
      __syncthreads();
    }
#pragma unroll
    for (int p = 0; p < PER; ++p) {
      if (!in[p]) continue;
      hist_row_table_counts<HALO, RS, RB>(
          sm, R4, lv[p], B, nf[p], mn[p], mx[p], [&](int k) -> float {
            if (!wide) return mtab[(unsigned)(cw[p][k >> 3] >> ((k & 7) << 3)) & 255u];
            return __fdiv_rn((float)((unsigned)(cw[p][k >> 2] >> ((k & 3) << 4)) & 0xFFFFu),
                             (float)N);
          });
    }
    return true;
  }
  if constexpr (hist_params(MODEL)) {
    const int B = f.B;
    float sc[PER];
    bool bin[PER];
    bool any = false;
#pragma unroll
    for (int p = 0; p < PER; ++p) {
      bin[p] = false;
      sc[p] = 0.f;
      if (!in[p]) continue;
      float *wq = sm + 2 * HALO + lv[p];
      for (int b = 0; b < B; ++b) wq[b * HALO] = nf[p] ? qnan() : 0.f;
      bin[p] = !nf[p] && mn[p] != mx[p];
      if (!nf[p] && !bin[p]) wq[0] = 1.f;
      sc[p] = bin[p] ? __fdiv_rn((float)B, __fsub_rn(mx[p], mn[p])) : 0.f;
      any |= bin[p];
    }
    // boxes in reverse order: the last one of the first pass is still there
    const int last = ((N - 1) / nc) * nc;
    for (int k0 = last; k0 >= 0; k0 -= nc) {
      if (k0 != last) {
        if (!load(k0)) {
          if (threadIdx.x == 0) mbar_wait(bar, phase ^ 1u);
          __syncthreads();
          return false;
        }
      }
      const int kn = min(nc, N - k0);
      if (any) {
#pragma unroll
        for (int p = 0; p < PER; ++p) {
          if (!bin[p]) continue;
          const int sh = shift0(p, k0);
          const float *col = box + off[p] + sh;
          float *w0 = sm + 2 * HALO + lv[p];
          for (int k = 0; k < kn; ++k)
            w0[hist_bin(col[k * PLANE + (((sh + k * pl) & 3) - sh)], mn[p], sc[p], B) * HALO] +=
                1.f;
        }
      }
      __syncthreads();
    }
#pragma unroll
    for (int p = 0; p < PER; ++p)
      if (bin[p])
        for (int b = 0; b < B; ++b) {
          float *w = sm + (2 + b) * HALO + lv[p];
          *w = __fdiv_rn(*w, (float)N);
        }
    if constexpr (MODEL == kHist) {
      // the owner also builds the vertex's tail table
#pragma unroll
      for (int p = 0; p < PER; ++p)
        if (in[p]) hist_tail_table<HALO>(sm, lv[p], B);
    }
  }
  return true;
}

// validity of one participant's parameters; returns status bits and the
// histogram total mass
template <int MODEL, int HALO, bool ROWS = false>
__device__ __forceinline__ uint8_t check_params(const float *sm, int l, int B, float &T) {
  if constexpr (MODEL == kHist && ROWS) {
    // precomputed with the per-bin rows
    T = sm[2 * HALO + l];
    return (uint8_t)sm[3 * HALO + l];
  }
  if constexpr (MODEL == kHist) {
    // precomputed by the tail-table pass
    T = sm[(4 + B) * HALO + l];
    return (uint8_t)sm[(5 + B) * HALO + l];
  }
  const float a = sm[l], b = sm[HALO + l];
  T = 1.f;
  if (!isfinite(a) || !isfinite(b)) return V_NONFINITE;
  if (MODEL == kUniform) return a > b ? V_BAD : (a == b ? V_DEGENERATE : 0);
  if (MODEL == kEpan || MODEL == kGauss) return b < 0.f ? V_BAD : (b == 0.f ? V_DEGENERATE : 0);
  uint8_t st = a > b ? V_BAD : (a == b ? V_DEGENERATE : 0);
  float t = 0.f;
  for (int q = 0; q < B; ++q) {
    const float w = sm[(2 + q) * HALO + l];
    if (!isfinite(w)) st |= V_NONFINITE;
    else if (w < 0.f) st |= V_BAD;
    t += w;
  }
  T = t;
  return st;
}

// NaN and the timeout flag for every vertex of a tile whose staging gave up
// (a bounded wait expired)
template <int TYv, bool SADDLE>
__device__ __forceinline__ void mark_tile_timeout(const Field &f, int ty0, int tx0) {
  constexpr int TX = 32;
  for (int v = threadIdx.x; v < TYv * TX; v += NTHREADS) {
    const int gy = ty0 + v / TX, gx = tx0 + v % TX;
    if (gy >= f.y1 || gx >= f.W) continue;
    const long long gi = (long long)gy * f.W + gx;
    if constexpr (SADDLE) {
      if (f.out_saddle) f.out_saddle[gi] = qnan();
    } else {
      if ((f.cptypes & kMin) && f.out_min) f.out_min[gi] = qnan();
      if ((f.cptypes & kMax) && f.out_max) f.out_max[gi] = qnan();
    }
    if (f.status) f.status[gi] = V_TIMEOUT;
  }
}

template <int MODEL, int TYv, bool SADDLE, bool TABLES_BUILT, bool ROWS>
__device__ __forceinline__ void integrate_tile(const Field &f, int ty0, int tx0, float *sm,
                                               float4 *R4);

// One tile of TYv x 32 vertices: phase 1 stages the parameters of the tile
// and its one-vertex halo ((TYv + 2) x 34) in shared memory -- fitted from the
// members or loaded -- and phase 2 (integrate_tile) integrates every vertex
// of the tile; returns false if the staging gave up (a bounded wait
// expired; the tile is then marked).  SADDLE selects the saddle probability (Eq. saddleProb)
// instead of the minimum / maximum: a separate instance, so neither pays for
// the other.  TMA: the members are staged through the tensor map tmap into
// `box`, with the mbarrier `bar` (FROM_MEMBERS only); with ASYNC as well,
// by asynchronous copies into the same box instead (members the tensor
// memory accelerator cannot address; tmap unused).  RB > 0 (histograms
// of at most RB bins): the walk runs over per-bin rows in R4 (hist_r4_rows
// rows of hist_r4_stride float4, 16-byte aligned; it may overlap `box`)
// instead of the segment walker's tail table; each kernel instance carries
// one of the two walks.
template <int MODEL, bool FROM_MEMBERS, int TYv, bool SADDLE = false, bool TMA = false,
          int RB = 0, bool ASYNC = false>
__device__ __forceinline__ bool process_tile(const Field &f, int ty0, int tx0, float *sm,
                                             const CUtensorMap *tmap = nullptr,
                                             float *box = nullptr, uint64_t *bar = nullptr,
                                             float4 *R4 = nullptr) {
  constexpr int TY = TYv, TX = 32, HY = TYv + 2, HX = TX + 2, HALO = HY * HX;
  // rows beyond y1 are neither computed nor needed (row y1 is a neighbour)
  const int ylim = min(f.H, f.y1 + 1);

  bool staged = true;
  if constexpr (FROM_MEMBERS && TMA) {
    staged = stage_members_tma<MODEL, TY, RB, ASYNC>(f, sm, box, bar, tmap, ty0, tx0, R4);
  } else if (FROM_MEMBERS) {
    // work items per halo row: the two halo columns (scalar) and eight
    // groups of four interior columns (one float4 per member when aligned)
    for (int it = threadIdx.x; it < HY * 10; it += NTHREADS) {
      const int r = it / 10, g = it - r * 10;
      const int gy = ty0 + r - 1;
      if (gy < 0 || gy >= ylim) continue;
      const long long rowi = (long long)gy * f.W;
      if (g == 0 || g == 9) {
        const int c = g == 0 ? 0 : HX - 1, gx = tx0 + c - 1;
        if (gx >= 0 && gx < f.W) stage_members<MODEL, 1, HALO>(f, sm, r * HX + c, rowi + gx);
      } else {
        const int c0 = 1 + 4 * (g - 1), gx0 = tx0 + 4 * (g - 1);
        if (f.vec4 && gx0 + 3 < f.W) {
          stage_members<MODEL, 4, HALO>(f, sm, r * HX + c0, rowi + gx0);
        } else {
          for (int q = 0; q < 4; ++q)
            if (gx0 + q < f.W) stage_members<MODEL, 1, HALO>(f, sm, r * HX + c0 + q, rowi + gx0 + q);
        }
      }
    }
  } else if constexpr (MODEL == kHist && RB > 0) {
    // per-bin rows straight from the parameters (masses in registers)
    constexpr int RS = hist_r4_stride(HALO);
    hist_rows_from_params_tile<HALO, RS, RB, HX, (RB > 8)>(f, sm, R4, ty0, tx0, ylim, f.B, false);
  } else {
    for (int l = threadIdx.x; l < HALO; l += NTHREADS) {
      const int r = l / HX, c = l - r * HX;
      const int gy = ty0 + r - 1, gx = tx0 + c - 1;
      if (gy < 0 || gy >= ylim || gx < 0 || gx >= f.W) continue;
      stage_vertex<MODEL, false, HALO>(f, sm, l, (long long)gy * f.W + gx);
    }
  }
  __syncthreads();
  if (!staged) {  // a bounded wait gave up (uniform over the CTA): NaN + flag
    mark_tile_timeout<TY, SADDLE>(f, ty0, tx0);
    return false;
  }
  integrate_tile<MODEL, TY, SADDLE, (FROM_MEMBERS && TMA) || (!FROM_MEMBERS && RB > 0),
                 (RB > 0)>(f, ty0, tx0, sm, R4);
  return true;
}

// Phase 2 of a tile whose parameters (and, if TABLES_BUILT, histogram tail
// tables or per-bin rows) are staged in shared memory: every vertex of the
// tile integrated.
template <int MODEL, int TYv, bool SADDLE, bool TABLES_BUILT, bool ROWS>
__device__ __forceinline__ void integrate_tile(const Field &f, int ty0, int tx0, float *sm,
                                               float4 *R4) {
  constexpr int TY = TYv, TX = 32, HY = TYv + 2, HX = TX + 2, HALO = HY * HX;
  constexpr int RS = hist_r4_stride(HALO);
  (void)HY;
  (void)R4;
  if constexpr (MODEL == kHist && !TABLES_BUILT) {
    // tail tables or rows of every staged vertex (the TMA staging builds
    // them itself)
    for (int l = threadIdx.x; l < HALO; l += NTHREADS) {
      if constexpr (ROWS) hist_row_table<HALO, RS>(sm, R4, l, f.B);
      else hist_tail_table<HALO>(sm, l, f.B);
    }
    __syncthreads();
  }
  if constexpr (MODEL == kSemi) {
    // running mass sums C_1..C_B of every staged vertex, in bin order
    for (int l = threadIdx.x; l < HALO; l += NTHREADS) {
      float c = 0.f;
      for (int q = 0; q < f.B; ++q) {
        c += sm[(2 + q) * HALO + l];
        sm[(2 + f.B + q) * HALO + l] = c;
      }
    }
    __syncthreads();
  }
  [[maybe_unused]] const unsigned short *order = nullptr;
  // the segment walker's lanes take walks of about equal length (an 8-row
  // tile of per-bin row walks gains nothing from the ordering)
  if constexpr (MODEL == kHist && !ROWS) order = hist_order<TY, HALO>(f, sm, ty0, tx0);

  for (int it = threadIdx.x; it < TY * TX; it += NTHREADS) {
    int v = it;
    if constexpr (MODEL == kHist && !ROWS) {
      // pass j of warp w takes the j-th group of eight 32-vertex blocks of
      // the ordered list, in reverse on odd passes, so that every warp gets
      // about the same total length
      const int j = it / NTHREADS, w = (threadIdx.x >> 5), nw = NTHREADS / 32;
      const int blk = j * nw + ((j & 1) ? nw - 1 - w : w);
      v = order[blk * 32 + (threadIdx.x & 31)];
    }
    const int r = v / TX + 1, c = v % TX + 1;
    const int gy = ty0 + r - 1, gx = tx0 + c - 1;
    if (gy >= f.y1 || gx >= f.W) continue;
    const int l = r * HX + c;
    bool present[4];
    int nl[4];
    int k = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int yy = gy + kDy[i], xx = gx + kDx[i];
      present[i] = (yy >= 0 && yy < f.H && xx >= 0 && xx < f.W);
      nl[i] = l + kDy[i] * HX + kDx[i];
      k += present[i];
    }
    float T[4], Tc;
    uint8_t st = check_params<MODEL, HALO, ROWS>(sm, l, f.B, Tc);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      T[i] = 1.f;
      if (present[i])
        st |= check_params<MODEL, HALO, ROWS>(sm, nl[i], f.B, T[i]) & (V_NONFINITE | V_BAD);
    }
    float pmin = 0.f, pmax = 0.f, psad = 0.f;
    int sg[4], sg2[4];
    const bool bad = (st & (V_NONFINITE | V_BAD)) != 0;
    const bool has_saddle = SADDLE && saddle_signs(present, f.H, f.W, sg);
#pragma unroll
    for (int i = 0; i < 4; ++i) sg2[i] = SADDLE ? -sg[i] : 0;
    if (bad) {
      pmin = pmax = psad = qnan();
    } else if constexpr (MODEL == kSemi) {
      SemiNb nb[4];
      const float lo1 = sm[l];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        nb[i].off = nl[i];
        nb[i].T = T[i];
        if (!present[i]) {
          nb[i].kind = 0;
          nb[i].lam = 0.f;
          nb[i].ih = 0.f;
          continue;
        }
        const float lo = sm[nl[i]], hi = sm[HALO + nl[i]];
        nb[i].lam = lo - lo1;
        nb[i].kind = lo == hi ? 2 : 1;
        nb[i].ih = lo == hi ? 0.f : (float)f.B / (hi - lo);
      }
      const PhiloxKeys K(f.seed_lo, f.seed_hi);
      if (!SADDLE || has_saddle)
        semi_vertex<HALO, SADDLE>(sm + 2 * HALO, sm + (2 + f.B) * HALO, l, lo1, sm[HALO + l], nb,
                                  f.B, f.samples, K, (uint32_t)((long long)gy * f.W + gx),
                                  f.field_id, sg, pmin, pmax, psad);
      if (!SADDLE && f.boundary == 1 && k < 4) pmin = pmax = 0.f;
    } else if (MODEL == kUniform) {
      UniParams cp{sm[l], sm[HALO + l]}, nb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) nb[i] = UniParams{sm[nl[i]], sm[HALO + nl[i]]};
      if constexpr (!SADDLE) {
        if (!(f.boundary == 1 && k < 4)) uniform_vertex(cp, nb, present, f.cptypes, pmin, pmax);
      } else if (has_saddle) {
        psad = uniform_mixed(cp, nb, sg) + uniform_mixed(cp, nb, sg2);
      }
    } else if (MODEL == kGauss) {
      GaussParams cp{sm[l], sm[HALO + l]}, nb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) nb[i] = GaussParams{sm[nl[i]], sm[HALO + nl[i]]};
      if constexpr (!SADDLE) {
        if (!(f.boundary == 1 && k < 4)) gauss_vertex(cp, nb, present, pmin, pmax);
      } else if (has_saddle) {
        psad = gauss_saddle(cp, nb, present, sg);
      }
    } else if (MODEL == kEpan) {
      EpanParams cp{sm[l], sm[HALO + l]}, nb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) nb[i] = EpanParams{sm[nl[i]], sm[HALO + nl[i]]};
      if constexpr (!SADDLE) {
        if (!(f.boundary == 1 && k < 4)) epan_vertex(cp, nb, present, f.cptypes, pmin, pmax);
      } else if (has_saddle) {
        psad = epan_mixed(cp, nb, sg) + epan_mixed(cp, nb, sg2);
      }
    } else {
      const int B = f.B;
      const float lo1 = sm[l], hi1 = sm[HALO + l];
      const bool do_mm = !SADDLE && !(f.boundary == 1 && k < 4);
      const bool do_sad = SADDLE && has_saddle;
      if (lo1 == hi1) {
        float gm = Tc, gM = Tc, t1 = Tc, t2 = Tc;
        for (int i = 0; i < 4; ++i) {
          if (!present[i]) continue;
          float gt, lt;
          if constexpr (ROWS)
            hist_tails_at_rows(R4 + nl[i], RS, B, sm[nl[i]], sm[HALO + nl[i]], T[i], lo1, gt, lt);
          else
            hist_tails_at(sm + 2 * HALO + nl[i], HALO, B, sm[nl[i]], sm[HALO + nl[i]], T[i], lo1,
                          gt, lt);
          gm *= gt;
          gM *= lt;
          if (sg[i] != 0) {
            t1 *= sg[i] > 0 ? gt : lt;
            t2 *= sg[i] > 0 ? lt : gt;
          }
        }
        if (do_mm) {
          pmin = gm;
          pmax = gM;
        }
        if (do_sad) psad = t1 + t2;
      } else if ((do_mm || do_sad) && ROWS) {
        HistRowWalker nw[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          HistRowWalker &h = nw[i];
          if (!present[i]) {
            h.init_absent();
            continue;
          }
          const float lo = sm[nl[i]], hi = sm[HALO + nl[i]];
          h.init(R4 + nl[i], lo - lo1, T[i]);
          // the bin width only estimates how many edges lie below 0 (seek0
          // checks the estimate against the edges of the rows), so it need
          // not be the rows' own (hi - lo) / B
          h.seek0<RS>(R4 + nl[i], B, lo == hi ? 0.f : (hi - lo) * (1.f / (float)B));
        }
        if constexpr (!SADDLE) {
          hist_walk_rows<RS>(R4 + l, B, hi1 - lo1, nw, pmin, pmax);
        } else {
          float t1, t2;
          hist_walk_rows<RS, true>(R4 + l, B, hi1 - lo1, nw, t1, t2, sg);
          psad = t1 + t2;
        }
      } else if ((do_mm || do_sad) && !ROWS) {
        const float *S0 = sm + 2 * HALO;
        HistSeg nw[4];
        float Tw[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          HistSeg &h = nw[i];
          if (!present[i]) {
            h.init_absent(l, (float)B);
            Tw[i] = 2.f;  // CDF complement 2 - 1 = 1 for an absent neighbour
            continue;
          }
          Tw[i] = T[i];
          const float lo = sm[nl[i]], hi = sm[HALO + nl[i]];
          h.init<HALO>(S0, nl[i], lo - lo1, lo == hi ? 0.f : (hi - lo) / (float)B, T[i]);
          h.seek0<HALO>(S0, B);  // to the segment that contains x = 0
        }
        if constexpr (!SADDLE) {
          hist_walk<HALO>(S0, l, B, hi1 - lo1, nw, Tw, f.cptypes, pmin, pmax);
        } else {
          float t1, t2;
          hist_walk<HALO, true>(S0, l, B, hi1 - lo1, nw, Tw, 0u, t1, t2, sg);
          psad = t1 + t2;
        }
      }
    }
    const long long gi = (long long)gy * f.W + gx;
    if constexpr (SADDLE) {
      if (f.out_saddle) f.out_saddle[gi] = psad;
    } else {
      if ((f.cptypes & kMin) && f.out_min) f.out_min[gi] = pmin;
      if ((f.cptypes & kMax) && f.out_max) f.out_max[gi] = pmax;
    }
    if (f.status) f.status[gi] = st;
  }
}

}  // namespace ucp
