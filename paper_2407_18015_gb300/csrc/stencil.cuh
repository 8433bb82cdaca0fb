// stencil.cuh -- minimum / maximum probabilities with larger neighbour sets:
// the six-neighbour stencil of a triangulated 2D grid, the eight-neighbour
// stencil, and the six axis neighbours of a 3D grid (the extension named in
// the paper's Sec. "Conclusion").  The integrals are those of Eq.
// localMinimumProb with K <= 8 neighbour factors instead of 4; the piece
// integration is the same as in device.cuh, generalised over K.
#pragma once

#include "device.cuh"

namespace ucp {

constexpr int kStencil4 = 0, kStencil6 = 1, kStencil8 = 2, kStencil3D6 = 3;
constexpr int kMaxK = 8;

__host__ __device__ constexpr int stencil_k(int st) {
  return st == kStencil8 ? 8 : (st == kStencil4 ? 4 : 6);
}

// neighbour offsets (dz, dy, dx) of each stencil, the axis ones (e, n, w, s)
// first; stencil 6 adds ne and sw (every cell cut along its lower-left to
// upper-right diagonal), stencil 8 all four diagonals, the 3D one the
// neighbours below (z - 1) and above (z + 1)
__device__ __constant__ const int kStencilOff[4][kMaxK][3] = {
    {{0, 0, 1}, {0, -1, 0}, {0, 0, -1}, {0, 1, 0}},
    {{0, 0, 1}, {0, -1, 0}, {0, 0, -1}, {0, 1, 0}, {0, -1, 1}, {0, 1, -1}},
    {{0, 0, 1}, {0, -1, 0}, {0, 0, -1}, {0, 1, 0}, {0, -1, 1}, {0, -1, -1}, {0, 1, -1},
     {0, 1, 1}},
    {{0, 0, 1}, {0, -1, 0}, {0, 0, -1}, {0, 1, 0}, {-1, 0, 0}, {1, 0, 0}}};

// integral over [0,1] of (1-t)^(K-j) t^j = 1 / ((K+1) C(K,j))
__host__ __device__ constexpr float bern_w(int K, int j) {
  return 1.0f / float((K + 1) * binom(K, j));
}

// exact mean over [0,1] of a product of K linear factors given by their end
// values (the Bernstein form of bern_mean, for K <= 8)
template <int K>
__device__ __forceinline__ float bern_mean_k(const float *L, const float *R) {
  float e[K + 1];
  e[0] = L[0];
  e[1] = R[0];
#pragma unroll
  for (int i = 1; i < K; ++i) {
    e[i + 1] = e[i] * R[i];
#pragma unroll
    for (int j = i; j >= 1; --j) e[j] = fmaf(e[j - 1], R[i], e[j] * L[i]);
    e[0] = e[0] * L[i];
  }
  float s = 0.f;
#pragma unroll
  for (int j = 0; j <= K; ++j) s = fmaf(e[j], bern_w(K, j), s);
  return s;
}

// bern_mean_k of two products at once, one per half of a float2 (the same
// operations per half, packed FP32 instructions)
template <int K>
__device__ __forceinline__ float2 bern_mean_k_x2(const float2 *L, const float2 *R) {
  float2 e[K + 1];
  e[0] = L[0];
  e[1] = R[0];
#pragma unroll
  for (int i = 1; i < K; ++i) {
    e[i + 1] = __fmul2_rn(e[i], R[i]);
#pragma unroll
    for (int j = i; j >= 1; --j) e[j] = __ffma2_rn(e[j - 1], R[i], __fmul2_rn(e[j], L[i]));
    e[0] = __fmul2_rn(e[0], L[i]);
  }
  float2 s = make_float2(0.f, 0.f);
#pragma unroll
  for (int j = 0; j <= K; ++j) s = __ffma2_rn(e[j], make_float2(bern_w(K, j), bern_w(K, j)), s);
  return s;
}

// ascending sort of K keys with NP payload rows (odd-even transposition)
template <int NP>
__device__ __forceinline__ void cswap_k(float *k, float (*p)[kMaxK], int a, int b) {
  const bool sw = k[b] < k[a];
  const float ka = k[a], kb = k[b];
  k[a] = sw ? kb : ka;
  k[b] = sw ? ka : kb;
#pragma unroll
  for (int q = 0; q < NP; ++q) {
    const float pa = p[q][a], pb = p[q][b];
    p[q][a] = sw ? pb : pa;
    p[q][b] = sw ? pa : pb;
  }
}
template <int K, int NP>
__device__ __forceinline__ void sort_k(float *k, float (*p)[kMaxK]) {
#pragma unroll
  for (int r = 0; r < K; ++r)
#pragma unroll
    for (int i = r & 1; i + 1 < K; i += 2) cswap_k<NP>(k, p, i, i + 1);
}

// ---------------------------------------------------------------------------
// uniform

// piece J of uniform_side_k: [x[J], x[J+1]], on which the sorted factors
// 0..J-1 have started
template <int J, int K>
__device__ __forceinline__ void uni_pieces(const float *x, const float (*pay)[kMaxK], float *Lv,
                                           float *Rv, Kahan &acc) {
  const float x0 = x[J], x1 = x[J + 1];
#pragma unroll
  for (int i = 0; i < J - 1; ++i) Lv[i] = Rv[i];
  Lv[J - 1] = fmaxf(fmaf(-(x0 - pay[0][J - 1]), pay[1][J - 1], 1.f), 0.f);
#pragma unroll
  for (int i = 0; i < J; ++i) Rv[i] = fmaxf(fmaf(-(x1 - pay[0][i]), pay[1][i], 1.f), 0.f);
  acc.add((x1 - x0) * bern_mean_k<J>(Lv, Rv));
  if constexpr (J < K) uni_pieces<J + 1, K>(x, pay, Lv, Rv, acc);
}

// uniform_side with K factors: int_0^R (1/W1) prod_i (1 - max(0, x - al_i) sl_i)
template <int K>
__device__ __forceinline__ float uniform_side_k(float W1, float R, const float *al,
                                                const float *sl) {
  if (!(R > 0.f)) return 0.f;
  float t[kMaxK], pay[2][kMaxK];
#pragma unroll
  for (int i = 0; i < K; ++i) {
    t[i] = fminf(fmaxf(al[i], 0.f), R);
    pay[0][i] = al[i];
    pay[1][i] = sl[i];
  }
  sort_k<K, 2>(t, pay);
  float x[K + 2];
  x[0] = 0.f;
#pragma unroll
  for (int i = 0; i < K; ++i) x[i + 1] = t[i];
  x[K + 1] = R;
  Kahan acc;
  acc.add(x[1]);  // piece 0: no factor has started
  float Lv[K], Rv[K];
  uni_pieces<1, K>(x, pay, Lv, Rv, acc);
  return acc.get() * frcp(W1);
}

// P_min and P_max of a uniform centre with K neighbours (present[i])
template <int K>
__device__ __forceinline__ void uniform_vertex_k(UniParams c, const UniParams *nb,
                                                 const bool *present, unsigned want,
                                                 float &pmin, float &pmax) {
  if (c.a == c.b) {
    const float v = c.a;
    float gm = 1.f, gM = 1.f;
#pragma unroll
    for (int i = 0; i < K; ++i) {
      if (!present[i]) continue;
      const float a = nb[i].a, b = nb[i].b;
      float gt, lt;
      if (a == b) {
        gt = a > v ? 1.f : 0.f;
        lt = a < v ? 1.f : 0.f;
      } else {
        const float r = 1.f / (b - a);
        gt = fminf(fmaxf((b - v) * r, 0.f), 1.f);
        lt = fminf(fmaxf((v - a) * r, 0.f), 1.f);
      }
      gm *= gt;
      gM *= lt;
    }
    pmin = gm;
    pmax = gM;
    return;
  }
  const float W1 = c.b - c.a;
  float sl[K];
#pragma unroll
  for (int i = 0; i < K; ++i)
    sl[i] = (present[i] && nb[i].a != nb[i].b) ? frcp(nb[i].b - nb[i].a) : 0.f;
  if (want & kMin) {
    float al[K], R = W1;
#pragma unroll
    for (int i = 0; i < K; ++i) {
      if (present[i]) {
        al[i] = nb[i].a - c.a;
        R = fminf(R, nb[i].b - c.a);
      } else {
        al[i] = kFar;
      }
    }
    pmin = uniform_side_k<K>(W1, R, al, sl);
  }
  if (want & kMax) {
    // negated variables: -X has support [-b, -a]; origin at -b1
    float al[K], R = W1;
#pragma unroll
    for (int i = 0; i < K; ++i) {
      if (present[i]) {
        al[i] = c.b - nb[i].b;
        R = fminf(R, c.b - nb[i].a);
      } else {
        al[i] = kFar;
      }
    }
    pmax = uniform_side_k<K>(W1, R, al, sl);
  }
}

// ---------------------------------------------------------------------------
// Epanechnikov: with K neighbours the integrand has degree <= 2 + 3K = 26 on
// a piece; each piece takes the smallest rule of {2, 3, 5, 6, 8, 16} nodes
// that is exact for its degree (the 16-point rule: to degree 31)

// Node / weight q (ascending) of the NG-point Gauss-Legendre rule, NG in
// {2, 3, 5, 6, 8, 16}.
template <int NG>
__device__ __forceinline__ float sgl_x(int q) {
  if constexpr (NG == 16) return q < 8 ? -kGL16x[7 - q] : kGL16x[q - 8];
  else return gl_x<NG>(q);
}
template <int NG>
__device__ __forceinline__ float sgl_w(int q) {
  if constexpr (NG == 16) return q < 8 ? kGL16w[7 - q] : kGL16w[q - 8];
  else return gl_w<NG>(q);
}

// Piece J of epan_side_k: the centre density (degree 2) times the J started
// survivals (degree 3 each), degree 2 + 3J; the n-point rule with 2n - 1 >=
// 2 + 3J is exact: n = 2, 3, 5, 6, 8, then 16 (J = 5..8 need 9..14).
template <int J>
struct StencilNodes {
  static constexpr int value = J <= 4 ? EpanNodes<J>::value : 16;
};
template <int J, int K>
__device__ __forceinline__ void epan_pieces_k(const float *x, const float (*pay)[kMaxK], float iw1,
                                              float c1, Kahan &acc) {
  constexpr int NG = StencilNodes<J>::value;
  const float x0 = x[J], x1 = x[J + 1];
  const float half = 0.5f * (x1 - x0), mid = 0.5f * (x0 + x1);
  // nodes in pairs, one per half of a float2 (packed FP32 instructions)
  const float2 one2 = make_float2(1.f, 1.f);
  float2 s2 = make_float2(0.f, 0.f);
#pragma unroll
  for (int q = 0; q + 1 < NG; q += 2) {
    const float2 xx = __ffma2_rn(make_float2(half, half),
                                 make_float2(sgl_x<NG>(q), sgl_x<NG>(q + 1)), make_float2(mid, mid));
    const float2 u1 = __fmul2_rn(xx, make_float2(iw1, iw1));
    const float2 g = __ffma2_rn(make_float2(-u1.x, -u1.y), u1, one2);
    float2 f = __fmul2_rn(make_float2(c1, c1), make_float2(fmaxf(g.x, 0.f), fmaxf(g.y, 0.f)));
#pragma unroll
    for (int i = 0; i < J; ++i) {
      // the started factors' arguments lie in [-1, 1] on this piece (as in
      // epan_pieces): epan_surv without its clamp
      const float2 u = __fmul2_rn(__fadd2_rn(xx, make_float2(-pay[0][i], -pay[0][i])),
                                  make_float2(pay[1][i], pay[1][i]));
      const float2 qq = __fadd2_rn(one2, make_float2(-u.x, -u.y));
      const float2 sv = __fmul2_rn(__fmul2_rn(make_float2(0.25f, 0.25f), __fmul2_rn(qq, qq)),
                                   __fadd2_rn(make_float2(2.f, 2.f), u));
      f = __fmul2_rn(f, sv);
    }
    s2 = __ffma2_rn(make_float2(sgl_w<NG>(q), sgl_w<NG>(q + 1)), f, s2);
  }
  float sum = s2.x + s2.y;
  if constexpr (NG & 1) {
    constexpr int q = NG - 1;
    const float xx = fmaf(half, sgl_x<NG>(q), mid);
    const float u1 = xx * iw1;
    float f = c1 * fmaxf(fmaf(-u1, u1, 1.f), 0.f);
#pragma unroll
    for (int i = 0; i < J; ++i) f *= epan_surv((xx - pay[0][i]) * pay[1][i]);
    sum = fmaf(sgl_w<NG>(q), f, sum);
  }
  acc.add(sum * half);
  if constexpr (J < K) epan_pieces_k<J + 1, K>(x, pay, iw1, c1, acc);
}

// epan_side with K factors (same frame and arguments)
template <int K>
__device__ __forceinline__ float epan_side_k(float w1, float L, float R, const float *al,
                                             const float *d, const float *iw) {
  if (!(R > L)) return 0.f;
  float t[kMaxK], pay[2][kMaxK];
#pragma unroll
  for (int i = 0; i < K; ++i) {
    t[i] = fminf(fmaxf(al[i], L), R);
    pay[0][i] = d[i];
    pay[1][i] = iw[i];
  }
  sort_k<K, 2>(t, pay);
  float x[K + 2];
  x[0] = L;
#pragma unroll
  for (int i = 0; i < K; ++i) x[i + 1] = t[i];
  x[K + 1] = R;
  const float iw1 = frcp(w1);
  const float c1 = 0.75f * iw1;
  Kahan acc;
  epan_pieces_k<0, K>(x, pay, iw1, c1, acc);
  return acc.get();
}

template <int K>
__device__ __forceinline__ void epan_vertex_k(EpanParams c, const EpanParams *nb,
                                              const bool *present, unsigned want, float &pmin,
                                              float &pmax) {
  if (c.w == 0.f) {
    const float v = c.m;
    float gm = 1.f, gM = 1.f;
#pragma unroll
    for (int i = 0; i < K; ++i) {
      if (!present[i]) continue;
      float gt, lt;
      if (nb[i].w == 0.f) {
        gt = nb[i].m > v ? 1.f : 0.f;
        lt = nb[i].m < v ? 1.f : 0.f;
      } else {
        gt = epan_surv((v - nb[i].m) / nb[i].w);
        lt = epan_surv((nb[i].m - v) / nb[i].w);
      }
      gm *= gt;
      gM *= lt;
    }
    pmin = gm;
    pmax = gM;
    return;
  }
  const float w1 = c.w;
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    if (!(want & (side == 0 ? kMin : kMax))) continue;
    // side 1: the negated variables, frame of -m1: d = m1 - m_n
    float al[K], d[K], iw[K], R = w1;
#pragma unroll
    for (int i = 0; i < K; ++i) {
      al[i] = kFar; d[i] = kFar; iw[i] = 0.f;
      if (!present[i]) continue;
      const float dn = side == 0 ? nb[i].m - c.m : c.m - nb[i].m, wn = nb[i].w;
      if (wn == 0.f) {  // point mass: survival 1 below it, and it caps R
        R = fminf(R, dn);
      } else {
        al[i] = dn - wn; d[i] = dn; iw[i] = frcp(wn);
        R = fminf(R, dn + wn);
      }
    }
    const float p = epan_side_k<K>(w1, -w1, R, al, d, iw);
    if (side == 0) pmin = p; else pmax = p;
  }
}

// ---------------------------------------------------------------------------
// histogram: tail tables in global memory, one row of R = B + 4 floats per
// vertex: S_0..S_{B+1} (S_k = T - (m_0 + ... + m_{k-1}), S_B = S_{B+1} = 0,
// all 0 for a point mass), the total mass T, the status bits

__host__ __device__ constexpr int hist_table_row(int B) { return B + 4; }

// HistSeg over a global tail-table row (see HistSeg in device.cuh): the
// read at the next crossing is at tab[addr]; a walker crosses at most B + 1
// edges, so addr stays within its row
struct HistSegG {
  long long addr;
  float kf, lam, h, invh;
  float el, nx, s, sn, sl;
  __device__ __forceinline__ void init_absent(long long a, float Bf) {
    addr = a; kf = Bf + 1.f; lam = h = invh = 0.f;
    el = -kFar; nx = kFar; s = sn = 1.f; sl = 0.f;
  }
  __device__ __forceinline__ void init(const float *tab, long long row, float lam_, float h_,
                                       float T) {
    addr = row + 1; kf = 0.f;
    lam = lam_; h = h_; invh = h_ > 0.f ? frcp(h_) : 0.f;
    el = -kFar; nx = lam_; s = T; sn = __ldg(tab + row); sl = 0.f;
  }
  __device__ __forceinline__ bool step(const float *tab, float x1, float Bf) {
    const bool c = nx <= x1;
    const float t = __ldg(tab + addr);
    s = c ? sn : s;
    sn = c ? t : sn;
    addr += c ? 1 : 0;
    sl = (s - sn) * invh;
    el = c ? x1 : el;
    kf = c ? kf + 1.f : kf;
    nx = c ? (kf <= Bf ? fmaf(kf, h, lam) : kFar) : nx;
    return c;
  }
  __device__ __forceinline__ float G(float x) const { return fmaf(-sl, x - el, s); }
};

// hist_walk with K neighbours (centre row crow of the tail table)
template <int K>
__device__ __forceinline__ void hist_walk_k(const float *tab, long long crow, int B, float W1,
                                            HistSegG *nw, const float *T, unsigned want,
                                            float &pmin, float &pmax) {
  if (!(W1 <= 1e38f)) {
    pmin = pmax = __int_as_float(0x7fc00000);
    return;
  }
  const float Bf = (float)B;
  const float h1 = W1 / Bf, ih1 = frcp(h1);
  long long addr_c = crow + 2;
  float kcf = 1.f;
  float sc = __ldg(tab + crow), scn = __ldg(tab + crow + 1);
  float dens = (sc - scn) * ih1;
  float nxc = B > 1 ? h1 : W1;
  // (G, F) of each factor at the piece's left and right ends
  float2 Pl[K];
#pragma unroll
  for (int i = 0; i < K; ++i) {
    const float g = nw[i].G(0.f);
    Pl[i] = make_float2(g, T[i] - g);
  }
  float2 acc = make_float2(0.f, 0.f);
  (void)want;
  float x0 = 0.f;
  const int max_steps = (K + 1) * (B + 2) + 4;
  for (int step = 0; step < max_steps && x0 < W1; ++step) {
    float x1 = nxc;
#pragma unroll
    for (int i = 0; i < K; ++i) x1 = fminf(x1, nw[i].nx);
    x1 = fmaxf(x1, x0);
    float2 Pr[K];
#pragma unroll
    for (int i = 0; i < K; ++i) {
      const float g = nw[i].G(x1);
      Pr[i] = make_float2(g, T[i] - g);
    }
    const float wgt = (x1 - x0) * dens;
    acc = __ffma2_rn(make_float2(wgt, wgt), bern_mean_k_x2<K>(Pl, Pr), acc);
#pragma unroll
    for (int i = 0; i < K; ++i) {
      const bool c = nw[i].step(tab, x1, Bf);
      const float g = c ? nw[i].s : Pr[i].x;
      Pl[i] = make_float2(g, T[i] - g);
    }
    {
      const bool c = nxc <= x1;
      const float t = __ldg(tab + addr_c);
      sc = c ? scn : sc;
      scn = c ? t : scn;
      addr_c += c ? 1 : 0;
      kcf = c ? kcf + 1.f : kcf;
      nxc = c ? (kcf < Bf ? kcf * h1 : (kcf == Bf ? W1 : kFar)) : nxc;
      dens = (sc - scn) * ih1;
    }
    x0 = x1;
  }
  pmin = fmaxf(acc.x, 0.f);
  pmax = fmaxf(acc.y, 0.f);
}

// survival and CDF of a histogram neighbour (tail-table row) at a point v
__device__ __forceinline__ void hist_tails_row(const float *tab, long long row, int B, float lo,
                                               float hi, float T, float v, float &gt,
                                               float &lt) {
  if (lo == hi) {
    gt = lo > v ? T : 0.f;
    lt = lo < v ? T : 0.f;
    return;
  }
  if (v <= lo) {
    gt = T; lt = 0.f;
    return;
  }
  if (v >= hi) {
    gt = 0.f; lt = T;
    return;
  }
  const float h = (hi - lo) / (float)B;
  const int j = min(max((int)floorf((v - lo) / h), 0), B - 1);
  const float fr = fminf(fmaxf((v - lo - (float)j * h) / h, 0.f), 1.f);
  const float sj = __ldg(tab + row + j), sj1 = __ldg(tab + row + j + 1);
  gt = fmaxf(fmaf(-fr, sj - sj1, sj), 0.f);
  lt = fmaxf(T - gt, 0.f);
}

}  // namespace ucp
