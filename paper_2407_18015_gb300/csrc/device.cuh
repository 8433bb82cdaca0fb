// device.cuh -- per-vertex device routines of libucp (sm_103a).
//
// Critical-point probabilities of a vertex with value X_1 and in-grid axis
// neighbours X_n (arXiv 2407.18015, Eq. localMinimumProb and the negation
// rule for maxima):
//   P_min = int pdf_1(x) prod_n G_n(x) dx,   P_max = int pdf_1(x) prod_n F_n(x) dx.
// On every piece between consecutive support starts (Task 1 of the paper's
// algorithm) each factor is one polynomial, so each piece integral is exact:
//   - uniform / histogram: pdf_1 is constant and every G_n is linear on a
//     piece, so the integral of the product is the Bernstein mean of its end
//     values (no quadrature, all terms non-negative, no cancellation);
//   - Epanechnikov: pdf_1 quadratic, G_n cubic, degree <= 14 on a piece,
//     integrated exactly by 8-point Gauss-Legendre (exact to degree 15).
// All arithmetic is FP32 in a vertex-local frame (the centre's lower support
// end or mean is the origin), pieces are summed with Kahan compensation.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace ucp {

constexpr int kUniform = 0, kEpan = 1, kHist = 2, kMvn = 3, kSemi = 4, kGauss = 5;

// histogram parameters (lo, hi, masses): the closed form and the estimator
__host__ __device__ constexpr bool hist_params(int model) { return model == kHist || model == kSemi; }
constexpr unsigned kMin = 1u, kMax = 2u, kSaddle = 4u;
constexpr int kMaxBins = 64;

enum : uint8_t {
  V_DEGENERATE = 1,
  V_NONFINITE = 2,
  V_BAD = 4,
  V_JITTER = 8,
  V_CHOLFAIL = 16,
  V_TIMEOUT = 32
};

// Neighbour directions e, n, w, s (same order as the MVN variable slots 1..4).
__device__ __constant__ const int kDy[4] = {0, -1, 0, 1};
__device__ __constant__ const int kDx[4] = {1, 0, -1, 0};

constexpr float kFar = 3.0e38f;  // "never starts" breakpoint (finite: 0*kFar = 0)

// ---------------------------------------------------------------------------
// small helpers

// Reciprocal of a positive, finite, normal width (2 ulp; no IEEE division
// sequence): support widths and bin widths only.
__device__ __forceinline__ float frcp(float x) { return __fdividef(1.0f, x); }

// NaN-propagating minimum / maximum (a NaN input gives NaN; otherwise the
// same value as fminf / fmaxf): a running min and max over members then
// flag a non-finite member by themselves (NaN: both NaN; +Inf: the max;
// -Inf: the min).
__device__ __forceinline__ float fmin_nan(float a, float b) {
  float r;
  asm("min.NaN.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ float fmax_nan(float a, float b) {
  float r;
  asm("max.NaN.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ float fmin3_nan(float a, float b, float c) {
  float r;
  asm("min.NaN.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}
__device__ __forceinline__ float fmax3_nan(float a, float b, float c) {
  float r;
  asm("max.NaN.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}

// Compensated (Kahan) summation: the running rounding error c is fed back
// into the next addend.
struct Kahan {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ float get() const { return s; }
};

__host__ __device__ constexpr int binom(int n, int k) {
  int r = 1;
  for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
  return r;
}

// integral over [0,1] of (1-t)^(K-j) t^j = 1 / ((K+1) C(K,j)), as a table
// built at compile time (index [K][j], K <= 4)
struct BernTable {
  float w[5][5];
  constexpr BernTable() : w{} {
    for (int K = 0; K <= 4; ++K)
      for (int j = 0; j <= K; ++j) w[K][j] = 1.0f / float((K + 1) * binom(K, j));
  }
};
constexpr BernTable kBern{};
template <int K, int J>
struct BernW {
  static constexpr float value = kBern.w[K][J];
};

// integral over tau in [0,1] of prod_{i<K} (L[i] (1-tau) + R[i] tau):
// the product in the Bernstein basis of degree K (coefficients e_j = sums of
// products of j right values and K-j left values), then its exact mean.
template <int K>
__device__ __forceinline__ float bern_mean(const float *L, const float *R) {
  if constexpr (K == 0) {
    return 1.0f;
  } else {
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
    // weights 1/((K+1) C(K,j)) are symmetric in j
    float s;
    if constexpr (K == 1) {
      s = 0.5f * (e[0] + e[1]);
    } else if constexpr (K == 2) {
      s = fmaf(e[0] + e[2], BernW<2, 0>::value, e[1] * BernW<2, 1>::value);
    } else if constexpr (K == 3) {
      s = fmaf(e[0] + e[3], BernW<3, 0>::value, (e[1] + e[2]) * BernW<3, 1>::value);
    } else {
      s = fmaf(e[0] + e[4], BernW<4, 0>::value,
               fmaf(e[1] + e[3], BernW<4, 1>::value, e[2] * BernW<4, 2>::value));
    }
    return s;
  }
}

// bern_mean<4> of two products at once, one in each half of a float2, with
// the packed FP32 instructions (each half rounds exactly as the scalar form)
__device__ __forceinline__ float2 bern_mean4_x2(const float2 *L, const float2 *R) {
  float2 e0 = L[0], e1 = R[0], e2, e3, e4;
  e2 = __fmul2_rn(e1, R[1]);
  e1 = __ffma2_rn(e0, R[1], __fmul2_rn(e1, L[1]));
  e0 = __fmul2_rn(e0, L[1]);
  e3 = __fmul2_rn(e2, R[2]);
  e2 = __ffma2_rn(e1, R[2], __fmul2_rn(e2, L[2]));
  e1 = __ffma2_rn(e0, R[2], __fmul2_rn(e1, L[2]));
  e0 = __fmul2_rn(e0, L[2]);
  e4 = __fmul2_rn(e3, R[3]);
  e3 = __ffma2_rn(e2, R[3], __fmul2_rn(e3, L[3]));
  e2 = __ffma2_rn(e1, R[3], __fmul2_rn(e2, L[3]));
  e1 = __ffma2_rn(e0, R[3], __fmul2_rn(e1, L[3]));
  e0 = __fmul2_rn(e0, L[3]);
  const float2 w0 = make_float2(BernW<4, 0>::value, BernW<4, 0>::value);
  const float2 w1 = make_float2(BernW<4, 1>::value, BernW<4, 1>::value);
  const float2 w2 = make_float2(BernW<4, 2>::value, BernW<4, 2>::value);
  return __ffma2_rn(__fadd2_rn(e0, e4), w0,
                    __ffma2_rn(__fadd2_rn(e1, e3), w1, __fmul2_rn(e2, w2)));
}

// bern_mean<4> of two products at once, from the factors taken in two pairs:
// with b0 = L0 L1, b2 = R0 R1, b1 = L0 R1 + R0 L1 (the pair's quadratic in
// the Bernstein basis, middle coefficient doubled) and c0, c1, c2 likewise
// for factors 2 and 3, the integral of the product of the two quadratics is
//   (b0 c0 + b2 c2) / 5 + ((b0 + b2) c1 + b1 (c0 + c2)) / 20
//   + (b0 c2 + b2 c0 + b1 c1) / 30,
// the same value as bern_mean4_x2 in exact arithmetic (every term a product
// of non-negative end values) with fewer operations.
__device__ __forceinline__ float2 bern_mean4_pairs_x2(const float2 *L, const float2 *R) {
  const float2 b0 = __fmul2_rn(L[0], L[1]), b2 = __fmul2_rn(R[0], R[1]);
  const float2 b1 = __ffma2_rn(L[0], R[1], __fmul2_rn(R[0], L[1]));
  const float2 c0 = __fmul2_rn(L[2], L[3]), c2 = __fmul2_rn(R[2], R[3]);
  const float2 c1 = __ffma2_rn(L[2], R[3], __fmul2_rn(R[2], L[3]));
  const float2 t1 = __ffma2_rn(b0, c0, __fmul2_rn(b2, c2));
  const float2 t2 = __ffma2_rn(__fadd2_rn(b0, b2), c1, __fmul2_rn(b1, __fadd2_rn(c0, c2)));
  const float2 t3 = __ffma2_rn(b0, c2, __ffma2_rn(b2, c0, __fmul2_rn(b1, c1)));
  return __ffma2_rn(make_float2(0.2f, 0.2f), t1,
                    __ffma2_rn(make_float2(0.05f, 0.05f), t2,
                               __fmul2_rn(make_float2(1.f / 30.f, 1.f / 30.f), t3)));
}

// bern_mean<K> (K <= 4) of two products at once, one per half of a float2
template <int K>
__device__ __forceinline__ float2 bern_mean_x2(const float2 *L, const float2 *R) {
  if constexpr (K == 4) {
    return bern_mean4_x2(L, R);
  } else {
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
    if constexpr (K == 1) {
      return __fmul2_rn(make_float2(0.5f, 0.5f), __fadd2_rn(e[0], e[1]));
    } else if constexpr (K == 2) {
      const float2 w0 = make_float2(BernW<2, 0>::value, BernW<2, 0>::value);
      const float2 w1 = make_float2(BernW<2, 1>::value, BernW<2, 1>::value);
      return __ffma2_rn(__fadd2_rn(e[0], e[2]), w0, __fmul2_rn(e[1], w1));
    } else {
      const float2 w0 = make_float2(BernW<3, 0>::value, BernW<3, 0>::value);
      const float2 w1 = make_float2(BernW<3, 1>::value, BernW<3, 1>::value);
      return __ffma2_rn(__fadd2_rn(e[0], e[3]), w0, __fmul2_rn(__fadd2_rn(e[1], e[2]), w1));
    }
  }
}

// Kahan summation of two sums at once
struct Kahan2 {
  float2 s = {0.f, 0.f}, c = {0.f, 0.f};
  __device__ __forceinline__ void add(float2 v) {
    const float2 y = __fadd2_rn(v, make_float2(-c.x, -c.y));
    const float2 t = __fadd2_rn(s, y);
    c = __fadd2_rn(__fadd2_rn(t, make_float2(-s.x, -s.y)), make_float2(-y.x, -y.y));
    s = t;
  }
};

// Sort four (key, payload...) tuples ascending by key with a 5-exchange network.
template <int NP>
__device__ __forceinline__ void cswap(float *k, float (*p)[4], int a, int b) {
  bool sw = k[b] < k[a];
  float ka = k[a], kb = k[b];
  k[a] = sw ? kb : ka;
  k[b] = sw ? ka : kb;
#pragma unroll
  for (int q = 0; q < NP; ++q) {
    float pa = p[q][a], pb = p[q][b];
    p[q][a] = sw ? pb : pa;
    p[q][b] = sw ? pa : pb;
  }
}
template <int NP>
__device__ __forceinline__ void sort4(float *k, float (*p)[4]) {
  cswap<NP>(k, p, 0, 1);
  cswap<NP>(k, p, 2, 3);
  cswap<NP>(k, p, 0, 2);
  cswap<NP>(k, p, 1, 3);
  cswap<NP>(k, p, 1, 2);
}

// ---------------------------------------------------------------------------
// fitting (the statistics pass)

// min / max over N members at stride `plane`; nonfinite set if any is NaN/Inf
__device__ __forceinline__ void members_minmax(const float *__restrict__ p, long long plane,
                                               int N, float &mn, float &mx, bool &nonfinite) {
  float a = p[0], b = p[0];
  bool nf = false;
  int k = 0;
  for (; k + 4 <= N; k += 4) {
    float v0 = __ldg(p + (long long)k * plane), v1 = __ldg(p + (long long)(k + 1) * plane);
    float v2 = __ldg(p + (long long)(k + 2) * plane), v3 = __ldg(p + (long long)(k + 3) * plane);
    nf |= !(isfinite(v0) && isfinite(v1) && isfinite(v2) && isfinite(v3));
    a = fminf(fminf(a, v0), fminf(v1, fminf(v2, v3)));
    b = fmaxf(fmaxf(b, v0), fmaxf(v1, fmaxf(v2, v3)));
  }
  for (; k < N; ++k) {
    float v = __ldg(p + (long long)k * plane);
    nf |= !isfinite(v);
    a = fminf(a, v);
    b = fmaxf(b, v);
  }
  mn = a;
  mx = b;
  nonfinite = nf;
}

// Epanechnikov fit: one pass, shifted by the first member, compensated sums
// of d = x - x_0 and d^2; m = x_0 + mean(d), var = (S2 - S1^2/N) / (N-1).
__device__ __forceinline__ void members_epan(const float *__restrict__ p, long long plane, int N,
                                             float scale, float &m, float &w, float &mn,
                                             float &mx, bool &nonfinite) {
  const float x0 = __ldg(p);
  Kahan s1, s2;
  float a = x0, b = x0;
  bool nf = false;
  for (int k = 0; k < N; ++k) {
    float v = __ldg(p + (long long)k * plane);
    nf |= !isfinite(v);
    a = fminf(a, v);
    b = fmaxf(b, v);
    float d = v - x0;
    s1.add(d);
    s2.add(d * d);
  }
  mn = a;
  mx = b;
  nonfinite = nf;
  if (a == b) {
    m = a;
    w = 0.f;
    return;
  }
  float S1 = s1.get(), S2 = s2.get();
  float md = S1 / (float)N;
  float var = fmaxf(S2 - S1 * md, 0.f) / (float)(N - 1);
  m = x0 + md;
  w = scale * sqrtf(var);
}

// histogram bin of x: floor((x - lo) * s), s = B / (hi - lo), one rounding per
// operation (no contraction), clamped to [0, B-1]
__device__ __forceinline__ int hist_bin(float x, float lo, float s, int B) {
  int i = (int)floorf(__fmul_rn(__fsub_rn(x, lo), s));
  return min(max(i, 0), B - 1);
}
// hist_bin for a finite member x >= lo (lo the members' minimum, s > 0):
// (x - lo) * s is then >= 0, so truncation is the floor and the lower clamp
// never acts -- the same bin as hist_bin
__device__ __forceinline__ int hist_bin_nonneg(float x, float lo, float s, int B) {
  return min(__float2int_rz(__fmul_rn(__fsub_rn(x, lo), s)), B - 1);
}

// ---------------------------------------------------------------------------
// closed-form integration, uniform model

// One-sided problem in a local frame: the centre is uniform on [0, W1]
// (W1 > 0), factor i is 1 - max(0, x - al[i]) * sl[i] (a neighbour survival
// that starts at al[i]; sl = 0 for absent or point-mass neighbours), the
// integration range is [0, R].  Returns int_0^R (1/W1) prod_i factor_i dx.
__device__ __forceinline__ float uniform_side(float W1, float R, float al[4], float sl[4]) {
  if (!(R > 0.f)) return 0.f;
  float t[4];
  float pay[2][4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    t[i] = fminf(fmaxf(al[i], 0.f), R);
    pay[0][i] = al[i];
    pay[1][i] = sl[i];
  }
  sort4<2>(t, pay);
  // breakpoints x_0 = 0 < t0 <= t1 <= t2 <= t3 <= x_5 = R; on piece j the
  // factors 0..j-1 (sorted) have started and the others are 1.
  float x[6] = {0.f, t[0], t[1], t[2], t[3], R};
  Kahan acc;
  acc.add(x[1]);  // piece 0: no factor has started
  float L[4], Rv[4];
#pragma unroll
  for (int j = 1; j <= 4; ++j) {
    const float x0 = x[j], x1 = x[j + 1];
    // left values: the previous piece's right values, plus the factor that
    // starts at x0 (1 there unless its start was clamped to 0)
#pragma unroll
    for (int i = 0; i < j - 1; ++i) L[i] = Rv[i];
    L[j - 1] = fmaxf(fmaf(-(x0 - pay[0][j - 1]), pay[1][j - 1], 1.f), 0.f);
#pragma unroll
    for (int i = 0; i < j; ++i) Rv[i] = fmaxf(fmaf(-(x1 - pay[0][i]), pay[1][i], 1.f), 0.f);
    float I;
    if (j == 1) I = bern_mean<1>(L, Rv);
    else if (j == 2) I = bern_mean<2>(L, Rv);
    else if (j == 3) I = bern_mean<3>(L, Rv);
    else I = bern_mean<4>(L, Rv);
    acc.add((x1 - x0) * I);
  }
  return acc.get() * frcp(W1);
}

// uniform_side for the minimum (.x) and the maximum (.y) problems at once:
// each half sorts its own breakpoints, then the pieces of both are integrated
// with packed FP32 instructions.  R <= 0 gives 0.
__device__ __forceinline__ float2 uniform_side2(float W1, float2 R, const float2 *al,
                                                const float *sl) {
  R = make_float2(fmaxf(R.x, 0.f), fmaxf(R.y, 0.f));
  float tx[4], ty[4], px[2][4], py[2][4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    tx[i] = fminf(fmaxf(al[i].x, 0.f), R.x);
    ty[i] = fminf(fmaxf(al[i].y, 0.f), R.y);
    px[0][i] = al[i].x; px[1][i] = sl[i];
    py[0][i] = al[i].y; py[1][i] = sl[i];
  }
  sort4<2>(tx, px);
  sort4<2>(ty, py);
  float2 x[6] = {make_float2(0.f, 0.f), make_float2(tx[0], ty[0]), make_float2(tx[1], ty[1]),
                 make_float2(tx[2], ty[2]), make_float2(tx[3], ty[3]), R};
  float2 a[4], sv[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    a[i] = make_float2(px[0][i], py[0][i]);
    sv[i] = make_float2(-px[1][i], -py[1][i]);
  }
  Kahan2 acc;
  acc.add(x[1]);  // piece 0: no factor has started
  float2 L[4], Rv[4];
  const float2 one2 = make_float2(1.f, 1.f);
  auto factor = [&](float2 xe, int i) {
    const float2 v = __ffma2_rn(__fadd2_rn(xe, make_float2(-a[i].x, -a[i].y)), sv[i], one2);
    return make_float2(fmaxf(v.x, 0.f), fmaxf(v.y, 0.f));
  };
#pragma unroll
  for (int j = 1; j <= 4; ++j) {
    const float2 x0 = x[j], x1 = x[j + 1];
#pragma unroll
    for (int i = 0; i < j - 1; ++i) L[i] = Rv[i];
    L[j - 1] = factor(x0, j - 1);
#pragma unroll
    for (int i = 0; i < j; ++i) Rv[i] = factor(x1, i);
    float2 I;
    if (j == 1) I = bern_mean_x2<1>(L, Rv);
    else if (j == 2) I = bern_mean_x2<2>(L, Rv);
    else if (j == 3) I = bern_mean_x2<3>(L, Rv);
    else I = bern_mean_x2<4>(L, Rv);
    acc.add(__fmul2_rn(__fadd2_rn(x1, make_float2(-x0.x, -x0.y)), I));
  }
  const float iw = frcp(W1);
  return make_float2(acc.s.x * iw, acc.s.y * iw);
}

struct UniParams {
  float a, b;
};

// P_min and P_max of a centre (a1,b1) with neighbours nb[0..3] (present[i]).
// Degenerate centre: products of strict tail probabilities.
__device__ __forceinline__ void uniform_vertex(UniParams c, const UniParams *nb,
                                               const bool *present, unsigned want, float &pmin,
                                               float &pmax) {
  if (c.a == c.b) {
    const float v = c.a;
    float gm = 1.f, gM = 1.f;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (!present[i]) continue;
      float a = nb[i].a, b = nb[i].b;
      float gt, lt;
      if (a == b) {
        gt = a > v ? 1.f : 0.f;
        lt = a < v ? 1.f : 0.f;
      } else {
        float r = 1.f / (b - a);
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
  float sl[4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
    sl[i] = (present[i] && nb[i].a != nb[i].b) ? frcp(nb[i].b - nb[i].a) : 0.f;
  if ((want & kMin) && (want & kMax)) {
    // both problems at once; maximum: negated variables, origin at -b1
    float2 al[4];
    float2 R = make_float2(W1, W1);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (present[i]) {
        al[i] = make_float2(nb[i].a - c.a, c.b - nb[i].b);
        R = make_float2(fminf(R.x, nb[i].b - c.a), fminf(R.y, c.b - nb[i].a));
      } else {
        al[i] = make_float2(kFar, kFar);
      }
    }
    const float2 p = uniform_side2(W1, R, al, sl);
    pmin = p.x;
    pmax = p.y;
    return;
  }
  if (want & kMin) {
    float al[4], s2[4], R = W1;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      s2[i] = sl[i];
      if (present[i]) {
        al[i] = nb[i].a - c.a;
        R = fminf(R, nb[i].b - c.a);
      } else {
        al[i] = kFar;
      }
    }
    pmin = uniform_side(W1, R, al, s2);
  }
  if (want & kMax) {
    // negated variables: -X has support [-b, -a]; origin at -b1
    float al[4], s2[4], R = W1;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      s2[i] = sl[i];
      if (present[i]) {
        al[i] = c.b - nb[i].b;
        R = fminf(R, c.b - nb[i].a);
      } else {
        al[i] = kFar;
      }
    }
    pmax = uniform_side(W1, R, al, s2);
  }
}

// ---------------------------------------------------------------------------
// closed-form integration, Epanechnikov model

// 8-point Gauss-Legendre rule on [-1, 1] (roots of P_8, weights
// 2 / ((1 - x^2) P_8'(x)^2)); exact for polynomials of degree <= 15.
__device__ __constant__ const float kGLx[4] = {0.18343464249564978f, 0.525532409916329f,
                                               0.7966664774136267f, 0.9602898564975362f};
__device__ __constant__ const float kGLw[4] = {0.36268378337836166f, 0.3137066458778869f,
                                               0.22238103445337443f, 0.10122853629037706f};

// Gauss-Legendre rules on [-1, 1] with 2, 3, 5 and 6 nodes (all nodes,
// ascending: the roots of P_n, weights 2 / ((1 - x^2) P_n'(x)^2)); the n-point
// rule is exact for polynomials of degree <= 2n - 1.
__device__ __constant__ const float kGL2x[2] = {-0.57735026918962573f, 0.57735026918962573f};
__device__ __constant__ const float kGL2w[2] = {1.f, 1.f};
__device__ __constant__ const float kGL3x[3] = {-0.7745966692414834f, 0.f, 0.7745966692414834f};
__device__ __constant__ const float kGL3w[3] = {0.55555555555555569f, 0.88888888888888884f,
                                                0.55555555555555569f};
__device__ __constant__ const float kGL5x[5] = {-0.90617984593866396f, -0.53846931010568311f, 0.f,
                                                0.53846931010568311f, 0.90617984593866396f};
__device__ __constant__ const float kGL5w[5] = {0.23692688505618928f, 0.4786286704993663f,
                                                0.56888888888888867f, 0.4786286704993663f,
                                                0.23692688505618928f};
__device__ __constant__ const float kGL6x[6] = {-0.93246951420315194f, -0.66120938646626448f,
                                                -0.2386191860831969f,  0.2386191860831969f,
                                                0.66120938646626448f,  0.93246951420315194f};
__device__ __constant__ const float kGL6w[6] = {0.17132449237917027f, 0.36076157304813872f,
                                                0.46791393457269104f, 0.46791393457269104f,
                                                0.36076157304813872f, 0.17132449237917027f};

// node / weight q (ascending) of the NG-point rule, NG in {2, 3, 5, 6, 8}
template <int NG>
__device__ __forceinline__ float gl_x(int q) {
  if constexpr (NG == 2) return kGL2x[q];
  else if constexpr (NG == 3) return kGL3x[q];
  else if constexpr (NG == 5) return kGL5x[q];
  else if constexpr (NG == 6) return kGL6x[q];
  else return q < 4 ? -kGLx[3 - q] : kGLx[q - 4];
}
template <int NG>
__device__ __forceinline__ float gl_w(int q) {
  if constexpr (NG == 2) return kGL2w[q];
  else if constexpr (NG == 3) return kGL3w[q];
  else if constexpr (NG == 5) return kGL5w[q];
  else if constexpr (NG == 6) return kGL6w[q];
  else return q < 4 ? kGLw[3 - q] : kGLw[q - 4];
}

// survival of the standard Epanechnikov kernel on [-1,1]: (1-u)^2 (2+u) / 4
__device__ __forceinline__ float epan_surv(float u) {
  u = fminf(fmaxf(u, -1.f), 1.f);
  const float q = 1.f - u;
  return 0.25f * q * q * (2.f + u);
}

// Piece J of epan_side: on [x[J], x[J+1]] the centre density (degree 2)
// times the J started survivals (degree 3 each) has degree 2 + 3J, so the
// n-point rule with 2n - 1 >= 2 + 3J is exact: n = 2, 3, 5, 6, 8.
template <int J>
struct EpanNodes {
  static constexpr int value = J == 0 ? 2 : (J == 1 ? 3 : (J == 2 ? 5 : (J == 3 ? 6 : 8)));
};
template <int J>
__device__ __forceinline__ void epan_pieces(const float *x, const float (*pay)[4], float iw1,
                                            float c1, Kahan &acc) {
  constexpr int NG = EpanNodes<J>::value;
  const float x0 = x[J], x1 = x[J + 1];
  const float half = 0.5f * (x1 - x0), mid = 0.5f * (x0 + x1);
  // nodes in pairs, one per half of a float2 (packed FP32 instructions)
  const float2 one2 = make_float2(1.f, 1.f);
  float2 s2 = make_float2(0.f, 0.f);
#pragma unroll
  for (int q = 0; q + 1 < NG; q += 2) {
    const float2 xx = __ffma2_rn(make_float2(half, half),
                                 make_float2(gl_x<NG>(q), gl_x<NG>(q + 1)), make_float2(mid, mid));
    const float2 u1 = __fmul2_rn(xx, make_float2(iw1, iw1));
    const float2 g = __ffma2_rn(make_float2(-u1.x, -u1.y), u1, one2);
    float2 f = __fmul2_rn(make_float2(c1, c1), make_float2(fmaxf(g.x, 0.f), fmaxf(g.y, 0.f)));
#pragma unroll
    for (int i = 0; i < J; ++i) {
      // epan_surv of both nodes, unclamped: on the piece where J factors
      // have started, each started factor's u lies in [-1, 1] (the piece
      // begins after the factor's start, and R is at most every present
      // neighbour's end); absent and point-mass factors start at R and so
      // only enter pieces of zero width
      const float2 u = __fmul2_rn(__fadd2_rn(xx, make_float2(-pay[0][i], -pay[0][i])),
                                  make_float2(pay[1][i], pay[1][i]));
      const float2 qq = __fadd2_rn(one2, make_float2(-u.x, -u.y));
      const float2 sv = __fmul2_rn(__fmul2_rn(make_float2(0.25f, 0.25f), __fmul2_rn(qq, qq)),
                                   __fadd2_rn(make_float2(2.f, 2.f), u));
      f = __fmul2_rn(f, sv);
    }
    s2 = __ffma2_rn(make_float2(gl_w<NG>(q), gl_w<NG>(q + 1)), f, s2);
  }
  float s = s2.x + s2.y;
  if constexpr (NG & 1) {
    constexpr int q = NG - 1;
    const float xx = fmaf(half, gl_x<NG>(q), mid);
    const float u1 = xx * iw1;
    float f = c1 * fmaxf(fmaf(-u1, u1, 1.f), 0.f);
#pragma unroll
    for (int i = 0; i < J; ++i) f *= epan_surv((xx - pay[0][i]) * pay[1][i]);
    s = fmaf(gl_w<NG>(q), f, s);
  }
  acc.add(s * half);
  if constexpr (J < 4) epan_pieces<J + 1>(x, pay, iw1, c1, acc);
}

// One-sided problem in the centre's frame (origin m1): centre pdf
// 3/(4 w1) (1 - (x/w1)^2) on [-w1, w1], factor i = epan_surv((x - d[i]) * iw[i])
// starting at al[i] = d[i] - 1/iw[i] (iw = 0, d = kFar for absent/point-mass
// neighbours).  Integrates over [L, R].
__device__ __forceinline__ float epan_side(float w1, float L, float R, float al[4], float d[4],
                                           float iw[4]) {
  if (!(R > L)) return 0.f;
  float t[4];
  float pay[2][4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    t[i] = fminf(fmaxf(al[i], L), R);
    pay[0][i] = d[i];
    pay[1][i] = iw[i];
  }
  sort4<2>(t, pay);
  const float x[6] = {L, t[0], t[1], t[2], t[3], R};
  const float iw1 = frcp(w1);
  const float c1 = 0.75f * iw1;
  Kahan acc;
  epan_pieces<0>(x, pay, iw1, c1, acc);
  return acc.get();
}

struct EpanParams {
  float m, w;
};

__device__ __forceinline__ void epan_vertex(EpanParams c, const EpanParams *nb,
                                            const bool *present, unsigned want, float &pmin,
                                            float &pmax) {
  if (c.w == 0.f) {
    const float v = c.m;
    float gm = 1.f, gM = 1.f;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
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
  if (want & kMin) {
    float al[4], d[4], iw[4], R = w1;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (present[i]) {
        const float dn = nb[i].m - c.m, wn = nb[i].w;
        if (wn == 0.f) {  // point mass: survival 1 below it, and it caps R
          al[i] = kFar; d[i] = kFar; iw[i] = 0.f;
          R = fminf(R, dn);
        } else {
          al[i] = dn - wn; d[i] = dn; iw[i] = frcp(wn);
          R = fminf(R, dn + wn);
        }
      } else {
        al[i] = kFar; d[i] = kFar; iw[i] = 0.f;
      }
    }
    pmin = epan_side(w1, -w1, R, al, d, iw);
  }
  if (want & kMax) {
    // negated variables: -X_n has mean -m_n; in the frame of -m1: d = m1 - m_n
    float al[4], d[4], iw[4], R = w1;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (present[i]) {
        const float dn = c.m - nb[i].m, wn = nb[i].w;
        if (wn == 0.f) {
          al[i] = kFar; d[i] = kFar; iw[i] = 0.f;
          R = fminf(R, dn);
        } else {
          al[i] = dn - wn; d[i] = dn; iw[i] = frcp(wn);
          R = fminf(R, dn + wn);
        }
      } else {
        al[i] = kFar; d[i] = kFar; iw[i] = 0.f;
      }
    }
    pmax = epan_side(w1, -w1, R, al, d, iw);
  }
}

// nodes (positive half, ascending) and weights of the 16-point rule on
// [-1, 1]: the roots of the Legendre polynomial P_16 and 2 / ((1 - x^2)
// P_16'(x)^2)
__device__ __constant__ const float kGL16x[8] = {
    0.095012509837637441f, 0.28160355077925892f, 0.45801677765722737f, 0.61787624440264377f,
    0.755404408355003f,    0.86563120238783176f, 0.9445750230732326f,  0.98940093499164994f};
__device__ __constant__ const float kGL16w[8] = {
    0.18945061045506864f, 0.18260341504492364f, 0.16915651939500265f, 0.14959598881657671f,
    0.12462897125553407f, 0.095158511682492605f, 0.062253523938647456f, 0.027152459411754176f};

// ---------------------------------------------------------------------------
// independent Gaussians (the parametric model the paper compares with by
// Monte Carlo, Sec. "Comparison of Parametric Vs. Nonparametric Models"):
// no finite support, so the one-dimensional integral
//   P = int phi(t) prod_n f_n(t) dt,  t = (x - m1) / s1,
// f_n = Q((t - a_n) / r_n) (survival) or Phi((t - a_n) / r_n) (CDF),
// a_n = (m_n - m1) / s1, r_n = s_n / s1, is evaluated by quadrature: the
// range |t| <= 8 (mass beyond it 1.2e-15) is cut at -3, 0, 3 and at every
// neighbour's a_n and a_n +- 8 r_n, and each piece takes the 16-point
// Gauss-Legendre rule (on such pieces the integrand is smooth and the rule
// converges to ~1e-15 in exact arithmetic).

struct GaussParams {
  float m, s;
};

constexpr float kGaussR = 8.f;
constexpr int kGaussBp = 5 + 3 * 4;

// 0.5 erfc(|z| / sqrt 2): the smaller of Q(z) and Phi(z), accurate in both
// tails; returns (Q(z), Phi(z))
__device__ __forceinline__ float2 gauss_tails(float z) {
  const float e = 0.5f * erfcf(fabsf(z) * 0.70710678118654752f);
  return z >= 0.f ? make_float2(e, 1.f - e) : make_float2(1.f - e, e);
}

// The minimum and maximum (SADDLE = false) or the saddle terms t1, t2
// (SADDLE = true, sg as in the mixed products) of a centre with sigma > 0.
template <bool SADDLE>
__device__ __forceinline__ float2 gauss_quad(GaussParams c, const GaussParams *nb,
                                             const bool *present, const int *sg) {
  float a[4], ir[4];
  bool step[4];
  float bp[kGaussBp];
  int nbp = 0;
  bp[nbp++] = -kGaussR; bp[nbp++] = -3.f; bp[nbp++] = 0.f; bp[nbp++] = 3.f; bp[nbp++] = kGaussR;
  const float is1 = 1.f / c.s;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const bool on = present[i] && (!SADDLE || sg[i] != 0);
    a[i] = on ? (nb[i].m - c.m) * is1 : 0.f;
    const float r = on ? nb[i].s * is1 : 0.f;
    step[i] = r == 0.f;
    ir[i] = step[i] ? 0.f : 1.f / r;
    const float lo = on ? fminf(fmaxf(a[i] - kGaussR * r, -kGaussR), kGaussR) : -kGaussR;
    const float mid = on ? fminf(fmaxf(a[i], -kGaussR), kGaussR) : -kGaussR;
    const float hi = on ? fminf(fmaxf(a[i] + kGaussR * r, -kGaussR), kGaussR) : -kGaussR;
    bp[nbp++] = lo; bp[nbp++] = mid; bp[nbp++] = hi;
  }
  // insertion sort of the breakpoints (kGaussBp values)
#pragma unroll
  for (int i = 1; i < kGaussBp; ++i)
#pragma unroll
    for (int j = i; j > 0; --j) {
      const float x = bp[j - 1], y = bp[j];
      bp[j - 1] = fminf(x, y);
      bp[j] = fmaxf(x, y);
    }
  const float inv_sqrt_2pi = 0.39894228040143268f;
  float2 tot = make_float2(0.f, 0.f), comp = make_float2(0.f, 0.f);
  for (int k = 0; k + 1 < kGaussBp; ++k) {
    const float x0 = bp[k], x1 = bp[k + 1];
    if (!(x1 > x0)) continue;
    const float half = 0.5f * (x1 - x0), mid = 0.5f * (x0 + x1);
    float2 sum = make_float2(0.f, 0.f);
    for (int q = 0; q < 16; ++q) {
      const float xi = (q < 8) ? -kGL16x[7 - q] : kGL16x[q - 8];
      const float wi = (q < 8) ? kGL16w[7 - q] : kGL16w[q - 8];
      const float t = fmaf(half, xi, mid);
      const float ph = inv_sqrt_2pi * expf(-0.5f * t * t);
      float u = ph, v = ph;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        if (!(present[i] && (!SADDLE || sg[i] != 0))) continue;
        float2 qp;
        if (step[i]) qp = t < a[i] ? make_float2(1.f, 0.f) : make_float2(0.f, 1.f);
        else qp = gauss_tails((t - a[i]) * ir[i]);
        if (SADDLE && sg[i] < 0) qp = make_float2(qp.y, qp.x);
        u *= qp.x;  // min: survival (saddle t1: its factor)
        v *= qp.y;  // max: CDF (saddle t2: the other factor)
      }
      sum.x = fmaf(wi, u, sum.x);
      sum.y = fmaf(wi, v, sum.y);
    }
    // Kahan over the pieces
    const float yx = sum.x * half - comp.x, yy = sum.y * half - comp.y;
    const float tx = tot.x + yx, ty = tot.y + yy;
    comp.x = (tx - tot.x) - yx;
    comp.y = (ty - tot.y) - yy;
    tot.x = tx;
    tot.y = ty;
  }
  return tot;
}

__device__ __forceinline__ void gauss_vertex(GaussParams c, const GaussParams *nb,
                                             const bool *present, float &pmin, float &pmax) {
  if (c.s == 0.f) {
    float gm = 1.f, gM = 1.f;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (!present[i]) continue;
      float2 qp;
      if (nb[i].s == 0.f)
        qp = make_float2(nb[i].m > c.m ? 1.f : 0.f, nb[i].m < c.m ? 1.f : 0.f);
      else
        qp = gauss_tails((c.m - nb[i].m) / nb[i].s);
      gm *= qp.x;
      gM *= qp.y;
    }
    pmin = gm;
    pmax = gM;
    return;
  }
  const float2 r = gauss_quad<false>(c, nb, present, nullptr);
  pmin = fminf(fmaxf(r.x, 0.f), 1.f);
  pmax = fminf(fmaxf(r.y, 0.f), 1.f);
}

// saddle t1 + t2 (sg: +1 survival, -1 CDF, 0 absent, for t1)
__device__ __forceinline__ float gauss_saddle(GaussParams c, const GaussParams *nb,
                                              const bool *present, const int *sg) {
  if (c.s == 0.f) {
    float t1 = 1.f, t2 = 1.f;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (sg[i] == 0) continue;
      float2 qp;
      if (nb[i].s == 0.f)
        qp = make_float2(nb[i].m > c.m ? 1.f : 0.f, nb[i].m < c.m ? 1.f : 0.f);
      else
        qp = gauss_tails((c.m - nb[i].m) / nb[i].s);
      t1 *= sg[i] > 0 ? qp.x : qp.y;
      t2 *= sg[i] > 0 ? qp.y : qp.x;
    }
    return t1 + t2;
  }
  const float2 r = gauss_quad<true>(c, nb, present, sg);
  return fmaxf(r.x, 0.f) + fmaxf(r.y, 0.f);
}

// ---------------------------------------------------------------------------
// saddle: products that mix survivals and CDFs (Eq. saddleProb)
//
// sg[i] = +1: the factor is the survival G_i (X_1 < X_i), -1: the CDF F_i
// (X_1 > X_i), 0: absent (the constant 1).  A survival factor is 1 below its
// support start and 0 above its end; a CDF factor is 0 below the start and 1
// above the end.  So the product vanishes outside [L, R], L = the largest
// start among CDF factors (and the centre's own), R = the smallest end among
// survival factors; inside, the breakpoints are the survival factors' starts
// and the CDF factors' ends.

// uniform: t = int pdf_1 prod_i f_i in the centre's frame (origin a1)
__device__ __forceinline__ float uniform_mixed(UniParams c, const UniParams *nb, const int *sg) {
  if (c.a == c.b) {
    const float v = c.a;
    float p = 1.f;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (sg[i] == 0) continue;
      const float a = nb[i].a, b = nb[i].b;
      float q;
      if (a == b) q = sg[i] > 0 ? (a > v ? 1.f : 0.f) : (a < v ? 1.f : 0.f);
      else {
        const float r = frcp(b - a);
        q = sg[i] > 0 ? (b - v) * r : (v - a) * r;
        q = fminf(fmaxf(q, 0.f), 1.f);
      }
      p *= q;
    }
    return p;
  }
  const float W1 = c.b - c.a;
  float L = 0.f, R = W1;
  float bp[4], al[4], be[4], sl[4];
  int kind[4];  // 0 constant 1, 1 survival, 2 CDF
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    kind[i] = 0; al[i] = 0.f; be[i] = 0.f; sl[i] = 0.f; bp[i] = kFar;
    if (sg[i] == 0) continue;
    const float a = nb[i].a - c.a, b = nb[i].b - c.a;
    if (sg[i] > 0) {
      R = fminf(R, b);
      if (nb[i].a != nb[i].b) { kind[i] = 1; bp[i] = a; }
    } else {
      L = fmaxf(L, a);
      if (nb[i].a != nb[i].b) { kind[i] = 2; bp[i] = b; }
    }
    al[i] = a; be[i] = b;
    sl[i] = nb[i].a != nb[i].b ? frcp(nb[i].b - nb[i].a) : 0.f;
  }
  if (!(R > L)) return 0.f;
  float t[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) t[i] = fminf(fmaxf(bp[i], L), R);
  float none[1][4];
  sort4<0>(t, none);
  const float x[6] = {L, t[0], t[1], t[2], t[3], R};
  Kahan acc;
  float Lv[4], Rv[4];
#pragma unroll
  for (int j = 0; j <= 4; ++j) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float x0 = x[j], x1 = x[j + 1];
      if (kind[i] == 1) {
        Lv[i] = fminf(fmaxf((be[i] - x0) * sl[i], 0.f), 1.f);
        Rv[i] = fminf(fmaxf((be[i] - x1) * sl[i], 0.f), 1.f);
      } else if (kind[i] == 2) {
        Lv[i] = fminf(fmaxf((x0 - al[i]) * sl[i], 0.f), 1.f);
        Rv[i] = fminf(fmaxf((x1 - al[i]) * sl[i], 0.f), 1.f);
      } else {
        Lv[i] = Rv[i] = 1.f;
      }
    }
    acc.add((x[j + 1] - x[j]) * bern_mean<4>(Lv, Rv));
  }
  return acc.get() * frcp(W1);
}

// Epanechnikov: the same, 8-point Gauss-Legendre on each piece (origin m1);
// F_i(x) = epan_surv((m_i - x)/w_i) by the kernel's symmetry
__device__ __forceinline__ float epan_mixed(EpanParams c, const EpanParams *nb, const int *sg) {
  if (c.w == 0.f) {
    const float v = c.m;
    float p = 1.f;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (sg[i] == 0) continue;
      float q;
      if (nb[i].w == 0.f) q = sg[i] > 0 ? (nb[i].m > v ? 1.f : 0.f) : (nb[i].m < v ? 1.f : 0.f);
      else q = epan_surv(sg[i] > 0 ? (v - nb[i].m) / nb[i].w : (nb[i].m - v) / nb[i].w);
      p *= q;
    }
    return p;
  }
  const float w1 = c.w;
  float L = -w1, R = w1;
  float bp[4], d[4], iw[4], sgn[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    bp[i] = kFar; d[i] = 0.f; iw[i] = 0.f; sgn[i] = 0.f;
    if (sg[i] == 0) continue;
    const float dn = nb[i].m - c.m, wn = nb[i].w;
    if (sg[i] > 0) {
      R = fminf(R, dn + wn);
      if (wn > 0.f) { bp[i] = dn - wn; d[i] = dn; iw[i] = frcp(wn); sgn[i] = 1.f; }
    } else {
      L = fmaxf(L, dn - wn);
      if (wn > 0.f) { bp[i] = dn + wn; d[i] = dn; iw[i] = frcp(wn); sgn[i] = -1.f; }
    }
  }
  if (!(R > L)) return 0.f;
  float t[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) t[i] = fminf(fmaxf(bp[i], L), R);
  float none[1][4];
  sort4<0>(t, none);
  const float x[6] = {L, t[0], t[1], t[2], t[3], R};
  const float iw1 = frcp(w1), c1 = 0.75f * iw1;
  Kahan acc;
  // the 8 nodes in the symmetric pairs (-x_k, x_k), which share the weight
  // w_k: one pair per float2 (packed FP32 instructions, the same operations
  // per node as the scalar form)
  const float2 one2 = make_float2(1.f, 1.f), two2 = make_float2(2.f, 2.f);
#pragma unroll
  for (int j = 0; j <= 4; ++j) {
    const float half = 0.5f * (x[j + 1] - x[j]), mid = 0.5f * (x[j] + x[j + 1]);
    float2 s2 = make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float2 xx = __ffma2_rn(make_float2(half, half), make_float2(-kGLx[k], kGLx[k]),
                                   make_float2(mid, mid));
      const float2 u1 = __fmul2_rn(xx, make_float2(iw1, iw1));
      const float2 g = __ffma2_rn(make_float2(-u1.x, -u1.y), u1, one2);
      float2 f = __fmul2_rn(make_float2(c1, c1), make_float2(fmaxf(g.x, 0.f), fmaxf(g.y, 0.f)));
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        if (sgn[i] == 0.f) continue;
        // epan_surv of sgn (x - d) / w at both nodes
        float2 u = __fmul2_rn(__fmul2_rn(make_float2(sgn[i], sgn[i]),
                                         __fadd2_rn(xx, make_float2(-d[i], -d[i]))),
                              make_float2(iw[i], iw[i]));
        u = make_float2(fminf(fmaxf(u.x, -1.f), 1.f), fminf(fmaxf(u.y, -1.f), 1.f));
        const float2 qq = __fadd2_rn(one2, make_float2(-u.x, -u.y));
        const float2 sv = __fmul2_rn(__fmul2_rn(__fmul2_rn(make_float2(0.25f, 0.25f), qq), qq),
                                     __fadd2_rn(two2, u));
        f = __fmul2_rn(f, sv);
      }
      s2 = __ffma2_rn(make_float2(kGLw[k], kGLw[k]), f, s2);
    }
    acc.add((s2.x + s2.y) * half);
  }
  return acc.get();
}

// saddle signs of the four slots (e, n, w, s) for t1, or all zero when the
// vertex has no saddle neighbourhood: all four neighbours present -> G F G F;
// a 1 x W (H x 1) grid with both line neighbours -> next (e / s) G, previous
// (w / n) F
__device__ __forceinline__ bool saddle_signs(const bool *present, int H, int W, int *sg) {
  const int k = (int)present[0] + present[1] + present[2] + present[3];
  sg[0] = sg[1] = sg[2] = sg[3] = 0;
  if (k == 4) {
    sg[0] = 1; sg[1] = -1; sg[2] = 1; sg[3] = -1;
    return true;
  }
  if (k == 2 && (H == 1 || W == 1)) {
    if (present[0]) sg[0] = 1;
    if (present[2]) sg[2] = -1;
    if (present[3]) sg[3] = 1;
    if (present[1]) sg[1] = -1;
    return true;
  }
  return false;
}

// ---------------------------------------------------------------------------
// counter-based generator: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11)

// key schedule (Weyl sequence), computed once per vertex
struct PhiloxKeys {
  uint32_t k0[10], k1[10];
  __device__ __forceinline__ PhiloxKeys(uint32_t a, uint32_t b) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
      k0[r] = a;
      k1[r] = b;
      a += 0x9E3779B9u;
      b += 0xBB67AE85u;
    }
  }
};

__device__ __forceinline__ void philox_round(uint4 &c, uint32_t k0, uint32_t k1) {
  const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
  const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
  c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
}

__device__ __forceinline__ uint4 philox_block(uint4 c, const PhiloxKeys &K) {
#pragma unroll
  for (int r = 0; r < 10; ++r) philox_round(c, K.k0[r], K.k1[r]);
  return c;
}

// ((r >> 8) + 0.5) * 2^-24 rounded to binary32 (one rounding: exact below
// 1/2, the nearest even multiple of 2^-24 above, 1.0 for the largest r):
// the semianalytical estimator's uniforms
__device__ __forceinline__ float u01(uint32_t r) {
  return fmaf(__uint2float_rn(r >> 8), 0x1p-24f, 0x1p-25f);
}
// ((r >> 9) + 0.5) * 2^-23, exact in binary32 and strictly inside (0, 1):
// the Monte Carlo path's uniforms (a logarithm of each is taken)
__device__ __forceinline__ float u01_23(uint32_t r) {
  return fmaf(__uint2float_rn(r >> 9), 0x1p-23f, 0x1p-24f);
}

// ---------------------------------------------------------------------------
// semianalytical histogram estimator (Sec. "Semianalytical Solution")
//
// c samples from the centre's histogram; for each sample x the probability
// of being below (above) every neighbour is exact -- the neighbours' mixture
// survivals G_n(x) (CDFs F_n(x)) from their bin and prefix mass -- and the
// estimate is T_1 times the mean of the products.  Sample s of vertex i uses
// the Philox block with counter (s >> 1, i, field, 2): words 0, 1 (s even) or
// 2, 3 (s odd) are (ua, ub).  Bin: the number of running mass sums C_1..C_B
// (binary32, bin order) that are <= ua * T_1, clamped to B - 1 (binary
// search over the prefix planes); position: (j + ub) h inside the bin.

struct SemiNb {
  float lam, ih, T;  // local support start, B / (hi - lo), total mass
  int off;           // shared-memory index of the vertex
  int kind;          // 0 absent, 1 bins, 2 point mass
};

// F_n(x) and G_n(x) = T_n - F_n(x) of a neighbour at the local position x.
// Branch-free, so that the lanes of a warp stay converged: the in-support
// value is formed for every kind (its reads stay inside the neighbour's
// rows: the bin index is clamped to [0, B-1]; an absent or point-mass
// neighbour has ih = 0) and the result selected by position and kind.
template <int WS>
__device__ __forceinline__ void semi_tails(const float *w, const float *C, const SemiNb &n, int B,
                                           float x, float &G, float &F) {
  const float v = (x - n.lam) * n.ih;
  const float fk = floorf(v);
  const int k = (int)fminf(fmaxf(fk, 0.f), (float)(B - 1));
  const float Ck = C[max(k - 1, 0) * WS + n.off];
  const float Fin = fmaf(w[k * WS + n.off], v - fk, k > 0 ? Ck : 0.f);
  F = fk < 0.f ? 0.f : (fk >= (float)B ? n.T : Fin);
  G = fk < 0.f ? n.T : (fk >= (float)B ? 0.f : n.T - Fin);
  if (n.kind != 1) {
    G = n.kind == 2 ? (x < n.lam ? n.T : 0.f) : 1.f;
    F = n.kind == 2 ? (x > n.lam ? n.T : 0.f) : 1.f;
  }
}

template <int WS, bool SADDLE>
__device__ __forceinline__ void semi_vertex(const float *w, const float *C, int l, float lo1,
                                            float hi1, const SemiNb *nb, int B, int S,
                                            const PhiloxKeys &K, uint32_t vid, uint32_t field,
                                            const int *sg, float &pmin, float &pmax,
                                            float &psad) {
  const float T1 = C[(B - 1) * WS + l];
  if (lo1 == hi1) {  // point-mass centre: every sample is its position
    float gm = T1, gM = T1, t1 = T1, t2 = T1;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      float G, F;
      semi_tails<WS>(w, C, nb[i], B, 0.f, G, F);
      gm *= G;
      gM *= F;
      if (SADDLE && sg[i] != 0) {
        t1 *= sg[i] > 0 ? G : F;
        t2 *= sg[i] > 0 ? F : G;
      }
    }
    pmin = gm;
    pmax = gM;
    psad = t1 + t2;
    return;
  }
  const float h1 = (hi1 - lo1) / (float)B;
  Kahan amin, amax;
  for (int s = 0; s < S; s += 2) {
    const uint4 r = philox_block(make_uint4((uint32_t)(s >> 1), vid, field, 2u), K);
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      if (s + half >= S) break;
      const float ua = u01(half ? r.z : r.x), ub = u01(half ? r.w : r.y);
      const float t = ua * T1;
      int lo = 0, hi = B;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (C[mid * WS + l] <= t) lo = mid + 1;
        else hi = mid;
      }
      const int j = min(lo, B - 1);
      const float x = ((float)j + ub) * h1;
      float pm = T1, pM = T1, t1 = T1, t2 = T1;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        float G, F;
        semi_tails<WS>(w, C, nb[i], B, x, G, F);
        if (SADDLE) {
          t1 *= sg[i] > 0 ? G : (sg[i] < 0 ? F : 1.f);
          t2 *= sg[i] > 0 ? F : (sg[i] < 0 ? G : 1.f);
        } else {
          pm *= G;
          pM *= F;
        }
      }
      if (SADDLE) {
        amin.add(t1 + t2);
      } else {
        amin.add(pm);
        amax.add(pM);
      }
    }
  }
  const float inv = 1.f / (float)S;
  pmin = amin.get() * inv;
  pmax = amax.get() * inv;
  psad = pmin;
}

// ---------------------------------------------------------------------------
// closed-form integration, histogram model (breakpoint merge)

// Shared-memory layout of a staged histogram vertex after the tail-table pass
// (row r at sm[r * WS + l]): 0 lo, 1 hi, 2 + k the tail S_k = T - (m_0 + ...
// + m_{k-1}) for k = 0..B+1 (S_0 = T, S_B = S_{B+1} = 0; all 0 for a point
// mass), 4 + B the total mass T, 5 + B the status bits.  On bin k the
// survival is G(x) = S_k - (S_k - S_{k+1}) (x - e_k) / h.
__host__ __device__ constexpr int hist_rows(int B) { return B + 6; }

// buckets of the per-tile ordering of histogram walks by length (a walk has
// at most B + 4 (B + 1) pieces)
constexpr int kSortBuckets = 5 * kMaxBins + 8;

// A neighbour's survival G(x) (mixture form) walked segment by segment over
// its edges lam + j h, j = 0..B: before the support G = T, on bin k the
// segment above, after the support 0.  A point mass has h = 0: all its edges
// coincide and G jumps from T to 0 there.  An absent neighbour is the
// constant 1 that never reaches an edge.
struct HistSeg {
  int addr;                 // table index of the tail read at the next crossing
  float kf;                 // index of the next edge (B + 1: none left)
  float lam, h, invh;       // support start, bin width, 1/h (0 for a point mass)
  float el, nx, s, sn, sl;  // segment start, next edge, S_k, S_{k+1}, slope
  __device__ __forceinline__ void init_absent(int off, float Bf) {
    addr = off; kf = Bf + 1.f; lam = h = invh = 0.f;
    el = -kFar; nx = kFar; s = sn = 1.f; sl = 0.f;
  }
  template <int WS>
  __device__ __forceinline__ void init(const float *S0, int off, float lam_, float h_, float T) {
    addr = off + WS; kf = 0.f;
    lam = lam_; h = h_; invh = h_ > 0.f ? frcp(h_) : 0.f;
    el = -kFar; nx = lam_; s = T; sn = S0[off]; sl = 0.f;
  }
  // One merge step at x1 (x1 < kFar): cross the next edge if it is at or
  // below x1 (then enter the next bin: S_k <- S_{k+1}, read S_{k+2}), else
  // keep the segment.  No branch; the table read always has a valid address:
  // after its last edge nx = kFar, so a walker crosses at most B + 1 edges,
  // and the table ends two rows after S_B.  Returns whether it crossed.
  template <int WS>
  __device__ __forceinline__ bool step(const float *S0, float x1, float Bf) {
    const bool c = nx <= x1;
    const float t = S0[addr];
    s = c ? sn : s;
    sn = c ? t : sn;
    addr += c ? WS : 0;
    sl = (s - sn) * invh;
    el = c ? x1 : el;
    kf = c ? kf + 1.f : kf;
    nx = c ? (kf <= Bf ? fmaf(kf, h, lam) : kFar) : nx;
    return c;
  }
  __device__ __forceinline__ float G(float x) const { return fmaf(-sl, x - el, s); }
  // From the initial state, cross every edge at or below 0 at once: the
  // state step() would reach edge by edge (the count of such edges comes
  // from -lam / h and is then checked against the edges themselves).
  template <int WS>
  __device__ __forceinline__ void seek0(const float *S0, int B) {
    if (nx > 0.f) return;  // the first edge is above 0 (also: absent)
    int j;                 // edges lam + i h <= 0 for i < j
    if (h > 0.f) {
      j = (int)fminf(fmaxf(floorf(-lam * invh), 0.f), (float)B) + 1;
      if (j <= B && fmaf((float)j, h, lam) <= 0.f) ++j;
      if (j >= 2 && fmaf((float)(j - 1), h, lam) > 0.f) --j;
    } else {
      j = B + 1;  // a point mass at or below 0: all its edges coincide
    }
    const int off = addr - WS;
    const int k = j - 1;  // the bin now entered
    s = S0[off + k * WS];
    sn = S0[off + j * WS];
    addr = off + (j + 1) * WS;
    sl = (s - sn) * invh;
    el = fmaf((float)k, h, lam);
    kf = (float)j;
    nx = j <= B ? fmaf((float)j, h, lam) : kFar;
  }
};

// Both probabilities of a non-degenerate histogram centre in one walk over
// [0, W1] (local frame at lo1, centre tail table Sc): all bin edges of the
// centre and of the neighbours are merged in increasing order; on each piece
// the centre pdf is the constant m_j / h1 and each factor is linear, so the
// piece integral is the Bernstein mean of the factor end values.  Beyond a
// neighbour's support its survival is 0, before it its CDF is 0, so both
// integrals run over the centre's whole support.  Every lane executes the
// same instructions on every step (the crossings are predicated, one edge or
// a tie per step), so a warp stays converged until its lanes run out of
// pieces.
// SADDLE = false: (pmin, pmax) = (int pdf prod G, int pdf prod F).
// SADDLE = true:  (pmin, pmax) = (t1, t2) with factor i = G_i if sg[i] > 0
// else F_i for t1, and the other one for t2 (absent neighbours are 1 in both).
template <int WS, bool SADDLE = false>
__device__ __forceinline__ void hist_walk(const float *S0, int coff, int B, float W1,
                                          HistSeg *nw, const float *T, unsigned want,
                                          float &pmin, float &pmax, const int *sg = nullptr) {
  // every breakpoint of the walk is at most W1, below kFar
  if (!(W1 <= 1e38f)) {
    pmin = pmax = __int_as_float(0x7fc00000);
    return;
  }
  const float Bf = (float)B;
  const float h1 = W1 / Bf, ih1 = frcp(h1);
  // centre: tails sc = S_k, scn = S_{k+1} of its bin k, next edge index kcf
  int addr_c = coff + 2 * WS;
  float kcf = 1.f;
  float sc = S0[coff], scn = S0[coff + WS];
  float dens = (sc - scn) * ih1;
  float nxc = B > 1 ? h1 : W1;
  // factor end values, two products per float2: (G, F) for the minimum and
  // maximum, (t1 factor, t2 factor) for the saddle
  auto pair = [&](int i, float g, float f) {
    if constexpr (SADDLE) return sg[i] > 0 ? make_float2(g, f) : make_float2(f, g);
    else return make_float2(g, f);
  };
  float2 Pl[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float g = nw[i].G(0.f);
    Pl[i] = pair(i, g, T[i] - g);
  }
  float2 acc = make_float2(0.f, 0.f);
  float x0 = 0.f;
  const int max_steps = 5 * (B + 2) + 4;
#pragma unroll 2
  for (int step = 0; step < max_steps && x0 < W1; ++step) {
    float x1 = fminf(fminf(nw[0].nx, nw[1].nx), fminf(nw[2].nx, nw[3].nx));
    x1 = fmaxf(fminf(x1, nxc), x0);
    float2 Pr[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float g = nw[i].G(x1);
      Pr[i] = pair(i, g, T[i] - g);
    }
    const float wgt = (x1 - x0) * dens;
    acc = __ffma2_rn(make_float2(wgt, wgt), bern_mean4_x2(Pl, Pr), acc);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      // the left value of the next piece is the new segment's value at x1
      // (the right value, except after a point mass)
      const bool c = nw[i].step<WS>(S0, x1, Bf);
      Pl[i] = c ? pair(i, nw[i].s, T[i] - nw[i].s) : Pr[i];
    }
    {
      const bool c = nxc <= x1;
      const float t = S0[addr_c];
      sc = c ? scn : sc;
      scn = c ? t : scn;
      addr_c += c ? WS : 0;
      kcf = c ? kcf + 1.f : kcf;
      nxc = c ? (kcf < Bf ? kcf * h1 : (kcf == Bf ? W1 : kFar)) : nxc;
      dens = (sc - scn) * ih1;
    }
    x0 = x1;
  }
  (void)want;
  pmin = fmaxf(acc.x, 0.f);
  pmax = fmaxf(acc.y, 0.f);
}

// Crossing step of a walker over shared-memory rows: if nx <= x1, read the
// 16-byte row at addr into v and advance addr by `stride` bytes; else leave
// both.  One comparison, one predicated read and one predicated add, no
// branch.  addr: a shared-state-space address.
template <unsigned stride>
__device__ __forceinline__ void lds128_cross(float nx, float x1, uint32_t &addr, float4 &v) {
  asm("{\n .reg .pred q;\n setp.le.f32 q, %5, %6;\n"
      " @q ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];\n"
      " @q add.u32 %4, %4, %7;\n}"
      : "+f"(v.x), "+f"(v.y), "+f"(v.z), "+f"(v.w), "+r"(addr)
      : "f"(nx), "f"(x1), "n"(stride));
}
template <unsigned stride>
__device__ __forceinline__ void lds64_cross(float nx, float x1, uint32_t &addr, float2 &v) {
  asm("{\n .reg .pred q;\n setp.le.f32 q, %3, %4;\n"
      " @q ld.shared.v2.f32 {%0, %1}, [%2];\n"
      " @q add.u32 %2, %2, %5;\n}"
      : "+f"(v.x), "+f"(v.y), "+r"(addr)
      : "f"(nx), "f"(x1), "n"(stride));
}

// Per-bin rows of a staged histogram vertex for the forward walk: float4
// rows at R[k * RS + l], k = 0..B.  Row k < B describes bin k: (S_k,
// T - S_k, slope_k, e_{k+1} - lo), with the tail S_k = T - (m_0 + ... +
// m_{k-1}), slope_k = (S_k - S_{k+1}) / h (the bin's density, m_k / h, in
// the mixture form) and e_{k+1} - lo = (k + 1) h (hi - lo for the last
// edge).  Row B is (0, T, 0, kFar), beyond the support.  A point mass has
// every row (0, T, 0, kFar): its one edge takes the survival from T to 0.
// A walker reads a row only when it crosses an edge, at most B + 1 times,
// so no row past B is ever read.
__host__ __device__ constexpr int hist_r4_rows(int B) { return B + 1; }

// Row stride of the per-bin rows of a halo of `halo` vertices, in float4:
// a multiple of 8 (128 bytes).  The 32 lanes of a warp walk 32 consecutive
// vertices and read the rows of the same neighbour direction, so lane i
// reads R[k_i * RS + l0 + i]; with RS a multiple of 128 bytes the bank of
// that 16-byte read depends on i alone, whatever row k_i each lane is on,
// and the eight lanes of a quarter warp never share a bank.
__host__ __device__ constexpr int hist_r4_stride(int halo) { return (halo + 7) & ~7; }

// A neighbour's survival G and CDF F walked bin by bin over the per-bin
// rows: before the support (G, F) = (T, 0); on bin k G falls and F rises by
// slope_k per unit of x; beyond it (0, T).  The walker holds the row of its
// current segment, (G, F, slope, next edge - lo) with G and F taken at the
// walk's current position, advances G and F by the step length and,
// crossing an edge, lets one predicated 16-byte read replace the whole state
// with the next row, whose (S_k, T - S_k) are the exact values at that edge
// (which also carries the jump of a point mass).  An absent neighbour is the
// constant G = F = 1 that never reaches an edge.
struct HistRowWalker {
  float4 r;       // (G, F at the current position, slope, next edge - lo)
  float lam;      // support start in the centre's frame
  uint32_t addr;  // shared-memory address of the row read at the next crossing
  __device__ __forceinline__ float nx() const { return lam + r.w; }
  __device__ __forceinline__ void init_absent() {
    r = make_float4(1.f, 1.f, 0.f, kFar); lam = 0.f; addr = 0u;
  }
  // before the support: (G, F) = (T, 0), the first edge is the support start
  __device__ __forceinline__ void init(const float4 *row0, float lam_, float T) {
    r = make_float4(T, 0.f, 0.f, 0.f); lam = lam_;
    addr = static_cast<uint32_t>(__cvta_generic_to_shared(row0));
  }
  // Move to x1 (G and F there given): cross the next edge if it is at or
  // below x1 -- it is then exactly at x1, the walk's next breakpoint being
  // the smallest next edge -- and take the new segment's row.
  template <int RS>
  __device__ __forceinline__ void step(float x1, float g1, float f1) {
    const float n = nx();
    r.x = g1;
    r.y = f1;
    lds128_cross<(unsigned)(RS * 16)>(n, x1, addr, r);
  }
  // From the initial state, cross every edge at or below 0 at once (the
  // state step() would reach edge by edge; the count of such edges comes
  // from -lam / h and is checked against the edges of the rows), and set G
  // and F to their values at 0.  Returns the number of edges crossed (a
  // point mass: 1), 0 if the first edge is above 0.
  template <int RS>
  __device__ __forceinline__ int seek0(const float4 *row0, int B, float h) {
    if (nx() > 0.f) return 0;  // the first edge is above 0 (also: absent)
    int j = 1;               // edges e_0 .. e_{j-1} are at or below 0
    float el;
    if (h > 0.f) {
      auto edge = [&](int i) { return i == 0 ? lam : lam + row0[(i - 1) * RS].w; };
      j = (int)fminf(fmaxf(floorf(-lam * frcp(h)), 0.f), (float)B) + 1;
      if (j <= B && edge(j) <= 0.f) ++j;
      if (j >= 2 && edge(j - 1) > 0.f) --j;
      el = edge(j - 1);
    } else {
      el = lam;              // a point mass: its one edge
    }
    r = row0[(j - 1) * RS];
    // on the segment that starts at el <= 0: G(x) = S - slope (x - el) and
    // F(x) = T - S + slope (x - el), taken at x = 0
    r.x = fmaf(r.z, el, r.x);
    r.y = fmaf(-r.z, el, r.y);
    addr = static_cast<uint32_t>(__cvta_generic_to_shared(row0 + j * RS));
    return j;
  }
};

// Both probabilities of a non-degenerate histogram centre in one walk over
// [0, W1] (local frame at lo1; the centre's rows from crow): all bin edges of
// the centre and of the four neighbours are merged in increasing order; on
// each piece the centre pdf is the constant m_j / h1 and each factor is
// linear, so the piece integral is the Bernstein mean of the factor end
// values (bern_mean4_pairs_x2).  Beyond a neighbour's support its survival is
// 0, before it its CDF is 0, so both integrals run over the centre's whole
// support.  Every lane executes the same instructions on every step; only the
// row reads of the crossings are predicated.
// SADDLE = false: (pmin, pmax) = (int pdf prod G, int pdf prod F).
// SADDLE = true:  (pmin, pmax) = (t1, t2) with factor i = G_i if sg[i] > 0
// else F_i for t1, and the other one for t2 (absent neighbours are 1 in both).
template <int RS, bool SADDLE = false>
__device__ __forceinline__ void hist_walk_rows(const float4 *crow, int B, float W1,
                                               HistRowWalker *nw, float &pmin, float &pmax,
                                               const int *sg = nullptr) {
  if (!(W1 <= 1e38f)) {
    pmin = pmax = __int_as_float(0x7fc00000);
    return;
  }
  // the centre needs only the density and the next edge of its bin: the
  // (z, w) half of each row
  uint32_t addr_c = static_cast<uint32_t>(__cvta_generic_to_shared(crow + RS)) + 8u;
  float2 dc;  // (density, next edge) of the centre's current bin
  {
    const float4 t = crow[0];
    dc = make_float2(t.z, t.w);
  }
  auto pair = [&](int i, float g, float ff) {
    if constexpr (SADDLE) return sg[i] > 0 ? make_float2(g, ff) : make_float2(ff, g);
    else return make_float2(g, ff);
  };
  float2 acc = make_float2(0.f, 0.f);
  float x0 = 0.f;
  const int max_steps = 5 * (B + 1) + 4;
#pragma unroll 1
  for (int step = 0; step < max_steps && x0 < W1; ++step) {
    const float x1 =
        fminf(fminf(fminf(nw[0].nx(), nw[1].nx()), fminf(nw[2].nx(), nw[3].nx())), dc.y);
    const float d = x1 - x0;
    float g1[4], f1[4];
    float2 L[4], Rv[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      g1[i] = fmaf(-nw[i].r.z, d, nw[i].r.x);
      f1[i] = fmaf(nw[i].r.z, d, nw[i].r.y);
      L[i] = pair(i, nw[i].r.x, nw[i].r.y);
      Rv[i] = pair(i, g1[i], f1[i]);
    }
    const float wgt = d * dc.x;
    acc = __ffma2_rn(make_float2(wgt, wgt), bern_mean4_pairs_x2(L, Rv), acc);
#pragma unroll
    for (int i = 0; i < 4; ++i) nw[i].step<RS>(x1, g1[i], f1[i]);
    lds64_cross<(unsigned)(RS * 16)>(dc.y, x1, addr_c, dc);
    x0 = x1;
  }
  pmin = fmaxf(acc.x, 0.f);
  pmax = fmaxf(acc.y, 0.f);
}

// survival and CDF of a histogram neighbour (tail table S, total T) at a
// point v (degenerate centre)
__device__ __forceinline__ void hist_tails_at(const float *S, int ws, int B, float lo, float hi,
                                              float T, float v, float &gt, float &lt) {
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
  const float sj = S[j * ws], sj1 = S[(j + 1) * ws];
  gt = fmaxf(fmaf(-fr, sj - sj1, sj), 0.f);
  lt = fmaxf(T - gt, 0.f);
}

// hist_tails_at with the tails read from per-bin rows (R at the vertex's
// row 0, rows ws apart)
__device__ __forceinline__ void hist_tails_at_rows(const float4 *R, int ws, int B, float lo,
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
  const float sj = R[j * ws].x, sj1 = R[(j + 1) * ws].x;
  gt = fmaxf(fmaf(-fr, sj - sj1, sj), 0.f);
  lt = fmaxf(T - gt, 0.f);
}

}  // namespace ucp
