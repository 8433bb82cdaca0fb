// backward.cu -- adjoint of L = sum_v W_v P_v with respect to every vertex's
// model parameters (uniform (a, b), Epanechnikov (m, w), histogram masses).
//
// P_v depends on the parameters of v and of its in-grid neighbours.  Each
// centre v gives the partials W_v dP_v/d(theta_u) for u = v and its four
// neighbours (slot 0 = v, 1..4 = e, n, w, s); every u's gradient is its own
// partial plus those its neighbours gave about it (u is the west neighbour
// of its east neighbour, and so on), summed in a fixed order, so the result
// is deterministic and needs no atomics.  The tile kernels (closed_adj_tile,
// hist_adj_tile) sum the partials of each tile's inner pairs in the CTA and
// hand the rest to the neighbouring tiles through a ring (hist_adj_fixup);
// histograms of more than 16 bins keep partial rows rows[slot][q][H][W] and a
// gather pass.
//
// Derivatives (exact, of the closed forms integrated in device.cuh):
//   neighbour n: d/dtheta_n int pdf_1 prod G = int pdf_1 (dG_n/dtheta_n) prod_{m!=n} G_m
//     uniform:       dG/da = s G, dG/db = s (1 - G) on the support (s = 1/(b-a))
//     Epanechnikov:  dG/dm = pdf_n, dG/dw = pdf_n (x - m)/w
//     histogram:     dG/dw_q = survival of the uniform kernel of bin q
//   centre: uniform adds the boundary terms of its moving support,
//     dP/da1 = (P - H(a1))/(b1-a1), dP/db1 = (H(b1) - P)/(b1-a1), H = prod G;
//     Epanechnikov differentiates the density (it vanishes at the ends);
//     histogram: dP/dw_j = (1/h) int_{bin j} prod G.
// Maxima use the negated variables (P_max(theta) = P_min(-theta)).
#include <algorithm>
#include <atomic>

#include "device.cuh"
#include "launch.h"
#include "tile.cuh"

namespace ucp {

namespace {

__device__ __forceinline__ float qnan_b() { return __int_as_float(0x7fc00000); }

// Leave-one-out products of four values.
__device__ __forceinline__ void loo4(const float *g, float *out) {
  const float p01 = g[0] * g[1], p23 = g[2] * g[3];
  out[0] = g[1] * p23;
  out[1] = g[0] * p23;
  out[2] = p01 * g[3];
  out[3] = p01 * g[2];
}

// ---------------------------------------------------------------------------
// uniform, minimum, in the frame of the centre's lower end

struct UniGrad {
  float ga, gb;      // centre
  float na[4], nb[4];  // neighbours (original slot order)
};

// al/sl/bl: neighbour start, slope (0 for point masses / absent), local end;
// kind: 0 absent, 1 continuous, 2 point mass (at al)
__device__ __forceinline__ void uniform_grad_side(float W1, float R, const float *al,
                                                  const float *sl, const int *kind,
                                                  UniGrad &g) {
#pragma unroll
  for (int i = 0; i < 4; ++i) g.na[i] = g.nb[i] = 0.f;
  // survival product at the centre's ends (point masses: step, strict)
  float H0 = 1.f, H1 = 1.f;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    if (kind[i] == 1) {
      H0 *= fminf(fmaxf(fmaf(-(0.f - al[i]), sl[i], 1.f), 0.f), 1.f);
      H1 *= fminf(fmaxf(fmaf(-(W1 - al[i]), sl[i], 1.f), 0.f), 1.f);
    } else if (kind[i] == 2) {
      H0 *= (0.f < al[i]) ? 1.f : 0.f;
      H1 *= (W1 < al[i]) ? 1.f : 0.f;
    }
  }
  if (R < W1) H1 = 0.f;
  if (!(R > 0.f)) {
    g.ga = -H0 / W1;
    g.gb = 0.f;
    return;
  }
  float t[4];
  float pay[3][4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const bool act = kind[i] == 1;
    t[i] = act ? fminf(fmaxf(al[i], 0.f), R) : R;
    pay[0][i] = act ? al[i] : kFar;
    pay[1][i] = act ? sl[i] : 0.f;
    pay[2][i] = (float)i;
  }
  sort4<3>(t, pay);
  const float x[6] = {0.f, t[0], t[1], t[2], t[3], R};
  float I[5];
  float Db[4] = {0.f, 0.f, 0.f, 0.f};  // per sorted factor: int of (1-G_i) prod_{m!=i} G
  I[0] = x[1];
  float L[4], Rv[4], L2[4], R2[4];
#pragma unroll
  for (int j = 1; j <= 4; ++j) {
    const float x0 = x[j], x1 = x[j + 1], len = x1 - x0;
#pragma unroll
    for (int i = 0; i < j; ++i) {
      L[i] = fmaxf(fmaf(-(x0 - pay[0][i]), pay[1][i], 1.f), 0.f);
      Rv[i] = fmaxf(fmaf(-(x1 - pay[0][i]), pay[1][i], 1.f), 0.f);
    }
    float Ij;
    if (j == 1) Ij = bern_mean<1>(L, Rv);
    else if (j == 2) Ij = bern_mean<2>(L, Rv);
    else if (j == 3) Ij = bern_mean<3>(L, Rv);
    else Ij = bern_mean<4>(L, Rv);
    I[j] = len * Ij;
#pragma unroll
    for (int i = 0; i < j; ++i) {
#pragma unroll
      for (int q = 0; q < j; ++q) {
        L2[q] = (q == i) ? 1.f - L[q] : L[q];
        R2[q] = (q == i) ? 1.f - Rv[q] : Rv[q];
      }
      float Bi;
      if (j == 1) Bi = bern_mean<1>(L2, R2);
      else if (j == 2) Bi = bern_mean<2>(L2, R2);
      else if (j == 3) Bi = bern_mean<3>(L2, R2);
      else Bi = bern_mean<4>(L2, R2);
      Db[i] += len * Bi;
    }
  }
  const float iW = 1.f / W1;
  const float P = (I[0] + I[1] + I[2] + I[3] + I[4]) * iW;
  g.ga = (P - H0) * iW;
  g.gb = (H1 - P) * iW;
  // factor i (sorted) is active on pieces j >= i + 1
  float tail = 0.f;
  float Da[4];
#pragma unroll
  for (int i = 3; i >= 0; --i) {
    tail += I[i + 1];
    Da[i] = tail;
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int o = (int)pay[2][i];
    const float s = pay[1][i] * iW;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (q == o) {
        g.na[q] = s * Da[i];
        g.nb[q] = s * Db[i];
      }
    }
  }
}

// full uniform gradient of one centre (min or max) -> rows
__device__ __forceinline__ void uniform_grad_vertex(float a1, float b1, const float *an,
                                                   const float *bn, const bool *present,
                                                   bool want_max, UniGrad &out) {
  // for the maximum, work on -X: (a, b) -> (-b, -a)
  const float A1 = want_max ? -b1 : a1, B1 = want_max ? -a1 : b1;
  float A[4], Bv[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    A[i] = want_max ? -bn[i] : an[i];
    Bv[i] = want_max ? -an[i] : bn[i];
  }
  UniGrad g;
  if (A1 == B1) {
    // point-mass centre: P = prod_n Pr[X_n > c]
    const float c = A1;
    float S[4], dsa[4], dsb[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      S[i] = 1.f; dsa[i] = 0.f; dsb[i] = 0.f;
      if (!present[i]) continue;
      if (A[i] == Bv[i]) {
        S[i] = A[i] > c ? 1.f : 0.f;
      } else {
        const float s = 1.f / (Bv[i] - A[i]);
        const float v = (Bv[i] - c) * s;
        S[i] = fminf(fmaxf(v, 0.f), 1.f);
        if (A[i] < c && c < Bv[i]) {
          dsa[i] = S[i] * s;
          dsb[i] = (1.f - S[i]) * s;
        }
      }
    }
    float lo[4];
    loo4(S, lo);
    g.ga = g.gb = 0.f;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      g.na[i] = dsa[i] * lo[i];
      g.nb[i] = dsb[i] * lo[i];
    }
  } else {
    const float W1 = B1 - A1;
    float al[4], sl[4], R = W1;
    int kind[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (!present[i]) {
        kind[i] = 0; al[i] = kFar; sl[i] = 0.f;
        continue;
      }
      al[i] = A[i] - A1;
      R = fminf(R, Bv[i] - A1);
      if (A[i] == Bv[i]) {
        kind[i] = 2; sl[i] = 0.f;
      } else {
        kind[i] = 1; sl[i] = 1.f / (Bv[i] - A[i]);
      }
    }
    uniform_grad_side(W1, R, al, sl, kind, g);
  }
  if (!want_max) {
    out = g;
    return;
  }
  // d/da = -d/db', d/db = -d/da'
  out.ga = -g.gb;
  out.gb = -g.ga;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    out.na[i] = -g.nb[i];
    out.nb[i] = -g.na[i];
  }
}

// ---------------------------------------------------------------------------
// Epanechnikov, minimum, Gauss-Legendre on the sorted pieces

struct EpanGrad {
  float gm, gw;
  float nm[4], nw[4];
};

__device__ __forceinline__ void epan_grad_vertex(float m1, float w1, const float *mn,
                                                const float *wn, const bool *present,
                                                bool want_max, EpanGrad &out) {
  // maximum: work on -X (m -> -m, w unchanged); d/dm flips sign
  const float M1 = want_max ? -m1 : m1;
  float M[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) M[i] = want_max ? -mn[i] : mn[i];
  EpanGrad g;
  g.gm = g.gw = 0.f;
#pragma unroll
  for (int i = 0; i < 4; ++i) g.nm[i] = g.nw[i] = 0.f;
  if (w1 == 0.f) {
    const float c = M1;
    float S[4], dm[4], dw[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      S[i] = 1.f; dm[i] = 0.f; dw[i] = 0.f;
      if (!present[i]) continue;
      if (wn[i] == 0.f) {
        S[i] = M[i] > c ? 1.f : 0.f;
      } else {
        const float u = (c - M[i]) / wn[i];
        S[i] = epan_surv(u);
        if (u > -1.f && u < 1.f) {
          const float pd = 0.75f / wn[i] * (1.f - u * u);
          dm[i] = pd;
          dw[i] = pd * u;
        }
      }
    }
    float lo[4];
    loo4(S, lo);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      g.nm[i] = dm[i] * lo[i];
      g.nw[i] = dw[i] * lo[i];
    }
  } else {
    float al[4], d[4], iw[4], R = w1;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      al[i] = kFar; d[i] = kFar; iw[i] = 0.f;
      if (!present[i]) continue;
      const float dn = M[i] - M1;
      if (wn[i] == 0.f) {
        R = fminf(R, dn);
      } else {
        al[i] = dn - wn[i]; d[i] = dn; iw[i] = 1.f / wn[i];
        R = fminf(R, dn + wn[i]);
      }
    }
    const float L0 = -w1;
    if (R > L0) {
      float t[4];
      float pay[3][4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        t[i] = fminf(fmaxf(al[i], L0), R);
        pay[0][i] = d[i];
        pay[1][i] = iw[i];
        pay[2][i] = (float)i;
      }
      sort4<3>(t, pay);
      const float x[6] = {L0, t[0], t[1], t[2], t[3], R};
      const float iw1 = 1.f / w1;
      const float c1 = 0.75f * iw1;
      const float cm = 1.5f * iw1 * iw1 * iw1;   // d pdf / dm1 = 1.5 x / w1^3
      const float cw = -0.75f * iw1 * iw1;       // d pdf / dw1 = -0.75/w1^2 (1 - 3u^2)
      float am[4] = {0, 0, 0, 0}, aw[4] = {0, 0, 0, 0};
      float gm = 0.f, gw = 0.f;
#pragma unroll
      for (int j = 0; j <= 4; ++j) {
        const float x0 = x[j], x1 = x[j + 1];
        const float half = 0.5f * (x1 - x0), mid = 0.5f * (x0 + x1);
        float pm = 0.f, pw = 0.f, qm[4] = {0, 0, 0, 0}, qw[4] = {0, 0, 0, 0};
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const float xi = (q < 4) ? -kGLx[3 - q] : kGLx[q - 4];
          const float wi = (q < 4) ? kGLw[3 - q] : kGLw[q - 4];
          const float xx = fmaf(half, xi, mid);
          const float u1 = xx * iw1;
          const float p1 = c1 * fmaxf(fmaf(-u1, u1, 1.f), 0.f);
          float G[4] = {1.f, 1.f, 1.f, 1.f}, pd[4] = {0, 0, 0, 0}, un[4] = {0, 0, 0, 0};
#pragma unroll
          for (int i = 0; i < j; ++i) {
            const float u = fminf(fmaxf((xx - pay[0][i]) * pay[1][i], -1.f), 1.f);
            G[i] = epan_surv(u);
            pd[i] = 0.75f * pay[1][i] * (1.f - u * u);
            un[i] = u;
          }
          float lo[4];
          loo4(G, lo);
          const float Hx = lo[0] * G[0];
          pm = fmaf(wi, cm * xx * Hx, pm);
          pw = fmaf(wi, cw * fmaf(-3.f * u1, u1, 1.f) * Hx, pw);
#pragma unroll
          for (int i = 0; i < j; ++i) {
            const float e = wi * p1 * pd[i] * lo[i];
            qm[i] += e;
            qw[i] = fmaf(e, un[i], qw[i]);
          }
        }
        gm = fmaf(pm, half, gm);
        gw = fmaf(pw, half, gw);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          am[i] = fmaf(qm[i], half, am[i]);
          aw[i] = fmaf(qw[i], half, aw[i]);
        }
      }
      g.gm = gm;
      g.gw = gw;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int o = (int)pay[2][i];
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (q == o) {
            g.nm[q] = am[i];
            g.nw[q] = aw[i];
          }
      }
    }
  }
  const float sgn = want_max ? -1.f : 1.f;
  out.gm = sgn * g.gm;
  out.gw = g.gw;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    out.nm[i] = sgn * g.nm[i];
    out.nw[i] = g.nw[i];
  }
}

// ---------------------------------------------------------------------------
// histogram, minimum (maximum through the negated histogram)

// read access to one vertex's histogram, optionally negated (X -> -X:
// support [-hi, -lo], bins reversed)
struct HistView {
  const float *p;
  long long plane;
  int B;
  bool neg;
  __device__ __forceinline__ float lo() const { return neg ? -p[plane] : p[0]; }
  __device__ __forceinline__ float hi() const { return neg ? -p[0] : p[plane]; }
  __device__ __forceinline__ float mass(int q) const {
    return p[(long long)(2 + (neg ? B - 1 - q : q)) * plane];
  }
  __device__ __forceinline__ int orig(int q) const { return neg ? B - 1 - q : q; }
};

struct NWalk {
  HistView v;
  int B, j;            // j: -1 before, B after
  float lam, h, ih, end, eleft, enext, S, slope, T;
  float C, Cstart, inbin;
};

__device__ __forceinline__ void nwalk_advance(NWalk &n, float *rows_n, long long ostride,
                                              float wv) {
  // leaving bin j (if inside the support): its partial is C(e_j) + within-bin
  if (n.j >= 0 && n.j < n.B) rows_n[(long long)n.v.orig(n.j) * ostride] = wv * (n.Cstart + n.inbin);
  ++n.j;
  n.Cstart = n.C;
  n.inbin = 0.f;
  if (n.j >= n.B) {
    n.j = n.B;
    n.S = 0.f;
    n.slope = 0.f;
    n.eleft = n.enext;
    n.enext = kFar;
    return;
  }
  if (n.j > 0) n.S -= n.v.mass(n.j - 1);
  n.slope = n.v.mass(n.j) * n.ih;
  n.eleft = n.enext;
  n.enext = (n.j + 1 < n.B) ? fmaf((float)(n.j + 1), n.h, n.lam) : n.end;
}

__device__ __forceinline__ float nwalk_G(const NWalk &n, float x) {
  return fmaxf(fmaf(-n.slope, x - n.eleft, n.S), 0.f);
}

// Partials of one centre vi (the point-mass path and the general walk in
// global memory): slot s (0 the centre, 1 + i neighbour i) and bin q go to
// out[(s * B + q) * ostride].
__device__ __noinline__ void hist_grad_vertex(const float *params, long long plane, long long vi,
                                 const long long *ni, const bool *present, int B, bool want_max,
                                 float wv, float *out, long long ostride) {
  const HistView cv{params + vi, plane, B, want_max};
  const float lo1 = cv.lo(), hi1 = cv.hi();
  float T[4];
  NWalk nw[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    T[i] = 1.f;
    if (!present[i]) continue;
    nw[i].v = HistView{params + ni[i], plane, B, want_max};
    float t = 0.f;
    for (int q = 0; q < B; ++q) t += nw[i].v.mass(q);
    T[i] = t;
  }
  float *own = out;  // slot 0
  if (lo1 == hi1) {
    // point-mass centre at c (total T1): P = T1 prod_n S_n(c)
    const float c = lo1;
    float S[4];
    float T1 = 0.f;
    for (int q = 0; q < B; ++q) T1 += cv.mass(q);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      S[i] = 1.f;
      if (!present[i]) continue;
      const HistView &v = nw[i].v;
      const float lo = v.lo(), hi = v.hi();
      if (lo == hi) {
        S[i] = lo > c ? T[i] : 0.f;
      } else if (c <= lo) {
        S[i] = T[i];
      } else if (c >= hi) {
        S[i] = 0.f;
      } else {
        const float h = (hi - lo) / (float)B;
        const int j = min(max((int)floorf((c - lo) / h), 0), B - 1);
        float Cs = 0.f;
        for (int q = 0; q < j; ++q) Cs += v.mass(q);
        const float fr = fminf(fmaxf((c - lo - (float)j * h) / h, 0.f), 1.f);
        S[i] = fmaxf(T[i] - Cs - fr * v.mass(j), 0.f);
      }
    }
    float lo4[4];
    loo4(S, lo4);
    const float Pn = lo4[0] * S[0];
    for (int q = 0; q < B; ++q) own[(long long)cv.orig(q) * ostride] = wv * Pn;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (!present[i]) continue;
      float *rn = out + (long long)(1 + i) * B * ostride;
      const HistView &v = nw[i].v;
      const float lo = v.lo(), hi = v.hi();
      const float h = (hi - lo) / (float)B;
      for (int q = 0; q < B; ++q) {
        float d;
        if (lo == hi) {
          d = c < lo ? 1.f : 0.f;
        } else {
          const float e0 = lo + (float)q * h, e1 = (q + 1 < B) ? lo + (float)(q + 1) * h : hi;
          d = c < e0 ? 1.f : (c >= e1 ? 0.f : (e1 - c) / (e1 - e0));
        }
        rn[(long long)v.orig(q) * ostride] = wv * T1 * d * lo4[i];
      }
    }
    return;
  }
  // walk over [0, W1] in the frame of lo1
  const float W1 = hi1 - lo1;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    if (!present[i]) continue;
    NWalk &n = nw[i];
    const float lo = n.v.lo(), hi = n.v.hi();
    n.lam = lo - lo1;
    n.B = (lo == hi) ? 0 : B;
    n.h = (lo == hi) ? 1.f : (hi - lo) / (float)B;
    n.ih = frcp(n.h);
    n.end = (lo == hi) ? n.lam : hi - lo1;
    n.j = -1;
    n.S = T[i];
    n.slope = 0.f;
    n.eleft = -kFar;
    n.enext = n.lam;
    n.C = n.Cstart = n.inbin = 0.f;
    n.T = T[i];
    float *rn = out + (long long)(1 + i) * B * ostride;
    if (n.B == 0) {
      // point mass: every mass partial is int_{x < c} pdf_1 prod_{m!=n} G; filled at the end
      continue;
    }
    for (int g = 0; g <= B && n.enext <= 0.f && n.j < n.B; ++g) nwalk_advance(n, rn, ostride, wv);
  }
  const float h1 = W1 / (float)B, ih1 = frcp(h1);
  int j1 = 0;
  float p1 = cv.mass(0) * ih1;
  float e1 = (B > 1) ? h1 : W1;
  float own_acc = 0.f;
  float x0 = 0.f;
  float Gl[4];
  float pmC[4] = {0, 0, 0, 0};  // point-mass neighbours: int up to their position
#pragma unroll
  for (int i = 0; i < 4; ++i) Gl[i] = present[i] ? nwalk_G(nw[i], 0.f) : 1.f;
  const int max_steps = 5 * (B + 2) + 4;
  for (int step = 0; step < max_steps; ++step) {
    float x1 = e1;
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (present[i]) x1 = fminf(x1, nw[i].enext);
    x1 = fminf(x1, W1);
    float Gr[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) Gr[i] = present[i] ? nwalk_G(nw[i], x1) : 1.f;
    const float len = x1 - x0;
    if (len > 0.f) {
      own_acc += len * bern_mean<4>(Gl, Gr);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        if (!present[i]) continue;
        float L3[4], R3[4];
        int q = 0;
#pragma unroll
        for (int m = 0; m < 4; ++m)
          if (m != i) {
            L3[q] = Gl[m];
            R3[q] = Gr[m];
            ++q;
          }
        const float A = len * p1 * bern_mean<3>(L3, R3);
        NWalk &n = nw[i];
        n.C += A;
        if (n.j >= 0 && n.j < n.B) {
          // within-bin factor (e_{j+1} - x) / h
          L3[3] = (n.enext - x0) * n.ih;
          R3[3] = (n.enext - x1) * n.ih;
          n.inbin += len * p1 * bern_mean<4>(L3, R3);
        }
      }
    }
    if (x1 >= W1) break;
    if (e1 <= x1) {
      own[(long long)cv.orig(j1) * ostride] = wv * own_acc * ih1;
      own_acc = 0.f;
      ++j1;
      p1 = (j1 < B) ? cv.mass(j1) * ih1 : 0.f;
      e1 = (j1 + 1 < B) ? (float)(j1 + 1) * h1 : W1;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (present[i] && nw[i].enext <= x1) {
        NWalk &n = nw[i];
        if (n.B == 0) pmC[i] = n.C;  // crossing a point mass
        nwalk_advance(n, out + (long long)(1 + i) * B * ostride, ostride, wv);
        Gr[i] = nwalk_G(n, x1);
      }
      Gl[i] = Gr[i];
    }
    x0 = x1;
  }
  if (j1 < B) own[(long long)cv.orig(j1) * ostride] = wv * own_acc * ih1;
  for (int q = j1 + 1; q < B; ++q) own[(long long)cv.orig(q) * ostride] = 0.f;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    if (!present[i]) continue;
    NWalk &n = nw[i];
    float *rn = out + (long long)(1 + i) * B * ostride;
    if (n.B == 0) {
      // point mass at lam: partial = int_{x < lam} ...; never crossed -> whole integral
      const float v = (n.j < 0) ? (n.lam <= 0.f ? 0.f : n.C) : pmC[i];
      for (int q = 0; q < B; ++q) rn[(long long)q * ostride] = wv * v;
      continue;
    }
    if (n.j >= 0 && n.j < n.B) rn[(long long)n.v.orig(n.j) * ostride] = wv * (n.Cstart + n.inbin);
    // bins entirely above the walk: the survival of the bin is 1 on [0, W1]
    for (int q = (n.j < 0 ? 0 : n.j + 1); q < n.B; ++q)
      rn[(long long)n.v.orig(q) * ostride] = wv * n.C;
  }
}

// ---------------------------------------------------------------------------
// histogram adjoint, tiled (non-degenerate centres)
//
// The partials of P_min = int pdf_1 prod_n G_n (mixture form) are
//   own bin j:        (1/h1) int_{bin j} prod_n G_n
//   neighbour n, k:   int pdf_1 S_nk LOO_n,  LOO_n = prod_{m != n} G_m,
// with S_nk = 1 below bin k of n, (e_{k+1} - x)/h_n on it, 0 above.  One
// merge walk (the forward's walkers over shared-memory tail tables) carries,
// per neighbour, the running integral C_n = int_0^x pdf_1 LOO_n and the
// in-bin integral of its current bin; leaving bin k stores C_n(e_k) + in-bin.
// On a piece every factor is linear, so the products (degree <= 4) are
// integrated exactly by the 3-point Gauss-Legendre rule at the same three
// nodes for all of them; the leave-one-out products come from prefix and
// suffix products at the nodes.  No branch depends on the lane's data except
// the end of the walk.  The maximum is the minimum of the mirrored problem
// (-X; bins reversed), staged mirrored.

constexpr int kGradTY = 16;

template <int HALO>
__device__ __forceinline__ void hist_grad_walk(const float *S0, int l, const int *nl,
                                               const bool *present, int B, bool mirrored,
                                               float wv, float *rows, long long plane,
                                               long long gi) {
  const float lo1 = S0[l - 2 * HALO], hi1 = S0[l - HALO];
  const float W1 = hi1 - lo1;
  auto row = [&](int slot, int q) -> float * {
    return rows + ((long long)slot * B + (mirrored ? B - 1 - q : q)) * plane + gi;
  };
  if (!(W1 <= 1e38f)) {  // a support too wide for the walk's frame: no partials
    for (int sl = 0; sl < 5; ++sl)
      if (sl == 0 || present[sl - 1])
        for (int q = 0; q < B; ++q) *row(sl, q) = __int_as_float(0x7fc00000);
    return;
  }
  const float Bf = (float)B;
  HistSeg nw[4];
  float T[4];
  int kb[4];  // bin of neighbour i after the seek
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    HistSeg &h = nw[i];
    if (!present[i]) {
      h.init_absent(l, Bf);
      T[i] = 1.f;
      kb[i] = -1;
      continue;
    }
    const float lo = S0[nl[i] - 2 * HALO], hi = S0[nl[i] - HALO];
    T[i] = S0[nl[i] + (2 + B) * HALO];
    h.init<HALO>(S0, nl[i], lo - lo1, lo == hi ? 0.f : (hi - lo) / Bf, T[i]);
    h.seek0<HALO>(S0, B);
    kb[i] = (int)h.kf - 1;
    // bins entirely below the centre's support: their survival is 0 there
    for (int q = 0; q < min(kb[i], B); ++q) *row(1 + i, q) = 0.f;
  }
  const float h1 = W1 / Bf, ih1 = frcp(h1);
  int addr_c = l + 2 * HALO;
  float kcf = 1.f;
  float sc = S0[l], scn = S0[l + HALO];
  float dens = (sc - scn) * ih1;
  float nxc = B > 1 ? h1 : W1;
  int jc = 0;
  float Gl[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) Gl[i] = nw[i].G(0.f);
  float own = 0.f, C[4] = {0.f, 0.f, 0.f, 0.f}, Cs[4] = {0.f, 0.f, 0.f, 0.f};
  float inb[4] = {0.f, 0.f, 0.f, 0.f};
  // 3-point Gauss-Legendre on [0, 1]
  const float t0 = 0.11270166537925831f, t2 = 0.88729833462074169f;
  const float wE = 5.f / 18.f, wM = 8.f / 18.f;
  float x0 = 0.f;
  const int max_steps = 5 * (B + 2) + 4;
  for (int step = 0; step < max_steps && x0 < W1; ++step) {
    float x1 = fminf(fminf(nw[0].nx, nw[1].nx), fminf(nw[2].nx, nw[3].nx));
    x1 = fmaxf(fminf(x1, nxc), x0);
    float Gr[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) Gr[i] = nw[i].G(x1);
    const float len = x1 - x0, a = len * dens;
    // factor values at the nodes
    float f[3][4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float d = Gr[i] - Gl[i];
      f[0][i] = fmaf(d, t0, Gl[i]);
      f[1][i] = fmaf(d, 0.5f, Gl[i]);
      f[2][i] = fmaf(d, t2, Gl[i]);
    }
    // in-bin weights (e_next - x) / h of each neighbour inside a bin
    float wl[4], wr[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const bool in = nw[i].kf >= 1.f && nw[i].kf <= Bf;
      wl[i] = in ? (nw[i].nx - x0) * nw[i].invh : 0.f;
      wr[i] = in ? (nw[i].nx - x1) * nw[i].invh : 0.f;
    }
    float full = 0.f, loo[4] = {0.f, 0.f, 0.f, 0.f}, loow[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const float wq = q == 1 ? wM : wE, tq = q == 0 ? t0 : (q == 1 ? 0.5f : t2);
      const float p2 = f[q][0] * f[q][1], p3 = p2 * f[q][2];
      const float s2 = f[q][3] * f[q][2], s3 = s2 * f[q][1];
      const float L[4] = {s3, f[q][0] * s2, p2 * f[q][3], p3};
      full = fmaf(wq, p3 * f[q][3], full);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        loo[i] = fmaf(wq, L[i], loo[i]);
        loow[i] = fmaf(wq * fmaf(wr[i] - wl[i], tq, wl[i]), L[i], loow[i]);
      }
    }
    own = fmaf(len, full, own);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      C[i] = fmaf(a, loo[i], C[i]);
      inb[i] = fmaf(a, loow[i], inb[i]);
    }
    // crossings: a neighbour leaving bin k stores its partial
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int k = (int)nw[i].kf - 1;  // the bin being left, if it crosses
      const bool c = nw[i].step<HALO>(S0, x1, Bf);
      if (c && present[i] && k >= 0 && k < B) *row(1 + i, k) = wv * (Cs[i] + inb[i]);
      Cs[i] = c ? C[i] : Cs[i];
      inb[i] = c ? 0.f : inb[i];
      Gl[i] = c ? nw[i].s : Gr[i];
    }
    {
      const bool c = nxc <= x1;
      if (c && jc < B) *row(0, jc) = wv * own * ih1;
      own = c ? 0.f : own;
      jc += c ? 1 : 0;
      const float t = S0[addr_c];
      sc = c ? scn : sc;
      scn = c ? t : scn;
      addr_c += c ? HALO : 0;
      kcf = c ? kcf + 1.f : kcf;
      nxc = c ? (kcf < Bf ? kcf * h1 : (kcf == Bf ? W1 : kFar)) : nxc;
      dens = (sc - scn) * ih1;
    }
    x0 = x1;
  }
  for (int q = jc; q < B; ++q) *row(0, q) = 0.f;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    if (!present[i]) continue;
    const int k = (int)nw[i].kf - 1;
    if (k >= 0 && k < B) *row(1 + i, k) = wv * (Cs[i] + inb[i]);
    // bins above the walk: their survival is 1 on the whole support
    for (int q = max(k + 1, 0); q < B; ++q) *row(1 + i, q) = wv * C[i];
  }
}

template <int TYv>
__global__ void __launch_bounds__(NTHREADS, 2)
    hist_partials_tile(Field f, int tiles_x, int want_max, const float *__restrict__ weight,
                       float *__restrict__ rows) {
  extern __shared__ float sm[];
  constexpr int TY = TYv, TX = 32, HY = TY + 2, HX = TX + 2, HALO = HY * HX;
  const int B = f.B;
  const long long plane = f.plane;
  const int ty0 = f.y0 + ((int)blockIdx.x / tiles_x) * TY, tx0 = ((int)blockIdx.x % tiles_x) * TX;
  const int ylim = min(f.H, f.y1 + 1);
  // stage the parameters (mirrored for the maximum: -X on [-hi, -lo], bins reversed)
  for (int l = threadIdx.x; l < HALO; l += NTHREADS) {
    const int r = l / HX, c = l - r * HX;
    const int gy = ty0 + r - 1, gx = tx0 + c - 1;
    if (gy < 0 || gy >= ylim || gx < 0 || gx >= f.W) continue;
    const long long gi = (long long)gy * f.W + gx;
    const float a = f.params[gi], b = f.params[plane + gi];
    sm[l] = want_max ? -b : a;
    sm[HALO + l] = want_max ? -a : b;
    for (int q = 0; q < B; ++q)
      sm[(2 + q) * HALO + l] = f.params[(long long)(2 + (want_max ? B - 1 - q : q)) * plane + gi];
  }
  __syncthreads();
  for (int l = threadIdx.x; l < HALO; l += NTHREADS) hist_tail_table<HALO>(sm, l, B);
  __syncthreads();
  const unsigned short *order = hist_order<TY, HALO>(f, sm, ty0, tx0);
  const float *S0 = sm + 2 * HALO;
  for (int it = threadIdx.x; it < TY * TX; it += NTHREADS) {
    const int j = it / NTHREADS, w = threadIdx.x >> 5, nwp = NTHREADS / 32;
    const int v = order[(j * nwp + ((j & 1) ? nwp - 1 - w : w)) * 32 + (threadIdx.x & 31)];
    const int r = v / TX + 1, c = v % TX + 1;
    const int gy = ty0 + r - 1, gx = tx0 + c - 1;
    if (gy >= f.y1 || gx >= f.W) continue;
    const int l = r * HX + c;
    const long long gi = (long long)gy * f.W + gx;
    bool present[4];
    int nl[4];
    long long ni[4];
    int k = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int yy = gy + kDy[i], xx = gx + kDx[i];
      present[i] = (yy >= 0 && yy < f.H && xx >= 0 && xx < f.W);
      nl[i] = l + kDy[i] * HX + kDx[i];
      ni[i] = present[i] ? (long long)yy * f.W + xx : gi;
      k += present[i];
    }
    int st = (int)sm[(5 + B) * HALO + l];
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (present[i]) st |= (int)sm[(5 + B) * HALO + nl[i]] & (V_NONFINITE | V_BAD);
    const float wv = weight[gi];
    if ((st & (V_NONFINITE | V_BAD)) || (f.boundary == 1 && k < 4)) {
      const float fill = (st & (V_NONFINITE | V_BAD)) ? qnan() : 0.f;
      for (int sl = 0; sl < 5; ++sl)
        for (int q = 0; q < B; ++q) rows[((long long)sl * B + q) * plane + gi] = fill;
      continue;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (!present[i])
        for (int q = 0; q < B; ++q) rows[((long long)(1 + i) * B + q) * plane + gi] = 0.f;
    if (sm[l] == sm[HALO + l]) {
      // a point-mass centre: the product of tails (global-memory path)
      hist_grad_vertex(f.params, plane, gi, ni, present, B, want_max != 0, wv, rows + gi, plane);
    } else {
      hist_grad_walk<HALO>(S0, l, nl, present, B, want_max != 0, wv, rows, plane, gi);
    }
  }
}

// ---------------------------------------------------------------------------
// histogram adjoint over per-bin rows (at most RB bins, non-degenerate
// centres): the forward's row tables and walkers (device.cuh), built here
// from the parameters, mirrored for the maximum as above.  Per piece all
// factors are linear; the own product (degree 4), each leave-one-out product
// LOO_n (degree 3) and LOO_n times the in-bin weight (e_{k+1} - x) / h_n
// (degree 4) are integrated exactly by the 3-point Gauss-Legendre rule at
// shared nodes, the leave-one-out products from pair products.  Every lane
// runs the same steps; row reads at crossings are predicated, partials are
// stored when a neighbour leaves a bin (or the centre leaves one of its own).

// the bin width of the rows of a support of width w (as hist_rows_build)
__device__ __forceinline__ float rows_bin_width(float w, int B) {
  return (B & (B - 1)) == 0 ? w * (1.f / (float)B) : w / (float)B;
}

// a 4-byte global store that happens only where p holds (one predicated
// instruction, no branch); the address is not touched where p is false
__device__ __forceinline__ void stg_if(bool p, float *ptr, float v) {
  asm volatile(
      "{\n .reg .pred q;\n setp.ne.b32 q, %2, 0;\n @q st.global.f32 [%0], %1;\n}" ::"l"(ptr),
      "f"(v), "r"((int)p)
      : "memory");
}

// One neighbour's crossing in the adjoint walk, without a branch: if its
// next edge nx is at or below x1 -- store `val` (its partial of the bin it
// leaves) at optr if it was inside a bin (ihe != 0), move optr to the next
// bin's partial, restart Cs = C and inb = 0, read the next row into r (and
// advance addr), and set ihe to 1/h inside a bin (ih) or 0 beyond the
// support (the beyond row's next edge is kFar).
template <unsigned stride>
__device__ __forceinline__ void adj_cross(float nx, float x1, float val, float *&optr,
                                          long long qs, float C, float &Cs, float &inb,
                                          uint32_t &addr, float4 &r, float ih, float &ihe) {
  asm volatile(
      "{\n .reg .pred q, e, n;\n"
      " setp.le.f32 q, %9, %10;\n"
      " setp.ne.and.f32 e, %8, 0f00000000, q;\n"
      " @e st.global.f32 [%4], %11;\n"
      " @q add.s64 %4, %4, %12;\n"
      " @q mov.f32 %6, %13;\n"
      " @q mov.f32 %7, 0f00000000;\n"
      " @q ld.shared.v4.f32 {%0, %1, %2, %3}, [%5];\n"
      " @q add.u32 %5, %5, %14;\n"
      " setp.lt.and.f32 n, %3, 0f7E61B1E6, q;\n"
      " @q selp.f32 %8, %15, 0f00000000, n;\n}"
      : "+f"(r.x), "+f"(r.y), "+f"(r.z), "+f"(r.w), "+l"(optr), "+r"(addr), "+f"(Cs),
        "+f"(inb), "+f"(ihe)
      : "f"(nx), "f"(x1), "f"(val), "l"(qs * (long long)sizeof(float)), "f"(C), "n"(stride),
        "f"(ih)
      : "memory");
}

template <int HALO, int RS>
__device__ __forceinline__ void hist_adj_walk(const float *sm, const float4 *R4, int l,
                                              const int *nl, const bool *present, int B,
                                              bool mirrored, float wv, float *outc,
                                              long long ostride) {
  const float lo1 = sm[l], hi1 = sm[HALO + l];
  const float W1 = hi1 - lo1;
  // partial of slot s (0 centre, 1 + i neighbour i) and bin q (mirrored:
  // the bins are reversed) at outc[(s * B + q) * ostride]
  const long long qstride = mirrored ? -ostride : ostride;
  float *const out0 = outc + (mirrored ? (long long)(B - 1) * ostride : 0);
  auto out = [&](int slot, int q) -> float * {
    return out0 + (long long)slot * B * ostride + (long long)q * qstride;
  };
  if (!(W1 <= 1e38f)) {  // a support too wide for the walk's frame: no partials
    for (int s = 0; s < 5; ++s)
      if (s == 0 || present[s - 1])
        for (int q = 0; q < B; ++q) *out(s, q) = __int_as_float(0x7fc00000);
    return;
  }
  HistRowWalker nw[4];
  // per neighbour: C = int_0^x pdf_1 LOO, Cs = C at the start of its current
  // bin, inb = the in-bin integral of that bin, ihe = 1/h inside a bin (0
  // before or beyond its support, and for a point mass), kb = its bin (-1
  // before the support, B beyond; a point mass moves from -1 to 0 at its
  // position and stays there)
  float2 C01 = {0.f, 0.f}, C23 = {0.f, 0.f}, inb01 = {0.f, 0.f}, inb23 = {0.f, 0.f};
  float Cs[4] = {0.f, 0.f, 0.f, 0.f}, ih[4], ihe[4];
  int kb[4];
  bool pm[4];
  float *optr[4];  // the partial of neighbour i's current bin (used inside a bin only)
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    pm[i] = false;
    ih[i] = ihe[i] = 0.f;
    optr[i] = outc;
    if (!present[i]) {
      nw[i].init_absent();
      kb[i] = B;
      continue;
    }
    const float lo = sm[nl[i]], hi = sm[HALO + nl[i]];
    pm[i] = lo == hi;
    const float h = pm[i] ? 0.f : rows_bin_width(hi - lo, B);
    ih[i] = pm[i] ? 0.f : frcp(h);
    nw[i].init(R4 + nl[i], lo - lo1, sm[2 * HALO + nl[i]]);
    const int j = nw[i].seek0<RS>(R4 + nl[i], B, h);
    kb[i] = j - 1;
    ihe[i] = (kb[i] >= 0 && kb[i] < B) ? ih[i] : 0.f;
    optr[i] = out(1 + i, 0) + (long long)kb[i] * qstride;
    // bins entirely below the centre's support: their survival is 0 there
    if (!pm[i])
      for (int q = 0; q < j - 1; ++q) *out(1 + i, q) = 0.f;
  }
  const float ih1 = frcp(rows_bin_width(W1, B));
  uint32_t addr_c = static_cast<uint32_t>(__cvta_generic_to_shared(R4 + l + RS)) + 8u;
  float2 dc;  // (density, next edge) of the centre's current bin
  {
    const float4 t = R4[l];
    dc = make_float2(t.z, t.w);
  }
  int jc = 0;
  float own = 0.f;
  const float wvh = wv * ih1;
  float x0 = 0.f;
  const int max_steps = 5 * (B + 1) + 4;
#pragma unroll 1
  for (int step = 0; step < max_steps && x0 < W1; ++step) {
    float e[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) e[i] = nw[i].nx();
    const float x1 = fminf(fminf(fminf(e[0], e[1]), fminf(e[2], e[3])), dc.y);
    const float d = x1 - x0, a = d * dc.x;
    // the four factors in the pairs (0, 2) and (1, 3): values at x0 (g0),
    // their change over the piece (dg); in-bin weights (e - x) / h at x0
    // (w0) and their change (dw)
    const float2 gA = make_float2(nw[0].r.x, nw[2].r.x), gB = make_float2(nw[1].r.x, nw[3].r.x);
    const float2 sA = make_float2(-nw[0].r.z, -nw[2].r.z), sB = make_float2(-nw[1].r.z, -nw[3].r.z);
    const float2 dd = make_float2(d, d);
    const float2 dgA = __fmul2_rn(sA, dd), dgB = __fmul2_rn(sB, dd);
    const float2 ihA = make_float2(ihe[0], ihe[2]), ihB = make_float2(ihe[1], ihe[3]);
    const float2 w0A = __fmul2_rn(__fadd2_rn(make_float2(e[0], e[2]), make_float2(-x0, -x0)), ihA);
    const float2 w0B = __fmul2_rn(__fadd2_rn(make_float2(e[1], e[3]), make_float2(-x0, -x0)), ihB);
    const float2 dwA = __fmul2_rn(ihA, make_float2(-d, -d)), dwB = __fmul2_rn(ihB, make_float2(-d, -d));
    // 3-point Gauss-Legendre on [0, 1]: nodes 1/2 -+ sqrt(3/5)/2, weights 5/18, 8/18
    float so = 0.f;
    float2 scA = {0.f, 0.f}, scB = {0.f, 0.f}, siA = {0.f, 0.f}, siB = {0.f, 0.f};
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const float tq = q == 0 ? 0.11270166537925831f : (q == 1 ? 0.5f : 0.88729833462074169f);
      const float wq = q == 1 ? 8.f / 18.f : 5.f / 18.f;
      const float2 tt = make_float2(tq, tq), ww = make_float2(wq, wq);
      const float2 fA = __ffma2_rn(dgA, tt, gA), fB = __ffma2_rn(dgB, tt, gB);  // (f0,f2),(f1,f3)
      const float2 P = __fmul2_rn(fA, fB);                                       // (p01, p23)
      const float2 Ps = make_float2(P.y, P.x);                                   // (p23, p01)
      // leave-one-out products: (L0, L2) = (f1 p23, f3 p01), (L1, L3) = (f0 p23, f2 p01)
      const float2 wLA = __fmul2_rn(ww, __fmul2_rn(fB, Ps));
      const float2 wLB = __fmul2_rn(ww, __fmul2_rn(fA, Ps));
      so = fmaf(wq, P.x * P.y, so);
      scA = __fadd2_rn(scA, wLA);
      scB = __fadd2_rn(scB, wLB);
      siA = __ffma2_rn(__ffma2_rn(dwA, tt, w0A), wLA, siA);
      siB = __ffma2_rn(__ffma2_rn(dwB, tt, w0B), wLB, siB);
    }
    own = fmaf(d, so, own);
    const float2 aa = make_float2(a, a);
    // back to the neighbour order (0, 1) and (2, 3)
    C01 = __ffma2_rn(aa, make_float2(scA.x, scB.x), C01);
    C23 = __ffma2_rn(aa, make_float2(scA.y, scB.y), C23);
    inb01 = __ffma2_rn(aa, make_float2(siA.x, siB.x), inb01);
    inb23 = __ffma2_rn(aa, make_float2(siA.y, siB.y), inb23);
    float C[4] = {C01.x, C01.y, C23.x, C23.y}, inb[4] = {inb01.x, inb01.y, inb23.x, inb23.y};
    // crossings: a neighbour leaving bin k stores its partial C(e_k) + in-bin
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      nw[i].r.x = fmaf(-nw[i].r.z, d, nw[i].r.x);
      adj_cross<(unsigned)(RS * 16)>(e[i], x1, wv * (Cs[i] + inb[i]), optr[i], qstride, C[i],
                                     Cs[i], inb[i], nw[i].addr, nw[i].r, ih[i], ihe[i]);
    }
    inb01 = make_float2(inb[0], inb[1]);
    inb23 = make_float2(inb[2], inb[3]);
    {
      const bool cr = dc.y <= x1;
      stg_if(cr && jc < B, out(0, jc), wvh * own);
      own = cr ? 0.f : own;
      jc += cr ? 1 : 0;
      lds64_cross<(unsigned)(RS * 16)>(dc.y, x1, addr_c, dc);
    }
    x0 = x1;
  }
  if (jc < B) *out(0, jc) = wvh * own;
  for (int q = jc + 1; q < B; ++q) *out(0, q) = 0.f;
  const float C[4] = {C01.x, C01.y, C23.x, C23.y}, inb[4] = {inb01.x, inb01.y, inb23.x, inb23.y};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    if (!present[i]) continue;
    kb[i] = (int)((optr[i] - out(1 + i, 0)) / qstride);  // the bin the walker ended in
    if (kb[i] >= 0 && kb[i] < B) *out(1 + i, kb[i]) = wv * (Cs[i] + inb[i]);
    // bins entirely above the walk: their survival is 1 on the whole support
    // (a point mass: every mass partial is the integral below its position,
    // Cs once it has been reached, else the whole integral)
    const float above = pm[i] && kb[i] >= 0 ? Cs[i] : C[i];
    for (int q = (kb[i] < 0 ? 0 : kb[i] + 1); q < B; ++q) *out(1 + i, q) = wv * above;
  }
}

// Tiles of 8 x 32 centres, one per CTA.  Each CTA claims one of nslots
// scratch blocks of partials [5][B][256] (slot, bin, centre of the tile) in
// global memory for its lifetime (a flag per block, taken with an atomic
// compare-and-swap and released at the end), so the blocks -- as many as the
// CTAs that can be resident at once, with room to spare -- are rewritten
// tile after tile and stay in L2.  After a tile's walks the same
// CTA sums, for every vertex u of the tile, its own partials and those that
// its neighbours inside the tile wrote about it -- in the fixed order own,
// e, n, w, s -- into grad.  The partials about vertices outside the tile
// (the n slot of the top row, s of the bottom row, w of the left column, e
// of the right column) go to the tile's ring (N, S: B x 32; W, E: B x 8 each,
// 80 B floats), which hist_adj_fixup adds to the edge vertices of the
// neighbouring tiles afterwards.  Deterministic, no atomics.
constexpr int kAdjTY = 8, kAdjTV = kAdjTY * 32, kAdjRing = 80;

// The partials of one centre (gy, gx), staged at l, into out[(s * B + q) *
// kAdjTV]: NaN or 0 for a centre whose probability is invalid or 0 by the
// boundary rule, 0 for absent neighbours, else the walk (or the point-mass
// path).
template <int HALO, int RS>
__device__ __forceinline__ void hist_adj_centre(const Field &f, const float *sm, const float4 *R4,
                                             int gy, int gx, int l, bool mirrored,
                                             const float *__restrict__ weight, float *out) {
  constexpr int HX = 34;
  const int B = f.B;
  const long long plane = f.plane;
  const long long gi = (long long)gy * f.W + gx;
  bool present[4];
  int nl[4];
  long long ni[4];
  int k = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int yy = gy + kDy[i], xx = gx + kDx[i];
    present[i] = (yy >= 0 && yy < f.H && xx >= 0 && xx < f.W);
    nl[i] = l + kDy[i] * HX + kDx[i];
    ni[i] = present[i] ? (long long)yy * f.W + xx : gi;
    k += present[i];
  }
  int st = (int)sm[3 * HALO + l];
#pragma unroll
  for (int i = 0; i < 4; ++i)
    if (present[i]) st |= (int)sm[3 * HALO + nl[i]] & (V_NONFINITE | V_BAD);
  const float wv = weight[gi];
  if ((st & (V_NONFINITE | V_BAD)) || (f.boundary == 1 && k < 4)) {
    const float fill = (st & (V_NONFINITE | V_BAD)) ? qnan() : 0.f;
    for (int q = 0; q < 5 * B; ++q) out[q * kAdjTV] = fill;
    return;
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
    if (!present[i])
      for (int q = 0; q < B; ++q) out[((1 + i) * B + q) * kAdjTV] = 0.f;
  if (sm[l] == sm[HALO + l]) {
    // a point-mass centre: the product of tails (global-memory path)
    hist_grad_vertex(f.params, plane, gi, ni, present, B, mirrored, wv, out, kAdjTV);
  } else {
    hist_adj_walk<HALO, RS>(sm, R4, l, nl, present, B, mirrored, wv, out, kAdjTV);
  }
}

template <int RB>
__global__ void __launch_bounds__(NTHREADS, 2)
    hist_adj_tile(Field f, int tiles_x, int want_max, const float *__restrict__ weight,
                  int *__restrict__ flags, int nslots, float *__restrict__ scratch,
                  float *__restrict__ ring, float *__restrict__ grad) {
  extern __shared__ __align__(16) float smem[];
  constexpr int TY = kAdjTY, TX = 32, HY = TY + 2, HX = TX + 2, HALO = HY * HX, TV = kAdjTV;
  constexpr int RS = hist_r4_stride(HALO);
  static_assert(TV == NTHREADS, "one centre and one gathered vertex per thread");
  const int B = f.B;
  const long long plane = f.plane;
  float4 *R4 = reinterpret_cast<float4 *>(smem);
  float *sm = smem + 4 * hist_r4_rows(B) * RS;  // lo, hi, T, status
  const bool mirrored = want_max != 0;
  const int tile = blockIdx.x;
  const int ty0 = f.y0 + (tile / tiles_x) * TY, tx0 = (tile % tiles_x) * TX;
  const int ylim = min(f.H, f.y1 + 1);
  // claim a scratch block: try the ones after 2 x (this SM's index) first;
  // the polls are bounded (a block is released when its CTA ends)
  __shared__ int slot_sm;
  if (threadIdx.x == 0) {
    unsigned smid;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
    int got = -1;
    for (int it = 0; it < (1 << 22) && got < 0; ++it) {
      for (int k = 0; k < nslots && got < 0; ++k) {
        const int sl = (int)((2u * smid + (unsigned)k) % (unsigned)nslots);
        if (atomicCAS(flags + sl, 0, 1) == 0) got = sl;
      }
      if (got < 0) __nanosleep(1000);
    }
    __threadfence();
    slot_sm = got;
  }
  hist_rows_from_params_tile<HALO, RS, RB, HX, true>(f, sm, R4, ty0, tx0, ylim, B, mirrored);
  __syncthreads();
  const int slot = slot_sm;
  const int v = threadIdx.x;
  const int r = v / TX + 1, c = v % TX + 1;
  const int gy = ty0 + r - 1, gx = tx0 + c - 1;
  const bool live = gy < f.y1 && gx < f.W;
  if (slot < 0) {  // no scratch block within the bound: NaN gradient
    if (live)
      for (int q = 0; q < B; ++q) grad[(long long)q * plane + (long long)gy * f.W + gx] = qnan();
    return;
  }
  float *const sc = scratch + (long long)slot * 5 * B * TV;
  // walks: one centre per thread, partials into the scratch block
  if (live) hist_adj_centre<HALO, RS>(f, sm, R4, gy, gx, r * HX + c, mirrored, weight, sc + v);
  __syncthreads();
  // gather: vertex u = v of the tile
  if (live) {
    const long long gi = (long long)gy * f.W + gx;
    const int lr = r - 1, lc = c - 1;  // local row and column
    bool in_tile[4];
    int vn[4];
#pragma unroll
    for (int d = 0; d < 4; ++d) {
      const int yy = gy + kDy[d], xx = gx + kDx[d];
      const int rr = lr + kDy[d], cc = lc + kDx[d];
      in_tile[d] = yy >= 0 && yy < f.y1 && xx >= 0 && xx < f.W && rr >= 0 && rr < TY &&
                   cc >= 0 && cc < TX;
      vn[d] = rr * TX + cc;
    }
    float *ring_t = ring + (long long)tile * kAdjRing * B;
    // four bins at a time: every read of the block first (independent L2
    // reads in flight together), then the sums and stores
    for (int q0 = 0; q0 < B; q0 += 4) {
      float own[4], nbv[4][4], rv[4][4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int q = min(q0 + j, B - 1);
        own[j] = sc[q * TV + v];
#pragma unroll
        for (int d = 0; d < 4; ++d) {
          const int opp = (d + 2) & 3;
          nbv[j][d] = in_tile[d] ? sc[((1 + opp) * B + q) * TV + vn[d]] : 0.f;
          rv[j][d] = sc[((1 + d) * B + q) * TV + v];
        }
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int q = q0 + j;
        if (q >= B) break;
        float acc = own[j];
#pragma unroll
        for (int d = 0; d < 4; ++d)
          if (in_tile[d]) acc += nbv[j][d];
        grad[(long long)q * plane + gi] = acc;
        // this centre's partials about vertices of other tiles
        if (lr == 0) ring_t[q * 32 + lc] = rv[j][1];               // n
        if (lr == TY - 1) ring_t[(B + q) * 32 + lc] = rv[j][3];    // s
        if (lc == 0) ring_t[64 * B + q * 8 + lr] = rv[j][2];       // w
        if (lc == TX - 1) ring_t[72 * B + q * 8 + lr] = rv[j][0];  // e
      }
    }
  }
  // every read of the block is done: release it
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicExch(flags + slot, 0);
  }
}

// Adds to every vertex on the edge of a tile the partials that centres of
// the neighbouring tiles wrote about it (their rings), in the order e, n,
// w, s: one thread per (tile, edge position); edge positions 0..31 top row,
// 32..63 bottom row, 64..69 left column rows 1..6, 70..75 right column.
__global__ void __launch_bounds__(256) hist_adj_fixup(Field f, int tiles_x, int ntiles,
                                                      const float *__restrict__ ring,
                                                      float *__restrict__ grad) {
  constexpr int TY = kAdjTY, TX = 32, NP = 2 * TX + 2 * (TY - 2);
  const int B = f.B;
  const long long plane = f.plane;
  const long long total = (long long)ntiles * NP;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int tile = (int)(t / NP), p = (int)(t % NP);
    const int tr = tile / tiles_x, tc = tile % tiles_x;
    int lr, lc;
    if (p < TX) { lr = 0; lc = p; }
    else if (p < 2 * TX) { lr = TY - 1; lc = p - TX; }
    else if (p < 2 * TX + TY - 2) { lr = 1 + (p - 2 * TX); lc = 0; }
    else { lr = 1 + (p - 2 * TX - (TY - 2)); lc = TX - 1; }
    const int gy = f.y0 + tr * TY + lr, gx = tc * TX + lc;
    if (gy >= f.y1 || gx >= f.W) continue;
    const long long gi = (long long)gy * f.W + gx;
    // the neighbouring tile's ring entry in direction d, if that neighbour
    // is in the grid but outside this tile
    const float *src[4];
    bool have[4];
#pragma unroll
    for (int d = 0; d < 4; ++d) {
      const int yy = gy + kDy[d], xx = gx + kDx[d];
      const int rr = lr + kDy[d], cc = lc + kDx[d];
      have[d] = yy >= 0 && yy < f.y1 && xx >= 0 && xx < f.W && !(rr >= 0 && rr < TY && cc >= 0 && cc < TX);
      src[d] = ring;
      if (!have[d]) continue;
      const int nt = tile + (rr < 0 ? -tiles_x : (rr >= TY ? tiles_x : 0)) + (cc < 0 ? -1 : (cc >= TX ? 1 : 0));
      const float *rt = ring + (long long)nt * kAdjRing * B;
      if (d == 0) src[d] = rt + 64 * B + lr;        // e: the right tile's w ring (its left column)
      else if (d == 1) src[d] = rt + B * 32 + lc;   // n: the upper tile's s ring (its bottom row)
      else if (d == 2) src[d] = rt + 72 * B + lr;   // w: the left tile's e ring (its right column)
      else src[d] = rt + lc;                        // s: the lower tile's n ring (its top row)
    }
    // eight parameters at a time, every read first (the compiler cannot
    // tell the planes' addresses apart, so a read after a store would wait
    // for it), then the sums in the order grad, e, n, w, s and the stores
    // (launched for at most 16 parameters: histograms of <= 16 bins, and
    // the two of uniform / Epanechnikov)
#pragma unroll
    for (int q0 = 0; q0 < 16; q0 += 8) {
      if (q0 >= B) break;
      float gv[8], rv[8][4];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int q = q0 + j;
        if (q < B) {
          gv[j] = grad[(long long)q * plane + gi];
#pragma unroll
          for (int d = 0; d < 4; ++d)
            rv[j][d] = have[d] ? src[d][(d == 0 || d == 2) ? q * 8 : q * 32] : 0.f;
        }
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int q = q0 + j;
        if (q < B) {
          float acc = gv[j];
#pragma unroll
          for (int d = 0; d < 4; ++d)
            if (have[d]) acc += rv[j][d];
          grad[(long long)q * plane + gi] = acc;
        }
      }
    }
  }
}

// Uniform and Epanechnikov adjoint, tiled as hist_adj_tile: one CTA per
// 8 x 32 tile, one centre per thread.  A centre's ten weighted partials
// (slot 0 the centre, 1 + i neighbour i; parameter q of two) go to shared
// memory; after the tile's centres are done each thread sums, for its own
// vertex u, u's partials and those its neighbours inside the tile wrote
// about u, in the fixed order own, e, n, w, s, and writes grad.  The
// partials about vertices of other tiles go to the tile's ring (80 x 2
// floats, the layout of hist_adj_tile's ring), which hist_adj_fixup adds to
// them afterwards.  No global scratch besides the ring, no atomics.
template <int MODEL>
__global__ void __launch_bounds__(NTHREADS) closed_adj_tile(Field f, int tiles_x, int want_max,
                                                            const float *__restrict__ weight,
                                                            float *__restrict__ ring,
                                                            float *__restrict__ grad) {
  static_assert(MODEL == kUniform || MODEL == kEpan, "two parameters per vertex");
  constexpr int TY = kAdjTY, TX = 32, TV = kAdjTV, Q = 2;
  __shared__ float sc[5 * Q * TV];
  const long long plane = f.plane;
  const int tile = blockIdx.x;
  const int ty0 = f.y0 + (tile / tiles_x) * TY, tx0 = (tile % tiles_x) * TX;
  const int v = threadIdx.x, lr = v / TX, lc = v % TX;
  const int y = ty0 + lr, x = tx0 + lc;
  const bool live = y < f.y1 && x < f.W;
  if (live) {
    const long long vi = (long long)y * f.W + x;
    bool present[4];
    long long ni[4];
    int k = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int yy = y + kDy[i], xx = x + kDx[i];
      present[i] = (yy >= 0 && yy < f.H && xx >= 0 && xx < f.W);
      ni[i] = present[i] ? (long long)yy * f.W + xx : vi;
      k += present[i];
    }
    // validity of every participant
    bool bad = false;
#pragma unroll
    for (int t = 0; t < 5; ++t) {
      if (t > 0 && !present[t - 1]) continue;
      const long long u = t == 0 ? vi : ni[t - 1];
      const float a = f.params[u], b = f.params[plane + u];
      if (!isfinite(a) || !isfinite(b)) bad = true;
      else if (MODEL == kEpan ? (b < 0.f) : (a > b)) bad = true;
    }
    float g[5 * Q];
    if (bad || (f.boundary == 1 && k < 4)) {
      const float fill = bad ? qnan_b() : 0.f;
#pragma unroll
      for (int t = 0; t < 5 * Q; ++t) g[t] = fill;
    } else {
      const float wv = weight[vi];
      float an[4], bn[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        an[i] = f.params[ni[i]];
        bn[i] = f.params[plane + ni[i]];
      }
      if constexpr (MODEL == kUniform) {
        UniGrad r;
        uniform_grad_vertex(f.params[vi], f.params[plane + vi], an, bn, present, want_max != 0,
                            r);
        g[0] = wv * r.ga;
        g[1] = wv * r.gb;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          g[2 + 2 * i] = wv * r.na[i];
          g[3 + 2 * i] = wv * r.nb[i];
        }
      } else {
        EpanGrad r;
        epan_grad_vertex(f.params[vi], f.params[plane + vi], an, bn, present, want_max != 0, r);
        g[0] = wv * r.gm;
        g[1] = wv * r.gw;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          g[2 + 2 * i] = wv * r.nm[i];
          g[3 + 2 * i] = wv * r.nw[i];
        }
      }
    }
#pragma unroll
    for (int t = 0; t < 5 * Q; ++t) sc[t * TV + v] = g[t];
  }
  __syncthreads();
  if (!live) return;
  // gather: vertex u = v of the tile
  const long long gi = (long long)y * f.W + x;
  bool in_tile[4];
  int vn[4];
#pragma unroll
  for (int d = 0; d < 4; ++d) {
    const int yy = y + kDy[d], xx = x + kDx[d];
    const int rr = lr + kDy[d], cc = lc + kDx[d];
    in_tile[d] = yy >= 0 && yy < f.y1 && xx >= 0 && xx < f.W && rr >= 0 && rr < TY && cc >= 0 &&
                 cc < TX;
    vn[d] = rr * TX + cc;
  }
  float *ring_t = ring + (long long)tile * kAdjRing * Q;
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    float acc = sc[q * TV + v];
#pragma unroll
    for (int d = 0; d < 4; ++d) {
      // u is the opposite-direction neighbour of v = u + dir d
      const int opp = (d + 2) & 3;
      if (in_tile[d]) acc += sc[((1 + opp) * Q + q) * TV + vn[d]];
    }
    grad[(long long)q * plane + gi] = acc;
    // this centre's partials about vertices of other tiles
    if (lr == 0) ring_t[q * 32 + lc] = sc[((1 + 1) * Q + q) * TV + v];               // n
    if (lr == TY - 1) ring_t[(Q + q) * 32 + lc] = sc[((1 + 3) * Q + q) * TV + v];    // s
    if (lc == 0) ring_t[64 * Q + q * 8 + lr] = sc[((1 + 2) * Q + q) * TV + v];       // w
    if (lc == TX - 1) ring_t[72 * Q + q * 8 + lr] = sc[((1 + 0) * Q + q) * TV + v];  // e
  }
}

// shared-memory bytes of hist_adj_tile at B bins
static size_t hist_adj_smem(int B) {
  constexpr int HALO = 10 * 34;
  return ((size_t)4 * hist_r4_rows(B) * hist_r4_stride(HALO) + 4 * HALO) * sizeof(float);
}

// pass 2: grad[q][u] = own row + the rows u's neighbours wrote about u
__global__ void __launch_bounds__(256) gather_kernel(Field f, int Q, const float *__restrict__ rows,
                                                     float *__restrict__ grad) {
  const long long plane = f.plane;
  const long long total = plane * Q;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int q = (int)(t / plane);
    const long long u = t - (long long)q * plane;
    const int y = (int)(u / f.W), x = (int)(u % f.W);
    float s = rows[(long long)q * plane + u];
#pragma unroll
    for (int d = 0; d < 4; ++d) {
      const int yy = y + kDy[d], xx = x + kDx[d];
      if (yy < 0 || yy >= f.H || xx < 0 || xx >= f.W) continue;
      const int opp = (d + 2) & 3;  // u is the opposite-direction neighbour of v
      s += rows[((long long)(1 + opp) * Q + q) * plane + (long long)yy * f.W + xx];
    }
    grad[t] = s;
  }
}

}  // namespace

// tiles of the per-bin-row histogram adjoint over the computed rows
static long long adj_tiles(const Field &f, int *tiles_x) {
  *tiles_x = (f.W + 31) / 32;
  const long long tiles_y = (f.y1 - f.y0 + kAdjTY - 1) / kAdjTY;
  return tiles_y > 0 ? (long long)*tiles_x * tiles_y : 0;
}

// scratch of the per-bin-row histogram adjoint: nslots claim flags (in 64
// floats' room each 64 flags), the ring, nslots partial blocks
static size_t adj_layout(long long nt, int B, long long nslots, long long *flags_f,
                         long long *ring_f) {
  *flags_f = (nslots + 63) / 64 * 64;
  *ring_f = nt * kAdjRing * B;
  return (size_t)(*flags_f + *ring_f + nslots * 5LL * B * kAdjTV);
}

size_t backward_scratch_floats(const Field &f, int model, int ctas) {
  if (model == kUniform || model == kEpan) {  // the tiles' rings
    int tx;
    return (size_t)adj_tiles(f, &tx) * kAdjRing * 2;
  }
  if (model == kHist && f.B <= 16) {
    int tx;
    const long long nt = adj_tiles(f, &tx);
    long long a, b;
    return adj_layout(nt, f.B, std::max(1, ctas), &a, &b);
  }
  const int Q = model == kHist ? f.B : 2;
  return (size_t)5 * Q * (size_t)f.plane;
}

cudaError_t launch_backward(const Field &f, int model, int cptype, const float *weight,
                            float *rows, size_t rows_floats, int max_ctas, float *grad,
                            cudaStream_t s) {
  const int Q = model == kHist ? f.B : 2;
  long long b = (f.plane + 127) / 128;
  if (b > (1LL << 30)) b = 1LL << 30;
  const int want_max = cptype == 2;
  if (model == kUniform || model == kEpan) {
    // tiled, partials in shared memory; ring partials after the tiles
    int tiles_x;
    const long long nt = adj_tiles(f, &tiles_x);
    if (nt > 0x7fffffffLL) return cudaErrorInvalidValue;
    if (nt == 0) return cudaSuccess;
    if ((size_t)nt * kAdjRing * 2 > rows_floats) return cudaErrorInvalidValue;
    if (model == kUniform)
      closed_adj_tile<kUniform><<<(int)nt, NTHREADS, 0, s>>>(f, tiles_x, want_max, weight, rows,
                                                             grad);
    else
      closed_adj_tile<kEpan><<<(int)nt, NTHREADS, 0, s>>>(f, tiles_x, want_max, weight, rows,
                                                          grad);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    Field g = f;
    g.B = 2;  // the ring's parameters per vertex
    const long long fx = (nt * (2 * 32 + 2 * (kAdjTY - 2)) + 255) / 256;
    hist_adj_fixup<<<(int)std::min<long long>(fx, 1LL << 30), 256, 0, s>>>(g, tiles_x, (int)nt,
                                                                          rows, grad);
    return cudaGetLastError();
  }
  switch (model) {
    case kHist: {
      if (f.B <= 16) {
        // per-bin rows, 8 x 32 tiles, two CTAs per SM; partials of a tile in
        // its CTA's scratch block, gathered in place; ring partials after the
        // tiles (see hist_adj_tile)
        static std::atomic<bool> attr_rows[2][128] = {};
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
        const int which = f.B <= 8 ? 0 : 1;
        if (!attr_rows[which][dev].load(std::memory_order_acquire)) {
          e = which == 0 ? cudaFuncSetAttribute(hist_adj_tile<8>,
                                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                (int)hist_adj_smem(8))
                         : cudaFuncSetAttribute(hist_adj_tile<16>,
                                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                (int)hist_adj_smem(16));
          if (e != cudaSuccess) {
            cudaGetLastError();
            return e;
          }
          attr_rows[which][dev].store(true, std::memory_order_release);
        }
        int tiles_x;
        const long long nt = adj_tiles(f, &tiles_x);
        if (nt > 0x7fffffffLL) return cudaErrorInvalidValue;
        if (nt == 0) return cudaSuccess;
        // as many scratch blocks as fit, at most max_ctas
        long long ns = std::max(1, max_ctas), flags_f, ring_f;
        while (ns > 1 && adj_layout(nt, f.B, ns, &flags_f, &ring_f) > rows_floats) --ns;
        if (adj_layout(nt, f.B, ns, &flags_f, &ring_f) > rows_floats) return cudaErrorInvalidValue;
        int *flags = reinterpret_cast<int *>(rows);
        float *ring = rows + flags_f, *scratch = ring + ring_f;
        e = cudaMemsetAsync(flags, 0, (size_t)ns * sizeof(int), s);
        if (e != cudaSuccess) return e;
        if (which == 0)
          hist_adj_tile<8><<<(int)nt, NTHREADS, hist_adj_smem(f.B), s>>>(
              f, tiles_x, want_max, weight, flags, (int)ns, scratch, ring, grad);
        else
          hist_adj_tile<16><<<(int)nt, NTHREADS, hist_adj_smem(f.B), s>>>(
              f, tiles_x, want_max, weight, flags, (int)ns, scratch, ring, grad);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        const long long fx = (nt * (2 * 32 + 2 * (kAdjTY - 2)) + 255) / 256;
        hist_adj_fixup<<<(int)std::min<long long>(fx, 1LL << 30), 256, 0, s>>>(f, tiles_x, (int)nt,
                                                                              ring, grad);
        return cudaGetLastError();
      }
      constexpr int TYg = kGradTY;
      // per device: the attribute is set once (host threads may race to set
      // it; setting it twice is harmless, the flag itself is atomic)
      static std::atomic<bool> attr_set[128] = {};
      int dev = 0;
      cudaError_t e = cudaGetDevice(&dev);
      if (e != cudaSuccess) return e;
      if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
      if (!attr_set[dev].load(std::memory_order_acquire)) {
        e = cudaFuncSetAttribute(hist_partials_tile<TYg>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(tile_floats(kHist, kMaxBins, TYg) * sizeof(float)));
        if (e != cudaSuccess) {
          cudaGetLastError();
          return e;
        }
        attr_set[dev].store(true, std::memory_order_release);
      }
      const int tiles_x = (f.W + TX - 1) / TX, tiles_y = (f.y1 - f.y0 + TYg - 1) / TYg;
      const long long tiles = (long long)tiles_x * tiles_y;
      if (tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
      if (tiles > 0)
        hist_partials_tile<TYg><<<(int)tiles, NTHREADS,
                                  (size_t)tile_floats(kHist, f.B, TYg) * sizeof(float), s>>>(
            f, tiles_x, want_max, weight, rows);
      break;
    }
    default: return cudaErrorInvalidValue;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  long long g = (f.plane * Q + 255) / 256;
  if (g > (1LL << 30)) g = 1LL << 30;
  gather_kernel<<<(int)g, 256, 0, s>>>(f, Q, rows, grad);
  return cudaGetLastError();
}

}  // namespace ucp
