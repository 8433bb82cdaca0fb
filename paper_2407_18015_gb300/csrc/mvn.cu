// mvn.cu -- multivariate Gaussian model over (X_v, X_e, X_n, X_w, X_s):
// per-vertex mean and covariance (the fit), Cholesky factor, and Monte
// Carlo estimates of P_min / P_max, the approach of the prior work the paper
// compares against (Sec. "Comparison of Parametric Vs. Nonparametric
// Models", multivariate Gaussian with Monte Carlo sampling).
//
// One warp per vertex.  Lanes split the samples; each sample draws two
// Philox4x32-10 blocks (counter (s, vertex, field, j), key = seed), maps the
// words to uniforms ((r >> 9) + 0.5) 2^-23 (exact in binary32, inside
// (0, 1)), and Box-Muller gives six
// normals, five of which are used.  The comparisons x_v < x_n are evaluated
// on the differences y_n = x_v - x_n = (mu_v - mu_n) + (L_v. - L_n.) z, and
// hits are counted with __ballot_sync + __popc.
#include "device.cuh"
#include "launch.h"

namespace ucp {

// The two blocks of one sample: counters (s, v, field, 0) and (s, v, field, 1)
// differ only in the last word, so the first round's products are shared.
__device__ __forceinline__ void philox_pair(uint32_t s, uint32_t v, uint32_t field,
                                            const PhiloxKeys &K, uint4 &r0, uint4 &r1) {
  const uint32_t hi0 = __umulhi(0xD2511F53u, s), lo0 = 0xD2511F53u * s;
  const uint32_t hi1 = __umulhi(0xCD9E8D57u, field), lo1 = 0xCD9E8D57u * field;
  const uint32_t a = hi1 ^ v ^ K.k0[0];
  r0 = make_uint4(a, lo1, hi0 ^ K.k1[0], lo0);
  r1 = make_uint4(a, lo1, hi0 ^ 1u ^ K.k1[0], lo0);
#pragma unroll
  for (int r = 1; r < 10; ++r) {
    philox_round(r0, K.k0[r], K.k1[r]);
    philox_round(r1, K.k0[r], K.k1[r]);
  }
}

// Box-Muller: radius sqrt(-2 ln ua), angle 2 pi ub.  The angle is taken as
// pi + t with t = 2 pi (ub - 1/2) in [-pi, pi), where the hardware sine and
// cosine are accurate to ~4e-7 absolute: cos(2 pi ub) = -cos t,
// sin(2 pi ub) = -sin t.  The logarithm keeps full accuracy (its error is
// not bounded relative to the radius near ub -> 1).
__device__ __forceinline__ void box_muller(float ua, float ub, float &z0, float &z1) {
  const float v = -2.f * logf(ua);
  const float rad = v * rsqrtf(v);
  float s, c;
  __sincosf(6.283185307179586f * (ub - 0.5f), &s, &c);
  z0 = -rad * c;
  z1 = -rad * s;
}

// Slots of the variables: 0 = v, 1..4 = e, n, w, s.  Returns the number of
// present variables and their slots in order.
__device__ __forceinline__ int mvn_slots(const Field &f, int y, int x, int *slot,
                                         long long *gidx) {
  int nv = 1;
  slot[0] = 0;
  gidx[0] = (long long)y * f.W + x;
#pragma unroll
  for (int d = 0; d < 4; ++d) {
    const int yy = y + kDy[d], xx = x + kDx[d];
    if (yy >= 0 && yy < f.H && xx >= 0 && xx < f.W) {
      slot[nv] = 1 + d;
      gidx[nv] = (long long)yy * f.W + xx;
      ++nv;
    }
  }
  return nv;
}

__device__ __forceinline__ int packed(int a, int b) {  // a >= b
  return a * (a + 1) / 2 + b;
}

// Cholesky of the nv x nv matrix A (row-major, 5x5 storage) into L.
__device__ __forceinline__ bool chol5(const float (&A)[5][5], int nv, float (&L)[5][5]) {
#pragma unroll
  for (int i = 0; i < 5; ++i)
#pragma unroll
    for (int j = 0; j < 5; ++j) L[i][j] = 0.f;
  bool ok = true;
#pragma unroll
  for (int j = 0; j < 5; ++j) {
    if (j >= nv) break;
    float s = A[j][j];
#pragma unroll
    for (int k = 0; k < j; ++k) s = fmaf(-L[j][k], L[j][k], s);
    if (!(s > 0.f)) {
      ok = false;
      break;
    }
    const float d = sqrtf(s);
    L[j][j] = d;
#pragma unroll
    for (int i = j + 1; i < 5; ++i) {
      if (i >= nv) break;
      float t = A[i][j];
#pragma unroll
      for (int k = 0; k < j; ++k) t = fmaf(-L[i][k], L[j][k], t);
      L[i][j] = t / d;
    }
  }
  return ok;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------------------
// fit: mean and covariance (N-1) of the present variables, thread per vertex

__global__ void __launch_bounds__(256) mvn_fit_kernel(Field f) {
  float *out = const_cast<float *>(f.params);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < f.plane;
       i += (long long)gridDim.x * blockDim.x) {
    const int y = (int)(i / f.W), x = (int)(i % f.W);
    int slot[5];
    long long g[5];
    const int nv = mvn_slots(f, y, x, slot, g);
    float mu[5] = {0, 0, 0, 0, 0};
    bool nf = false;
    for (int a = 0; a < nv; ++a) {
      float s = 0.f;
      for (int k = 0; k < f.N; ++k) {
        const float v = __ldg(f.ens + (long long)k * f.plane + g[a]);
        nf |= !isfinite(v);
        s += v;
      }
      mu[a] = s / (float)f.N;
    }
    float full_mu[5] = {0, 0, 0, 0, 0};
    for (int a = 0; a < nv; ++a) full_mu[slot[a]] = mu[a];
    for (int q = 0; q < 5; ++q) out[q * f.plane + i] = nf ? __int_as_float(0x7fc00000) : full_mu[q];
    float C[15];
    for (int q = 0; q < 15; ++q) C[q] = 0.f;
    if (f.N > 1) {
      for (int k = 0; k < f.N; ++k) {
        float dv[5];
        for (int a = 0; a < nv; ++a) dv[a] = __ldg(f.ens + (long long)k * f.plane + g[a]) - mu[a];
        for (int a = 0; a < nv; ++a)
          for (int b = 0; b <= a; ++b) C[packed(slot[a], slot[b])] += dv[a] * dv[b];
      }
      for (int q = 0; q < 15; ++q) C[q] /= (float)(f.N - 1);
    }
    for (int q = 0; q < 15; ++q)
      out[(5 + q) * f.plane + i] = nf ? __int_as_float(0x7fc00000) : C[q];
    if (f.status) f.status[i] = nf ? V_NONFINITE : 0;
  }
}

// ---------------------------------------------------------------------------
// Monte Carlo, warp per vertex

template <bool FROM_MEMBERS, bool SADDLE>
__global__ void __launch_bounds__(256) mvn_mc_kernel(Field f, int S, uint32_t k0, uint32_t k1,
                                                     uint32_t field) {
  const int lane = threadIdx.x & 31;
  const long long warp0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const long long vbeg = (long long)f.y0 * f.W, vend = (long long)f.y1 * f.W;
  for (long long v = vbeg + warp0; v < vend; v += nwarps) {
    const int y = (int)(v / f.W), x = (int)(v % f.W);
    int slot[5];
    long long g[5];
    const int nv = mvn_slots(f, y, x, slot, g);
    float mu[5] = {0, 0, 0, 0, 0};
    float A[5][5];
#pragma unroll
    for (int a = 0; a < 5; ++a)
#pragma unroll
      for (int b = 0; b < 5; ++b) A[a][b] = 0.f;
    bool nf = false;
    if (FROM_MEMBERS) {
      float s[5] = {0, 0, 0, 0, 0};
      for (int k = lane; k < f.N; k += 32)
#pragma unroll
        for (int a = 0; a < 5; ++a)
          if (a < nv) {
            const float t = __ldg(f.ens + (long long)k * f.plane + g[a]);
            nf |= !isfinite(t);
            s[a] += t;
          }
#pragma unroll
      for (int a = 0; a < 5; ++a) mu[a] = warp_sum(s[a]) / (float)f.N;
      nf = __any_sync(0xffffffffu, nf);
      float c[15];
#pragma unroll
      for (int q = 0; q < 15; ++q) c[q] = 0.f;
      for (int k = lane; k < f.N; k += 32) {
        float dv[5];
#pragma unroll
        for (int a = 0; a < 5; ++a)
          dv[a] = (a < nv) ? __ldg(f.ens + (long long)k * f.plane + g[a]) - mu[a] : 0.f;
#pragma unroll
        for (int a = 0; a < 5; ++a)
#pragma unroll
          for (int b = 0; b <= a; ++b) c[packed(a, b)] = fmaf(dv[a], dv[b], c[packed(a, b)]);
      }
      const float inv = f.N > 1 ? 1.f / (float)(f.N - 1) : 0.f;
#pragma unroll
      for (int a = 0; a < 5; ++a)
#pragma unroll
        for (int b = 0; b <= a; ++b) {
          const float t = warp_sum(c[packed(a, b)]) * inv;
          A[a][b] = t;
          A[b][a] = t;
        }
    } else {
#pragma unroll
      for (int a = 0; a < 5; ++a) {
        if (a >= nv) break;
        mu[a] = __ldg(f.params + (long long)slot[a] * f.plane + v);
      }
#pragma unroll
      for (int a = 0; a < 5; ++a)
#pragma unroll
        for (int b = 0; b <= a; ++b) {
          if (a < nv) {
            const int sa = slot[a], sb = slot[b];
            const int q = sa >= sb ? packed(sa, sb) : packed(sb, sa);
            const float t = __ldg(f.params + (long long)(5 + q) * f.plane + v);
            A[a][b] = t;
            A[b][a] = t;
          }
        }
    }
    float tr = 0.f;
#pragma unroll
    for (int a = 0; a < 5; ++a) {
      if (a < nv) {
        nf |= !isfinite(mu[a]);
        tr += A[a][a];
#pragma unroll
        for (int b = 0; b < 5; ++b)
          if (b < nv) nf |= !isfinite(A[a][b]);
      }
    }
    uint8_t st = nf ? V_NONFINITE : 0;
    float pmin = 0.f, pmax = 0.f, psad = 0.f;
    // saddle sign of each present variable (+1: t1 wants x_v < x_n); a vertex
    // without a saddle neighbourhood counts no saddle hits
    float ssg[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    const bool line = (f.H == 1 || f.W == 1) && nv == 3;
    const bool has_saddle = (nv == 5) || line;
#pragma unroll
    for (int a = 1; a < 5; ++a)
      if (a < nv) {
        const int sl = slot[a];  // 1 e, 2 n, 3 w, 4 s
        ssg[a] = (nv == 5) ? ((sl == 1 || sl == 3) ? 1.f : -1.f)
                           : ((sl == 1 || sl == 4) ? 1.f : -1.f);
      }
    const bool zero_mm = f.boundary == 1 && nv < 5;
    if (nf) {
      pmin = pmax = psad = __int_as_float(0x7fc00000);
    } else if (tr == 0.f) {
      bool lt = true, gt = true, t1 = has_saddle, t2 = has_saddle;
#pragma unroll
      for (int a = 1; a < 5; ++a)
        if (a < nv) {
          lt &= mu[0] < mu[a];
          gt &= mu[0] > mu[a];
          t1 &= ssg[a] > 0.f ? mu[0] < mu[a] : mu[0] > mu[a];
          t2 &= ssg[a] > 0.f ? mu[0] > mu[a] : mu[0] < mu[a];
        }
      pmin = (lt && !zero_mm) ? 1.f : 0.f;
      pmax = (gt && !zero_mm) ? 1.f : 0.f;
      psad = (t1 || t2) ? 1.f : 0.f;
      st |= V_DEGENERATE;
    } else {
      float L[5][5];
      bool ok = chol5(A, nv, L);
      if (!ok) {
        float eps = 1e-6f * tr / (float)nv;
        for (int r = 0; r < 3 && !ok; ++r) {
          float Aj[5][5];
#pragma unroll
          for (int a = 0; a < 5; ++a)
#pragma unroll
            for (int b = 0; b < 5; ++b) Aj[a][b] = A[a][b] + (a == b ? eps : 0.f);
          ok = chol5(Aj, nv, L);
          eps *= 10.f;
        }
        st |= ok ? V_JITTER : V_CHOLFAIL;
      }
      if (!ok) {
        pmin = pmax = psad = __int_as_float(0x7fc00000);
      } else {
        // y_n = x_0 - x_n = D_n + sum_b M[n][b] z_b
        float D[5], M[5][5];
#pragma unroll
        for (int n = 0; n < 5; ++n) {
          D[n] = mu[0] - mu[n];
#pragma unroll
          for (int b = 0; b < 5; ++b) M[n][b] = (b == 0 ? L[0][0] : 0.f) - L[n][b];
        }
        unsigned cmin = 0, cmax = 0, csad = 0;
        const int iters = (S + 31) >> 5;
        const uint32_t vid = (uint32_t)v;
        const PhiloxKeys K(k0, k1);
        for (int it = 0; it < iters; ++it) {
          const int s = (it << 5) + lane;
          uint4 r0, r1;
          philox_pair((uint32_t)s, vid, field, K, r0, r1);
          float z[6];
          box_muller(u01_23(r0.x), u01_23(r0.y), z[0], z[1]);
          box_muller(u01_23(r0.z), u01_23(r0.w), z[2], z[3]);
          box_muller(u01_23(r1.x), u01_23(r1.y), z[4], z[5]);
          // x_v below every neighbour: the largest y_n = x_v - x_n is < 0;
          // above every one: the smallest is > 0
          float ymax = -kFar, ymin = kFar;
          bool t1 = has_saddle, t2 = has_saddle;
#pragma unroll
          for (int n = 1; n < 5; ++n) {
            if (n < nv) {
              float yv = D[n];
#pragma unroll
              for (int b = 0; b <= n; ++b) yv = fmaf(M[n][b], z[b], yv);
              ymax = fmaxf(ymax, yv);
              ymin = fminf(ymin, yv);
              if constexpr (SADDLE) {
                // y = x_v - x_n: t1 wants x_v < x_n where the sign is +1
                const float sy = ssg[n] * yv;
                t1 &= sy < 0.f;
                t2 &= sy > 0.f;
              }
            }
          }
          const bool valid = s < S;
          if constexpr (!SADDLE) {
            cmin += __popc(__ballot_sync(0xffffffffu, valid && ymax < 0.f));
            cmax += __popc(__ballot_sync(0xffffffffu, valid && ymin > 0.f));
          } else {
            csad += __popc(__ballot_sync(0xffffffffu, valid && (t1 || t2)));
          }
        }
        pmin = zero_mm ? 0.f : (float)cmin / (float)S;
        pmax = zero_mm ? 0.f : (float)cmax / (float)S;
        psad = (float)csad / (float)S;
      }
    }
    if (lane == 0) {
      // each instance writes its own outputs; the status once (by the
      // minimum / maximum instance when it runs)
      if constexpr (!SADDLE) {
        if ((f.cptypes & kMin) && f.out_min) f.out_min[v] = pmin;
        if ((f.cptypes & kMax) && f.out_max) f.out_max[v] = pmax;
        if (f.status) f.status[v] = st;
      } else {
        if (f.out_saddle) f.out_saddle[v] = psad;
        if (f.status && !(f.cptypes & (kMin | kMax))) f.status[v] = st;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// launchers

cudaError_t launch_mvn_fit(const Field &f, cudaStream_t s) {
  long long b = (f.plane + 255) / 256;
  if (b > (1LL << 30)) b = 1LL << 30;
  mvn_fit_kernel<<<(int)b, 256, 0, s>>>(f);
  return cudaGetLastError();
}

cudaError_t launch_mvn_mc(const Field &f, bool from_members, int samples, uint64_t seed,
                          uint32_t field_id, cudaStream_t s) {
  // one warp per vertex, 8 warps per CTA, grid-stride over vertices
  const long long nvtx = (long long)(f.y1 - f.y0) * f.W;
  if (nvtx <= 0) return cudaSuccess;
  long long b = (nvtx + 7) / 8;
  if (b > (1LL << 30)) b = 1LL << 30;
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  // minimum / maximum and the saddle are separate instances, so that
  // neither pays for the other's tests in the sample loop
  cudaError_t e = cudaSuccess;
  if (f.cptypes & (kMin | kMax)) {
    if (from_members)
      mvn_mc_kernel<true, false><<<(int)b, 256, 0, s>>>(f, samples, k0, k1, field_id);
    else
      mvn_mc_kernel<false, false><<<(int)b, 256, 0, s>>>(f, samples, k0, k1, field_id);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && (f.cptypes & kSaddle)) {
    if (from_members)
      mvn_mc_kernel<true, true><<<(int)b, 256, 0, s>>>(f, samples, k0, k1, field_id);
    else
      mvn_mc_kernel<false, true><<<(int)b, 256, 0, s>>>(f, samples, k0, k1, field_id);
    e = cudaGetLastError();
  }
  return e;
}

}  // namespace ucp
