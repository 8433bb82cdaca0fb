// stencil.cu -- minimum / maximum probability fields with the six- or
// eight-neighbour stencil of a 2D grid or the six axis neighbours of a 3D
// grid (the extension named in the paper's Sec. "Conclusion").
//
// The parameters come from the statistics pass (fit_kernel over all D*H*W
// vertices) or from the caller.  For histograms a table pass turns every
// vertex's masses into its tail table (stencil.cuh).  The probability kernel
// gives one vertex to each thread; a vertex reads its own and its K
// neighbours' parameters through the read-only cache, where a neighbour's
// values are shared by the K+1 threads that read them.
#include "device.cuh"
#include "launch.h"
#include "stencil.cuh"

namespace ucp {

namespace {

__device__ __forceinline__ float nanf_() { return __int_as_float(0x7fc00000); }

// tail table of every vertex (one row of hist_table_row(B) floats each)
__global__ void __launch_bounds__(256) hist_table_kernel(const float *__restrict__ params,
                                                         long long V, int B,
                                                         float *__restrict__ tab) {
  const int R = hist_table_row(B);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < V;
       i += (long long)gridDim.x * blockDim.x) {
    const float a = params[i], b = params[V + i];
    uint8_t st = (!isfinite(a) || !isfinite(b)) ? V_NONFINITE
                                               : (a > b ? V_BAD : (a == b ? V_DEGENERATE : 0));
    float t = 0.f;
    for (int q = 0; q < B; ++q) {
      const float w = params[(2 + q) * V + i];
      if (!isfinite(w)) st |= V_NONFINITE;
      else if (w < 0.f) st |= V_BAD;
      t += w;
    }
    float *row = tab + i * R;
    const bool point = a == b;
    float c = 0.f;
    for (int q = 0; q < B; ++q) {
      row[q] = point ? 0.f : t - c;
      c += params[(2 + q) * V + i];
    }
    row[B] = 0.f;
    row[B + 1] = 0.f;
    row[B + 2] = t;
    row[B + 3] = (float)st;
  }
}

// status bits of uniform / Epanechnikov parameters (a, b) = (p0, p1)
template <int MODEL>
__device__ __forceinline__ uint8_t check2(float a, float b) {
  if (!isfinite(a) || !isfinite(b)) return V_NONFINITE;
  if (MODEL == kUniform) return a > b ? V_BAD : (a == b ? V_DEGENERATE : 0);
  return b < 0.f ? V_BAD : (b == 0.f ? V_DEGENERATE : 0);
}

template <int MODEL, int ST>
__global__ void __launch_bounds__(128) stencil_kernel(StencilField f) {
  constexpr int K = stencil_k(ST);
  const long long V = f.V, HW = (long long)f.H * f.W;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < V;
       i += (long long)gridDim.x * blockDim.x) {
    const int z = (int)(i / HW);
    const long long r = i - (long long)z * HW;
    const int y = (int)(r / f.W), x = (int)(r - (long long)y * f.W);
    long long nidx[K];
    bool present[K];
    int k = 0;
#pragma unroll
    for (int n = 0; n < K; ++n) {
      const int dz = kStencilOff[ST][n][0], dy = kStencilOff[ST][n][1],
                dx = kStencilOff[ST][n][2];
      const int zz = z + dz, yy = y + dy, xx = x + dx;
      present[n] = zz >= 0 && zz < f.D && yy >= 0 && yy < f.H && xx >= 0 && xx < f.W;
      nidx[n] = present[n] ? i + dz * HW + (long long)dy * f.W + dx : i;
      k += present[n];
    }
    const bool zero = f.boundary == 1 && k < K;
    float pmin = 0.f, pmax = 0.f;
    uint8_t st;
    if constexpr (MODEL == kHist) {
      const int B = f.B, R = hist_table_row(B);
      const long long crow = i * R;
      st = (uint8_t)__ldg(f.tab + crow + B + 3);
      float T[K];
#pragma unroll
      for (int n = 0; n < K; ++n) {
        T[n] = 2.f;  // CDF complement 2 - 1 = 1 for an absent neighbour
        if (!present[n]) continue;
        st |= (uint8_t)__ldg(f.tab + nidx[n] * R + B + 3) & (V_NONFINITE | V_BAD);
        T[n] = __ldg(f.tab + nidx[n] * R + B + 2);
      }
      if (st & (V_NONFINITE | V_BAD)) {
        pmin = pmax = nanf_();
      } else if (!zero) {
        const float lo1 = __ldg(f.params + i), hi1 = __ldg(f.params + V + i);
        if (lo1 == hi1) {
          float gm = __ldg(f.tab + crow + B + 2), gM = gm;
#pragma unroll
          for (int n = 0; n < K; ++n) {
            if (!present[n]) continue;
            float gt, lt;
            hist_tails_row(f.tab, nidx[n] * R, B, __ldg(f.params + nidx[n]),
                           __ldg(f.params + V + nidx[n]), T[n], lo1, gt, lt);
            gm *= gt;
            gM *= lt;
          }
          pmin = gm;
          pmax = gM;
        } else {
          HistSegG nw[K];
#pragma unroll
          for (int n = 0; n < K; ++n) {
            HistSegG &h = nw[n];
            if (!present[n]) {
              h.init_absent(crow, (float)B);
              continue;
            }
            const float lo = __ldg(f.params + nidx[n]), hi = __ldg(f.params + V + nidx[n]);
            h.init(f.tab, nidx[n] * R, lo - lo1, lo == hi ? 0.f : (hi - lo) / (float)B, T[n]);
            // move to the segment that contains x = 0
            for (int g = 0; g <= B && h.nx <= 0.f; ++g)
              if (!h.step(f.tab, h.nx, (float)B)) break;
          }
          hist_walk_k<K>(f.tab, crow, B, hi1 - lo1, nw, T, f.cptypes, pmin, pmax);
        }
      }
    } else {
      const float c0 = __ldg(f.params + i), c1 = __ldg(f.params + V + i);
      st = check2<MODEL>(c0, c1);
      float p0[K], p1[K];
#pragma unroll
      for (int n = 0; n < K; ++n) {
        p0[n] = __ldg(f.params + nidx[n]);
        p1[n] = __ldg(f.params + V + nidx[n]);
        if (present[n]) st |= check2<MODEL>(p0[n], p1[n]) & (V_NONFINITE | V_BAD);
      }
      if (st & (V_NONFINITE | V_BAD)) {
        pmin = pmax = nanf_();
      } else if (!zero) {
        if constexpr (MODEL == kUniform) {
          UniParams nb[K];
#pragma unroll
          for (int n = 0; n < K; ++n) nb[n] = UniParams{p0[n], p1[n]};
          uniform_vertex_k<K>(UniParams{c0, c1}, nb, present, f.cptypes, pmin, pmax);
        } else {
          EpanParams nb[K];
#pragma unroll
          for (int n = 0; n < K; ++n) nb[n] = EpanParams{p0[n], p1[n]};
          epan_vertex_k<K>(EpanParams{c0, c1}, nb, present, f.cptypes, pmin, pmax);
        }
      }
    }
    if ((f.cptypes & kMin) && f.out_min) f.out_min[i] = pmin;
    if ((f.cptypes & kMax) && f.out_max) f.out_max[i] = pmax;
    if (f.status) f.status[i] = st;
  }
}

int grid_blocks(long long n, int threads, int sm_count, int per_sm) {
  long long b = (n + threads - 1) / threads;
  const long long cap = (long long)sm_count * per_sm;
  if (b > cap) b = cap;
  return (int)(b < 1 ? 1 : b);
}

template <int MODEL>
cudaError_t launch_model(const StencilField &f, int stencil, int blocks, cudaStream_t s) {
  switch (stencil) {
    case kStencil6: stencil_kernel<MODEL, kStencil6><<<blocks, 128, 0, s>>>(f); break;
    case kStencil8: stencil_kernel<MODEL, kStencil8><<<blocks, 128, 0, s>>>(f); break;
    case kStencil3D6: stencil_kernel<MODEL, kStencil3D6><<<blocks, 128, 0, s>>>(f); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_hist_table(const float *params, long long V, int B, float *tab, int sm_count,
                              cudaStream_t s) {
  hist_table_kernel<<<grid_blocks(V, 256, sm_count, 8), 256, 0, s>>>(params, V, B, tab);
  return cudaGetLastError();
}

cudaError_t launch_stencil(const StencilField &f, int model, int stencil, int sm_count,
                           cudaStream_t s) {
  const int blocks = grid_blocks(f.V, 128, sm_count, 16);
  switch (model) {
    case kUniform: return launch_model<kUniform>(f, stencil, blocks, s);
    case kEpan: return launch_model<kEpan>(f, stencil, blocks, s);
    case kHist: return launch_model<kHist>(f, stencil, blocks, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ucp
