// closed.cu -- closed-form critical-point probability kernels (uniform,
// Epanechnikov, histogram) and the statistics pass.
//
// Tile kernel: one CTA per TY x 32 tile of vertices (TY = 8 or 16, see
// TileH).  Phase 1 stages the parameters of the tile and its one-vertex halo
// ((TY + 2) x 34) in shared memory, either fitted from the members (the
// statistics pass fused into the same launch, so parameters never reach HBM)
// or loaded from a parameter array.  Phase 2 gives each of the 256 threads
// TY / 8 vertices; a vertex reads its own and its four neighbours'
// parameters from shared memory (the neighbourhood access of the paper's
// VTK-m worklet, Sec. "Integration with VTK-m and ParaView") and integrates
// P_min / P_max exactly (device.cuh).
#include <atomic>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>

#include "device.cuh"
#include "launch.h"
#include "tile.cuh"

namespace ucp {

// ---------------------------------------------------------------------------
// statistics pass alone: params[P][H][W] + status

template <int MODEL>
__global__ void __launch_bounds__(256) fit_kernel(Field f) {
  const long long plane = f.plane;
  // histogram masses count / N of up to 255 members, as a table
  __shared__ float mtab[256];
  if (MODEL == kHist && f.N <= 255) {
    for (int c = threadIdx.x; c <= f.N; c += blockDim.x) mtab[c] = __fdiv_rn((float)c, (float)f.N);
    __syncthreads();
  }
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < plane;
       i += (long long)gridDim.x * blockDim.x) {
    const float *p = f.ens + i;
    float *out = const_cast<float *>(f.params);
    uint8_t st = 0;
    if (MODEL == kUniform) {
      float mn, mx;
      bool nf;
      members_minmax(p, plane, f.N, mn, mx, nf);
      if (nf) {
        mn = mx = __int_as_float(0x7fc00000);
        st |= V_NONFINITE;
      } else if (mn == mx) {
        st |= V_DEGENERATE;
      }
      out[i] = mn;
      out[plane + i] = mx;
    } else if (MODEL == kEpan || MODEL == kGauss) {
      float m, w, mn, mx;
      bool nf;
      members_epan(p, plane, f.N, MODEL == kGauss ? 1.f : f.epan_scale, m, w, mn, mx, nf);
      if (nf) {
        m = w = __int_as_float(0x7fc00000);
        st |= V_NONFINITE;
      } else if (mn == mx) {
        st |= V_DEGENERATE;
      }
      out[i] = m;
      out[plane + i] = w;
    } else {
      float mn, mx;
      bool nf;
      members_minmax(p, plane, f.N, mn, mx, nf);
      const int B = f.B;
      if (nf) {
        for (int q = 0; q < 2 + B; ++q) out[q * plane + i] = __int_as_float(0x7fc00000);
        st |= V_NONFINITE;
      } else if (B <= 16 && f.N <= 255) {
        // 8-bit bin counters packed in two 64-bit registers (no local memory)
        unsigned long long c0 = 0ull, c1 = 0ull;
        if (mn == mx) {
          c0 = (unsigned long long)f.N;
          st |= V_DEGENERATE;
        } else {
          const float s = __fdiv_rn((float)B, __fsub_rn(mx, mn));
#pragma unroll 4
          for (int k = 0; k < f.N; ++k) {
            const int j = hist_bin_nonneg(__ldg(p + (long long)k * plane), mn, s, B);
            const unsigned long long inc = 1ull << ((j & 7) << 3);
            c0 += j < 8 ? inc : 0ull;
            c1 += j < 8 ? 0ull : inc;
          }
        }
        out[i] = mn;
        out[plane + i] = mx;
        for (int q = 0; q < B; ++q) {
          const unsigned c = (unsigned)((q < 8 ? c0 : c1) >> ((q & 7) << 3)) & 255u;
          out[(2 + q) * plane + i] = mtab[c];
        }
      } else {
        int cnt[kMaxBins];
        for (int q = 0; q < B; ++q) cnt[q] = 0;
        if (mn == mx) {
          cnt[0] = f.N;
          st |= V_DEGENERATE;
        } else {
          const float s = __fdiv_rn((float)B, __fsub_rn(mx, mn));
          for (int k = 0; k < f.N; ++k) cnt[hist_bin(__ldg(p + (long long)k * plane), mn, s, B)]++;
        }
        out[i] = mn;
        out[plane + i] = mx;
        for (int q = 0; q < B; ++q)
          out[(2 + q) * plane + i] = __fdiv_rn((float)cnt[q], (float)f.N);
      }
    }
    if (f.status) f.status[i] = st;
  }
}

// Histogram fit of at most 16 bins and MAXN members in one pass over the
// members: a thread holds its vertex's members in registers (every load in
// flight at once), takes their minimum and maximum (NaN-propagating: a
// non-finite member shows in them) and bins them from the registers, where
// fit_kernel reads them twice.  The same values as fit_kernel: the same
// bins, counters and count / N table.
template <int MAXN>
__global__ void __launch_bounds__(128) fit_hist_regs(Field f) {
  __shared__ float mtab[MAXN + 1];
  const int N = f.N, B = f.B;
  for (int c = threadIdx.x; c <= N; c += blockDim.x) mtab[c] = __fdiv_rn((float)c, (float)N);
  __syncthreads();
  const long long plane = f.plane;
  float *out = const_cast<float *>(f.params);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < plane;
       i += (long long)gridDim.x * blockDim.x) {
    const float *p = f.ens + i;
    float v[MAXN];
    v[0] = __ldg(p);
#pragma unroll
    for (int k = 1; k < MAXN; ++k) v[k] = k < N ? __ldg(p + (long long)k * plane) : v[0];
    // members past N repeat member 0: they change neither minimum nor maximum
    float mn = v[0], mx = v[0];
#pragma unroll
    for (int k = 1; k + 1 < MAXN; k += 2) {
      mn = fmin3_nan(mn, v[k], v[k + 1]);
      mx = fmax3_nan(mx, v[k], v[k + 1]);
    }
    if constexpr ((MAXN & 1) == 0) {
      mn = fmin_nan(mn, v[MAXN - 1]);
      mx = fmax_nan(mx, v[MAXN - 1]);
    }
    uint8_t st = 0;
    if (!(isfinite(mn) && isfinite(mx))) {
      for (int q = 0; q < 2 + B; ++q) out[q * plane + i] = __int_as_float(0x7fc00000);
      st |= V_NONFINITE;
    } else {
      unsigned long long c0 = 0ull, c1 = 0ull;
      if (mn == mx) {
        c0 = (unsigned long long)N;
        st |= V_DEGENERATE;
      } else {
        const float sc = __fdiv_rn((float)B, __fsub_rn(mx, mn));
#pragma unroll
        for (int k = 0; k < MAXN; ++k) {
          if (k < N) {
            const int j = hist_bin_nonneg(v[k], mn, sc, B);
            const unsigned long long inc = 1ull << ((j & 7) << 3);
            c0 += j < 8 ? inc : 0ull;
            c1 += j < 8 ? 0ull : inc;
          }
        }
      }
      out[i] = mn;
      out[plane + i] = mx;
      for (int q = 0; q < B; ++q) {
        const unsigned c = (unsigned)((q < 8 ? c0 : c1) >> ((q & 7) << 3)) & 255u;
        out[(2 + q) * plane + i] = mtab[c];
      }
    }
    if (f.status) f.status[i] = st;
  }
}

// ---------------------------------------------------------------------------
// tile kernel

// tile height: 8 rows for the uniform and histogram models and the
// estimator (a 20-member box fits next to the parameter tile, and the
// histogram's per-bin rows fit), 16 for the Gaussian and, from parameters,
// Epanechnikov models (a smaller halo share).  The fused Epanechnikov kernel
// takes 8 rows when all members fit one box of 8 rows, else 16: with several
// boxes either way, the halo's share of the compensated sums outweighs the
// extra boxes.  Histograms without per-bin rows take 16 rows.
template <int MODEL>
struct TileH {
  static constexpr int value = (MODEL == kGauss || MODEL == kEpan) ? TY : 8;
};

// Shared memory: the parameter tile, then (RB > 0) the per-bin rows,
// 16-byte aligned.
template <int MODEL, bool FROM_MEMBERS, bool SADDLE, int TYm, int RB>
__global__ void __launch_bounds__(NTHREADS, (TileOcc<MODEL, RB>::value))
    tile_kernel(Field f, int tiles_x) {
  extern __shared__ __align__(16) float sm[];
  const int tile = blockIdx.x;
  constexpr bool ROWS = RB > 0;
  float4 *R4 = nullptr;
  // the per-thread staging counts into masses held in the tile; from
  // parameters the rows are built from registers (small tile)
  if constexpr (ROWS)
    R4 = reinterpret_cast<float4 *>(
        sm + ((param_tile_floats<MODEL, TYm, ROWS>(f.B, FROM_MEMBERS) + 3) & ~3LL));
  process_tile<MODEL, FROM_MEMBERS, TYm, SADDLE, false, RB>(
      f, f.y0 + (tile / tiles_x) * TYm, (tile % tiles_x) * TX, sm, nullptr, nullptr, nullptr, R4);
}

// The same with the members staged in a box: shared memory holds the
// member box (nc x (TYm + 2) x 40 floats, 128-byte aligned), filled by the
// tensor memory accelerator or (ASYNC, members it cannot address) by
// asynchronous copies -- for per-bin-row histograms the same room then
// takes the rows, once the box is no longer read -- then the parameter
// tile, then the mbarrier.
// resident CTAs per SM the register budget of a box-staged tile kernel is
// set for: the model's, at most four for the Epanechnikov saddle (its
// mixed-factor integrals in packed node pairs need more registers than the
// minimum / maximum: at five CTAs they spilled)
template <int MODEL, bool SADDLE, int RB>
struct TmaOcc {
  static constexpr int value = SADDLE && MODEL == kEpan && TileOcc<MODEL, RB>::value > 4
                                   ? 4
                                   : TileOcc<MODEL, RB>::value;
};

template <int MODEL, bool SADDLE, int TYm, int RB, bool ASYNC>
__global__ void __launch_bounds__(NTHREADS, (TmaOcc<MODEL, SADDLE, RB>::value))
    tile_kernel_tma(Field f, int tiles_x, const __grid_constant__ CUtensorMap tmap) {
  extern __shared__ __align__(128) float smem[];
  const int tile = blockIdx.x;
  const int box_floats = f.tma_nc * (TYm + 2) * kBoxW;
  constexpr bool ROWS = RB > 0;
  const int r4 = ROWS ? r4_floats(f.B, TYm) : 0;
  float *sm = smem + max(box_floats, r4);
  const long long tile_f = param_tile_floats<MODEL, TYm, ROWS>(f.B, false);
  uint64_t *bar = reinterpret_cast<uint64_t *>(sm + ((tile_f + 1) & ~1LL));
  process_tile<MODEL, true, TYm, SADDLE, true, RB, ASYNC>(
      f, f.y0 + (tile / tiles_x) * TYm, (tile % tiles_x) * TX, sm, &tmap, smem, bar,
      ROWS ? reinterpret_cast<float4 *>(smem) : nullptr);
}

// ---------------------------------------------------------------------------
// uniform parameters from a decompressed field and an error bound

__global__ void eb_params_kernel(const float *__restrict__ d, float eb, long long n,
                                 float *__restrict__ params) {
  const float h = 0.5f * eb;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float v = d[i];
    params[i] = v - h;
    params[n + i] = v + h;
  }
}

// ---------------------------------------------------------------------------
// launchers

static int grid_for(long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  if (b > (1LL << 30)) b = 1LL << 30;
  return (int)(b < 1 ? 1 : b);
}

cudaError_t launch_fit(const Field &f, int model, cudaStream_t s) {
  const int g = grid_for(f.plane, 256);
  switch (model) {
    case kUniform: fit_kernel<kUniform><<<g, 256, 0, s>>>(f); break;
    case kEpan: fit_kernel<kEpan><<<g, 256, 0, s>>>(f); break;
    case kGauss: fit_kernel<kGauss><<<g, 256, 0, s>>>(f); break;
    case kHist:
    case kSemi:
      if (f.B <= 16 && f.N >= 1 && f.N <= 64) {
        const int g2 = grid_for(f.plane, 128);
        if (f.N <= 32) fit_hist_regs<32><<<g2, 128, 0, s>>>(f);
        else fit_hist_regs<64><<<g2, 128, 0, s>>>(f);
      } else {
        fit_kernel<kHist><<<g, 256, 0, s>>>(f);
      }
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// cuTensorMapEncodeTiled, from the driver (no link-time dependency); looked
// up once (thread-safe static initialisation)
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = []() {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    PFN_cuTensorMapEncodeTiled_v12000 f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      f = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    cudaGetLastError();
    return f;
  }();
  return fn;
}

void *tensor_map_encoder_fn() { return reinterpret_cast<void *>(tensor_map_encoder()); }

// Members per TMA box next to a TYm-row parameter tile at the model's
// occupancy (0: not even one), capped at N and at the box limit of 256.
template <int MODEL, int TYm, int RB>
static int tma_box_members(int N, int B) {
  constexpr bool ROWS = RB > 0;
  const size_t tile_b =
      (size_t)((param_tile_floats<MODEL, TYm, ROWS>(B, false) + 1) & ~1LL) * sizeof(float) + 16;
  const size_t per_member = (size_t)(TYm + 2) * kBoxW * sizeof(float);
  const size_t budget = (size_t)227 * 1024 / TileOcc<MODEL, RB>::value - 1024;
  if (budget < tile_b + per_member) return 0;
  const size_t nc = (budget - tile_b) / per_member;
  return (int)std::min<size_t>(nc, (size_t)std::min(N, 256));
}

// Launch with member staging into a shared-memory box when a box of at
// least one member fits next to the parameter tile at the model's
// occupancy; returns false to fall back.  The box is filled by the tensor
// memory accelerator when the members allow it (W % 4 == 0, a 16-byte
// aligned base: f.vec4), else by 4-byte asynchronous copies (the tensor map
// is then left empty and never used).
template <int MODEL, bool SADDLE, int TYm, int RB>
static bool launch_tile_tma(const Field &f, int tiles_x, int tiles, cudaStream_t s,
                            cudaError_t *err) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (f.vec4 && !enc) return false;
  // histogram per-bin rows, in the room of the member box
  constexpr bool ROWS = RB > 0;
  const size_t tile_b =
      (size_t)((param_tile_floats<MODEL, TYm, ROWS>(f.B, false) + 1) & ~1LL) * sizeof(float) + 16;
  const size_t per_member = (size_t)(TYm + 2) * kBoxW * sizeof(float);
  const size_t budget = (size_t)227 * 1024 / TileOcc<MODEL, RB>::value - 1024;
  const int nc = tma_box_members<MODEL, TYm, RB>(f.N, f.B);
  if (nc < 1) return false;
  const size_t r4_b = ROWS ? (size_t)r4_floats(f.B, TYm) * sizeof(float) : 0;
  if (tile_b + r4_b > budget) return false;
  CUtensorMap map;
  memset(&map, 0, sizeof(map));
  if (f.vec4) {
    const cuuint64_t dims[3] = {(cuuint64_t)f.W, (cuuint64_t)f.H, (cuuint64_t)f.N};
    const cuuint64_t strides[2] = {(cuuint64_t)f.W * sizeof(float),
                                   (cuuint64_t)f.plane * sizeof(float)};
    const cuuint32_t box[3] = {(cuuint32_t)kBoxW, (cuuint32_t)(TYm + 2), (cuuint32_t)nc};
    const cuuint32_t estr[3] = {1, 1, 1};
    if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(f.ens), dims, strides,
            box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
  }
  // per device: the attribute is set once (several host threads may race to
  // set it; setting it twice is harmless, the flag itself is atomic)
  static std::atomic<bool> attr_set[128] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) {
    cudaGetLastError();
    return false;
  }
  if (!attr_set[dev].load(std::memory_order_acquire)) {
    if (cudaFuncSetAttribute(tile_kernel_tma<MODEL, SADDLE, TYm, RB, false>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024) !=
            cudaSuccess ||
        cudaFuncSetAttribute(tile_kernel_tma<MODEL, SADDLE, TYm, RB, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024) !=
            cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    attr_set[dev].store(true, std::memory_order_release);
  }
  Field g = f;
  g.tma_nc = nc;
  const size_t smem = std::max((size_t)nc * per_member, r4_b) + tile_b;
  if (f.vec4)
    tile_kernel_tma<MODEL, SADDLE, TYm, RB, false><<<tiles, NTHREADS, smem, s>>>(g, tiles_x, map);
  else
    tile_kernel_tma<MODEL, SADDLE, TYm, RB, true><<<tiles, NTHREADS, smem, s>>>(g, tiles_x, map);
  *err = cudaGetLastError();
  return true;
}

// Box staging of one field's members with TYm-row tiles at the occupancy
// of (MODEL, RB): members per box (0: not possible) and the CTA's shared
// memory bytes, as launch_tile_tma sets them up (by the tensor memory
// accelerator or, for members it cannot address, by asynchronous copies).
template <int MODEL, int TYm, int RB>
static int tma_plan_t(const Field &f, size_t *smem) {
  constexpr bool ROWS = RB > 0;
  const size_t tile_b =
      (size_t)((param_tile_floats<MODEL, TYm, ROWS>(f.B, false) + 1) & ~1LL) * sizeof(float) + 16;
  const size_t per_member = (size_t)(TYm + 2) * kBoxW * sizeof(float);
  const size_t budget = (size_t)227 * 1024 / TileOcc<MODEL, RB>::value - 1024;
  const int nc = tma_box_members<MODEL, TYm, RB>(f.N, f.B);
  const size_t r4_b = ROWS ? (size_t)r4_floats(f.B, TYm) * sizeof(float) : 0;
  if (nc < 1 || tile_b + r4_b > budget) return 0;
  *smem = std::max((size_t)nc * per_member, r4_b) + tile_b;
  return nc;
}

int tma_plan(int model, int TYm, int RB, const Field &f, size_t *smem) {
  if (model == kUniform && RB == 0) return TYm == 8 ? tma_plan_t<kUniform, 8, 0>(f, smem)
                                                    : tma_plan_t<kUniform, 16, 0>(f, smem);
  if (model == kEpan && RB == 0) return TYm == 8 ? tma_plan_t<kEpan, 8, 0>(f, smem)
                                                 : tma_plan_t<kEpan, 16, 0>(f, smem);
  if (model == kHist && TYm == 8 && RB == 8 && f.B <= 8 && f.N <= 65535)
    return tma_plan_t<kHist, 8, 8>(f, smem);
  if (model == kHist && TYm == 8 && RB == 16 && f.B <= 16 && f.N <= 65535)
    return tma_plan_t<kHist, 8, 16>(f, smem);
  return 0;
}

bool encode_member_map(void *map, const Field &f, int TYm, int nc) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)f.W, (cuuint64_t)f.H, (cuuint64_t)f.N};
  const cuuint64_t strides[2] = {(cuuint64_t)f.W * sizeof(float),
                                 (cuuint64_t)f.plane * sizeof(float)};
  const cuuint32_t box[3] = {(cuuint32_t)kBoxW, (cuuint32_t)(TYm + 2), (cuuint32_t)nc};
  const cuuint32_t estr[3] = {1, 1, 1};
  return enc(static_cast<CUtensorMap *>(map), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
             const_cast<float *>(f.ens), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int MODEL, bool FM, bool SADDLE, int TYm, int RB>
static cudaError_t launch_tile_h(const Field &f, cudaStream_t s) {
  size_t smem = (size_t)tile_floats(MODEL, f.B, TYm) * sizeof(float);
  // histogram per-bin rows after the tile (launch_tile checked that they fit)
  if constexpr (RB > 0)
    smem = (size_t)((param_tile_floats<MODEL, TYm, true>(f.B, FM) + 3) & ~3LL) * sizeof(float) +
           (size_t)r4_floats(f.B, TYm) * sizeof(float);
  // per device: the attribute is set once (several host threads may race to
  // set it; setting it twice is harmless, the flag itself is atomic)
  static std::atomic<bool> attr_set[128] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
  if (!attr_set[dev].load(std::memory_order_acquire)) {
    // the largest tile of this model (64 bins; the histogram adds its tail
    // table, total, status and ordering scratch, the estimator its running
    // mass sums: 95 KB and 173 KB at 10 x 34), or the per-bin rows' bound
    const size_t most = std::max((size_t)tile_floats(MODEL, kMaxBins, TYm) * sizeof(float),
                                 MODEL == kHist ? (size_t)227 * 1024 : (size_t)0);
    e = cudaFuncSetAttribute(tile_kernel<MODEL, FM, SADDLE, TYm, RB>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)most);
    if (e != cudaSuccess) {
      cudaGetLastError();  // do not leave the failed call as the last error
      return e;
    }
    attr_set[dev].store(true, std::memory_order_release);
  }
  Field g = f;
  g.vec4 = (f.ens != nullptr) && (f.W % 4 == 0) && ((reinterpret_cast<uintptr_t>(f.ens) & 15) == 0);
  const int tiles_x = (f.W + TX - 1) / TX, tiles_y = (f.y1 - f.y0 + TYm - 1) / TYm;
  if (tiles_y <= 0) return cudaSuccess;
  const long long tiles = (long long)tiles_x * tiles_y;
  if (tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
  if constexpr (FM) {
    cudaError_t te = cudaSuccess;
    if (launch_tile_tma<MODEL, SADDLE, TYm, RB>(g, tiles_x, (int)tiles, s, &te)) return te;
  }
  tile_kernel<MODEL, FM, SADDLE, TYm, RB><<<(int)tiles, NTHREADS, smem, s>>>(g, tiles_x);
  return cudaGetLastError();
}

// bytes of a per-bin-row histogram tile of TYm rows at B bins, the fused
// kernel's layout (members counted in registers: small parameter tile)
static size_t hist_rows_bytes(int B, int TYm) {
  return (size_t)((hist_rows_tile_floats(B, TYm, false) + 3) & ~3LL) * sizeof(float) +
         (size_t)r4_floats(B, TYm) * sizeof(float) + 16;
}

template <int MODEL, bool FM, bool SADDLE>
static cudaError_t launch_tile(const Field &f, cudaStream_t s) {
  if constexpr (MODEL == kEpan && FM) {
    if (f.N <= tma_box_members<kEpan, 8, 0>(f.N, f.B))
      return launch_tile_h<MODEL, FM, SADDLE, 8, 0>(f, s);
  }
  if constexpr (MODEL == kHist) {
    // Per-bin rows on 8-row tiles: up to 8 bins at four CTAs per SM, up to
    // 16 at two (members counted in registers: at most 65535 of them);
    // otherwise the segment walker on 16-row tiles, where the smaller halo
    // wins.  From members the box staging (tensor memory accelerator or
    // asynchronous copies) applies to every field; from parameters the rows
    // are built from registers.
    const bool counts_ok = !FM || f.N <= 65535;
    if (counts_ok && f.B <= 8 &&
        hist_rows_bytes(f.B, 8) <= (size_t)227 * 1024 / TileOcc<kHist, 8>::value - 1024)
      return launch_tile_h<MODEL, FM, SADDLE, 8, 8>(f, s);
    if (counts_ok && f.B <= 16 &&
        hist_rows_bytes(f.B, 8) <= (size_t)227 * 1024 / TileOcc<kHist, 16>::value - 1024)
      return launch_tile_h<MODEL, FM, SADDLE, 8, 16>(f, s);
    return launch_tile_h<MODEL, FM, SADDLE, TY, 0>(f, s);
  }
  return launch_tile_h<MODEL, FM, SADDLE, TileH<MODEL>::value, 0>(f, s);
}

template <bool SADDLE>
static cudaError_t launch_closed_t(const Field &f, int model, bool fm, cudaStream_t s) {
  if (model == kUniform) return fm ? launch_tile<kUniform, true, SADDLE>(f, s)
                                   : launch_tile<kUniform, false, SADDLE>(f, s);
  if (model == kEpan) return fm ? launch_tile<kEpan, true, SADDLE>(f, s)
                                : launch_tile<kEpan, false, SADDLE>(f, s);
  if (model == kGauss) return fm ? launch_tile<kGauss, true, SADDLE>(f, s)
                                 : launch_tile<kGauss, false, SADDLE>(f, s);
  if (model == kHist) return fm ? launch_tile<kHist, true, SADDLE>(f, s)
                                : launch_tile<kHist, false, SADDLE>(f, s);
  if (model == kSemi) return fm ? launch_tile<kSemi, true, SADDLE>(f, s)
                                : launch_tile<kSemi, false, SADDLE>(f, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_closed(const Field &f, int model, bool from_members, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  if (f.cptypes & (kMin | kMax)) e = launch_closed_t<false>(f, model, from_members, s);
  if (e == cudaSuccess && (f.cptypes & kSaddle))
    e = launch_closed_t<true>(f, model, from_members, s);
  return e;
}

cudaError_t launch_eb_params(const float *d, float eb, long long n, float *params,
                             cudaStream_t s) {
  eb_params_kernel<<<grid_for(n, 256), 256, 0, s>>>(d, eb, n, params);
  return cudaGetLastError();
}

}  // namespace ucp
