// fused.cu -- the uniform, Epanechnikov and histogram models of one ensemble
// in one kernel.
//
// Each model's own tile kernel (closed.cu) stages the members of its tile
// through the tensor memory accelerator, reduces them, and integrates; run
// one after another, the three read the same members three times and wait
// for three sets of copies.  Here one CTA stages a tile's members once: the
// first pass over the member box gives the minimum and maximum (uniform
// parameters, histogram range) and the compensated sums of the
// Epanechnikov fit, the second pass the histogram's bin counts; then every
// vertex of the tile is integrated under the three models.  Every model's
// arithmetic is that of its own kernel (the same member order, sums, rows
// and walks), so the probabilities are the same bit for bit.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <atomic>

#include "device.cuh"
#include "launch.h"
#include "tile.cuh"

namespace ucp {

namespace {

constexpr int kTY3 = 8, kHALO3 = (kTY3 + 2) * 34, kRS3 = hist_r4_stride(kHALO3);
constexpr int kOcc3 = 3;  // resident CTAs per SM

// Shared memory of a fused tile, in floats: the member box, whose room the
// histogram's per-bin rows take after the last read of the box; the
// histogram tile (lo, hi, total, status; then the count / N table), whose lo
// and hi are also the uniform parameters; the Epanechnikov tile (m, w); the
// mbarrier.
__host__ __device__ constexpr long long rows3_floats(int B) {
  return 4LL * hist_r4_rows(B) * kRS3;
}
__host__ __device__ constexpr long long htile3_floats() { return 4LL * kHALO3 + ROWS_MASS_TABLE; }
__host__ __device__ constexpr long long etile3_floats() { return 2LL * kHALO3; }

// Staging of one fused tile (see stage_members_tma: the same box walk, the
// same per-vertex arithmetic for each model; ASYNC: the box filled by
// asynchronous copies, members the tensor memory accelerator cannot
// address).  Returns false if a bounded wait gave up.
template <bool ASYNC>
__device__ __forceinline__ bool stage3(const Field &f, float *smh, float *sme, float *box,
                                       uint64_t *bar, const CUtensorMap *tmap, int ty0, int tx0,
                                       float4 *R4) {
  constexpr int HY = kTY3 + 2, HX = 34, HALO = kHALO3;
  constexpr int PER = (HALO + NTHREADS - 1) / NTHREADS;
  constexpr int PLANE = HY * kBoxW;
  const int N = f.N, nc = f.tma_nc, B = f.B;
  const unsigned box_bytes = (unsigned)(PLANE * nc * sizeof(float));
  const int ylim = min(f.H, f.y1 + 1);
  // element shifts of the asynchronous-copy box (all 0 for the accelerator)
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
  auto shift0 = [&](int p, int k0) { return (eb + (k0 & 3) * pl + rq[p]) & 3; };
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    mbar_init_fence();
  }
  // the histogram masses count / N of up to 255 members
  if (N <= 255)
    for (int c = threadIdx.x; c <= N; c += NTHREADS) smh[4 * HALO + c] = __fdiv_rn((float)c, (float)N);
  __syncthreads();
  unsigned phase = 0;
  // one warp polls the barrier, the others wait at the CTA barrier; every
  // thread then tests the completed phase once (its own acquire)
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
  auto give_up = [&]() {
    // the copy that timed out may still land: wait for it (bounded) before
    // the shared memory is left to another CTA
    if (threadIdx.x == 0) mbar_wait(bar, phase ^ 1u);
    __syncthreads();
    return false;
  };
  // pass 1: minimum, maximum, non-finite flag, compensated sums
  float mn[PER], mx[PER], x0[PER];
  bool nf[PER];
  Kahan s1[PER], s2[PER];
  for (int k0 = 0; k0 < N; k0 += nc) {
    if (!load(k0)) return give_up();
    const int kn = min(nc, N - k0);
#pragma unroll
    for (int p = 0; p < PER; ++p) {
      if (!in[p]) continue;
      const int sh = shift0(p, k0);
      const float *col = box + off[p] + sh;
      // member k of the box at col[at(k)]
      auto at = [&](int k) { return k * PLANE + (pl == 0 ? 0 : ((sh + k * pl) & 3) - sh); };
      // as stage_members_tma: member 0 starts min / max (and adds 0 to the
      // sums), the others in pairs into NaN-propagating min / max
      int k = 0;
      if (k0 == 0) {
        x0[p] = mn[p] = mx[p] = col[0];
        k = 1;
      }
      auto add = [&](float v) {
        const float d = v - x0[p];
        s1[p].add(d);
        s2[p].add(d * d);
      };
#pragma unroll 4
      for (; k + 1 < kn; k += 2) {
        const float v1 = col[at(k)], v2 = col[at(k + 1)];
        mn[p] = fmin3_nan(mn[p], v1, v2);
        mx[p] = fmax3_nan(mx[p], v1, v2);
        add(v1);
        add(v2);
      }
      if (k < kn) {
        const float v = col[at(k)];
        mn[p] = fmin_nan(mn[p], v);
        mx[p] = fmax_nan(mx[p], v);
        add(v);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int p = 0; p < PER; ++p) nf[p] = !(isfinite(mn[p]) && isfinite(mx[p]));
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    if (!in[p]) continue;
    const int l = lv[p];
    smh[l] = nf[p] ? qnan() : mn[p];
    smh[HALO + l] = nf[p] ? qnan() : mx[p];
    float m, w;
    if (mn[p] == mx[p]) {
      m = mn[p];
      w = 0.f;
    } else {
      const float S1 = s1[p].get(), S2 = s2[p].get();
      const float md = S1 / (float)N;
      m = x0[p] + md;
      w = f.epan_scale * sqrtf(fmaxf(S2 - S1 * md, 0.f) / (float)(N - 1));
    }
    sme[l] = nf[p] ? qnan() : m;
    sme[HALO + l] = nf[p] ? qnan() : w;
  }
  // pass 2 (boxes in reverse: the last one of pass 1 is still there): bin
  // counts, 8-bit counters packed in a 64-bit word for up to 255 members,
  // 16-bit ones in two words for more
  const bool wide = N > 255;
  const float *mtab = smh + 4 * HALO;
  float sc[PER];
  bool bin[PER];
  bool any = false;
  unsigned long long cw[PER][2];
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    cw[p][0] = cw[p][1] = 0ull;
    bin[p] = in[p] && !nf[p] && mn[p] != mx[p];
    sc[p] = bin[p] ? __fdiv_rn((float)B, __fsub_rn(mx[p], mn[p])) : 0.f;
    any |= bin[p];
  }
  const int last = ((N - 1) / nc) * nc;
  for (int k0 = last; k0 >= 0; k0 -= nc) {
    if (k0 != last && !load(k0)) return give_up();
    const int kn = min(nc, N - k0);
    if (any) {
#pragma unroll
      for (int p = 0; p < PER; ++p) {
        if (!bin[p]) continue;
        const int sh = shift0(p, k0);
        const float *col = box + off[p] + sh;
        auto at = [&](int k) { return k * PLANE + (pl == 0 ? 0 : ((sh + k * pl) & 3) - sh); };
        if (!wide) {
#pragma unroll 4
          for (int k = 0; k < kn; ++k)
            cw[p][0] += 1ull << (hist_bin_nonneg(col[at(k)], mn[p], sc[p], B) << 3);
        } else {
          for (int k = 0; k < kn; ++k) {
            const int j = hist_bin_nonneg(col[at(k)], mn[p], sc[p], B);
            const unsigned long long inc = 1ull << ((j & 3) << 4);
            cw[p][0] += (j >> 2) == 0 ? inc : 0ull;
            cw[p][1] += (j >> 2) == 1 ? inc : 0ull;
          }
        }
      }
    }
    __syncthreads();
  }
  // the histogram rows take the box's room
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    if (!in[p]) continue;
    hist_row_table_counts<HALO, kRS3, 8>(
        smh, R4, lv[p], B, nf[p], mn[p], mx[p], [&](int k) -> float {
          if (!wide) return mtab[(unsigned)(cw[p][0] >> (k << 3)) & 255u];
          return __fdiv_rn((float)((unsigned)(cw[p][k >> 2] >> ((k & 3) << 4)) & 0xFFFFu),
                           (float)N);
        });
  }
  return true;
}

// Every vertex of a staged fused tile under the three models (the uniform,
// Epanechnikov and histogram branches of integrate_tile).
__device__ __forceinline__ void integrate3(const Field3 &F, int ty0, int tx0, const float *smh,
                                           const float *sme, const float4 *R4) {
  constexpr int TX = 32, HX = 34, HALO = kHALO3, RS = kRS3;
  const Field &f = F.f;
  const int B = f.B;
  const int v = threadIdx.x;
  const int r = v / TX + 1, c = v % TX + 1;
  const int gy = ty0 + r - 1, gx = tx0 + c - 1;
  if (gy >= f.y1 || gx >= f.W) return;
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
  const long long gi = (long long)gy * f.W + gx;
  const bool zero_b = f.boundary == 1 && k < 4;
  auto put = [&](int m, float pmin, float pmax, uint8_t st) {
    if ((f.cptypes & kMin) && F.out_min[m]) F.out_min[m][gi] = pmin;
    if ((f.cptypes & kMax) && F.out_max[m]) F.out_max[m][gi] = pmax;
    if (F.status[m]) F.status[m][gi] = st;
  };
  // uniform (parameters: the histogram tile's lo, hi)
  {
    float T[4], Tc;
    uint8_t st = check_params<kUniform, HALO>(smh, l, B, Tc);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      T[i] = 1.f;
      if (present[i]) st |= check_params<kUniform, HALO>(smh, nl[i], B, T[i]) & (V_NONFINITE | V_BAD);
    }
    float pmin = 0.f, pmax = 0.f;
    if (st & (V_NONFINITE | V_BAD)) {
      pmin = pmax = qnan();
    } else if (!zero_b) {
      UniParams cp{smh[l], smh[HALO + l]}, nb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) nb[i] = UniParams{smh[nl[i]], smh[HALO + nl[i]]};
      uniform_vertex(cp, nb, present, f.cptypes, pmin, pmax);
    }
    put(0, pmin, pmax, st);
  }
  // Epanechnikov
  {
    float T[4], Tc;
    uint8_t st = check_params<kEpan, HALO>(sme, l, B, Tc);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      T[i] = 1.f;
      if (present[i]) st |= check_params<kEpan, HALO>(sme, nl[i], B, T[i]) & (V_NONFINITE | V_BAD);
    }
    float pmin = 0.f, pmax = 0.f;
    if (st & (V_NONFINITE | V_BAD)) {
      pmin = pmax = qnan();
    } else if (!zero_b) {
      EpanParams cp{sme[l], sme[HALO + l]}, nb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) nb[i] = EpanParams{sme[nl[i]], sme[HALO + nl[i]]};
      epan_vertex(cp, nb, present, f.cptypes, pmin, pmax);
    }
    put(1, pmin, pmax, st);
  }
  // histogram: the per-bin row walk
  {
    float T[4], Tc;
    uint8_t st = check_params<kHist, HALO, true>(smh, l, B, Tc);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      T[i] = 1.f;
      if (present[i]) st |= check_params<kHist, HALO, true>(smh, nl[i], B, T[i]) & (V_NONFINITE | V_BAD);
    }
    float pmin = 0.f, pmax = 0.f;
    const float lo1 = smh[l], hi1 = smh[HALO + l];
    if (st & (V_NONFINITE | V_BAD)) {
      pmin = pmax = qnan();
    } else if (lo1 == hi1) {
      float gm = Tc, gM = Tc;
      for (int i = 0; i < 4; ++i) {
        if (!present[i]) continue;
        float gt, lt;
        hist_tails_at_rows(R4 + nl[i], RS, B, smh[nl[i]], smh[HALO + nl[i]], T[i], lo1, gt, lt);
        gm *= gt;
        gM *= lt;
      }
      if (!zero_b) {
        pmin = gm;
        pmax = gM;
      }
    } else if (!zero_b) {
      HistRowWalker nw[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        HistRowWalker &h = nw[i];
        if (!present[i]) {
          h.init_absent();
          continue;
        }
        const float lo = smh[nl[i]], hi = smh[HALO + nl[i]];
        h.init(R4 + nl[i], lo - lo1, T[i]);
        h.seek0<RS>(R4 + nl[i], B, lo == hi ? 0.f : (hi - lo) * (1.f / (float)B));
      }
      hist_walk_rows<RS>(R4 + l, B, hi1 - lo1, nw, pmin, pmax);
    }
    put(2, pmin, pmax, st);
  }
}

template <bool ASYNC>
__global__ void __launch_bounds__(NTHREADS, kOcc3)
    tile3_kernel(Field3 F, int tiles_x, const __grid_constant__ CUtensorMap tmap) {
  extern __shared__ __align__(128) float smem[];
  const Field &f = F.f;
  const int tile = blockIdx.x;
  const int ty0 = f.y0 + (tile / tiles_x) * kTY3, tx0 = (tile % tiles_x) * 32;
  const long long box_floats = (long long)f.tma_nc * (kTY3 + 2) * kBoxW;
  float *smh = smem + max(box_floats, rows3_floats(f.B));
  float *sme = smh + htile3_floats();
  uint64_t *bar = reinterpret_cast<uint64_t *>(sme + ((etile3_floats() + 1) & ~1LL));
  float4 *R4 = reinterpret_cast<float4 *>(smem);
  const bool ok = stage3<ASYNC>(f, smh, sme, smem, bar, &tmap, ty0, tx0, R4);
  __syncthreads();
  if (!ok) {  // a bounded wait gave up: NaN and the timeout flag, every model
    const int v = threadIdx.x, gy = ty0 + v / 32, gx = tx0 + v % 32;
    if (gy < f.y1 && gx < f.W) {
      const long long gi = (long long)gy * f.W + gx;
      for (int m = 0; m < 3; ++m) {
        if ((f.cptypes & kMin) && F.out_min[m]) F.out_min[m][gi] = qnan();
        if ((f.cptypes & kMax) && F.out_max[m]) F.out_max[m][gi] = qnan();
        if (F.status[m]) F.status[m][gi] = V_TIMEOUT;
      }
    }
    return;
  }
  integrate3(F, ty0, tx0, smh, sme, R4);
}

}  // namespace

cudaError_t launch_closed3(const Field3 &F, cudaStream_t s, bool *launched) {
  *launched = false;
  const Field &f = F.f;
  if (f.B < 1 || f.B > 8 || f.N < 1 || f.N > 65535) return cudaSuccess;
  // members the tensor memory accelerator cannot address (W not a multiple
  // of 4, a base not 16-byte aligned) are staged by asynchronous copies
  const bool tma = f.W % 4 == 0 && (reinterpret_cast<uintptr_t>(f.ens) & 15) == 0;
  auto enc = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(tensor_map_encoder_fn());
  if (tma && !enc) return cudaSuccess;
  const size_t fixed_b =
      (size_t)(htile3_floats() + ((etile3_floats() + 1) & ~1LL)) * sizeof(float) + 16;
  const size_t rows_b = (size_t)rows3_floats(f.B) * sizeof(float);
  const size_t per_member = (size_t)(kTY3 + 2) * kBoxW * sizeof(float);
  const size_t budget = (size_t)227 * 1024 / kOcc3 - 1024;
  if (fixed_b + std::max(rows_b, per_member) > budget) return cudaSuccess;
  const int nc = (int)std::min<size_t>((budget - fixed_b) / per_member, (size_t)std::min(f.N, 256));
  const int tiles_x = (f.W + 31) / 32, tiles_y = (f.y1 - f.y0 + kTY3 - 1) / kTY3;
  if (tiles_y <= 0) {
    *launched = true;
    return cudaSuccess;
  }
  const long long tiles = (long long)tiles_x * tiles_y;
  if (tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
  CUtensorMap map;
  memset(&map, 0, sizeof(map));
  if (tma) {
    const cuuint64_t dims[3] = {(cuuint64_t)f.W, (cuuint64_t)f.H, (cuuint64_t)f.N};
    const cuuint64_t strides[2] = {(cuuint64_t)f.W * sizeof(float),
                                   (cuuint64_t)f.plane * sizeof(float)};
    const cuuint32_t box[3] = {(cuuint32_t)kBoxW, (cuuint32_t)(kTY3 + 2), (cuuint32_t)nc};
    const cuuint32_t estr[3] = {1, 1, 1};
    if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(f.ens), dims, strides,
            box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return cudaSuccess;
  }
  // per device: the attribute is set once (host threads may race to set it;
  // setting it twice is harmless, the flag itself is atomic)
  static std::atomic<bool> attr_set[128] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
  if (!attr_set[dev].load(std::memory_order_acquire)) {
    e = cudaFuncSetAttribute(tile3_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             227 * 1024);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(tile3_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               227 * 1024);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return e;
    }
    attr_set[dev].store(true, std::memory_order_release);
  }
  Field3 G = F;
  G.f.tma_nc = nc;
  const size_t smem = std::max((size_t)nc * per_member, rows_b) + fixed_b;
  if (tma)
    tile3_kernel<false><<<(int)tiles, NTHREADS, smem, s>>>(G, tiles_x, map);
  else
    tile3_kernel<true><<<(int)tiles, NTHREADS, smem, s>>>(G, tiles_x, map);
  *launched = true;
  return cudaGetLastError();
}

}  // namespace ucp
