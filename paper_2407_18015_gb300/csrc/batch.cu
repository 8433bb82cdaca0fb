// batch.cu -- many fields (different sizes, member counts, models and
// critical-point types) in one persistent kernel launch.
//
// Work list: every field is cut into tiles of TY x 32 vertices (TY chosen per
// model by the autotuner, 8, 16 or 32).  Fields are ordered by estimated cost
// per tile, most expensive first, so the dynamic hand-out below runs the long
// tiles early and the tail is short.  The persistent kernel (a few CTAs per
// SM, sized by the occupancy calculator) takes tile indices from a global
// atomic counter until the list is exhausted, finds the tile's field by
// binary search over the fields' first-tile indices, and runs the same tile
// body as the single-field kernel (tile.cuh).  ucp_batch_run enqueues a
// counter reset and one launch, so a whole batch can be captured into a CUDA
// graph and replayed.
//
// Autotuner: for each model present, every candidate tile height is timed on
// a batch of that model's fields alone (CUDA events on the caller's stream,
// best of three), and the fastest is kept; results are cached in a small JSON
// file keyed by model, bin count and a member-count class.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <sys/stat.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "device.cuh"
#include "launch.h"
#include "tile.cuh"
#include "ucp_internal.h"

using namespace ucp;

namespace {

constexpr int kTileHeights[3] = {8, 16, 32};

struct BatchItem {
  Field f;
  int model;
  int th;            // index into kTileHeights
  int tiles_x;
  long long first;   // index of the field's first tile in the work list
};

template <int MODEL, int TH>
__device__ __forceinline__ void run_tile(const Field &f, long long local, int tiles_x, float *sm) {
  constexpr int TYv = kTileHeights[TH];
  const int ty0 = f.y0 + (int)(local / tiles_x) * TYv;
  const int tx0 = (int)(local % tiles_x) * 32;
  process_tile<MODEL, true, TYv>(f, ty0, tx0, sm);
}

// three resident CTAs per SM: 80 registers, the histogram walk's budget
__global__ void __launch_bounds__(NTHREADS, 3)
    batch_kernel(const BatchItem *__restrict__ items, int nitems, long long total,
                 unsigned long long *__restrict__ counter) {
  extern __shared__ float sm[];
  __shared__ long long s_tile;
  __shared__ int s_item;
  for (;;) {
    if (threadIdx.x == 0) {
      const long long t = (long long)atomicAdd(counter, 1ull);
      int lo = 0, hi = nitems - 1;
      if (t < total) {
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (items[mid].first <= t) lo = mid;
          else hi = mid - 1;
        }
      }
      s_tile = t;
      s_item = lo;
    }
    __syncthreads();
    const long long t = s_tile;
    const int it = s_item;
    if (t >= total) break;
    const BatchItem &bi = items[it];
    const Field f = bi.f;
    const long long local = t - bi.first;
    switch (bi.model * 3 + bi.th) {
      case 0: run_tile<kUniform, 0>(f, local, bi.tiles_x, sm); break;
      case 1: run_tile<kUniform, 1>(f, local, bi.tiles_x, sm); break;
      case 2: run_tile<kUniform, 2>(f, local, bi.tiles_x, sm); break;
      case 3: run_tile<kEpan, 0>(f, local, bi.tiles_x, sm); break;
      case 4: run_tile<kEpan, 1>(f, local, bi.tiles_x, sm); break;
      case 5: run_tile<kEpan, 2>(f, local, bi.tiles_x, sm); break;
      case 6: run_tile<kHist, 0>(f, local, bi.tiles_x, sm); break;
      case 7: run_tile<kHist, 1>(f, local, bi.tiles_x, sm); break;
      default: run_tile<kHist, 2>(f, local, bi.tiles_x, sm); break;
    }
    __syncthreads();  // shared tile and s_tile are reused by the next tile
  }
}

// ---------------------------------------------------------------------------
// classes of fields whose members the tensor memory accelerator stages: one
// persistent kernel per class (model, tile height, per-bin rows), each at
// its own occupancy, with the single-field kernels' layout and tile body;
// every field carries the tensor map of its members in the device work list

struct alignas(64) TmaItem {
  CUtensorMap tmap;  // the members' box of this field (64-byte aligned)
  Field f;           // f.tma_nc: members per box
  int tiles_x;
  long long first;   // index of the field's first tile in the class's list
};

struct TmaClass {
  int model, ty, rb;
};
// classes 0..5 stage members by the tensor memory accelerator, 6..11 (the
// same kinds) by asynchronous copies (members it cannot address)
constexpr int kNumKinds = 6, kNumTmaCls = 2 * kNumKinds;
constexpr TmaClass kTmaCls[kNumKinds] = {{kUniform, 8, 0}, {kUniform, 16, 0}, {kEpan, 8, 0},
                                         {kEpan, 16, 0},    {kHist, 8, 8},     {kHist, 8, 16}};

// resident CTAs per SM of a class kernel: the single-field kernel's, at
// most four (the persistent loop's own registers do not fit beside the
// tile body's at five)
template <int MODEL, int RB>
struct BatchOcc {
  static constexpr int value = TileOcc<MODEL, RB>::value > 4 ? 4 : TileOcc<MODEL, RB>::value;
};

template <int MODEL, int TYm, int RB, bool ASYNC>
__global__ void __launch_bounds__(NTHREADS, (BatchOcc<MODEL, RB>::value))
    batch_tma_kernel(const TmaItem *__restrict__ items, int nitems, long long total,
                     unsigned long long *__restrict__ counter) {
  extern __shared__ __align__(128) float smem[];
  __shared__ long long s_tile;
  __shared__ int s_item;
  // the current field's description, read from shared memory where used
  // (as the single-field kernel reads its parameter), not held in registers
  __shared__ __align__(16) Field s_f;
  constexpr bool ROWS = RB > 0;
  static_assert(sizeof(Field) % 4 == 0, "copied as words");
  for (;;) {
    if (threadIdx.x == 0) {
      const long long t = (long long)atomicAdd(counter, 1ull);
      int lo = 0, hi = nitems - 1;
      if (t < total) {
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (items[mid].first <= t) lo = mid;
          else hi = mid - 1;
        }
      }
      s_tile = t;
      s_item = lo;
    }
    __syncthreads();
    const long long t = s_tile;
    if (t >= total) break;
    const TmaItem &it = items[s_item];
    for (int w = threadIdx.x; w < (int)(sizeof(Field) / 4); w += NTHREADS)
      reinterpret_cast<int *>(&s_f)[w] = reinterpret_cast<const int *>(&it.f)[w];
    __syncthreads();
    const Field &f = s_f;
    const long long local = t - it.first;
    const int ty0 = f.y0 + (int)(local / it.tiles_x) * TYm, tx0 = (int)(local % it.tiles_x) * 32;
    // the single-field kernel's layout: member box (per-bin rows in its
    // room), parameter tile, mbarrier
    const int box_floats = f.tma_nc * (TYm + 2) * kBoxW;
    const int r4 = ROWS ? r4_floats(f.B, TYm) : 0;
    float *sm = smem + max(box_floats, r4);
    const long long tile_f = param_tile_floats<MODEL, TYm, ROWS>(f.B, false);
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + ((tile_f + 1) & ~1LL));
    const bool ok = process_tile<MODEL, true, TYm, false, true, RB, ASYNC>(
        f, ty0, tx0, sm, &it.tmap, smem, bar, ROWS ? reinterpret_cast<float4 *>(smem) : nullptr);
    __syncthreads();
    // a copy that gave up may still land: this CTA takes no further tile
    if (!ok) break;
    // the barrier's room may hold other data in the next tile
    if (threadIdx.x == 0) mbar_inval(bar);
    __syncthreads();
  }
}

// relative cost of one vertex (bench-calibrated magnitudes; only the order
// of fields matters)
double vertex_cost(int model, int N, int B) {
  if (model == kUniform) return 1.0 + 0.25 * N;
  if (model == kEpan) return 12.0 + 0.3 * N;
  return 8.0 * (B + 1) + 0.5 * N;
}

std::string cache_path() {
  const char *p = getenv("UCP_TUNE_CACHE");
  if (p && *p) return p;
  const char *home = getenv("HOME");
  return std::string(home ? home : "/tmp") + "/.cache/ucp_tune.json";
}

std::string tune_key(int model, int B, int N) {
  const int ncls = N <= 16 ? 0 : (N <= 32 ? 1 : (N <= 64 ? 2 : 3));
  char k[64];
  snprintf(k, sizeof(k), "m%d_b%d_n%d", model, model == kHist ? B : 0, ncls);
  return k;
}

// the cache is a flat JSON object {"key": tile_height_index, ...}
std::map<std::string, int> read_cache() {
  std::map<std::string, int> m;
  FILE *fp = fopen(cache_path().c_str(), "r");
  if (!fp) return m;
  char buf[8192];
  const size_t n = fread(buf, 1, sizeof(buf) - 1, fp);
  fclose(fp);
  buf[n] = 0;
  const char *s = buf;
  while ((s = strchr(s, '"')) != nullptr) {
    const char *e = strchr(s + 1, '"');
    if (!e) break;
    std::string key(s + 1, e - s - 1);
    const char *c = strchr(e, ':');
    if (!c) break;
    const int v = atoi(c + 1);
    if (v >= 0 && v < 3) m[key] = v;
    s = c + 1;
  }
  return m;
}

void write_cache(const std::map<std::string, int> &m) {
  const std::string path = cache_path();
  const size_t slash = path.rfind('/');
  if (slash != std::string::npos && slash > 0) mkdir(path.substr(0, slash).c_str(), 0755);
  FILE *fp = fopen(path.c_str(), "w");
  if (!fp) return;
  fprintf(fp, "{");
  bool first = true;
  for (const auto &kv : m) {
    fprintf(fp, "%s\"%s\": %d", first ? "" : ", ", kv.first.c_str(), kv.second);
    first = false;
  }
  fprintf(fp, "}\n");
  fclose(fp);
}

std::mutex g_cache_mutex;

}  // namespace

struct ucp_batch {
  ucp_ctx *ctx = nullptr;
  std::vector<BatchItem> items;  // in insertion order
  int th[3] = {1, 1, 1};        // tile-height index per model
  bool tuned[3] = {false, false, false};
  bool dirty = true;
  BatchItem *d_items = nullptr;
  size_t d_cap = 0;
  unsigned long long *d_counter = nullptr;  // generic list, then one per TMA class
  long long total = 0;
  int nitems = 0;
  size_t smem = 0;
  int grid = 0;
  // TMA classes: items of class c at d_tma[tma_off[c] .. + tma_n[c])
  TmaItem *d_tma = nullptr;
  size_t d_tma_cap = 0;
  size_t tma_off[kNumTmaCls] = {};
  int tma_n[kNumTmaCls] = {};
  long long tma_total[kNumTmaCls] = {};
  size_t tma_smem[kNumTmaCls] = {};
  int tma_grid[kNumTmaCls] = {};
  // the kernels of one run go to their own streams, forked from and joined
  // back into the caller's, so that one kernel's last tiles overlap the next
  // one's first (capturable: the graph gets parallel branches)
  cudaStream_t lane[1 + kNumTmaCls] = {};
  cudaEvent_t fork_ev = nullptr;
  cudaEvent_t join_ev[1 + kNumTmaCls] = {};
};

namespace {

size_t tile_smem(const BatchItem &b) {
  return (size_t)tile_floats(b.model, b.f.B, kTileHeights[b.th]) * sizeof(float);
}

// dynamic shared memory one CTA may use on this architecture (227 KB)
constexpr size_t kSmemPerBlock = 227 * 1024;

// the class kernel of class c
const void *tma_kernel(int c) {
  switch (c) {
    case 0: return reinterpret_cast<const void *>(batch_tma_kernel<kUniform, 8, 0, false>);
    case 1: return reinterpret_cast<const void *>(batch_tma_kernel<kUniform, 16, 0, false>);
    case 2: return reinterpret_cast<const void *>(batch_tma_kernel<kEpan, 8, 0, false>);
    case 3: return reinterpret_cast<const void *>(batch_tma_kernel<kEpan, 16, 0, false>);
    case 4: return reinterpret_cast<const void *>(batch_tma_kernel<kHist, 8, 8, false>);
    case 5: return reinterpret_cast<const void *>(batch_tma_kernel<kHist, 8, 16, false>);
    case 6: return reinterpret_cast<const void *>(batch_tma_kernel<kUniform, 8, 0, true>);
    case 7: return reinterpret_cast<const void *>(batch_tma_kernel<kUniform, 16, 0, true>);
    case 8: return reinterpret_cast<const void *>(batch_tma_kernel<kEpan, 8, 0, true>);
    case 9: return reinterpret_cast<const void *>(batch_tma_kernel<kEpan, 16, 0, true>);
    case 10: return reinterpret_cast<const void *>(batch_tma_kernel<kHist, 8, 8, true>);
    default: return reinterpret_cast<const void *>(batch_tma_kernel<kHist, 8, 16, true>);
  }
}

// the TMA class of an item at the tuned tile heights, -1 for none
int tma_class_of(const BatchItem &it, const int *th) {
  const int async = it.f.vec4 ? 0 : kNumKinds;
  if (it.model == kUniform || it.model == kEpan) {
    const int ty = kTileHeights[th[it.model]];
    if (ty > 16) return -1;
    return (it.model == kUniform ? 0 : 2) + (ty == 16 ? 1 : 0) + async;
  }
  if (it.f.B <= 8) return 4 + async;
  return it.f.B <= 16 ? 5 + async : -1;
}

// order, tile and upload a list (synchronous: not inside a stream capture).
// Fields whose members fit a box staging go to their class (tile heights of
// uniform and Epanechnikov as tuned, 8 or 16; 8 for histograms of up to 16
// bins) -- with a tensor map when the tensor memory accelerator can address
// them (f.vec4), else with an empty one, staged by asynchronous copies --
// the rest to the generic list; a generic
// item whose tile at the requested height would not fit in shared memory
// (histograms with many bins) takes the next lower height.
int finalize(ucp_batch *b, std::vector<BatchItem> all, const int *th) {
  std::vector<BatchItem> list;
  std::vector<TmaItem> cls[kNumTmaCls];
  size_t csm[kNumTmaCls] = {};
  for (const auto &it : all) {
    const int c = tma_class_of(it, th);
    size_t sm = 0;
    const TmaClass *k = c < 0 ? nullptr : &kTmaCls[c % kNumKinds];
    const int nc = k ? tma_plan(k->model, k->ty, k->rb, it.f, &sm) : 0;
    TmaItem ti{};
    ti.f = it.f;
    ti.f.tma_nc = nc;
    if (nc > 0 && (!ti.f.vec4 || encode_member_map(&ti.tmap, ti.f, k->ty, nc))) {
      ti.tiles_x = (it.f.W + 31) / 32;
      cls[c].push_back(ti);
      csm[c] = std::max(csm[c], sm);
    } else {
      list.push_back(it);
    }
  }
  std::vector<TmaItem> flat;
  for (int c = 0; c < kNumTmaCls; ++c) {
    const TmaClass &k = kTmaCls[c % kNumKinds];
    std::stable_sort(cls[c].begin(), cls[c].end(), [&k](const TmaItem &x, const TmaItem &y) {
      return vertex_cost(k.model, x.f.N, x.f.B) > vertex_cost(k.model, y.f.N, y.f.B);
    });
    long long first = 0;
    for (auto &ti : cls[c]) {
      ti.first = first;
      first += (long long)ti.tiles_x * ((ti.f.H + k.ty - 1) / k.ty);
    }
    b->tma_off[c] = flat.size();
    b->tma_n[c] = (int)cls[c].size();
    b->tma_total[c] = first;
    b->tma_smem[c] = csm[c];
    flat.insert(flat.end(), cls[c].begin(), cls[c].end());
    b->tma_grid[c] = 0;
    if (cls[c].empty()) continue;
    // the plan keeps 1 KB of each CTA's share free, room for the kernel's
    // static shared variables (the field and the claimed tile)
    cudaError_t e = cudaFuncSetAttribute(tma_kernel(c), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)csm[c]);
    int per_sm = 0;
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tma_kernel(c), NTHREADS, csm[c]);
    if (e != cudaSuccess) return ucp_set_error(b->ctx, e);
    b->tma_grid[c] = std::max(per_sm, 1) * b->ctx->sm_count;
  }
  if (flat.size() > b->d_tma_cap) {
    if (b->d_tma) cudaFree(b->d_tma);
    b->d_tma = nullptr;
    b->d_tma_cap = 0;
    cudaError_t e = cudaMalloc(&b->d_tma, flat.size() * sizeof(TmaItem));
    if (e != cudaSuccess) return ucp_set_error(b->ctx, e);
    b->d_tma_cap = flat.size();
  }
  if (!flat.empty()) {
    cudaError_t e = cudaMemcpy(b->d_tma, flat.data(), flat.size() * sizeof(TmaItem),
                               cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return ucp_set_error(b->ctx, e);
  }
  for (auto &it : list) {
    it.th = th[it.model];
    while (it.th > 0 && tile_smem(it) > kSmemPerBlock - 1024) --it.th;
    it.tiles_x = (it.f.W + 31) / 32;
  }
  std::stable_sort(list.begin(), list.end(), [](const BatchItem &x, const BatchItem &y) {
    const double cx = vertex_cost(x.model, x.f.N, x.f.B) * kTileHeights[x.th];
    const double cy = vertex_cost(y.model, y.f.N, y.f.B) * kTileHeights[y.th];
    return cx > cy;
  });
  long long first = 0;
  size_t smem = 0;
  for (auto &it : list) {
    it.first = first;
    const int TYv = kTileHeights[it.th];
    first += (long long)it.tiles_x * ((it.f.H + TYv - 1) / TYv);
    smem = std::max(smem, tile_smem(it));
  }
  if (list.size() > b->d_cap) {
    if (b->d_items) cudaFree(b->d_items);
    b->d_items = nullptr;
    b->d_cap = 0;
    cudaError_t e = cudaMalloc(&b->d_items, list.size() * sizeof(BatchItem));
    if (e != cudaSuccess) return ucp_set_error(b->ctx, e);
    b->d_cap = list.size();
  }
  if (!list.empty()) {
    cudaError_t e = cudaMemcpy(b->d_items, list.data(), list.size() * sizeof(BatchItem),
                               cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return ucp_set_error(b->ctx, e);
  }
  cudaError_t e = cudaFuncSetAttribute(batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)std::max(smem, (size_t)1));
  if (e != cudaSuccess) return ucp_set_error(b->ctx, e);
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel, NTHREADS, smem);
  if (e != cudaSuccess) return ucp_set_error(b->ctx, e);
  if (per_sm < 1) per_sm = 1;
  b->grid = per_sm * b->ctx->sm_count;
  b->total = first;
  b->nitems = (int)list.size();
  b->smem = smem;
  return UCP_OK;
}

// launch one class kernel (c < kNumTmaCls) or the generic kernel (c ==
// kNumTmaCls) on stream s
cudaError_t launch_one(ucp_batch *b, int c, cudaStream_t s) {
  if (c == kNumTmaCls) {
    const long long want = std::min<long long>(b->total, b->grid);
    batch_kernel<<<(int)want, NTHREADS, b->smem, s>>>(b->d_items, b->nitems, b->total,
                                                      b->d_counter);
    return cudaGetLastError();
  }
  const int g = (int)std::min<long long>(b->tma_total[c], b->tma_grid[c]);
  const TmaItem *items = b->d_tma + b->tma_off[c];
  const int n = b->tma_n[c];
  const long long tot = b->tma_total[c];
  unsigned long long *ctr = b->d_counter + 1 + c;
  const size_t sm = b->tma_smem[c];
  switch (c) {
#define UCP_CLS(M, T, R, A) \
  batch_tma_kernel<M, T, R, A><<<g, NTHREADS, sm, s>>>(items, n, tot, ctr); \
  break
    case 0: UCP_CLS(kUniform, 8, 0, false);
    case 1: UCP_CLS(kUniform, 16, 0, false);
    case 2: UCP_CLS(kEpan, 8, 0, false);
    case 3: UCP_CLS(kEpan, 16, 0, false);
    case 4: UCP_CLS(kHist, 8, 8, false);
    case 5: UCP_CLS(kHist, 8, 16, false);
    case 6: UCP_CLS(kUniform, 8, 0, true);
    case 7: UCP_CLS(kUniform, 16, 0, true);
    case 8: UCP_CLS(kEpan, 8, 0, true);
    case 9: UCP_CLS(kEpan, 16, 0, true);
    case 10: UCP_CLS(kHist, 8, 8, true);
    default: UCP_CLS(kHist, 8, 16, true);
#undef UCP_CLS
  }
  return cudaGetLastError();
}

int launch(ucp_batch *b, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(b->d_counter, 0, (1 + kNumTmaCls) * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return ucp_set_error(b->ctx, e);
  // the most expensive classes first: histograms, then Epanechnikov, then
  // uniform, then the generic list
  int order[1 + kNumTmaCls], n = 0;
  for (int c = kNumKinds - 1; c >= 0; --c)
    for (int a = 0; a < 2; ++a)
      if (b->tma_total[c + a * kNumKinds] > 0) order[n++] = c + a * kNumKinds;
  if (b->total > 0) order[n++] = kNumTmaCls;
  if (n == 1) return ucp_set_error(b->ctx, launch_one(b, order[0], s));
  if (n == 0) return UCP_OK;
  e = cudaEventRecord(b->fork_ev, s);
  for (int i = 0; i < n && e == cudaSuccess; ++i) {
    cudaStream_t l = b->lane[i];
    e = cudaStreamWaitEvent(l, b->fork_ev, 0);
    if (e == cudaSuccess) e = launch_one(b, order[i], l);
    if (e == cudaSuccess) e = cudaEventRecord(b->join_ev[i], l);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, b->join_ev[i], 0);
  }
  return ucp_set_error(b->ctx, e);
}

int apply_cache(ucp_batch *b) {
  std::lock_guard<std::mutex> lock(g_cache_mutex);
  const auto m = read_cache();
  for (const auto &it : b->items) {
    if (b->tuned[it.model]) continue;
    auto f = m.find(tune_key(it.model, it.f.B, it.f.N));
    if (f != m.end()) b->th[it.model] = f->second;
  }
  return UCP_OK;
}

}  // namespace

extern "C" {

int ucp_batch_create(ucp_ctx *ctx, ucp_batch **batch) {
  if (!ctx || !batch) return UCP_ERR_ARG;
  *batch = nullptr;
  ucp_batch *b = new (std::nothrow) ucp_batch();
  if (!b) return UCP_ERR_NOMEM;
  b->ctx = ctx;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(ctx->device);
  cudaError_t e = cudaMalloc(&b->d_counter, (1 + kNumTmaCls) * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork_ev, cudaEventDisableTiming);
  for (int i = 0; i <= kNumTmaCls && e == cudaSuccess; ++i) {
    e = cudaStreamCreateWithFlags(&b->lane[i], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join_ev[i], cudaEventDisableTiming);
  }
  if (prev >= 0) cudaSetDevice(prev);
  if (e != cudaSuccess) {
    ucp_set_error(ctx, e);
    ucp_batch_destroy(b);
    return UCP_ERR_CUDA;
  }
  *batch = b;
  return UCP_OK;
}

int ucp_batch_add(ucp_batch *batch, const float *ens, int N, int H, int W,
                  const ucp_model_desc *desc, unsigned cptypes, float *out_min, float *out_max) {
  if (!batch || !ens || !desc) return UCP_ERR_ARG;
  if (desc->model == UCP_MVN_MC || desc->model == UCP_HISTOGRAM_SEMI ||
      desc->model == UCP_GAUSSIAN)
    return UCP_ERR_UNSUPPORTED;
  if (desc->model < UCP_UNIFORM || desc->model > UCP_HISTOGRAM) return UCP_ERR_ARG;
  if (desc->model == UCP_HISTOGRAM && (desc->bins < 1 || desc->bins > kMaxBinsHost))
    return UCP_ERR_ARG;
  if (desc->boundary != UCP_BOUNDARY_INGRID && desc->boundary != UCP_BOUNDARY_ZERO)
    return UCP_ERR_ARG;
  if (desc->stencil != UCP_STENCIL_4 || desc->depth > 1) return UCP_ERR_UNSUPPORTED;
  if (N < 1 || H < 1 || W < 1 || (long long)H * W > 0xFFFFFFFFLL) return UCP_ERR_SHAPE;
  if (cptypes == 0 || (cptypes & ~3u)) return UCP_ERR_ARG;
  if (((cptypes & 1u) && !out_min) || ((cptypes & 2u) && !out_max)) return UCP_ERR_ARG;
  BatchItem it{};
  it.f.ens = ens;
  it.f.out_min = out_min;
  it.f.out_max = out_max;
  it.f.plane = (long long)H * W;
  it.f.N = N;
  it.f.H = H;
  it.f.W = W;
  it.f.B = desc->bins;
  it.f.y0 = 0;
  it.f.y1 = H;
  it.f.boundary = desc->boundary;
  it.f.epan_scale = desc->epan_width_scale > 0.f ? desc->epan_width_scale : 2.2360679774997896f;
  it.f.cptypes = cptypes;
  it.f.vec4 = (W % 4 == 0) && ((reinterpret_cast<uintptr_t>(ens) & 15) == 0);
  it.model = desc->model;
  batch->items.push_back(it);
  batch->dirty = true;
  return UCP_OK;
}

int ucp_batch_tune(ucp_batch *batch, ucp_stream stream) {
  if (!batch) return UCP_ERR_ARG;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(batch->ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = UCP_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    rc = UCP_ERR_CUDA;
  }
  std::map<std::string, int> results;
  for (int model = 0; model < 3 && rc == UCP_OK; ++model) {
    std::vector<BatchItem> sub;
    for (const auto &it : batch->items)
      if (it.model == model) sub.push_back(it);
    if (sub.empty()) continue;
    float best = 1e30f;
    int best_th = batch->th[model];
    for (int th = 0; th < 3 && rc == UCP_OK; ++th) {
      int ths[3] = {th, th, th};
      rc = finalize(batch, sub, ths);
      if (rc != UCP_OK) break;
      float t_min = 1e30f;
      for (int rep = 0; rep < 4 && rc == UCP_OK; ++rep) {  // first run warms up
        cudaEventRecord(e0, s);
        rc = launch(batch, s);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) rc = UCP_ERR_CUDA;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) t_min = std::min(t_min, ms);
      }
      if (t_min < best) {
        best = t_min;
        best_th = th;
      }
    }
    batch->th[model] = best_th;
    batch->tuned[model] = true;
    for (const auto &it : sub) results[tune_key(model, it.f.B, it.f.N)] = best_th;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (rc == UCP_OK) {
    std::lock_guard<std::mutex> lock(g_cache_mutex);
    auto m = read_cache();
    for (const auto &kv : results) m[kv.first] = kv.second;
    write_cache(m);
    rc = finalize(batch, batch->items, batch->th);
    if (rc == UCP_OK) batch->dirty = false;
  }
  if (prev >= 0) cudaSetDevice(prev);
  return rc;
}

int ucp_batch_run(ucp_batch *batch, ucp_stream stream) {
  if (!batch) return UCP_ERR_ARG;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(batch->ctx->device);
  int rc = UCP_OK;
  if (batch->dirty) {
    apply_cache(batch);
    rc = finalize(batch, batch->items, batch->th);
    if (rc == UCP_OK) batch->dirty = false;
  }
  if (rc == UCP_OK) rc = launch(batch, (cudaStream_t)stream);
  if (prev >= 0) cudaSetDevice(prev);
  return rc;
}

int ucp_batch_destroy(ucp_batch *batch) {
  if (!batch) return UCP_ERR_ARG;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(batch->ctx->device);
  if (batch->d_items) cudaFree(batch->d_items);
  if (batch->d_tma) cudaFree(batch->d_tma);
  if (batch->d_counter) cudaFree(batch->d_counter);
  for (int i = 0; i <= kNumTmaCls; ++i) {
    if (batch->lane[i]) cudaStreamDestroy(batch->lane[i]);
    if (batch->join_ev[i]) cudaEventDestroy(batch->join_ev[i]);
  }
  if (batch->fork_ev) cudaEventDestroy(batch->fork_ev);
  if (prev >= 0) cudaSetDevice(prev);
  delete batch;
  return UCP_OK;
}

}  // extern "C"
