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
  unsigned long long *d_counter = nullptr;
  long long total = 0;
  int nitems = 0;
  size_t smem = 0;
  int grid = 0;
};

namespace {

size_t tile_smem(const BatchItem &b) {
  return (size_t)tile_floats(b.model, b.f.B, kTileHeights[b.th]) * sizeof(float);
}

// dynamic shared memory one CTA may use on this architecture (227 KB)
constexpr size_t kSmemPerBlock = 227 * 1024;

// order, tile and upload a list (synchronous: not inside a stream capture);
// an item whose tile at the requested height would not fit in shared memory
// (histograms with many bins) takes the next lower height
int finalize(ucp_batch *b, std::vector<BatchItem> list, const int *th) {
  for (auto &it : list) {
    it.th = th[it.model];
    while (it.th > 0 && tile_smem(it) > kSmemPerBlock) --it.th;
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

int launch(ucp_batch *b, cudaStream_t s) {
  if (b->total == 0) return UCP_OK;
  cudaError_t e = cudaMemsetAsync(b->d_counter, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return ucp_set_error(b->ctx, e);
  const long long want = std::min<long long>(b->total, b->grid);
  batch_kernel<<<(int)want, NTHREADS, b->smem, s>>>(b->d_items, b->nitems, b->total,
                                                    b->d_counter);
  return ucp_set_error(b->ctx, cudaGetLastError());
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
  cudaError_t e = cudaMalloc(&b->d_counter, sizeof(unsigned long long));
  if (prev >= 0) cudaSetDevice(prev);
  if (e != cudaSuccess) {
    delete b;
    return ucp_set_error(ctx, e);
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
  if (batch->d_counter) cudaFree(batch->d_counter);
  if (prev >= 0) cudaSetDevice(prev);
  delete batch;
  return UCP_OK;
}

}  // extern "C"
