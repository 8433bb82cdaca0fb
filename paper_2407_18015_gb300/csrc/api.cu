// api.cu -- the C ABI declared in include/ucp.h.
//
// Host code only: argument validation (before anything is enqueued), the
// context (device, workspace, last CUDA error), and the kernel launches of
// closed.cu, mvn.cu, backward.cu and batch.cu.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <new>

#include "device.cuh"
#include "launch.h"
#include "ucp.h"
#include "ucp_internal.h"

using namespace ucp;

namespace {

const char *kStatusText[] = {
    "ok",
    "invalid argument",
    "invalid shape",
    "CUDA error",
    "out of device memory",
    "bounded device-side wait expired",
    "unsupported combination",
};

struct DeviceGuard {
  int prev = -1;
  cudaError_t err = cudaSuccess;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) err = cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

// the larger-stencil path (stencil.cu) instead of the four-neighbour one
bool uses_stencil(const ucp_model_desc *d) { return d->stencil != UCP_STENCIL_4; }

int slices(const ucp_model_desc *d) { return d->depth > 1 ? d->depth : 1; }

int valid_types(unsigned cptypes, const float *out_min, const float *out_max) {
  if (cptypes == 0 || (cptypes & ~3u)) return UCP_ERR_ARG;
  if ((cptypes & 1u) && !out_min) return UCP_ERR_ARG;
  if ((cptypes & 2u) && !out_max) return UCP_ERR_ARG;
  return UCP_OK;
}

float epan_scale(const ucp_model_desc *d) {
  return d->epan_width_scale > 0.f ? d->epan_width_scale : 2.2360679774997896f;
}

}  // namespace

int ucp_valid_desc(const ucp_model_desc *d, bool allow_sampled) {
  if (!d) return UCP_ERR_ARG;
  if (d->model < UCP_UNIFORM || d->model > UCP_GAUSSIAN) return UCP_ERR_ARG;
  const bool sampled = d->model == UCP_MVN_MC || d->model == UCP_HISTOGRAM_SEMI;
  if (sampled && !allow_sampled) return UCP_ERR_UNSUPPORTED;
  if ((d->model == UCP_HISTOGRAM || d->model == UCP_HISTOGRAM_SEMI) &&
      (d->bins < 1 || d->bins > kMaxBinsHost))
    return UCP_ERR_ARG;
  if (sampled && d->mc_samples < 1) return UCP_ERR_ARG;
  if (d->boundary != UCP_BOUNDARY_INGRID && d->boundary != UCP_BOUNDARY_ZERO) return UCP_ERR_ARG;
  if (d->stencil < UCP_STENCIL_4 || d->stencil > UCP_STENCIL_3D6 || d->depth < 0)
    return UCP_ERR_ARG;
  if (d->depth > 1 && d->stencil != UCP_STENCIL_3D6) return UCP_ERR_ARG;
  if (d->stencil != UCP_STENCIL_4 && d->model > UCP_HISTOGRAM) return UCP_ERR_UNSUPPORTED;
  return UCP_OK;
}

int ucp_valid_shape(long long N, long long H, long long W) {
  if (N < 1 || H < 1 || W < 1) return UCP_ERR_SHAPE;
  // vertex indices are 32-bit (Philox counter word 1); members 64-bit
  if (H * W > 0xFFFFFFFFLL) return UCP_ERR_SHAPE;
  if (H > 0x7FFFFFFFLL || W > 0x7FFFFFFFLL) return UCP_ERR_SHAPE;
  return UCP_OK;
}

// the checks ucp_backward and ucp_backward_static share, before any CUDA call
int ucp_valid_backward(const ucp_model_desc *desc, int cptype, int H, int W) {
  int rc = ucp_valid_desc(desc, false);
  if (rc) return rc;
  if (desc->model == UCP_GAUSSIAN) return UCP_ERR_UNSUPPORTED;
  if (desc->stencil != UCP_STENCIL_4) return UCP_ERR_UNSUPPORTED;
  if (cptype != UCP_MIN && cptype != UCP_MAX) return UCP_ERR_ARG;
  return ucp_valid_shape(1, H, W);
}

int ucp_set_error(ucp_ctx *ctx, cudaError_t e) {
  if (e == cudaSuccess) return UCP_OK;
  if (ctx) snprintf(ctx->last_error, sizeof(ctx->last_error), "%s: %s", cudaGetErrorName(e),
                    cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? UCP_ERR_NOMEM : UCP_ERR_CUDA;
}

int ucp_ensure_work(ucp_ctx *ctx, size_t bytes) {
  if (bytes <= ctx->work_bytes) return UCP_OK;
  if (ctx->work) cudaFree(ctx->work);
  ctx->work = nullptr;
  ctx->work_bytes = 0;
  cudaError_t e = cudaMalloc(&ctx->work, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return ucp_set_error(ctx, e);
  }
  ctx->work_bytes = bytes;
  return UCP_OK;
}

// The fused three-model kernel (fused.cu) when `descs` are one uniform, one
// Epanechnikov and one histogram of at most 8 bins with one boundary rule:
// order[m] = the kernel's model slot of descs[m] (0 uniform, 1
// Epanechnikov, 2 histogram); false otherwise.
bool ucp_fusable3(const ucp_model_desc *descs, int nmodels, int order[3]) {
  if (nmodels != 3) return false;
  bool seen[3] = {false, false, false};
  for (int m = 0; m < 3; ++m) {
    const ucp_model_desc &d = descs[m];
    int slot = d.model == UCP_UNIFORM ? 0 : d.model == UCP_EPANECHNIKOV ? 1
             : d.model == UCP_HISTOGRAM ? 2 : -1;
    if (slot < 0 || seen[slot] || d.stencil != UCP_STENCIL_4 || d.depth > 1) return false;
    if (slot == 2 && d.bins > 8) return false;
    if (d.boundary != descs[0].boundary) return false;
    seen[slot] = true;
    order[m] = slot;
  }
  return true;
}

// Fused launch of the three models on rows [y0, y1) of ens; *launched tells
// whether it applied.
int ucp_launch_fused3(ucp_ctx *ctx, const float *ens, int N, int H, int W,
                      const ucp_model_desc *descs, const int order[3], unsigned cptypes,
                      float *const *out_min, float *const *out_max, uint8_t *const *status,
                      int y0, int y1, cudaStream_t stream, bool *launched) {
  Field3 F{};
  Field &f = F.f;
  f.ens = ens;
  f.plane = (long long)H * W;
  f.N = N; f.H = H; f.W = W;
  f.y0 = y0; f.y1 = y1;
  f.boundary = descs[0].boundary;
  f.cptypes = cptypes;
  for (int m = 0; m < 3; ++m) {
    const int sl = order[m];
    if (sl == 1) f.epan_scale = epan_scale(descs + m);
    if (sl == 2) f.B = descs[m].bins;
    F.out_min[sl] = (cptypes & 1u) ? out_min[m] : nullptr;
    F.out_max[sl] = (cptypes & 2u) ? out_max[m] : nullptr;
    F.status[sl] = status ? status[m] : nullptr;
  }
  return ucp_set_error(ctx, launch_closed3(F, stream, launched));
}

extern "C" {

const char *ucp_status_string(int status) {
  if (status < 0 || status >= (int)(sizeof(kStatusText) / sizeof(kStatusText[0])))
    return "unknown status";
  return kStatusText[status];
}

const char *ucp_version(void) { return "ucp 1.0"; }

int ucp_param_count(const ucp_model_desc *desc) {
  if (ucp_valid_desc(desc, true) != UCP_OK) return 0;
  return param_planes(desc->model, desc->bins);
}

int ucp_create(ucp_ctx **ctx, int device) {
  if (!ctx) return UCP_ERR_ARG;
  *ctx = nullptr;
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return UCP_ERR_CUDA;
  }
  if (device < 0 || device >= n) return UCP_ERR_ARG;
  ucp_ctx *c = new (std::nothrow) ucp_ctx();
  if (!c) return UCP_ERR_NOMEM;
  c->device = device;
  DeviceGuard g(device);
  if (g.err != cudaSuccess) {
    delete c;
    return UCP_ERR_CUDA;
  }
  e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
  if (e != cudaSuccess) {
    delete c;
    return UCP_ERR_CUDA;
  }
  *ctx = c;
  return UCP_OK;
}

int ucp_destroy(ucp_ctx *ctx) {
  if (!ctx) return UCP_ERR_ARG;
  {
    DeviceGuard g(ctx->device);
    if (ctx->work) cudaFree(ctx->work);
    if (ctx->host_ens) cudaFree(ctx->host_ens);
    if (ctx->host_out) cudaFree(ctx->host_out);
    if (ctx->pipe_ready) {
      for (int i = 0; i < 2 + ucp_ctx::kPipeCompute; ++i) cudaStreamDestroy(ctx->pipe[i]);
      for (int k = 0; k < 1 + ucp_ctx::kPipeCompute; ++k)
        for (int i = 0; i < 64; ++i) cudaEventDestroy(ctx->pipe_ev[k][i]);
      if (ctx->fork_ev) cudaEventDestroy(ctx->fork_ev);
      for (int k = 0; k < ucp_ctx::kPipeCompute; ++k)
        if (ctx->join_ev[k]) cudaEventDestroy(ctx->join_ev[k]);
    }
  }
  delete ctx;
  return UCP_OK;
}

const char *ucp_last_error(const ucp_ctx *ctx) { return ctx ? ctx->last_error : ""; }

int ucp_fit(ucp_ctx *ctx, const float *ens, int N, int H, int W, const ucp_model_desc *desc,
            float *params, uint8_t *vertex_status, ucp_stream stream) {
  if (!ctx || !ens || !params) return UCP_ERR_ARG;
  int rc = ucp_valid_desc(desc, true);
  if (rc) return rc;
  if ((rc = ucp_valid_shape(N, (long long)slices(desc) * H, W))) return rc;
  H *= slices(desc);  // the fit is per vertex: D slices are D * H rows
  DeviceGuard g(ctx->device);
  if (g.err != cudaSuccess) return ucp_set_error(ctx, g.err);
  Field f{};
  f.ens = ens;
  f.params = params;
  f.status = vertex_status;
  f.plane = (long long)H * W;
  f.N = N; f.H = H; f.W = W; f.B = desc->bins;
  f.y0 = 0; f.y1 = H;
  f.boundary = desc->boundary;
  f.epan_scale = epan_scale(desc);
  cudaError_t e = desc->model == UCP_MVN_MC ? launch_mvn_fit(f, (cudaStream_t)stream)
                                            : launch_fit(f, desc->model, (cudaStream_t)stream);
  return ucp_set_error(ctx, e);
}

static int probability_impl(ucp_ctx *ctx, const float *ens, const float *params, int N, int H,
                            int W, const ucp_model_desc *desc, unsigned cptypes, float *out_min,
                            float *out_max, uint8_t *vertex_status, cudaStream_t stream) {
  Field f{};
  f.ens = ens;
  f.params = params;
  f.out_min = out_min;
  f.out_max = out_max;
  f.status = vertex_status;
  f.plane = (long long)H * W;
  f.N = N; f.H = H; f.W = W; f.B = desc->bins;
  f.y0 = 0; f.y1 = H;
  f.boundary = desc->boundary;
  f.epan_scale = epan_scale(desc);
  f.cptypes = cptypes;
  f.samples = desc->mc_samples;
  f.seed_lo = (uint32_t)desc->seed;
  f.seed_hi = (uint32_t)(desc->seed >> 32);
  f.field_id = desc->field_id;
  cudaError_t e;
  if (desc->model == UCP_MVN_MC)
    e = launch_mvn_mc(f, ens != nullptr, desc->mc_samples, desc->seed, desc->field_id, stream);
  else
    e = launch_closed(f, desc->model, ens != nullptr, stream);
  return ucp_set_error(ctx, e);
}

// minimum / maximum with a larger stencil: statistics pass into workspace
// (from members), tail tables (histogram), then one thread per vertex
static int stencil_impl(ucp_ctx *ctx, const float *ens, const float *params, int N, int H,
                        int W, const ucp_model_desc *desc, unsigned cptypes, float *out_min,
                        float *out_max, uint8_t *vertex_status, cudaStream_t stream) {
  const int D = slices(desc);
  const long long V = (long long)D * H * W;
  const int B = desc->bins;
  const int P = param_planes(desc->model, B);
  const size_t fit_floats = ens ? (size_t)P * V : 0;
  const size_t tab_floats = desc->model == UCP_HISTOGRAM ? (size_t)(B + 4) * V : 0;
  int rc = ucp_ensure_work(ctx, (fit_floats + tab_floats) * sizeof(float) + 256);
  if (rc) return rc;
  float *work = static_cast<float *>(ctx->work);
  cudaError_t e = cudaSuccess;
  if (ens) {
    Field f{};
    f.ens = ens;
    f.params = work;
    f.plane = V;
    f.N = N; f.H = D * H; f.W = W; f.B = B;
    f.y0 = 0; f.y1 = D * H;
    f.epan_scale = epan_scale(desc);
    e = launch_fit(f, desc->model, stream);
    params = work;
  }
  float *tab = nullptr;
  if (e == cudaSuccess && desc->model == UCP_HISTOGRAM) {
    tab = work + fit_floats;
    e = launch_hist_table(params, V, B, tab, ctx->sm_count, stream);
  }
  if (e == cudaSuccess) {
    StencilField s{};
    s.params = params;
    s.tab = tab;
    s.out_min = out_min;
    s.out_max = out_max;
    s.status = vertex_status;
    s.V = V;
    s.D = D; s.H = H; s.W = W; s.B = B;
    s.boundary = desc->boundary;
    s.cptypes = cptypes;
    e = launch_stencil(s, desc->model, desc->stencil, ctx->sm_count, stream);
  }
  return ucp_set_error(ctx, e);
}

int ucp_probability_from_params(ucp_ctx *ctx, const float *params, int H, int W,
                                const ucp_model_desc *desc, unsigned cptypes, float *out_min,
                                float *out_max, uint8_t *vertex_status, ucp_stream stream) {
  if (!ctx || !params) return UCP_ERR_ARG;
  int rc = ucp_valid_desc(desc, true);
  if (rc) return rc;
  if ((rc = ucp_valid_shape(1, (long long)slices(desc) * H, W))) return rc;
  if ((rc = valid_types(cptypes, out_min, out_max))) return rc;
  DeviceGuard g(ctx->device);
  if (g.err != cudaSuccess) return ucp_set_error(ctx, g.err);
  if (uses_stencil(desc))
    return stencil_impl(ctx, nullptr, params, 1, H, W, desc, cptypes, out_min, out_max,
                        vertex_status, (cudaStream_t)stream);
  return probability_impl(ctx, nullptr, params, 1, H, W, desc, cptypes, out_min, out_max,
                          vertex_status, (cudaStream_t)stream);
}

int ucp_probability(ucp_ctx *ctx, const float *ens, int N, int H, int W,
                    const ucp_model_desc *desc, unsigned cptypes, float *out_min, float *out_max,
                    uint8_t *vertex_status, ucp_stream stream) {
  if (!ctx || !ens) return UCP_ERR_ARG;
  int rc = ucp_valid_desc(desc, true);
  if (rc) return rc;
  if ((rc = ucp_valid_shape(N, (long long)slices(desc) * H, W))) return rc;
  if ((rc = valid_types(cptypes, out_min, out_max))) return rc;
  DeviceGuard g(ctx->device);
  if (g.err != cudaSuccess) return ucp_set_error(ctx, g.err);
  if (uses_stencil(desc))
    return stencil_impl(ctx, ens, nullptr, N, H, W, desc, cptypes, out_min, out_max,
                        vertex_status, (cudaStream_t)stream);
  return probability_impl(ctx, ens, nullptr, N, H, W, desc, cptypes, out_min, out_max,
                          vertex_status, (cudaStream_t)stream);
}

static int saddle_impl(ucp_ctx *ctx, const float *ens, const float *params, int N, int H, int W,
                       const ucp_model_desc *desc, float *out_saddle, uint8_t *vertex_status,
                       cudaStream_t stream) {
  Field f{};
  f.ens = ens;
  f.params = params;
  f.out_saddle = out_saddle;
  f.status = vertex_status;
  f.plane = (long long)H * W;
  f.N = N; f.H = H; f.W = W; f.B = desc->bins;
  f.y0 = 0; f.y1 = H;
  f.boundary = desc->boundary;
  f.epan_scale = epan_scale(desc);
  f.cptypes = kSaddle;
  f.samples = desc->mc_samples;
  f.seed_lo = (uint32_t)desc->seed;
  f.seed_hi = (uint32_t)(desc->seed >> 32);
  f.field_id = desc->field_id;
  cudaError_t e;
  if (desc->model == UCP_MVN_MC)
    e = launch_mvn_mc(f, ens != nullptr, desc->mc_samples, desc->seed, desc->field_id, stream);
  else
    e = launch_closed(f, desc->model, ens != nullptr, stream);
  return ucp_set_error(ctx, e);
}

int ucp_saddle(ucp_ctx *ctx, const float *ens, int N, int H, int W, const ucp_model_desc *desc,
               float *out_saddle, uint8_t *vertex_status, ucp_stream stream) {
  if (!ctx || !ens || !out_saddle) return UCP_ERR_ARG;
  int rc = ucp_valid_desc(desc, true);
  if (rc) return rc;
  if (uses_stencil(desc)) return UCP_ERR_UNSUPPORTED;
  if ((rc = ucp_valid_shape(N, H, W))) return rc;
  DeviceGuard g(ctx->device);
  if (g.err != cudaSuccess) return ucp_set_error(ctx, g.err);
  return saddle_impl(ctx, ens, nullptr, N, H, W, desc, out_saddle, vertex_status,
                     (cudaStream_t)stream);
}

int ucp_saddle_from_params(ucp_ctx *ctx, const float *params, int H, int W,
                           const ucp_model_desc *desc, float *out_saddle,
                           uint8_t *vertex_status, ucp_stream stream) {
  if (!ctx || !params || !out_saddle) return UCP_ERR_ARG;
  int rc = ucp_valid_desc(desc, true);
  if (rc) return rc;
  if (uses_stencil(desc)) return UCP_ERR_UNSUPPORTED;
  if ((rc = ucp_valid_shape(1, H, W))) return rc;
  DeviceGuard g(ctx->device);
  if (g.err != cudaSuccess) return ucp_set_error(ctx, g.err);
  return saddle_impl(ctx, nullptr, params, 1, H, W, desc, out_saddle, vertex_status,
                     (cudaStream_t)stream);
}

int ucp_probability_host(ucp_ctx *ctx, const float *ens_host, int N, int H, int W,
                         const ucp_model_desc *desc, unsigned cptypes, float *out_min_host,
                         float *out_max_host, uint8_t *status_host, ucp_stream stream) {
  if (!ctx || !ens_host) return UCP_ERR_ARG;
  int rc = ucp_valid_desc(desc, true);
  if (rc) return rc;
  if (uses_stencil(desc)) return UCP_ERR_UNSUPPORTED;
  if ((rc = ucp_valid_shape(N, H, W))) return rc;
  if ((rc = valid_types(cptypes, out_min_host, out_max_host))) return rc;
  DeviceGuard g(ctx->device);
  if (g.err != cudaSuccess) return ucp_set_error(ctx, g.err);
  return ucp_host_pipeline(ctx, ens_host, N, H, W, desc, 1, cptypes, &out_min_host,
                           &out_max_host, &status_host, (cudaStream_t)stream);
}

int ucp_probability_models(ucp_ctx *ctx, const float *ens, int N, int H, int W,
                           const ucp_model_desc *descs, int nmodels, unsigned cptypes,
                           float *const *out_min, float *const *out_max,
                           uint8_t *const *vertex_status, ucp_stream stream) {
  if (!ctx || !ens || !descs || !out_min || !out_max) return UCP_ERR_ARG;
  if (nmodels < 1 || nmodels > UCP_MAX_MODELS) return UCP_ERR_ARG;
  int rc = ucp_valid_shape(N, H, W);
  if (rc) return rc;
  if (cptypes == 0 || (cptypes & ~3u)) return UCP_ERR_ARG;
  for (int m = 0; m < nmodels; ++m) {
    if ((rc = ucp_valid_desc(descs + m, true))) return rc;
    if (uses_stencil(descs + m)) return UCP_ERR_UNSUPPORTED;
  }
  DeviceGuard g(ctx->device);
  if (g.err != cudaSuccess) return ucp_set_error(ctx, g.err);
  // uniform + Epanechnikov + histogram: one fused kernel on `stream`
  int order[3];
  if (ucp_fusable3(descs, nmodels, order)) {
    bool launched = false;
    rc = ucp_launch_fused3(ctx, ens, N, H, W, descs, order, cptypes, out_min, out_max,
                           vertex_status, 0, H, (cudaStream_t)stream, &launched);
    if (rc || launched) return rc;
  }
  if ((rc = ucp_ensure_pipe(ctx))) return rc;
  const int ncs = nmodels < ucp_ctx::kPipeCompute ? nmodels : ucp_ctx::kPipeCompute;
  // fork: every compute stream starts after the work queued on `stream`
  cudaError_t e = cudaEventRecord(ctx->fork_ev, (cudaStream_t)stream);
  for (int c = 0; c < ncs && e == cudaSuccess; ++c)
    e = cudaStreamWaitEvent(ctx->pipe[2 + c], ctx->fork_ev, 0);
  if (e != cudaSuccess) return ucp_set_error(ctx, e);
  for (int m = 0; m < nmodels && rc == UCP_OK; ++m)
    rc = probability_impl(ctx, ens, nullptr, N, H, W, descs + m, cptypes,
                          (cptypes & 1u) ? out_min[m] : nullptr,
                          (cptypes & 2u) ? out_max[m] : nullptr,
                          vertex_status ? vertex_status[m] : nullptr, ctx->pipe[2 + m % ncs]);
  // join: `stream` continues after every model (also after a failed launch,
  // so that nothing already queued outlives the call's ordering)
  for (int c = 0; c < ncs && e == cudaSuccess; ++c) {
    e = cudaEventRecord(ctx->join_ev[c], ctx->pipe[2 + c]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent((cudaStream_t)stream, ctx->join_ev[c], 0);
  }
  if (rc != UCP_OK) return rc;
  return ucp_set_error(ctx, e);
}

int ucp_probability_host_models(ucp_ctx *ctx, const float *ens_host, int N, int H, int W,
                                const ucp_model_desc *descs, int nmodels, unsigned cptypes,
                                float *const *out_min_host, float *const *out_max_host,
                                uint8_t *const *status_host, ucp_stream stream) {
  if (!ctx || !ens_host || !descs || !out_min_host || !out_max_host) return UCP_ERR_ARG;
  if (nmodels < 1 || nmodels > UCP_MAX_MODELS) return UCP_ERR_ARG;
  int rc = ucp_valid_shape(N, H, W);
  if (rc) return rc;
  if (cptypes == 0 || (cptypes & ~3u)) return UCP_ERR_ARG;
  for (int m = 0; m < nmodels; ++m) {
    if ((rc = ucp_valid_desc(descs + m, true))) return rc;
    if (uses_stencil(descs + m)) return UCP_ERR_UNSUPPORTED;
  }
  DeviceGuard g(ctx->device);
  if (g.err != cudaSuccess) return ucp_set_error(ctx, g.err);
  return ucp_host_pipeline(ctx, ens_host, N, H, W, descs, nmodels, cptypes, out_min_host,
                           out_max_host, status_host, (cudaStream_t)stream);
}

int ucp_params_from_error_bound(ucp_ctx *ctx, const float *decompressed, float eb, int H,
                                int W, float *params, ucp_stream stream) {
  if (!ctx || !decompressed || !params) return UCP_ERR_ARG;
  if (!(eb >= 0.f) || !isfinite(eb)) return UCP_ERR_ARG;
  int rc = ucp_valid_shape(1, H, W);
  if (rc) return rc;
  DeviceGuard g(ctx->device);
  if (g.err != cudaSuccess) return ucp_set_error(ctx, g.err);
  return ucp_set_error(ctx, launch_eb_params(decompressed, eb, (long long)H * W, params,
                                             (cudaStream_t)stream));
}

int ucp_backward(ucp_ctx *ctx, const float *params, int H, int W, const ucp_model_desc *desc,
                 int cptype, const float *weight, float *grad_params, ucp_stream stream) {
  if (!ctx || !params || !weight || !grad_params) return UCP_ERR_ARG;
  int rc = ucp_valid_backward(desc, cptype, H, W);
  if (rc) return rc;
  DeviceGuard g(ctx->device);
  if (g.err != cudaSuccess) return ucp_set_error(ctx, g.err);
  Field f{};
  f.params = params;
  f.plane = (long long)H * W;
  f.N = 1; f.H = H; f.W = W; f.B = desc->bins;
  f.y0 = 0; f.y1 = H;
  f.boundary = desc->boundary;
  f.cptypes = (unsigned)cptype;
  // scratch blocks of the histogram adjoint: twice the CTAs that can be
  // resident at once (two per SM)
  const int ctas = 4 * ctx->sm_count;
  const size_t floats = backward_scratch_floats(f, desc->model, ctas);
  if ((rc = ucp_ensure_work(ctx, floats * sizeof(float)))) return rc;
  return ucp_set_error(ctx, launch_backward(f, desc->model, cptype, weight, (float *)ctx->work,
                                            floats, ctas, grad_params, (cudaStream_t)stream));
}

}  // extern "C"
