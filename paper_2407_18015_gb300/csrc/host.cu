// host.cu -- ucp_probability_host: host arrays in, host arrays out.
//
// The grid is cut into row strips.  Strip i's members (rows [r0, r1] -- one
// extra row for the south neighbours of its last row) are copied on a copy
// stream, the strip is computed on a compute stream once its copy event has
// fired, and its output rows go back on a third stream.  Copies of strip i+1
// overlap the compute of strip i and the read-back of strip i-1.
#include <cuda_runtime.h>

#include "launch.h"
#include "ucp_internal.h"

using namespace ucp;

namespace {

constexpr int kMaxStrips = 64;
constexpr size_t kStripBytes = 8u << 20;

int ensure_buffer(ucp_ctx *ctx, void **p, size_t *have, size_t need) {
  if (need <= *have) return UCP_OK;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *have = 0;
  cudaError_t e = cudaMalloc(p, need);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return ucp_set_error(ctx, e);
  }
  *have = need;
  return UCP_OK;
}

int ensure_pipe(ucp_ctx *ctx) {
  if (ctx->pipe_ready) return UCP_OK;
  for (int i = 0; i < 3; ++i) {
    cudaError_t e = cudaStreamCreateWithFlags(&ctx->pipe[i], cudaStreamNonBlocking);
    if (e != cudaSuccess) return ucp_set_error(ctx, e);
  }
  for (int k = 0; k < 2; ++k)
    for (int i = 0; i < kMaxStrips; ++i) {
      cudaError_t e = cudaEventCreateWithFlags(&ctx->pipe_ev[k][i], cudaEventDisableTiming);
      if (e != cudaSuccess) return ucp_set_error(ctx, e);
    }
  ctx->pipe_ready = true;
  return UCP_OK;
}

}  // namespace

int ucp_host_pipeline(ucp_ctx *ctx, const float *ens_host, int N, int H, int W,
                      const ucp_model_desc *desc, unsigned cptypes, float *out_min_host,
                      float *out_max_host, uint8_t *status_host, cudaStream_t stream) {
  const long long plane = (long long)H * W;
  const size_t ens_bytes = (size_t)N * plane * sizeof(float);
  int rc = ensure_buffer(ctx, (void **)&ctx->host_ens, &ctx->host_ens_bytes, ens_bytes);
  if (rc) return rc;
  const size_t out_bytes = (size_t)plane * (2 * sizeof(float) + 1);
  if ((rc = ensure_buffer(ctx, &ctx->host_out, &ctx->host_out_bytes, out_bytes))) return rc;
  if ((rc = ensure_pipe(ctx))) return rc;

  float *d_min = (float *)ctx->host_out;
  float *d_max = d_min + plane;
  uint8_t *d_st = (uint8_t *)(d_max + plane);
  cudaStream_t s_in = ctx->pipe[0], s_cmp = ctx->pipe[1], s_out = ctx->pipe[2];

  // start after the work already queued on the caller's stream
  cudaError_t e = cudaEventRecord(ctx->pipe_ev[0][0], stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s_in, ctx->pipe_ev[0][0], 0);
  if (e != cudaSuccess) return ucp_set_error(ctx, e);

  long long strips = (long long)((ens_bytes + kStripBytes - 1) / kStripBytes);
  if (strips < 1) strips = 1;
  if (strips > kMaxStrips) strips = kMaxStrips;
  if (strips > H) strips = H;
  const int rows = (int)((H + strips - 1) / strips);
  const size_t pitch = (size_t)plane * sizeof(float);

  Field f{};
  f.ens = ctx->host_ens;
  f.out_min = d_min;
  f.out_max = d_max;
  f.status = d_st;
  f.plane = plane;
  f.N = N; f.H = H; f.W = W; f.B = desc->bins;
  f.boundary = desc->boundary;
  f.epan_scale = desc->epan_width_scale > 0.f ? desc->epan_width_scale : 2.2360679774997896f;
  f.cptypes = cptypes;
  f.samples = desc->mc_samples;
  f.seed_lo = (uint32_t)desc->seed;
  f.seed_hi = (uint32_t)(desc->seed >> 32);
  f.field_id = desc->field_id;

  int i = 0;
  for (int r0 = 0; r0 < H && e == cudaSuccess; r0 += rows, ++i) {
    const int r1 = r0 + rows < H ? r0 + rows : H;
    const int c1 = r1 < H ? r1 + 1 : H;  // copy one extra row: south neighbours
    const size_t width = (size_t)(c1 - r0) * W * sizeof(float);
    const size_t off = (size_t)r0 * W;
    if (pitch <= 0x7fffffffu) {
      e = cudaMemcpy2DAsync(ctx->host_ens + off, pitch, ens_host + off, pitch, width, N,
                            cudaMemcpyHostToDevice, s_in);
    } else {
      for (int k = 0; k < N && e == cudaSuccess; ++k)
        e = cudaMemcpyAsync(ctx->host_ens + off + (size_t)k * plane,
                            ens_host + off + (size_t)k * plane, width, cudaMemcpyHostToDevice,
                            s_in);
    }
    if (e != cudaSuccess) break;
    if ((e = cudaEventRecord(ctx->pipe_ev[0][i], s_in)) != cudaSuccess) break;
    if ((e = cudaStreamWaitEvent(s_cmp, ctx->pipe_ev[0][i], 0)) != cudaSuccess) break;
    f.y0 = r0;
    f.y1 = r1;
    e = desc->model == UCP_MVN_MC
            ? launch_mvn_mc(f, true, desc->mc_samples, desc->seed, desc->field_id, s_cmp)
            : launch_closed(f, desc->model, true, s_cmp);
    if (e != cudaSuccess) break;
    if ((e = cudaEventRecord(ctx->pipe_ev[1][i], s_cmp)) != cudaSuccess) break;
    if ((e = cudaStreamWaitEvent(s_out, ctx->pipe_ev[1][i], 0)) != cudaSuccess) break;
    const size_t nb = (size_t)(r1 - r0) * W;
    if ((cptypes & 1u) && out_min_host)
      e = cudaMemcpyAsync(out_min_host + off, d_min + off, nb * sizeof(float),
                          cudaMemcpyDeviceToHost, s_out);
    if (e == cudaSuccess && (cptypes & 2u) && out_max_host)
      e = cudaMemcpyAsync(out_max_host + off, d_max + off, nb * sizeof(float),
                          cudaMemcpyDeviceToHost, s_out);
    if (e == cudaSuccess && status_host)
      e = cudaMemcpyAsync(status_host + off, d_st + off, nb, cudaMemcpyDeviceToHost, s_out);
  }
  cudaError_t e2 = cudaStreamSynchronize(s_in);
  cudaError_t e3 = cudaStreamSynchronize(s_cmp);
  cudaError_t e4 = cudaStreamSynchronize(s_out);
  if (e == cudaSuccess) e = e2 != cudaSuccess ? e2 : (e3 != cudaSuccess ? e3 : e4);
  return ucp_set_error(ctx, e);
}
