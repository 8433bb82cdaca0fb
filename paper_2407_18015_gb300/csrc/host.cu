// host.cu -- ucp_probability_host / ucp_probability_host_models: host arrays
// in, host arrays out.
//
// The grid is cut into row strips.  Strip i's members (the rows not copied
// yet, up to one row past its last computed row, the south neighbours of its
// last row) are copied on a copy stream; every model is computed on its own
// compute stream once that copy has landed, and the strip's output rows of
// every model go back on a read-back stream.  The copy of strip i+1 overlaps the
// compute of strip i and the read-back of strip i-1.  Each member row is
// copied once, whatever the number of models.
#include <cuda_runtime.h>

#include "launch.h"
#include "ucp_internal.h"

using namespace ucp;

namespace {

constexpr int kMaxStrips = 64;
// strips of at least 8 MiB of members, and at most 7 of them: a strip's
// kernels then still cover a few waves of tiles, and the host's work per
// strip (launches, events, read-backs) stays off the critical path (1024 x
// 1024 x 20, three models: 8 strips 0.515 ms, 7 0.503, 12 0.530, 16 0.539)
constexpr size_t kStripBytes = 8u << 20;
constexpr int kPipeStrips = 7;

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

// The device address of mapped pinned host memory p (cudaHostAlloc, or
// cudaHostRegister with mapping), else nullptr.
void *mapped_host(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

}  // namespace

int ucp_ensure_pipe(ucp_ctx *ctx) {
  if (ctx->pipe_ready) return UCP_OK;
  for (int i = 0; i < 2 + ucp_ctx::kPipeCompute; ++i) {
    cudaError_t e = cudaStreamCreateWithFlags(&ctx->pipe[i], cudaStreamNonBlocking);
    if (e != cudaSuccess) return ucp_set_error(ctx, e);
  }
  for (int k = 0; k < 1 + ucp_ctx::kPipeCompute; ++k)
    for (int i = 0; i < kMaxStrips; ++i) {
      cudaError_t e = cudaEventCreateWithFlags(&ctx->pipe_ev[k][i], cudaEventDisableTiming);
      if (e != cudaSuccess) return ucp_set_error(ctx, e);
    }
  for (int k = 0; k <= ucp_ctx::kPipeCompute; ++k) {
    cudaEvent_t *ev = k == 0 ? &ctx->fork_ev : &ctx->join_ev[k - 1];
    cudaError_t e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return ucp_set_error(ctx, e);
  }
  ctx->pipe_ready = true;
  return UCP_OK;
}

int ucp_host_pipeline(ucp_ctx *ctx, const float *ens_host, int N, int H, int W,
                      const ucp_model_desc *descs, int nmodels, unsigned cptypes,
                      float *const *out_min_host, float *const *out_max_host,
                      uint8_t *const *status_host, cudaStream_t stream) {
  const long long plane = (long long)H * W;
  const size_t ens_bytes = (size_t)N * plane * sizeof(float);
  int rc = ensure_buffer(ctx, (void **)&ctx->host_ens, &ctx->host_ens_bytes, ens_bytes);
  if (rc) return rc;
  // per model: P_min and P_max planes, then all status planes
  const size_t out_bytes = (size_t)nmodels * plane * (2 * sizeof(float) + 1);
  if ((rc = ensure_buffer(ctx, &ctx->host_out, &ctx->host_out_bytes, out_bytes))) return rc;
  if ((rc = ucp_ensure_pipe(ctx))) return rc;

  float *d_out = (float *)ctx->host_out;
  uint8_t *d_st = (uint8_t *)(d_out + (size_t)2 * nmodels * plane);
  // the models of a strip run on their own compute streams, so that their
  // kernels share the GPU (one strip's tiles alone are about one wave)
  cudaStream_t s_in = ctx->pipe[0], s_out = ctx->pipe[1];
  const int ncs = nmodels < ucp_ctx::kPipeCompute ? nmodels : ucp_ctx::kPipeCompute;

  // start after the work already queued on the caller's stream
  cudaError_t e = cudaEventRecord(ctx->pipe_ev[0][0], stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s_in, ctx->pipe_ev[0][0], 0);
  if (e != cudaSuccess) return ucp_set_error(ctx, e);

  long long strips = (long long)((ens_bytes + kStripBytes - 1) / kStripBytes);
  if (strips < 1) strips = 1;
  if (strips > kPipeStrips) strips = kPipeStrips;
  if (strips > H) strips = H;
  // strip i computes rows [start[i], start[i+1])
  int start[kMaxStrips + 1];
  int nst = 0;
  const int rows = (int)((H + strips - 1) / strips);
  for (int r = 0; r < H; r += rows) start[nst++] = r;
  start[nst] = H;
  const size_t pitch = (size_t)plane * sizeof(float);

  // every strip's copy first (the copy stream then runs back to back,
  // whatever the host's launch latency), then every strip's kernels and
  // read-backs, each waiting for its copy
  int nstrips = 0, copied = 0;  // rows [0, copied) are on the device
  for (; nstrips < nst && e == cudaSuccess; ++nstrips) {
    const int r1 = start[nstrips + 1];
    const int c1 = r1 < H ? r1 + 1 : H;  // one row past: the south neighbours
    if (c1 > copied) {
      const size_t width = (size_t)(c1 - copied) * W * sizeof(float);
      const size_t off = (size_t)copied * W;
      if (pitch <= 0x7fffffffu) {
        e = cudaMemcpy2DAsync(ctx->host_ens + off, pitch, ens_host + off, pitch, width, N,
                              cudaMemcpyHostToDevice, s_in);
      } else {
        for (int k = 0; k < N && e == cudaSuccess; ++k)
          e = cudaMemcpyAsync(ctx->host_ens + off + (size_t)k * plane,
                              ens_host + off + (size_t)k * plane, width,
                              cudaMemcpyHostToDevice, s_in);
      }
      copied = c1;
    }
    if (e == cudaSuccess) e = cudaEventRecord(ctx->pipe_ev[0][nstrips], s_in);
  }
  // uniform + Epanechnikov + histogram: the fused kernel, one launch per strip
  int order[3];
  const bool fuse = ucp_fusable3(descs, nmodels, order);
  // When every wanted output array is mapped pinned host memory, the fused
  // kernel writes the probabilities straight into it (stores over the host
  // link, concurrent with the member copies): no read-back copies and no
  // read-back after the last strip.
  float *dmin[3] = {}, *dmax[3] = {};
  uint8_t *dst[3] = {};
  bool direct = fuse;
  for (int m = 0; m < nmodels && direct; ++m) {
    if ((cptypes & 1u) && out_min_host[m])
      direct = (dmin[m] = static_cast<float *>(mapped_host(out_min_host[m]))) != nullptr;
    if (direct && (cptypes & 2u) && out_max_host[m])
      direct = (dmax[m] = static_cast<float *>(mapped_host(out_max_host[m]))) != nullptr;
    if (direct && status_host && status_host[m])
      direct = (dst[m] = static_cast<uint8_t *>(mapped_host(status_host[m]))) != nullptr;
  }
  int fused_rc = UCP_OK;
  for (int i = 0; i < nstrips && e == cudaSuccess; ++i) {
    const int r0 = start[i], r1 = start[i + 1];
    for (int c = 0; c < ncs && e == cudaSuccess; ++c)
      e = cudaStreamWaitEvent(ctx->pipe[2 + c], ctx->pipe_ev[0][i], 0);
    bool fused = false;
    if (fuse && e == cudaSuccess) {
      float *omin[3], *omax[3];
      uint8_t *ost[3];
      for (int m = 0; m < 3; ++m) {
        omin[m] = direct ? dmin[m] : d_out + (size_t)(2 * m) * plane;
        omax[m] = direct ? dmax[m] : d_out + (size_t)(2 * m + 1) * plane;
        ost[m] = direct ? dst[m] : d_st + (size_t)m * plane;
      }
      fused_rc = ucp_launch_fused3(ctx, ctx->host_ens, N, H, W, descs, order, cptypes, omin,
                                   omax, ost, r0, r1, ctx->pipe[2], &fused);
      if (fused_rc) break;
    }
    for (int m = 0; m < nmodels && e == cudaSuccess && !fused; ++m) {
      cudaStream_t s_cmp = ctx->pipe[2 + m % ncs];
      const ucp_model_desc *desc = descs + m;
      Field f{};
      f.ens = ctx->host_ens;
      f.out_min = d_out + (size_t)(2 * m) * plane;
      f.out_max = d_out + (size_t)(2 * m + 1) * plane;
      f.status = d_st + (size_t)m * plane;
      f.plane = plane;
      f.N = N; f.H = H; f.W = W; f.B = desc->bins;
      f.boundary = desc->boundary;
      f.epan_scale = desc->epan_width_scale > 0.f ? desc->epan_width_scale : 2.2360679774997896f;
      f.cptypes = cptypes;
      f.samples = desc->mc_samples;
      f.seed_lo = (uint32_t)desc->seed;
      f.seed_hi = (uint32_t)(desc->seed >> 32);
      f.field_id = desc->field_id;
      f.y0 = r0;
      f.y1 = r1;
      e = desc->model == UCP_MVN_MC
              ? launch_mvn_mc(f, true, desc->mc_samples, desc->seed, desc->field_id, s_cmp)
              : launch_closed(f, desc->model, true, s_cmp);
    }
    for (int c = 0; c < ncs && e == cudaSuccess; ++c) {
      e = cudaEventRecord(ctx->pipe_ev[1 + c][i], ctx->pipe[2 + c]);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(s_out, ctx->pipe_ev[1 + c][i], 0);
    }
    if (e != cudaSuccess) break;
    if (fused && direct) continue;  // the kernel wrote the caller's arrays
    const size_t off = (size_t)r0 * W, nb = (size_t)(r1 - r0) * W;
    for (int m = 0; m < nmodels && e == cudaSuccess; ++m) {
      const float *dmin = d_out + (size_t)(2 * m) * plane, *dmax = dmin + plane;
      if ((cptypes & 1u) && out_min_host[m])
        e = cudaMemcpyAsync(out_min_host[m] + off, dmin + off, nb * sizeof(float),
                            cudaMemcpyDeviceToHost, s_out);
      if (e == cudaSuccess && (cptypes & 2u) && out_max_host[m])
        e = cudaMemcpyAsync(out_max_host[m] + off, dmax + off, nb * sizeof(float),
                            cudaMemcpyDeviceToHost, s_out);
      if (e == cudaSuccess && status_host && status_host[m])
        e = cudaMemcpyAsync(status_host[m] + off, d_st + (size_t)m * plane + off, nb,
                            cudaMemcpyDeviceToHost, s_out);
    }
  }
  for (int k = 0; k < 2 + ncs; ++k) {
    const cudaError_t ek = cudaStreamSynchronize(ctx->pipe[k]);
    if (e == cudaSuccess) e = ek;
  }
  if (fused_rc) return fused_rc;
  return ucp_set_error(ctx, e);
}
