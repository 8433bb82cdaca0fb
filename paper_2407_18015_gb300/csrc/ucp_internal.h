// ucp_internal.h -- host-side internals shared by the C ABI translation units.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "ucp.h"

constexpr int kMaxBinsHost = 64;

struct ucp_ctx {
  int device = 0;
  int sm_count = 0;
  char last_error[256] = {0};
  // backward partial rows and other scratch (grown on demand)
  void *work = nullptr;
  size_t work_bytes = 0;
  // device copies for the host-buffer entry point
  float *host_ens = nullptr;
  size_t host_ens_bytes = 0;
  void *host_out = nullptr;
  size_t host_out_bytes = 0;
  // host-buffer pipeline: pipe[0] copies in, pipe[1] copies out,
  // pipe[2..] compute (one per model, up to kPipeCompute); events per strip:
  // copy landed (pipe_ev[0]), and each compute stream done (pipe_ev[1 + c])
  static constexpr int kPipeCompute = 4;
  cudaStream_t pipe[2 + kPipeCompute] = {};
  cudaEvent_t pipe_ev[1 + kPipeCompute][64] = {};
  // fork of the caller's stream into the compute streams and the joins back
  // (ucp_probability_models)
  cudaEvent_t fork_ev = nullptr;
  cudaEvent_t join_ev[kPipeCompute] = {};
  bool pipe_ready = false;
};

int ucp_set_error(ucp_ctx *ctx, cudaError_t e);
// argument checks of the C ABI (status codes of include/ucp.h), made before
// anything is enqueued: a model description (sampled models allowed or
// not), a grid shape, and the whole argument set of the adjoint
int ucp_valid_desc(const ucp_model_desc *d, bool allow_sampled);
int ucp_valid_shape(long long N, long long H, long long W);
int ucp_valid_backward(const ucp_model_desc *desc, int cptype, int H, int W);
// the fused three-model kernel (uniform, Epanechnikov, histogram of at most 8
// bins, one boundary rule): whether `descs` qualify, with each one's model
// slot, and its launch on rows [y0, y1)
bool ucp_fusable3(const ucp_model_desc *descs, int nmodels, int order[3]);
int ucp_launch_fused3(ucp_ctx *ctx, const float *ens, int N, int H, int W,
                      const ucp_model_desc *descs, const int order[3], unsigned cptypes,
                      float *const *out_min, float *const *out_max, uint8_t *const *status,
                      int y0, int y1, cudaStream_t stream, bool *launched);
int ucp_ensure_work(ucp_ctx *ctx, size_t bytes);
// the context's streams and events of the multi-model entry points (once)
int ucp_ensure_pipe(ucp_ctx *ctx);
// models of one ensemble from host arrays (ucp_probability_host[_models])
int ucp_host_pipeline(ucp_ctx *ctx, const float *ens_host, int N, int H, int W,
                      const ucp_model_desc *descs, int nmodels, unsigned cptypes,
                      float *const *out_min_host, float *const *out_max_host,
                      uint8_t *const *status_host, cudaStream_t stream);
