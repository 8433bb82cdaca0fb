// batch.cu -- batched launch of many fields (persistent kernel).
#include "launch.h"
#include "ucp_internal.h"

extern "C" {
int ucp_batch_create(ucp_ctx *ctx, ucp_batch **batch) {
  if (!ctx || !batch) return UCP_ERR_ARG;
  *batch = nullptr;
  return UCP_ERR_UNSUPPORTED;
}
int ucp_batch_add(ucp_batch *batch, const float *, int, int, int, const ucp_model_desc *,
                  unsigned, float *, float *) {
  return batch ? UCP_ERR_UNSUPPORTED : UCP_ERR_ARG;
}
int ucp_batch_tune(ucp_batch *batch, ucp_stream) { return batch ? UCP_ERR_UNSUPPORTED : UCP_ERR_ARG; }
int ucp_batch_run(ucp_batch *batch, ucp_stream) { return batch ? UCP_ERR_UNSUPPORTED : UCP_ERR_ARG; }
int ucp_batch_destroy(ucp_batch *batch) { return batch ? UCP_ERR_UNSUPPORTED : UCP_ERR_ARG; }
}
