// noalloc.cu -- ucp_backward_static: the adjoint without any device
// allocation, for callers that must not allocate device memory once they are
// running (for example an application whose own allocator already owns the
// device memory budget, or a latency-critical path on which cudaMalloc /
// cudaFree, which may synchronise the whole device, are not acceptable).
//
// The adjoint scratch that ucp_backward keeps in context workspace (the
// tiles' rings, partial blocks and, for histograms of more than 16 bins,
// partial rows) lives here in a file-scope device array of fixed size
// instead.  Every device that loads
// this library holds the array until the process exits.  Host code may not
// use the array's name as a device address (in host code it names a host
// stand-in), so the device address is looked up once per device with
// cudaGetSymbolAddress, with that device current, on the first call made on
// that device; that first call should therefore come before any stream
// capture.  The address is cached for the life of the process, so the entry
// point must not be used on a device after a reset of its primary context
// (cudaDeviceReset), which reloads the module.  Every call on a device shares
// the one array: calls whose work
// overlaps on the GPU (different streams, no ordering between them) race on
// it.  The array keeps the last call's contents; the histogram adjoint's
// block flags, which must start at zero, are cleared by every call (a memset
// on the stream, no allocation); every other entry read is first written by
// the same call.
#include <cuda_runtime.h>

#include <mutex>

#include "launch.h"
#include "ucp.h"
#include "ucp_internal.h"

using namespace ucp;

namespace {

// 16 MiB of adjoint scratch: for uniform / Epanechnikov the rings (160
// floats per 8 x 32 tile); for histograms of at most 16 bins the block
// flags, the ring (80 * B floats per tile) and at least one partial block of
// 1280 * B floats; for more bins 5 * B * H * W floats of partial rows.
constexpr size_t kStaticRowsFloats = size_t(4) << 20;

__device__ __align__(256) float g_static_rows[kStaticRowsFloats];

constexpr int kMaxDevices = 128;
float *g_rows_dev[kMaxDevices] = {};
int g_sms_dev[kMaxDevices] = {};
std::mutex g_rows_mutex;

// the array's device address and the device's SM count, looked up once per
// device (with that device current)
int static_rows(int dev, float **out, int *sms) {
  if (dev < 0 || dev >= kMaxDevices) return UCP_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_rows_mutex);
  if (!g_rows_dev[dev]) {
    void *p = nullptr;
    int n = 0;
    if (cudaGetSymbolAddress(&p, g_static_rows) != cudaSuccess || p == nullptr ||
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaGetLastError();
      return UCP_ERR_CUDA;
    }
    g_rows_dev[dev] = static_cast<float *>(p);
    g_sms_dev[dev] = n;
  }
  *out = g_rows_dev[dev];
  *sms = g_sms_dev[dev];
  return UCP_OK;
}

}  // namespace

extern "C" size_t ucp_backward_static_capacity(void) { return kStaticRowsFloats; }

extern "C" int ucp_backward_static(const float *params, int H, int W,
                                   const ucp_model_desc *desc, int cptype, const float *weight,
                                   float *grad_params, ucp_stream stream) {
  if (!params || !weight || !grad_params) return UCP_ERR_ARG;
  // the same checks, in the same order, as ucp_backward
  const int vrc = ucp_valid_backward(desc, cptype, H, W);
  if (vrc) return vrc;
  Field f{};
  f.params = params;
  f.plane = (long long)H * W;
  f.N = 1;
  f.H = H;
  f.W = W;
  f.B = desc->bins;
  f.y0 = 0;
  f.y1 = H;
  f.boundary = desc->boundary;
  f.cptypes = (unsigned)cptype;
  // the adjoint's scratch with a single CTA must fit the array (more CTAs
  // take what is left)
  if (backward_scratch_floats(f, desc->model, 1) > kStaticRowsFloats) return UCP_ERR_SHAPE;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return UCP_ERR_CUDA;
  }
  float *rows = nullptr;
  int sms = 0;
  const int rc = static_rows(dev, &rows, &sms);
  if (rc) return rc;
  const cudaError_t e = launch_backward(f, desc->model, cptype, weight, rows, kStaticRowsFloats,
                                        4 * sms, grad_params, (cudaStream_t)stream);
  return e == cudaSuccess ? UCP_OK : UCP_ERR_CUDA;
}
