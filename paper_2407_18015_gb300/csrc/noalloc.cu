// noalloc.cu -- ucp_backward_static: the adjoint without any device
// allocation, for callers that must not allocate device memory once they are
// running (for example an application whose own allocator already owns the
// device memory budget, or a latency-critical path on which cudaMalloc /
// cudaFree, which may synchronise the whole device, are not acceptable).
//
// The partial rows that ucp_backward keeps in context workspace live here in
// a file-scope device array of fixed size instead.  Every device that loads
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
// it.  The array keeps the last call's contents; nothing in it needs to start
// at zero, because the partials pass writes every entry the gather pass reads.
#include <cuda_runtime.h>

#include <mutex>

#include "launch.h"
#include "ucp.h"
#include "ucp_internal.h"

using namespace ucp;

namespace {

// 16 MiB of partial rows: 5 * Q * H * W floats must fit (Q = 2 for uniform /
// Epanechnikov, Q = bins for histograms).
constexpr size_t kStaticRowsFloats = size_t(4) << 20;

__device__ __align__(256) float g_static_rows[kStaticRowsFloats];

constexpr int kMaxDevices = 128;
float *g_rows_dev[kMaxDevices] = {};
std::mutex g_rows_mutex;

int static_rows(int dev, float **out) {
  if (dev < 0 || dev >= kMaxDevices) return UCP_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_rows_mutex);
  if (!g_rows_dev[dev]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_rows);
    if (e != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return UCP_ERR_CUDA;
    }
    g_rows_dev[dev] = static_cast<float *>(p);
  }
  *out = g_rows_dev[dev];
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
  const size_t Q = desc->model == UCP_HISTOGRAM ? (size_t)desc->bins : 2;
  if ((size_t)H * (size_t)W > kStaticRowsFloats / (5 * Q)) return UCP_ERR_SHAPE;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return UCP_ERR_CUDA;
  }
  float *rows = nullptr;
  const int rc = static_rows(dev, &rows);
  if (rc) return rc;
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
  const cudaError_t e = launch_backward(f, desc->model, cptype, weight, rows, grad_params,
                                        (cudaStream_t)stream);
  return e == cudaSuccess ? UCP_OK : UCP_ERR_CUDA;
}
