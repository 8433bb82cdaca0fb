// launch.h -- internal launch interface between the C ABI (api.cu) and the
// kernel translation units.  Host and device visible; no torch types.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ucp {

// One field of work for the closed-form and Monte Carlo kernels.
struct Field {
  const float *ens;     // [N][H][W] members, or nullptr
  const float *params;  // [P][H][W] parameters, or nullptr
  float *out_min;       // [H][W] or nullptr
  float *out_max;       // [H][W] or nullptr
  float *out_saddle;    // [H][W] or nullptr
  uint8_t *status;      // [H][W] or nullptr
  long long plane;      // H * W
  int N, H, W, B;
  int y0, y1;           // rows [y0, y1) are computed (the arrays cover all H rows)
  int boundary;         // 0 in-grid neighbours, 1 zero at the boundary
  float epan_scale;
  unsigned cptypes;     // bit 1 min, bit 2 max, bit 4 saddle
  bool vec4;            // members may be read as aligned float4 (W % 4 == 0, 16B base)
  int tma_nc;           // members per tensor-memory-accelerator box (TMA staging)
  int samples;          // Monte Carlo / semianalytical samples per vertex
  uint32_t seed_lo, seed_hi, field_id;
};

// Tile of the closed-form kernels: TY x TX vertices plus a one-vertex halo.
constexpr int TY = 16, TX = 32, HY = TY + 2, HX = TX + 2, HALO = HY * HX, NTHREADS = 256;

inline int param_planes(int model, int B) {
  return (model == 2 || model == 4) ? 2 + B : (model == 3 ? 20 : 2);
}

// The uniform, Epanechnikov and histogram (at most 8 bins) models of one
// ensemble in one kernel (fused.cu): the members staged once, every model
// integrated per tile with the arithmetic of its own kernel.  f carries the
// ensemble, grid, rows, boundary, Epanechnikov scale and types; the outputs
// and status arrays of model m (0 uniform, 1 Epanechnikov, 2 histogram) are
// out_min[m], out_max[m], status[m] (each may be null when not wanted).
struct Field3 {
  Field f;
  float *out_min[3];
  float *out_max[3];
  uint8_t *status[3];
};
// Launches the fused kernel when it applies (any member alignment, at most 8
// bins and 65535 members); *launched tells whether it did.
cudaError_t launch_closed3(const Field3 &f, cudaStream_t s, bool *launched);
// cuTensorMapEncodeTiled from the driver (nullptr if unavailable)
void *tensor_map_encoder_fn();
// TMA staging plan of one field for the single-field tile kernels' layout
// (model, TYm-row tiles, RB: per-bin rows of at most RB bins, 0 none): the
// members per box, 0 if TMA staging does not apply; *smem = the CTA's
// dynamic shared memory.  encode_member_map writes the tensor map of the
// field's members for that box (map: a 64-byte aligned CUtensorMap).
int tma_plan(int model, int TYm, int RB, const Field &f, size_t *smem);
bool encode_member_map(void *map, const Field &f, int TYm, int nc);

cudaError_t launch_fit(const Field &f, int model, cudaStream_t s);
cudaError_t launch_closed(const Field &f, int model, bool from_members, cudaStream_t s);
cudaError_t launch_eb_params(const float *d, float eb, long long n, float *params,
                             cudaStream_t s);

// Monte Carlo for the multivariate Gaussian model.
cudaError_t launch_mvn_fit(const Field &f, cudaStream_t s);
cudaError_t launch_mvn_mc(const Field &f, bool from_members, int samples, uint64_t seed,
                          uint32_t field_id, cudaStream_t s);

// Larger neighbour sets (stencil.cu): one thread per vertex of a D x H x W
// grid, parameters [P][D][H][W] in global memory, histogram tail tables
// [D*H*W][B+4] (see stencil.cuh).
struct StencilField {
  const float *params;  // [P][D][H][W]
  const float *tab;     // histogram tail-table rows, or nullptr
  float *out_min;       // [D][H][W] or nullptr
  float *out_max;       // [D][H][W] or nullptr
  uint8_t *status;      // [D][H][W] or nullptr
  long long V;          // D * H * W
  int D, H, W, B;
  int boundary;
  unsigned cptypes;
};
cudaError_t launch_hist_table(const float *params, long long V, int B, float *tab, int sm_count,
                              cudaStream_t s);
cudaError_t launch_stencil(const StencilField &f, int model, int stencil, int sm_count,
                           cudaStream_t s);

// Adjoint.  Scratch `rows` of rows_floats floats: uniform, Epanechnikov and
// histograms of more than 16 bins write partial rows [5][Q][H][W], then
// gather them into grad; histograms of at most 16 bins use a ring of 80 B
// floats per 8 x 32 tile plus a partial block of 5 * B * 256 floats per CTA
// (at most max_ctas CTAs, fewer if the scratch is smaller).
// backward_scratch_floats: the scratch the adjoint uses with `ctas` CTAs.
size_t backward_scratch_floats(const Field &f, int model, int ctas);
cudaError_t launch_backward(const Field &f, int model, int cptype, const float *weight,
                            float *rows, size_t rows_floats, int max_ctas, float *grad,
                            cudaStream_t s);

}  // namespace ucp
