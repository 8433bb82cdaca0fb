/*
 * ucp.h -- C ABI of libucp: per-vertex critical-point probability fields of
 * 2D uncertain scalar fields on one GB300 (sm_103a).
 *
 * Method: Athawale et al., "Uncertainty Visualization of Critical Points of
 * 2D Scalar Fields for Parametric and Nonparametric Probabilistic Models"
 * (arXiv 2407.18015).  Problem statement (Sec. "Background and Problem
 * Setting"): a regular H x W grid; at every vertex p a random variable X_1
 * with finite support [a_1, b_1]; its axis neighbours e, n, w, s carry X_2..X_5;
 * the variables are independent (except for the multivariate Gaussian model).
 * The library returns, per vertex,
 *
 *   P_min = Pr[X_1 < X_n for every neighbour n] = int pdf_1(x) prod_n G_n(x) dx
 *   P_max = Pr[X_1 > X_n for every neighbour n] = int pdf_1(x) prod_n F_n(x) dx
 *
 * (Eq. localMinimumProb; the local maximum by negation, Sec. "Local Maximum
 * Probability"), with F_n the CDF and G_n = 1 - F_n the survival of X_n.
 *
 * Conventions shared by every call
 *   - Arrays are row-major and plane-major.  An ensemble is ens[N][H][W]
 *     float32 (member k of vertex (y,x) at ens[(k*H + y)*W + x]).  Model
 *     parameters are params[P][H][W] float32 (see UCP_* model comments).
 *     Probability fields are [H][W] float32; vertex status is [H][W] uint8.
 *   - Unless a call says "host", every array pointer is a DEVICE pointer on
 *     the context's device, owned by the caller and borrowed for the
 *     stream-ordered duration of the call (the library never frees it).
 *     Work is enqueued on `stream` (NULL = the legacy default stream) and the
 *     call returns without synchronising.
 *   - Neighbours of (y,x): e=(y,x+1), n=(y-1,x), w=(y,x-1), s=(y+1,x).
 *     UCP_BOUNDARY_INGRID uses the in-grid ones (2 at a corner, 3 on an edge;
 *     a 1 x W grid is the paper's two-neighbour case, Sec. "Critical Point
 *     Probability (Two-Pixel Neighborhood)"); UCP_BOUNDARY_ZERO writes 0 at
 *     every vertex that lacks a neighbour.  The paper ignores the boundary.
 *   - Every call returns a ucp_status.  Arguments are validated on the host
 *     before anything is enqueued; UCP_ERR_ARG / UCP_ERR_SHAPE mean nothing
 *     ran.  UCP_ERR_CUDA keeps the CUDA error text (ucp_last_error).
 *     Per-vertex numerical problems never fail a call: they set bits of the
 *     optional vertex_status array (ucp_vertex_flag); P is NaN only for
 *     UCP_V_NONFINITE, UCP_V_BAD_PARAMS, UCP_V_CHOL_FAIL and UCP_V_TIMEOUT.
 *   - No kernel of this library traps, asserts or waits without a bound.
 */
#ifndef UCP_H
#define UCP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ucp_ctx ucp_ctx;
typedef struct ucp_batch ucp_batch;
/* identical to cudaStream_t */
typedef struct CUstream_st *ucp_stream;

typedef enum {
  /* independent uniform, params (a, b): pdf 1/(b-a) on [a, b]
   * (Sec. "Parametric Noise Models").  Fit: a = min, b = max of the members
   * (Sec. "Validation and Performance of Proposed Algorithms"). */
  UCP_UNIFORM = 0,
  /* independent Epanechnikov, params (m, w): pdf 3/(4w)(1-((x-m)/w)^2) on
   * [m-w, m+w] (Sec. "Parametric Noise Models", m=(a+b)/2, w=(b-a)/2).  Fit:
   * m = sample mean, w = epan_width_scale * sample std (N-1 divisor); the
   * paper fixes no constant, the default sqrt(5) matches the variance. */
  UCP_EPANECHNIKOV = 1,
  /* independent B-bin histogram, params (lo, hi, w_0 .. w_{B-1}): B equal
   * bins on [lo, hi], pdf = sum_j w_j/h on bin j (a mixture of
   * non-overlapping uniform kernels, Sec. "Closed-Form Formulation").  Fit:
   * lo = min, hi = max, bin of member x = floor((x - lo) * (B / (hi - lo)))
   * in IEEE binary32 (one rounding per operation), clamped to [0, B-1],
   * w_j = count_j / N.  Masses need not sum to 1: the survival is used in the
   * mixture form sum_j w_j S_j(x). */
  UCP_HISTOGRAM = 2,
  /* multivariate Gaussian over (X_v, X_e, X_n, X_w, X_s) (the prior work the
   * paper compares with, Sec. "Comparison of Parametric Vs. Nonparametric
   * Models"), evaluated by Monte Carlo.  params: planes 0..4 = means of
   * (v, e, n, w, s); planes 5..19 = their covariance (N-1 divisor), packed
   * lower triangle row by row ((0,0),(1,0),(1,1),(2,0),...); entries of
   * absent neighbours are 0.  Sampling contract: sample s of the vertex with
   * linear index i draws two Philox4x32-10 blocks (Salmon et al., SC'11) with
   * counter (s, i, field_id, j), j = 0, 1, and key (seed & 0xffffffff,
   * seed >> 32); words r give uniforms ((r >> 9) + 0.5) * 2^-23 (exact in
   * binary32, strictly inside (0, 1)); Box-Muller
   * on (u0,u1), (u2,u3), (u4,u5) gives z_0..z_5; x = mu + L z with L the
   * Cholesky factor of the covariance of the vertex and its present
   * neighbours in the order v, e, n, w, s (z_0..z_k used).  If the
   * factorisation fails, eps*I is added, eps = 1e-6 * trace / (k+1), times
   * 10 per retry, three retries (UCP_V_CHOL_JITTER), else UCP_V_CHOL_FAIL.
   * A zero-trace covariance is deterministic (UCP_V_DEGENERATE). */
  UCP_MVN_MC = 3,
  /* the histogram model (same parameters, same fit) evaluated by the paper's
   * semianalytical estimator (Sec. "Semianalytical Solution"): mc_samples
   * samples x_s from the centre's histogram; the probability of each being
   * below (above) every neighbour is exact from the neighbours' histograms
   * (bin of x_s plus the prefix sum of the masses); the estimate is the
   * centre's total mass times the mean over the samples.  Sampling contract:
   * sample s of the vertex with linear index i uses the Philox4x32-10 block
   * with counter (s >> 1, i, field_id, 2) and the seed as key; words 0, 1 (s
   * even) or 2, 3 (s odd) give uniforms ua, ub as above; the bin is the
   * number of running mass sums C_1..C_B (IEEE binary32, bin order) that are
   * <= ua * T (T = C_B), clamped to B-1; x_s = lo + (bin + ub) h.  A
   * point-mass centre is exact.  Minimum, maximum and saddle; no adjoint,
   * no batch. */
  UCP_HISTOGRAM_SEMI = 4,
  /* independent Gaussian, params (m, s): pdf N(m, s^2) -- the parametric
   * model the paper compares the closed forms with (Sec. "Comparison of
   * Parametric Vs. Nonparametric Models", there by Monte Carlo).  Fit:
   * m = sample mean, s = sample std (N-1 divisor).  Without a finite support
   * the integral over t = (x - m_v)/s_v is taken by quadrature: |t| <= 8,
   * cut at -3, 0, 3 and at every neighbour's centre and centre +- 8 of its
   * standard deviations (in t), the 16-point Gauss-Legendre rule on each
   * piece (|dP| ~ 1e-6 in FP32).  Minimum, maximum and saddle; no adjoint,
   * no batch, four-neighbour stencil only. */
  UCP_GAUSSIAN = 5
} ucp_model;

typedef enum { UCP_MIN = 1, UCP_MAX = 2 } ucp_cptype; /* bit mask */

typedef enum { UCP_BOUNDARY_INGRID = 0, UCP_BOUNDARY_ZERO = 1 } ucp_boundary;

/* Neighbour set of a vertex.  UCP_STENCIL_4 is the paper's (e, n, w, s).
 * The others are the extension the paper names in Sec. "Conclusion"
 * (six- or eight-pixel neighbourhoods of a triangulated grid, and 3D
 * grids); offsets (dz, dy, dx):
 *   UCP_STENCIL_6:   e, n, w, s, ne (0,-1,+1), sw (0,+1,-1) -- the grid with
 *                    every cell cut along its lower-left to upper-right
 *                    diagonal (y grows southwards)
 *   UCP_STENCIL_8:   e, n, w, s, ne, nw (0,-1,-1), sw, se (0,+1,+1)
 *   UCP_STENCIL_3D6: e, n, w, s, below (-1,0,0), above (+1,0,0) on a
 *                    D x H x W grid (ucp_model_desc.depth = D)
 * The larger stencils give P_min / P_max of the closed-form models
 * (uniform, Epanechnikov, histogram) through ucp_probability,
 * ucp_probability_from_params and ucp_fit; other entry points and models
 * return UCP_ERR_UNSUPPORTED for them.  UCP_BOUNDARY_ZERO writes 0 wherever
 * the stencil is incomplete. */
typedef enum {
  UCP_STENCIL_4 = 0,
  UCP_STENCIL_6 = 1,
  UCP_STENCIL_8 = 2,
  UCP_STENCIL_3D6 = 3
} ucp_stencil;

typedef enum {
  UCP_OK = 0,
  UCP_ERR_ARG = 1,         /* null pointer, bad enum, bins/samples out of range */
  UCP_ERR_SHAPE = 2,       /* N, H or W < 1, or sizes beyond the index limits   */
  UCP_ERR_CUDA = 3,        /* a CUDA call failed; see ucp_last_error              */
  UCP_ERR_NOMEM = 4,       /* device workspace could not be allocated             */
  UCP_ERR_TIMEOUT = 5,     /* a bounded device-side wait expired                  */
  UCP_ERR_UNSUPPORTED = 6  /* the combination is not implemented                  */
} ucp_status;

typedef enum {
  UCP_V_DEGENERATE = 1,  /* the vertex is a point mass (min == max of members)  */
  UCP_V_NONFINITE = 2,   /* a participating member or parameter is NaN/Inf      */
  UCP_V_BAD_PARAMS = 4,  /* a participating parameter set is invalid
                            (a > b, w < 0, lo > hi, a negative mass)            */
  UCP_V_CHOL_JITTER = 8, /* MVN covariance needed diagonal jitter               */
  UCP_V_CHOL_FAIL = 16,  /* MVN covariance could not be factorised              */
  UCP_V_TIMEOUT = 32     /* a bounded device-side wait while staging this
                            vertex's tile expired; P is NaN                     */
} ucp_vertex_flag;

typedef struct {
  int model;              /* ucp_model                                          */
  int bins;               /* histogram bin count B, 1..64 (ignored otherwise)   */
  float epan_width_scale; /* Epanechnikov w = scale * std; <= 0 means sqrt(5)   */
  int mc_samples;         /* samples per vertex, MVN and semianalytical (>= 1)  */
  uint64_t seed;          /* MVN Philox key                                     */
  uint32_t field_id;      /* MVN Philox counter word 2                          */
  int boundary;           /* ucp_boundary                                       */
  int stencil;            /* ucp_stencil (0 = the paper's four neighbours)      */
  int depth;              /* slices D of a 3D grid (UCP_STENCIL_3D6 only; 0 or
                             1 = a 2D grid).  With D > 1 every array of a call
                             has D slices: ens[N][D][H][W], params[P][D][H][W],
                             outputs and status [D][H][W]; H and W are the
                             slice sizes.                                       */
} ucp_model_desc;

/* Text of a status code (static storage). */
const char *ucp_status_string(int status);

/* Library version string "ucp <major>.<minor>". */
const char *ucp_version(void);

/* Number of parameter planes P of a model: 2 (uniform, Epanechnikov),
 * 2 + bins (histogram, both evaluations), 20 (MVN); 0 for an invalid
 * descriptor. */
int ucp_param_count(const ucp_model_desc *desc);

/* Create a context bound to CUDA device `device`.  The context owns its
 * device workspace (grown on demand, freed by ucp_destroy) and caches
 * kernel attributes.  One context may be used from one host thread at a
 * time.  Errors: UCP_ERR_ARG (ctx NULL), UCP_ERR_CUDA (no such device). */
int ucp_create(ucp_ctx **ctx, int device);
int ucp_destroy(ucp_ctx *ctx);

/* Text of the last CUDA error seen by this context ("" if none). */
const char *ucp_last_error(const ucp_ctx *ctx);

/* Fit the per-vertex model (the statistics pass only): reads ens[N][H][W],
 * writes params[P][H][W] and, if vertex_status is not NULL, status[H][W]
 * (UCP_V_DEGENERATE, UCP_V_NONFINITE; non-finite members give NaN params).
 * Models: Sec. "Parametric Noise Models" / "Nonparametric Noise Models"
 * (fit rules in ucp_model).  For UCP_MVN_MC the covariance involves the
 * neighbours' members. */
int ucp_fit(ucp_ctx *ctx, const float *ens, int N, int H, int W, const ucp_model_desc *desc,
            float *params, uint8_t *vertex_status, ucp_stream stream);

/* Probability fields from parameters supplied directly, e.g. the uniform
 * model [d' - eb/2, d' + eb/2] of a decompressed field d' with error bound eb
 * (Sec. "Real Datasets", climate data).  cptypes: UCP_MIN | UCP_MAX; out_min
 * (out_max) must be non-NULL when its bit is set.  vertex_status may be
 * NULL. */
int ucp_probability_from_params(ucp_ctx *ctx, const float *params, int H, int W,
                                const ucp_model_desc *desc, unsigned cptypes, float *out_min,
                                float *out_max, uint8_t *vertex_status, ucp_stream stream);

/* Fused fit + probability from an ensemble (one pass over the members; the
 * parameters never reach global memory).  Arguments as above. */
int ucp_probability(ucp_ctx *ctx, const float *ens, int N, int H, int W,
                    const ucp_model_desc *desc, unsigned cptypes, float *out_min,
                    float *out_max, uint8_t *vertex_status, ucp_stream stream);

/* Saddle probability field (Eq. saddleProb): with the neighbours e, n, w, s
 * as X_2..X_5, P_s = Pr[X_1 < X_e, X_1 > X_n, X_1 < X_w, X_1 > X_s]
 * + Pr[X_1 > X_e, X_1 < X_n, X_1 > X_w, X_1 < X_s].  A vertex without all four
 * neighbours has no alternating neighbourhood and gets 0, except on a 1 x W
 * or H x 1 grid, where the two-neighbour form (Eq. 1D-saddleProb) is used:
 * X_1 between its next (e, or s) and previous (w, or n) neighbour, either
 * way round.  The boundary mode does not apply.  All four models
 * (UCP_MVN_MC by Monte Carlo with the same sampling contract).  out_saddle:
 * [H][W] device array; vertex_status may be NULL. */
int ucp_saddle(ucp_ctx *ctx, const float *ens, int N, int H, int W, const ucp_model_desc *desc,
               float *out_saddle, uint8_t *vertex_status, ucp_stream stream);
int ucp_saddle_from_params(ucp_ctx *ctx, const float *params, int H, int W,
                           const ucp_model_desc *desc, float *out_saddle,
                           uint8_t *vertex_status, ucp_stream stream);

/* Same as ucp_probability with HOST arrays: copies ens_host to a
 * context-owned device buffer in row strips overlapped with the computation,
 * copies the fields back and returns once the context's streams are
 * synchronised (the work starts after what is queued on `stream`).  Pinned
 * host memory gives the full copy bandwidth; pageable memory works too.
 * out_min_host / out_max_host follow cptypes; status_host may be NULL.  The
 * one-model case of ucp_probability_host_models. */
int ucp_probability_host(ucp_ctx *ctx, const float *ens_host, int N, int H, int W,
                         const ucp_model_desc *desc, unsigned cptypes, float *out_min_host,
                         float *out_max_host, uint8_t *status_host, ucp_stream stream);

#define UCP_MAX_MODELS 16

/* Several models of one ensemble, device arrays: one uniform, one
 * Epanechnikov and one histogram model of at most 8 bins (in any order, one
 * boundary rule) run as one fused kernel on `stream` that stages the
 * members once for all three (by the tensor memory accelerator when the
 * members are 16-byte aligned with W a multiple of 4, else by asynchronous
 * copies);
 * otherwise the models' kernels run concurrently on the context's compute
 * streams, forked from `stream` and joined back into it (asynchronous
 * either way; the results are those of ucp_probability for each model, bit
 * for bit).  descs[0..nmodels-1], 1 <= nmodels <=
 * UCP_MAX_MODELS, none with a larger stencil (UCP_ERR_UNSUPPORTED);
 * cptypes applies to every model.  out_min[m] / out_max[m]: [H][W] device
 * arrays of model m for the types in cptypes, an entry may be NULL (that
 * field is not written); vertex_status may be NULL, or nmodels pointers any
 * of which may be NULL.  Calls on one context must not overlap (they share
 * its streams).  The paper evaluates its models on the same ensemble
 * (Sec. "Comparison of Parametric Vs. Nonparametric Models"). */
int ucp_probability_models(ucp_ctx *ctx, const float *ens, int N, int H, int W,
                           const ucp_model_desc *descs, int nmodels, unsigned cptypes,
                           float *const *out_min, float *const *out_max,
                           uint8_t *const *vertex_status, ucp_stream stream);

/* Several models of one ensemble with HOST arrays (the paper compares its
 * models on the same ensemble, Sec. "Comparison of Parametric Vs.
 * Nonparametric Models"): the members are copied to the device once, in row
 * strips whose copies overlap the computation of the previous strip (every
 * model) and the read-back of the one before; synchronises the stream before
 * returning.  descs[0..nmodels-1], 1 <= nmodels <= UCP_MAX_MODELS, none
 * with a larger stencil (UCP_ERR_UNSUPPORTED); cptypes applies to every
 * model.  out_min_host[m] / out_max_host[m]: [H][W] host arrays of model m
 * for the types in cptypes; an entry may be NULL, and that field of that
 * model is then not copied back (the pointer arrays themselves must not be
 * NULL).  status_host may be NULL, or an array of nmodels pointers any of
 * which may be NULL.  When the models fuse (see ucp_probability_models) and
 * every wanted output array is mapped pinned host memory (cudaHostAlloc, or
 * cudaHostRegister with mapping), the fused kernel writes the probabilities
 * straight into those arrays over the host link, and nothing is read back.
 * Context-owned device buffers: N*H*W floats of members and
 * 9*nmodels*H*W bytes of outputs.  Results are those of ucp_probability. */
int ucp_probability_host_models(ucp_ctx *ctx, const float *ens_host, int N, int H, int W,
                                const ucp_model_desc *descs, int nmodels, unsigned cptypes,
                                float *const *out_min_host, float *const *out_max_host,
                                uint8_t *const *status_host, ucp_stream stream);

/* Uniform parameters [d' - eb/2, d' + eb/2] from a decompressed field
 * d'[H][W] and an absolute error bound eb >= 0 (Sec. "Real Datasets").
 * params: [2][H][W]. */
int ucp_params_from_error_bound(ucp_ctx *ctx, const float *decompressed, float eb, int H,
                                int W, float *params, ucp_stream stream);

/* Adjoint: gradient of L = sum_v weight_v * P_v (P_min if cptype ==
 * UCP_MIN, P_max if UCP_MAX) with respect to every vertex's parameters.
 * grad_params: [Q][H][W] with Q = 2 for uniform (d/da, d/db) and
 * Epanechnikov (d/dm, d/dw), Q = bins for histogram (d/dw_j, the masses;
 * lo and hi are held fixed).  The paper has no gradients; this is the exact
 * derivative of its closed form: each P_v depends on the parameters of v and
 * of its neighbours; neighbour factors are differentiated under the
 * integral, the uniform centre adds the boundary terms of its moving support.
 * Point masses get zero derivatives for their own (a, b) / (m, w).  Uses
 * context workspace: 160 floats per tile of 8 x 32 vertices for uniform
 * and Epanechnikov, 80 * bins per tile plus partial blocks for histograms
 * of at most 16 bins, 5*Q*H*W floats for more bins.  Not available for
 * UCP_MVN_MC (UCP_ERR_UNSUPPORTED). */
int ucp_backward(ucp_ctx *ctx, const float *params, int H, int W, const ucp_model_desc *desc,
                 int cptype, const float *weight, float *grad_params, ucp_stream stream);

/* The adjoint without any device allocation (the paper has no counterpart:
 * it has no gradients).  Some callers cannot call cudaMalloc once they are
 * running -- an application whose own allocator already owns the device
 * memory budget, or a latency-critical path on which cudaMalloc / cudaFree,
 * which may synchronise the whole device, are not acceptable.  This entry
 * point takes no context and allocates nothing: its scratch is a fixed
 * file-scope device array of ucp_backward_static_capacity() floats (16 MiB),
 * held by every device that loads the library until exit.  Inputs and
 * outputs are as for ucp_backward, on the CURRENT device.  The scratch must
 * fit the array, else UCP_ERR_SHAPE and nothing runs: 160 floats per tile
 * of 8 x 32 vertices for uniform and Epanechnikov (and 5 * bins * H * W for
 * histograms of more than 16 bins); for histograms of at most 16 bins 80 *
 * bins floats per tile
 * of 8 x 32 vertices plus one block of 1280 * bins floats (more blocks, up to
 * four per SM, when they fit; fewer make the call slower, not wrong) plus
 * 64 floats of block flags.  The first call on a device looks up the
 * array's device address and the device's SM count (once, with that device
 * current); make that first call before any stream capture.  All calls on a
 * device share the array: calls that can overlap on the GPU (unordered
 * streams) race on it.  It keeps the last call's contents; the block flags,
 * which must start at zero, are cleared on the stream by every call.  The
 * looked-up address is kept for the life of the process: do not call this
 * entry point on a device after cudaDeviceReset (or any other reset of its
 * primary context) in the same process, since the array then lives at a new
 * address.  Argument checks (and their status codes) are those of
 * ucp_backward. */
size_t ucp_backward_static_capacity(void);
int ucp_backward_static(const float *params, int H, int W, const ucp_model_desc *desc,
                        int cptype, const float *weight, float *grad_params, ucp_stream stream);

/* Batched launch: many fields of different sizes, member counts, models
 * (uniform, Epanechnikov, histogram) and types in a few persistent kernels:
 * one per class of fields (model, tile height, histogram row bound, members
 * staged by the tensor memory accelerator or by asynchronous copies) and
 * one generic kernel for the rest (more than 16 bins, 32-row tiles).
 * ucp_batch_add records a field (device pointers, borrowed until the batch
 * is destroyed); ucp_batch_tune times the tile shapes on `stream` and keeps
 * the fastest per model (optional; call before any stream capture);
 * ucp_batch_run enqueues the whole batch: a counter reset on `stream`, then
 * the kernels on the batch's own streams, forked from `stream` and joined
 * back into it (no allocation or synchronisation, so it can be captured
 * into a CUDA graph). */
int ucp_batch_create(ucp_ctx *ctx, ucp_batch **batch);
int ucp_batch_add(ucp_batch *batch, const float *ens, int N, int H, int W,
                  const ucp_model_desc *desc, unsigned cptypes, float *out_min, float *out_max);
int ucp_batch_tune(ucp_batch *batch, ucp_stream stream);
int ucp_batch_run(ucp_batch *batch, ucp_stream stream);
int ucp_batch_destroy(ucp_batch *batch);

#ifdef __cplusplus
}
#endif

#endif /* UCP_H */
