"""FP64 CPU oracle for critical-point probabilities (arXiv 2407.18015).

TEST INFRASTRUCTURE ONLY: the test-suite, the smoke check and the benchmark's
CPU-baseline leg are the only callers.  The product path never imports this
package, and this package never imports the product package.

Functions whose parity is pinned by the CPU test-suite (tests/test_oracle_*):
  fit, prob, prob_at, prob_hist_h5_at, mvn_mc_at, philox4x32_10, grad, saddle, semi_at,
  prob_stencil, gauss.
"""
from .oracle import (  # noqa: F401
    UNIFORM, EPANECHNIKOV, HISTOGRAM, MVN,
    ST_DEGENERATE, ST_NONFINITE, ST_BAD_PARAMS, ST_CHOL_JITTER, ST_CHOL_FAIL,
    build, lib, set_threads, get_threads,
    fit, prob, prob_at, prob_hist_h5_at, mvn_mc_at, philox4x32_10, grad,
    nparams, saddle, semi_at,
    STENCIL_4, STENCIL_6, STENCIL_8, STENCIL_3D6, prob_stencil, GAUSSIAN, gauss,
)
