"""ctypes wrapper around ucp_oracle.c (plain C, FP64, OpenMP over rows).

TEST INFRASTRUCTURE ONLY (see the package docstring).  All arrays are numpy;
parameters are float64 planes [P][H][W] in the same layout the CUDA library
uses for float32 parameters.
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

UNIFORM, EPANECHNIKOV, HISTOGRAM, MVN = 0, 1, 2, 3
GAUSSIAN = 5
ST_DEGENERATE, ST_NONFINITE, ST_BAD_PARAMS, ST_CHOL_JITTER, ST_CHOL_FAIL = 1, 2, 4, 8, 16

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ucp_oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_d = ctypes.POINTER(ctypes.c_double)
_f = ctypes.POINTER(ctypes.c_float)
_u8 = ctypes.POINTER(ctypes.c_uint8)
_i64 = ctypes.POINTER(ctypes.c_int64)
_u32 = ctypes.POINTER(ctypes.c_uint32)


def build(force=False):
    """Compile liboracle.so next to its source (gcc, OpenMP, no FP contraction)."""
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    tmp = _SO + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_SO)
            L.orc_set_threads.argtypes = [ctypes.c_int]
            L.orc_get_threads.restype = ctypes.c_int
            L.orc_fit.argtypes = [_f, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                  ctypes.c_int, ctypes.c_double, _d, _u8]
            L.orc_prob.argtypes = [_d, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                   ctypes.c_int, _d, _d, _u8]
            L.orc_prob_at.argtypes = [_d, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_int, _i64, ctypes.c_int64, _d, _d, _u8]
            L.orc_prob_hist_h5_at.argtypes = [_d, ctypes.c_int, ctypes.c_int, ctypes.c_int, _i64,
                                              ctypes.c_int64, _d, _d]
            L.orc_mvn_mc_at.argtypes = [_d, ctypes.c_int, ctypes.c_int, ctypes.c_int, _i64,
                                        ctypes.c_int64, ctypes.c_int, ctypes.c_uint64,
                                        ctypes.c_uint32, _i64, _i64, _i64, _i64, _u8]
            L.orc_saddle.argtypes = [_d, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     _i64, ctypes.c_int64, _d, _u8]
            L.orc_philox4x32_10.argtypes = [_u32, _u32, _u32]
            L.orc_semi_at.argtypes = [_d, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                      _i64, ctypes.c_int64, ctypes.c_int, ctypes.c_uint64,
                                      ctypes.c_uint32, _d, _d, _d, _d, _d]
            L.orc_grad.argtypes = [_d, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                   ctypes.c_int, ctypes.c_int, _d, _d]
            L.orc_gauss.argtypes = [_d, ctypes.c_int, ctypes.c_int, ctypes.c_int, _i64,
                                    ctypes.c_int64, _d, _d, _d, _u8]
            L.orc_prob_stencil.argtypes = [_d, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                           _i64, ctypes.c_int64, _d, _d, _u8]
            for fn in ("orc_fit", "orc_prob", "orc_prob_at", "orc_prob_hist_h5_at",
                       "orc_mvn_mc_at", "orc_grad", "orc_saddle", "orc_semi_at",
                       "orc_prob_stencil", "orc_gauss"):
                getattr(L, fn).restype = ctypes.c_int
            _lib = L
    return _lib


def set_threads(n):
    lib().orc_set_threads(int(n))


def get_threads():
    return int(lib().orc_get_threads())


def nparams(model, bins=0):
    if model == HISTOGRAM:
        return 2 + bins
    if model == MVN:
        return 20
    return 2


def _p(a, t):
    return a.ctypes.data_as(t)


def _c64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def fit(ens, model, bins=0, epan_scale=5.0 ** 0.5):
    """Per-vertex model parameters from an ensemble ens[N][H][W] (float32).
    Returns (params[P][H][W] float64, status[H][W] uint8)."""
    ens = np.ascontiguousarray(ens, dtype=np.float32)
    N, H, W = ens.shape
    out = np.empty((nparams(model, bins), H, W), np.float64)
    st = np.empty((H, W), np.uint8)
    rc = lib().orc_fit(_p(ens, _f), N, H, W, model, bins, float(epan_scale), _p(out, _d),
                       _p(st, _u8))
    if rc != 0:
        raise ValueError("orc_fit rejected its arguments")
    return out, st


def prob(params, model, bins=0, boundary=0):
    """Whole-field P_min, P_max (float64 [H][W]) and status."""
    params = _c64(params)
    _, H, W = params.shape
    pmin = np.empty((H, W), np.float64)
    pmax = np.empty((H, W), np.float64)
    st = np.empty((H, W), np.uint8)
    rc = lib().orc_prob(_p(params, _d), H, W, model, bins, boundary, _p(pmin, _d),
                        _p(pmax, _d), _p(st, _u8))
    if rc != 0:
        raise ValueError("orc_prob rejected its arguments")
    return pmin, pmax, st


def prob_at(params, model, idx, bins=0, boundary=0):
    """P_min, P_max at the linear vertex indices idx."""
    params = _c64(params)
    _, H, W = params.shape
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    n = idx.size
    pmin = np.empty(n, np.float64)
    pmax = np.empty(n, np.float64)
    st = np.empty(n, np.uint8)
    rc = lib().orc_prob_at(_p(params, _d), H, W, model, bins, boundary, _p(idx, _i64), n,
                           _p(pmin, _d), _p(pmax, _d), _p(st, _u8))
    if rc != 0:
        raise ValueError("orc_prob_at rejected its arguments")
    return pmin, pmax, st


STENCIL_4, STENCIL_6, STENCIL_8, STENCIL_3D6 = 0, 1, 2, 3


def prob_stencil(params, model, stencil, bins=0, boundary=0, idx=None):
    """P_min, P_max and status with the neighbour set of a stencil.  params:
    [P][H][W] (2D stencils) or [P][D][H][W] (any stencil; D > 1 only for the
    3D one).  Whole field (outputs shaped like one plane) or, with idx, the
    linear vertex indices idx (outputs 1D)."""
    params = _c64(params)
    if params.ndim == 3:
        D, (H, W) = 1, params.shape[1:]
    else:
        D, H, W = params.shape[1:]
    if idx is None:
        shape = params.shape[1:]
        n = D * H * W
        ip = None
    else:
        idx = np.ascontiguousarray(idx, dtype=np.int64)
        shape = (idx.size,)
        n = idx.size
        ip = _p(idx, _i64)
    pmin = np.empty(shape, np.float64)
    pmax = np.empty(shape, np.float64)
    st = np.empty(shape, np.uint8)
    rc = lib().orc_prob_stencil(_p(params, _d), D, H, W, model, bins, stencil, boundary, ip, n,
                                _p(pmin, _d), _p(pmax, _d), _p(st, _u8))
    if rc != 0:
        raise ValueError("orc_prob_stencil rejected its arguments")
    return pmin, pmax, st


def gauss(params, boundary=0, idx=None):
    """Independent-Gaussian P_min, P_max, P_saddle and status (params (m, s)
    planes [2][H][W]); whole field, or at the linear indices idx (1D)."""
    params = _c64(params)
    _, H, W = params.shape
    if idx is None:
        shape, n, ip = (H, W), H * W, None
    else:
        idx = np.ascontiguousarray(idx, dtype=np.int64)
        shape, n, ip = (idx.size,), idx.size, _p(idx, _i64)
    out = [np.empty(shape, np.float64) for _ in range(3)]
    st = np.empty(shape, np.uint8)
    rc = lib().orc_gauss(_p(params, _d), H, W, boundary, ip, n, _p(out[0], _d), _p(out[1], _d),
                         _p(out[2], _d), _p(st, _u8))
    if rc != 0:
        raise ValueError("orc_gauss rejected its arguments")
    return out[0], out[1], out[2], st


def prob_hist_h5_at(params, bins, idx):
    """The paper's sum-over-bin-combinations route for histograms."""
    params = _c64(params)
    _, H, W = params.shape
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    n = idx.size
    pmin = np.empty(n, np.float64)
    pmax = np.empty(n, np.float64)
    rc = lib().orc_prob_hist_h5_at(_p(params, _d), H, W, bins, _p(idx, _i64), n, _p(pmin, _d),
                                   _p(pmax, _d))
    if rc != 0:
        raise ValueError("orc_prob_hist_h5_at rejected its arguments")
    return pmin, pmax


def mvn_mc_at(params, idx, samples, seed, field=0, boundary=0, with_saddle=False):
    """Multivariate-Gaussian Monte Carlo at vertices idx.
    Returns (hits_min, hits_max, near_ties, status) as int64/uint8 arrays, and
    the saddle hits as a fifth array when with_saddle."""
    params = _c64(params)
    _, H, W = params.shape
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    n = idx.size
    hmin = np.empty(n, np.int64)
    hmax = np.empty(n, np.int64)
    hsad = np.empty(n, np.int64)
    ties = np.empty(n, np.int64)
    st = np.empty(n, np.uint8)
    rc = lib().orc_mvn_mc_at(_p(params, _d), H, W, boundary, _p(idx, _i64), n, int(samples),
                             int(seed) & 0xFFFFFFFFFFFFFFFF, int(field) & 0xFFFFFFFF,
                             _p(hmin, _i64), _p(hmax, _i64), _p(hsad, _i64), _p(ties, _i64),
                             _p(st, _u8))
    if rc != 0:
        raise ValueError("orc_mvn_mc_at rejected its arguments")
    if with_saddle:
        return hmin, hmax, ties, st, hsad
    return hmin, hmax, ties, st


def saddle(params, model, bins=0, idx=None):
    """Saddle probability (Eq. saddleProb) of every vertex, [H][W], or of the
    linear indices idx; and the status."""
    params = _c64(params)
    _, H, W = params.shape
    if idx is None:
        out = np.empty((H, W), np.float64)
        st = np.empty((H, W), np.uint8)
        rc = lib().orc_saddle(_p(params, _d), H, W, model, bins, None, 0, _p(out, _d),
                              _p(st, _u8))
    else:
        idx = np.ascontiguousarray(idx, dtype=np.int64)
        out = np.empty(idx.size, np.float64)
        st = np.empty(idx.size, np.uint8)
        rc = lib().orc_saddle(_p(params, _d), H, W, model, bins, _p(idx, _i64), idx.size,
                              _p(out, _d), _p(st, _u8))
    if rc != 0:
        raise ValueError("orc_saddle rejected its arguments")
    return out, st


def philox4x32_10(counter, key):
    """One Philox4x32-10 block: counter (4 x u32), key (2 x u32) -> 4 x u32."""
    c = np.ascontiguousarray(counter, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.empty(4, np.uint32)
    lib().orc_philox4x32_10(_p(c, _u32), _p(k, _u32), _p(out, _u32))
    return out


def grad(params, model, weight, cptype=1, bins=0, boundary=0):
    """Gradient of sum_v weight_v * P_v (P_min for cptype 1, P_max for 2)
    with respect to every vertex's parameters: [Q][H][W], Q = 2 or bins."""
    params = _c64(params)
    _, H, W = params.shape
    weight = _c64(weight)
    Q = bins if model == HISTOGRAM else 2
    out = np.empty((Q, H, W), np.float64)
    rc = lib().orc_grad(_p(params, _d), H, W, model, bins, boundary, cptype, _p(weight, _d),
                        _p(out, _d))
    if rc != 0:
        raise ValueError("orc_grad rejected its arguments")
    return out


def semi_at(params, bins, idx, samples, seed, field=0, boundary=0):
    """Semianalytical histogram estimator at vertices idx: (P_min, P_max,
    P_saddle, sd_min, sd_max) (sd: standard deviation of the mean)."""
    params = _c64(params)
    _, H, W = params.shape
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    n = idx.size
    out = [np.empty(n, np.float64) for _ in range(5)]
    rc = lib().orc_semi_at(_p(params, _d), H, W, bins, boundary, _p(idx, _i64), n, int(samples),
                           int(seed) & 0xFFFFFFFFFFFFFFFF, int(field) & 0xFFFFFFFF,
                           *[_p(o, _d) for o in out])
    if rc != 0:
        raise ValueError("orc_semi_at rejected its arguments")
    return tuple(out)
