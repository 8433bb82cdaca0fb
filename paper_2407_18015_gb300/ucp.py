"""Python binding of libucp (include/ucp.h): argument marshalling only.

Every function named ``ucp_*`` here calls the C entry point of the same name
with the device pointers of torch tensors and the current CUDA stream; all
computation happens in the library's kernels.  There is no CPU fallback: if
libucp.so is missing or a call fails, an exception is raised.

Convenience wrappers (``Context``, ``probability``, ``UcpProbability``)
allocate outputs with torch and call the same entry points.
"""
import ctypes
import os
import threading

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libucp.so")

UCP_UNIFORM, UCP_EPANECHNIKOV, UCP_HISTOGRAM, UCP_MVN_MC, UCP_HISTOGRAM_SEMI = 0, 1, 2, 3, 4
UCP_GAUSSIAN = 5
UCP_MIN, UCP_MAX = 1, 2
UCP_BOUNDARY_INGRID, UCP_BOUNDARY_ZERO = 0, 1
UCP_STENCIL_4, UCP_STENCIL_6, UCP_STENCIL_8, UCP_STENCIL_3D6 = 0, 1, 2, 3
UCP_OK, UCP_ERR_ARG, UCP_ERR_SHAPE, UCP_ERR_CUDA, UCP_ERR_NOMEM, UCP_ERR_TIMEOUT, \
    UCP_ERR_UNSUPPORTED = range(7)
UCP_V_DEGENERATE, UCP_V_NONFINITE, UCP_V_BAD_PARAMS, UCP_V_CHOL_JITTER, UCP_V_CHOL_FAIL = \
    1, 2, 4, 8, 16
UCP_V_TIMEOUT = 32

MODELS = {"uniform": UCP_UNIFORM, "epanechnikov": UCP_EPANECHNIKOV,
          "histogram": UCP_HISTOGRAM, "mvn": UCP_MVN_MC,
          "histogram_semi": UCP_HISTOGRAM_SEMI, "gaussian": UCP_GAUSSIAN}


class ucp_model_desc(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int), ("bins", ctypes.c_int),
                ("epan_width_scale", ctypes.c_float), ("mc_samples", ctypes.c_int),
                ("seed", ctypes.c_uint64), ("field_id", ctypes.c_uint32),
                ("boundary", ctypes.c_int), ("stencil", ctypes.c_int), ("depth", ctypes.c_int)]


class UcpError(RuntimeError):
    def __init__(self, status, where, detail=""):
        self.status = status
        msg = f"{where}: {status_string(status)}"
        if detail:
            msg += f" ({detail})"
        super().__init__(msg)


_lock = threading.Lock()
_lib = None

_P = ctypes.c_void_p
_I = ctypes.c_int


def lib():
    """The loaded libucp.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"libucp.so not built ({LIB_PATH}); run "
                                  "`python -m paper_2407_18015_gb300.build`")
            L = ctypes.CDLL(LIB_PATH)
            D = ctypes.POINTER(ucp_model_desc)
            sig = {
                "ucp_status_string": ([_I], ctypes.c_char_p),
                "ucp_version": ([], ctypes.c_char_p),
                "ucp_param_count": ([D], _I),
                "ucp_create": ([ctypes.POINTER(_P), _I], _I),
                "ucp_destroy": ([_P], _I),
                "ucp_last_error": ([_P], ctypes.c_char_p),
                "ucp_fit": ([_P, _P, _I, _I, _I, D, _P, _P, _P], _I),
                "ucp_probability_from_params": ([_P, _P, _I, _I, D, ctypes.c_uint, _P, _P, _P,
                                                 _P], _I),
                "ucp_probability": ([_P, _P, _I, _I, _I, D, ctypes.c_uint, _P, _P, _P, _P], _I),
                "ucp_probability_host": ([_P, _P, _I, _I, _I, D, ctypes.c_uint, _P, _P, _P, _P],
                                         _I),
                "ucp_probability_host_models": ([_P, _P, _I, _I, _I, D, _I, ctypes.c_uint, _P, _P,
                                                 _P, _P], _I),
                "ucp_probability_models": ([_P, _P, _I, _I, _I, D, _I, ctypes.c_uint, _P, _P, _P,
                                            _P], _I),
                "ucp_saddle": ([_P, _P, _I, _I, _I, D, _P, _P, _P], _I),
                "ucp_saddle_from_params": ([_P, _P, _I, _I, D, _P, _P, _P], _I),
                "ucp_params_from_error_bound": ([_P, _P, ctypes.c_float, _I, _I, _P, _P], _I),
                "ucp_backward": ([_P, _P, _I, _I, D, _I, _P, _P, _P], _I),
                "ucp_backward_static": ([_P, _I, _I, D, _I, _P, _P, _P], _I),
                "ucp_backward_static_capacity": ([], ctypes.c_size_t),
                "ucp_batch_create": ([_P, ctypes.POINTER(_P)], _I),
                "ucp_batch_add": ([_P, _P, _I, _I, _I, D, ctypes.c_uint, _P, _P], _I),
                "ucp_batch_tune": ([_P, _P], _I),
                "ucp_batch_run": ([_P, _P], _I),
                "ucp_batch_destroy": ([_P], _I),
            }
            for name, (args, res) in sig.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = res
            _lib = L
    return _lib


def status_string(status):
    return lib().ucp_status_string(int(status)).decode()


# ---------------------------------------------------------------------------
# marshalling helpers


def _ptr(t, dtype=None, device=None, name="tensor"):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t.data_ptr()


def _hptr(a, name="array"):
    """Host pointer of a CPU tensor (pinned or pageable) or numpy array."""
    if a is None:
        return None
    if isinstance(a, torch.Tensor):
        if a.is_cuda or not a.is_contiguous():
            raise ValueError(f"{name} must be a contiguous CPU tensor")
        return a.data_ptr()
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError(f"{name} must be C-contiguous")
    return a.ctypes.data


def _stream(stream=None, device=None):
    s = stream if stream is not None else torch.cuda.current_stream(device)
    return s.cuda_stream


def make_desc(model="uniform", bins=8, epan_width_scale=0.0, mc_samples=10000, seed=0x5EED,
              field_id=0, boundary=UCP_BOUNDARY_INGRID, stencil=UCP_STENCIL_4, depth=0):
    m = MODELS[model] if isinstance(model, str) else int(model)
    return ucp_model_desc(m, int(bins), float(epan_width_scale), int(mc_samples),
                          int(seed) & 0xFFFFFFFFFFFFFFFF, int(field_id) & 0xFFFFFFFF,
                          int(boundary), int(stencil), int(depth))


def _grid(t, desc, name):
    """(H, W) of a [lead][H][W] or [lead][D][H][W] tensor; D must be the
    descriptor's depth (a 2D tensor needs depth 0 or 1)."""
    D = desc.depth if desc.depth > 1 else 1
    if t.dim() == 4:
        if t.shape[1] != D:
            raise ValueError(f"{name}: {t.shape[1]} slices but desc.depth = {desc.depth}")
        return t.shape[2], t.shape[3]
    if t.dim() != 3 or D != 1:
        raise ValueError(f"{name}: expected [.][H][W] or [.][D][H][W] with D = desc.depth")
    return t.shape[1], t.shape[2]


def _check(rc, where, ctx=None):
    if rc != UCP_OK:
        detail = ""
        if ctx is not None and rc in (UCP_ERR_CUDA, UCP_ERR_NOMEM):
            detail = lib().ucp_last_error(ctx).decode()
        raise UcpError(rc, where, detail)


# ---------------------------------------------------------------------------
# same-name entry points (tensor arguments)


def ucp_create(device=0):
    h = _P()
    _check(lib().ucp_create(ctypes.byref(h), int(device)), "ucp_create")
    return h


def ucp_destroy(ctx):
    _check(lib().ucp_destroy(ctx), "ucp_destroy")


def ucp_param_count(desc):
    return lib().ucp_param_count(ctypes.byref(desc))


def ucp_fit(ctx, ens, desc, params, vertex_status=None, stream=None):
    N = ens.shape[0]
    H, W = _grid(ens, desc, "ens")
    rc = lib().ucp_fit(ctx, _ptr(ens, torch.float32, name="ens"), N, H, W, ctypes.byref(desc),
                       _ptr(params, torch.float32, name="params"),
                       _ptr(vertex_status, torch.uint8, name="vertex_status"),
                       _stream(stream, ens.device))
    _check(rc, "ucp_fit", ctx)


def ucp_probability_from_params(ctx, params, desc, cptypes, out_min, out_max,
                                vertex_status=None, stream=None):
    H, W = _grid(params, desc, "params")
    rc = lib().ucp_probability_from_params(
        ctx, _ptr(params, torch.float32, name="params"), H, W, ctypes.byref(desc), int(cptypes),
        _ptr(out_min, torch.float32, name="out_min"), _ptr(out_max, torch.float32, name="out_max"),
        _ptr(vertex_status, torch.uint8, name="vertex_status"), _stream(stream, params.device))
    _check(rc, "ucp_probability_from_params", ctx)


def ucp_probability(ctx, ens, desc, cptypes, out_min, out_max, vertex_status=None,
                    stream=None):
    N = ens.shape[0]
    H, W = _grid(ens, desc, "ens")
    rc = lib().ucp_probability(
        ctx, _ptr(ens, torch.float32, name="ens"), N, H, W, ctypes.byref(desc), int(cptypes),
        _ptr(out_min, torch.float32, name="out_min"), _ptr(out_max, torch.float32, name="out_max"),
        _ptr(vertex_status, torch.uint8, name="vertex_status"), _stream(stream, ens.device))
    _check(rc, "ucp_probability", ctx)


def ucp_saddle(ctx, ens, desc, out_saddle, vertex_status=None, stream=None):
    N, H, W = ens.shape
    rc = lib().ucp_saddle(ctx, _ptr(ens, torch.float32, name="ens"), N, H, W, ctypes.byref(desc),
                          _ptr(out_saddle, torch.float32, name="out_saddle"),
                          _ptr(vertex_status, torch.uint8, name="vertex_status"),
                          _stream(stream, ens.device))
    _check(rc, "ucp_saddle", ctx)


def ucp_saddle_from_params(ctx, params, desc, out_saddle, vertex_status=None, stream=None):
    _, H, W = params.shape
    rc = lib().ucp_saddle_from_params(
        ctx, _ptr(params, torch.float32, name="params"), H, W, ctypes.byref(desc),
        _ptr(out_saddle, torch.float32, name="out_saddle"),
        _ptr(vertex_status, torch.uint8, name="vertex_status"), _stream(stream, params.device))
    _check(rc, "ucp_saddle_from_params", ctx)


def ucp_probability_host(ctx, ens_host, desc, cptypes, out_min_host, out_max_host,
                         status_host=None, stream=None):
    N, H, W = ens_host.shape
    rc = lib().ucp_probability_host(
        ctx, _hptr(ens_host, "ens_host"), N, H, W, ctypes.byref(desc), int(cptypes),
        _hptr(out_min_host, "out_min_host"), _hptr(out_max_host, "out_max_host"),
        _hptr(status_host, "status_host"), _stream(stream))
    _check(rc, "ucp_probability_host", ctx)


def ucp_probability_models(ctx, ens, descs, cptypes, out_min, out_max, vertex_status=None,
                           stream=None):
    """Several models of one ensemble (device tensors): uniform,
    Epanechnikov and a histogram of at most 8 bins in one fused kernel on the
    current stream, other sets as kernels concurrent on the context's
    streams, forked from and joined back into the current stream.  descs,
    out_min, out_max (and vertex_status, if given) are sequences of the same
    length; an output entry may be None."""
    H, W = _grid(ens, descs[0], "ens")
    n = len(descs)
    if len(out_min) != n or len(out_max) != n or \
            (vertex_status is not None and len(vertex_status) != n):
        raise ValueError("one output per model")
    darr = (ucp_model_desc * n)(*descs)
    arr = lambda ts, dt, nm: ctypes.cast((ctypes.c_void_p * n)(
        *[_ptr(t, dt, name=nm) for t in ts]), ctypes.c_void_p)
    rc = lib().ucp_probability_models(
        ctx, _ptr(ens, torch.float32, name="ens"), ens.shape[0], H, W, darr, n, int(cptypes),
        arr(out_min, torch.float32, "out_min"), arr(out_max, torch.float32, "out_max"),
        None if vertex_status is None else arr(vertex_status, torch.uint8, "vertex_status"),
        _stream(stream, ens.device))
    _check(rc, "ucp_probability_models", ctx)


def ucp_probability_host_models(ctx, ens_host, descs, cptypes, out_min_host, out_max_host,
                                status_host=None, stream=None):
    """Several models of one ensemble with host arrays: descs, out_min_host,
    out_max_host (and status_host, if given) are sequences of the same length;
    an output entry may be None when cptypes leaves it out."""
    N, H, W = ens_host.shape
    n = len(descs)
    if len(out_min_host) != n or len(out_max_host) != n or \
            (status_host is not None and len(status_host) != n):
        raise ValueError("one output per model")
    darr = (ucp_model_desc * n)(*descs)
    pmin = (ctypes.c_void_p * n)(*[_hptr(a, "out_min_host") for a in out_min_host])
    pmax = (ctypes.c_void_p * n)(*[_hptr(a, "out_max_host") for a in out_max_host])
    pst = None if status_host is None else \
        (ctypes.c_void_p * n)(*[_hptr(a, "status_host") for a in status_host])
    addr = lambda a: None if a is None else ctypes.cast(a, ctypes.c_void_p)
    rc = lib().ucp_probability_host_models(
        ctx, _hptr(ens_host, "ens_host"), N, H, W, darr, n, int(cptypes), addr(pmin), addr(pmax),
        addr(pst), _stream(stream))
    _check(rc, "ucp_probability_host_models", ctx)


def ucp_params_from_error_bound(ctx, decompressed, eb, params, stream=None):
    H, W = decompressed.shape
    rc = lib().ucp_params_from_error_bound(
        ctx, _ptr(decompressed, torch.float32, name="decompressed"), float(eb), H, W,
        _ptr(params, torch.float32, name="params"), _stream(stream, decompressed.device))
    _check(rc, "ucp_params_from_error_bound", ctx)


def _backward_args(params, desc, weight, grad_params):
    """Shape, dtype and device checks of the adjoint's tensors, made before
    any launch: params [P][H][W] (P the model's parameter planes), weight
    [H][W], grad_params [Q][H][W] (Q = 2, or bins for histograms), float32,
    contiguous, all on one CUDA device.  A short output or weight would
    otherwise be written or read out of bounds on the device."""
    for name, t in (("params", params), ("weight", weight), ("grad_params", grad_params)):
        if not isinstance(t, torch.Tensor):
            raise TypeError(f"{name} must be a torch.Tensor")
        if not t.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor")
        if t.dtype != torch.float32:
            raise TypeError(f"{name} must be torch.float32, got {t.dtype}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    if params.dim() != 3:
        raise ValueError(f"params must be [P][H][W], got {tuple(params.shape)}")
    P, H, W = params.shape
    if desc.model not in (UCP_UNIFORM, UCP_EPANECHNIKOV, UCP_HISTOGRAM) or \
            desc.stencil != UCP_STENCIL_4:
        # the C entry point rejects these models and stencils with its own
        # status before anything is launched
        return H, W
    planes = lib().ucp_param_count(ctypes.byref(desc))
    if planes <= 0:
        raise UcpError(UCP_ERR_ARG, "ucp_backward", "invalid model description")
    Q = desc.bins if desc.model == UCP_HISTOGRAM else 2
    if P != planes:
        raise ValueError(f"params has {P} planes, the model has {planes}")
    if tuple(weight.shape) != (H, W):
        raise ValueError(f"weight must be [{H}][{W}], got {tuple(weight.shape)}")
    if tuple(grad_params.shape) != (Q, H, W):
        raise ValueError(f"grad_params must be [{Q}][{H}][{W}], got {tuple(grad_params.shape)}")
    if weight.device != params.device or grad_params.device != params.device:
        raise ValueError("params, weight and grad_params must be on one device")
    return H, W


def ucp_backward(ctx, params, desc, cptype, weight, grad_params, stream=None):
    H, W = _backward_args(params, desc, weight, grad_params)
    rc = lib().ucp_backward(ctx, params.data_ptr(), H, W, ctypes.byref(desc), int(cptype),
                            weight.data_ptr(), grad_params.data_ptr(),
                            _stream(stream, params.device))
    _check(rc, "ucp_backward", ctx)


def ucp_backward_static(params, desc, cptype, weight, grad_params, stream=None):
    """The adjoint without device allocation (no context; scratch is a fixed
    device array inside the library; see include/ucp.h).  The C entry point
    works on the current device, so the call is made with params' device
    current."""
    H, W = _backward_args(params, desc, weight, grad_params)
    with torch.cuda.device(params.device):
        rc = lib().ucp_backward_static(params.data_ptr(), H, W, ctypes.byref(desc), int(cptype),
                                       weight.data_ptr(), grad_params.data_ptr(),
                                       _stream(stream, params.device))
    _check(rc, "ucp_backward_static")


def ucp_backward_static_capacity():
    return int(lib().ucp_backward_static_capacity())


def ucp_batch_create(ctx):
    h = _P()
    _check(lib().ucp_batch_create(ctx, ctypes.byref(h)), "ucp_batch_create")
    return h


def ucp_batch_add(batch, ens, desc, cptypes, out_min, out_max):
    N, H, W = ens.shape
    rc = lib().ucp_batch_add(batch, _ptr(ens, torch.float32, name="ens"), N, H, W,
                             ctypes.byref(desc), int(cptypes),
                             _ptr(out_min, torch.float32, name="out_min"),
                             _ptr(out_max, torch.float32, name="out_max"))
    _check(rc, "ucp_batch_add")


def ucp_batch_tune(batch, stream=None, ctx=None):
    _check(lib().ucp_batch_tune(batch, _stream(stream)), "ucp_batch_tune", ctx)


def ucp_batch_run(batch, stream=None, ctx=None):
    _check(lib().ucp_batch_run(batch, _stream(stream)), "ucp_batch_run", ctx)


def ucp_batch_destroy(batch):
    _check(lib().ucp_batch_destroy(batch), "ucp_batch_destroy")


# ---------------------------------------------------------------------------
# convenience layer


class Context:
    """Owns a ucp_ctx on one CUDA device."""

    def __init__(self, device=None):
        if device is None:
            device = torch.cuda.current_device()
        self.device = torch.device("cuda", int(device) if not isinstance(device, torch.device)
                                   else device.index or 0)
        self.handle = ucp_create(self.device.index)

    def close(self):
        if self.handle is not None:
            ucp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def fit(self, ens, desc, with_status=False):
        grid = tuple(ens.shape[1:])
        params = torch.empty((ucp_param_count(desc),) + grid, dtype=torch.float32,
                             device=ens.device)
        st = torch.empty(grid, dtype=torch.uint8, device=ens.device) if with_status else None
        ucp_fit(self.handle, ens, desc, params, st)
        return (params, st) if with_status else params

    def _outs(self, grid, device, cptypes):
        pmin = torch.empty(grid, dtype=torch.float32, device=device) if cptypes & 1 else None
        pmax = torch.empty(grid, dtype=torch.float32, device=device) if cptypes & 2 else None
        st = torch.empty(grid, dtype=torch.uint8, device=device)
        return pmin, pmax, st

    def probability(self, ens, desc, cptypes=UCP_MIN | UCP_MAX):
        pmin, pmax, st = self._outs(tuple(ens.shape[1:]), ens.device, cptypes)
        ucp_probability(self.handle, ens, desc, cptypes, pmin, pmax, st)
        return pmin, pmax, st

    def probability_from_params(self, params, desc, cptypes=UCP_MIN | UCP_MAX):
        pmin, pmax, st = self._outs(tuple(params.shape[1:]), params.device, cptypes)
        ucp_probability_from_params(self.handle, params, desc, cptypes, pmin, pmax, st)
        return pmin, pmax, st

    def saddle(self, ens, desc):
        _, H, W = ens.shape
        out = torch.empty((H, W), dtype=torch.float32, device=ens.device)
        st = torch.empty((H, W), dtype=torch.uint8, device=ens.device)
        ucp_saddle(self.handle, ens, desc, out, st)
        return out, st

    def saddle_from_params(self, params, desc):
        _, H, W = params.shape
        out = torch.empty((H, W), dtype=torch.float32, device=params.device)
        st = torch.empty((H, W), dtype=torch.uint8, device=params.device)
        ucp_saddle_from_params(self.handle, params, desc, out, st)
        return out, st

    def backward(self, params, desc, cptype, weight):
        Q = desc.bins if desc.model in (UCP_HISTOGRAM, UCP_HISTOGRAM_SEMI) else 2
        _, H, W = params.shape
        grad = torch.empty((Q, H, W), dtype=torch.float32, device=params.device)
        ucp_backward(self.handle, params, desc, cptype, weight.contiguous(), grad)
        return grad


_ctx_cache = {}


def default_context(device=None):
    if device is None:
        device = torch.cuda.current_device()
    idx = device.index if isinstance(device, torch.device) else int(device)
    if idx not in _ctx_cache:
        _ctx_cache[idx] = Context(idx)
    return _ctx_cache[idx]


def probability(ens, model="uniform", types=("min", "max"), **kw):
    """P_min / P_max fields of an ensemble ens[N][H][W] (float32, CUDA)."""
    desc = make_desc(model, **kw)
    cp = (UCP_MIN if "min" in types else 0) | (UCP_MAX if "max" in types else 0)
    return default_context(ens.device).probability(ens, desc, cp)


class UcpProbability(torch.autograd.Function):
    """P = probability field from parameters; backward is the library's
    adjoint kernel (ucp_backward) with the incoming gradient as the weight."""

    @staticmethod
    def forward(ctx, params, model="uniform", bins=8, cptype=UCP_MIN, boundary=0):
        desc = make_desc(model, bins=bins, boundary=boundary)
        c = default_context(params.device)
        pmin, pmax, _ = c.probability_from_params(params.contiguous(), desc, cptype)
        ctx.save_for_backward(params)
        ctx.desc_args = (model, bins, boundary)
        ctx.cptype = cptype
        return pmin if cptype == UCP_MIN else pmax

    @staticmethod
    def backward(ctx, grad_out):
        (params,) = ctx.saved_tensors
        model, bins, boundary = ctx.desc_args
        desc = make_desc(model, bins=bins, boundary=boundary)
        c = default_context(params.device)
        grad = c.backward(params.contiguous(), desc, ctx.cptype,
                          grad_out.to(torch.float32).contiguous())
        if desc.model == UCP_HISTOGRAM:
            full = torch.zeros_like(params)
            full[2:] = grad
            grad = full
        return grad, None, None, None, None


class Batch:
    """Many fields in one persistent launch (ucp_batch_*).  Tensors passed to
    add() are kept alive until close()."""

    def __init__(self, ctx):
        self.ctx = ctx
        self.handle = ucp_batch_create(ctx.handle)
        self._keep = []

    def add(self, ens, desc, cptypes, out_min, out_max):
        ucp_batch_add(self.handle, ens, desc, cptypes, out_min, out_max)
        self._keep.append((ens, out_min, out_max))

    def tune(self, stream=None):
        ucp_batch_tune(self.handle, stream, self.ctx.handle)

    def run(self, stream=None):
        ucp_batch_run(self.handle, stream, self.ctx.handle)

    def close(self):
        if self.handle is not None:
            ucp_batch_destroy(self.handle)
            self.handle = None
            self._keep = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
