"""CPU-side checks of the C ABI: the library builds, loads without a GPU and
exports every entry point that include/ucp.h declares; host-side validation
rejects bad arguments before touching CUDA; device constants are right."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ucp.h")


@pytest.fixture(scope="module")
def L():
    from paper_2407_18015_gb300 import build, ucp
    build.build()
    return ucp.lib()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ucp_[a-z_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert len(names) >= 17
    for n in names:
        assert hasattr(L, n), n


def test_status_strings(L):
    from paper_2407_18015_gb300 import ucp
    assert ucp.status_string(0) == "ok"
    assert "argument" in ucp.status_string(1)
    assert ucp.status_string(99) == "unknown status"
    assert L.ucp_version().decode().startswith("ucp ")


def test_param_counts(L):
    from paper_2407_18015_gb300 import ucp
    assert ucp.ucp_param_count(ucp.make_desc("uniform")) == 2
    assert ucp.ucp_param_count(ucp.make_desc("epanechnikov")) == 2
    assert ucp.ucp_param_count(ucp.make_desc("histogram", bins=16)) == 18
    assert ucp.ucp_param_count(ucp.make_desc("mvn")) == 20
    assert ucp.ucp_param_count(ucp.make_desc("histogram", bins=0)) == 0
    assert ucp.ucp_param_count(ucp.make_desc("histogram", bins=65)) == 0


def test_validation_happens_before_cuda(L):
    """Null context / pointers and bad descriptors fail with UCP_ERR_ARG on a
    machine without a GPU, i.e. before any CUDA call."""
    from paper_2407_18015_gb300 import ucp
    d = ucp.make_desc("uniform")
    P = ctypes.c_void_p
    assert L.ucp_fit(None, P(16), 4, 4, 4, ctypes.byref(d), P(16), None, None) == ucp.UCP_ERR_ARG
    assert L.ucp_probability(None, P(16), 4, 4, 4, ctypes.byref(d), 3, P(16), P(16), None,
                             None) == ucp.UCP_ERR_ARG
    assert L.ucp_backward(None, P(16), 4, 4, ctypes.byref(d), 1, P(16), P(16), None) == \
        ucp.UCP_ERR_ARG
    assert L.ucp_create(None, 0) == ucp.UCP_ERR_ARG
    assert L.ucp_destroy(None) == ucp.UCP_ERR_ARG
    assert L.ucp_batch_create(None, None) == ucp.UCP_ERR_ARG
    assert L.ucp_batch_run(None, None) == ucp.UCP_ERR_ARG
    outs = (P * 1)(P(16))
    assert L.ucp_probability_host_models(None, P(16), 4, 4, 4, ctypes.byref(d), 1, 3, outs,
                                         outs, None, None) == ucp.UCP_ERR_ARG
    assert L.ucp_probability_models(None, P(16), 4, 4, 4, ctypes.byref(d), 1, 3, outs, outs,
                                    None, None) == ucp.UCP_ERR_ARG
    # a context-sized zeroed buffer stands in for the context: these calls
    # fail validation (no models, bad types, larger stencil) before any CUDA
    fake = ctypes.create_string_buffer(1 << 16)
    ctx = ctypes.cast(fake, ctypes.c_void_p)
    for fn in (L.ucp_probability_models, L.ucp_probability_host_models):
        assert fn(ctx, P(16), 4, 4, 4, ctypes.byref(d), 0, 3, outs, outs, None,
                  None) == ucp.UCP_ERR_ARG
        assert fn(ctx, P(16), 4, 4, 4, ctypes.byref(d), 17, 3, outs, outs, None,
                  None) == ucp.UCP_ERR_ARG
        assert fn(ctx, P(16), 4, 4, 4, ctypes.byref(d), 1, 4, outs, outs, None,
                  None) == ucp.UCP_ERR_ARG
        d6 = ucp.make_desc("uniform", stencil=ucp.UCP_STENCIL_6)
        assert fn(ctx, P(16), 4, 4, 4, ctypes.byref(d6), 1, 3, outs, outs, None,
                  None) == ucp.UCP_ERR_UNSUPPORTED


def test_gauss_legendre_constants_match_numpy():
    src = open(os.path.join(ROOT, "paper_2407_18015_gb300", "csrc", "device.cuh")).read()
    xs = re.search(r"kGLx\[4\] = \{([^}]*)\}", src).group(1)
    ws = re.search(r"kGLw\[4\] = \{([^}]*)\}", src).group(1)
    x = np.array([float(v.strip().rstrip("f")) for v in xs.split(",")])
    w = np.array([float(v.strip().rstrip("f")) for v in ws.split(",")])
    rx, rw = np.polynomial.legendre.leggauss(8)
    np.testing.assert_allclose(x, rx[4:], rtol=0, atol=1e-15)
    np.testing.assert_allclose(w, rw[4:], rtol=0, atol=1e-15)
