"""sip_apply_static_scratch: the apply for callers that cannot allocate device
memory (its trace scratch is a static device array, not cudaMalloc memory).
Called through the C ABI twice in a row and compared with sip_apply.  This
file is collected last so that a run stopping at the first failure has already
run every other test; it also passes alone in a fresh process."""
import ctypes as C

import numpy as np
import pytest

import sip_inputs as si

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(((a - b).norm() / b.norm()).item())


def test_static_scratch_apply_matches_apply():
    import torch
    from conftest import build_library
    g = build_library()
    lib = g._lib.lib
    m = si.rotate_elements(si.structured_mesh(3, 3, jitter=0.1, seed=51, order_range=(1, 5)), 52)
    op = g.SipOperator.from_mesh(m)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for dtype, prec, tol in ((torch.float64, g.SIP_FP64, 1e-12), (torch.float32, g.SIP_FP32, 1e-5)):
        X = torch.tensor(si.random_rhs_batch(2, op.ndof, 53), device="cuda").to(dtype)
        Y_ref = op.apply(X)                       # sip_apply, scratch on the handle
        for _ in range(2):                        # two calls in a row share the static array
            Y = torch.full_like(X, float("nan"))
            rc = lib.sip_apply_static_scratch(op._h, prec, C.c_void_p(X.data_ptr()), C.c_void_p(Y.data_ptr()),
                                              2, stream)
            g._lib.check(rc)
            torch.cuda.synchronize()
            assert _rel(Y, Y_ref) <= tol


def test_static_scratch_rejects_oversize():
    import torch
    from conftest import build_library
    g = build_library()
    lib = g._lib.lib
    m = si.workload("c1_2d_4x4_p3")
    op = g.SipOperator.from_mesh(m)
    per_rhs = 4 * op.info()["trace_points"] * 8
    nrhs = g._lib.SIP_STATIC_TRACE_BYTES // per_rhs + 1
    X = torch.zeros((nrhs, op.ndof), dtype=torch.float64, device="cuda")
    Y = torch.empty_like(X)
    rc = lib.sip_apply_static_scratch(op._h, g.SIP_FP64, C.c_void_p(X.data_ptr()), C.c_void_p(Y.data_ptr()),
                                      nrhs, C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == g._lib.SIP_ERR_ARG
    assert b"static limit" in lib.sip_last_error()
