"""sip_apply_static_scratch: the apply for callers that cannot allocate device
memory (its trace scratch is a static device array, not cudaMalloc memory).
Called through the C ABI twice in a row and compared with sip_apply, which
runs the same kernels on the same schedule and so must agree bit for bit.
This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes alone in a fresh process."""
import ctypes as C

import numpy as np
import pytest

import sip_inputs as si

pytestmark = pytest.mark.gpu


def _static_apply(g, op, prec, X, nrhs):
    import torch
    Y = torch.full_like(X, float("nan"))
    rc = g._lib.lib.sip_apply_static_scratch(op._h, prec, C.c_void_p(X.data_ptr()), C.c_void_p(Y.data_ptr()),
                                             nrhs, C.c_void_p(torch.cuda.current_stream().cuda_stream))
    g._lib.check(rc)
    torch.cuda.synchronize()
    return Y


def _fill_with_larger_mesh(g):
    """A static apply on a larger mesh with several right-hand sides first, so
    that the shared array holds stale values of another mesh when the small
    mesh's calls come (nothing in it may be read before it is written)."""
    import torch
    big = g.SipOperator.from_mesh(si.structured_mesh(3, 6, jitter=0.1, seed=55, order_range=(2, 5)))
    X = torch.tensor(si.random_rhs_batch(3, big.ndof, 56), device="cuda")
    _static_apply(g, big, g.SIP_FP64, X, 3)


@pytest.mark.parametrize("faces", ["shared", "p2p"])
def test_static_scratch_apply_matches_apply(faces):
    import torch
    from conftest import build_library
    g = build_library()
    _fill_with_larger_mesh(g)
    m = si.rotate_elements(si.structured_mesh(3, 3, jitter=0.1, seed=51, order_range=(1, 5)), 52)
    opts = g.options(face_scheme=g.SIP_FACES_P2P) if faces == "p2p" else None
    op = g.SipOperator.from_mesh(m, opts=opts)
    for dtype, prec in ((torch.float64, g.SIP_FP64), (torch.float32, g.SIP_FP32)):
        X = torch.tensor(si.random_rhs_batch(2, op.ndof, 53), device="cuda").to(dtype)
        Y_ref = op.apply(X)                       # sip_apply, scratch on the handle
        for _ in range(2):                        # two calls in a row share the static array
            Y = _static_apply(g, op, prec, X, 2)
            assert torch.equal(Y, Y_ref)


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
