"""GB300 library for the matrix-free symmetric interior penalty (SIP) Helmholtz
operator with per-element polynomial order (unified interface flux evaluation
on a shared trace space, Sec. 3.3).

The compute path is libsip.so (CUDA for sm_103a) behind the C ABI of
include/sip.h; this package only marshals arguments.  PyTorch supplies device
memory and the current CUDA stream.  There is no CPU fallback: without the
shared library or a GPU every call raises.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib
from ._lib import (SIP_CG_FP32_REFINED, SIP_CG_FP64, SIP_FACES_P2P, SIP_FACES_SHARED, SIP_FP32, SIP_FP64,
                   SIP_CTAS_SEQUENTIAL, SIP_CTAS_SM_MAJOR, SIP_RULE_GAUSS, SIP_RULE_GLL, SipError, check, lib,
                   sip_mesh, sip_options, sip_plan_info, sip_stats, sip_work)

__all__ = ["SipOperator", "plan_info", "options", "fp_peak", "SipError", "SIP_FP64", "SIP_FP32", "SIP_CG_FP64",
           "SIP_CG_FP32_REFINED", "SIP_FACES_SHARED", "SIP_FACES_P2P", "SIP_RULE_GAUSS", "SIP_RULE_GLL",
           "SIP_CTAS_SM_MAJOR", "SIP_CTAS_SEQUENTIAL",
           "SipApplyFn", "SipSolveFn", "lib"]


def options(**kw) -> sip_options:
    """sip_options with the library's defaults and the given fields;
    qorders (points per direction of each element) is kept alive with the
    struct."""
    o = sip_options()
    lib.sip_options_default(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        if k == "qorders" and v is not None:
            arr = np.ascontiguousarray(v, dtype=np.int32)
            o._qorders = arr
            v = arr.ctypes.data_as(C.POINTER(C.c_int32))
        setattr(o, k, v)
    return o


def fp_peak(precision=SIP_FP64, iters=1 << 14) -> float:
    """Measured FP64 / FP32 arithmetic peak of the current GPU, TFLOP/s
    (sip_fp_peak: FMA chains on every SM, CUDA-event timed)."""
    out = C.c_double()
    check(lib.sip_fp_peak(int(precision), int(iters), _stream(), C.byref(out)))
    return float(out.value)


def _mesh_struct(dim, vert, elem_vert):
    vert = np.ascontiguousarray(vert, dtype=np.float64)
    elem_vert = np.ascontiguousarray(elem_vert, dtype=np.int64)
    m = sip_mesh()
    m.dim = int(dim)
    m.n_vert = vert.shape[0]
    m.vert = vert.ctypes.data_as(C.POINTER(C.c_double))
    m.n_elem = elem_vert.shape[0]
    m.elem_vert = elem_vert.ctypes.data_as(C.POINTER(C.c_int64))
    return m, (vert, elem_vert)


def plan_info(dim, vert, elem_vert, orders, opts: sip_options | None = None) -> dict:
    """Host-only mesh analysis (face pairing, orientations, geometry); no GPU."""
    m, keep = _mesh_struct(dim, vert, elem_vert)
    orders = np.ascontiguousarray(orders, dtype=np.int32)
    h = C.c_void_p()
    check(lib.sip_plan_create(C.byref(m), orders.ctypes.data_as(C.POINTER(C.c_int32)),
                              C.byref(opts) if opts is not None else None, C.byref(h)))
    try:
        info = sip_plan_info()
        check(lib.sip_plan_info_get(h, C.byref(info)))
        return info.as_dict()
    finally:
        lib.sip_plan_destroy(h)


def _torch():
    import torch
    return torch


def _stream():
    torch = _torch()
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr())


class SipOperator:
    """One mesh + orders + lambda on the current CUDA device.

    Vectors are torch CUDA tensors, contiguous, float64 (or float32 for the
    FP32 apply), shape [ndof] or [nrhs, ndof].
    """

    def __init__(self, dim, vert, elem_vert, orders, lam=1.0, opts: sip_options | None = None):
        torch = _torch()
        if not torch.cuda.is_available():
            raise SipError(_lib.SIP_ERR_NO_DEVICE, "CUDA is not available")
        torch.cuda.init()
        m, keep = _mesh_struct(dim, vert, elem_vert)
        self.orders = np.ascontiguousarray(orders, dtype=np.int32)
        self.dim = int(dim)
        h = C.c_void_p()
        check(lib.sip_create(C.byref(m), self.orders.ctypes.data_as(C.POINTER(C.c_int32)), float(lam),
                             C.byref(opts) if opts is not None else None, C.byref(h)))
        self._h = h
        self.lam = float(lam)
        self.ndof = int(lib.sip_num_dofs(h))
        self.nquad = int(lib.sip_num_quad(h))
        E = len(self.orders)
        self.dof_off = np.zeros(E + 1, dtype=np.int64)
        self.quad_off = np.zeros(E + 1, dtype=np.int64)
        check(lib.sip_dof_offsets(h, self.dof_off.ctypes.data_as(C.POINTER(C.c_int64))))
        check(lib.sip_quad_offsets(h, self.quad_off.ctypes.data_as(C.POINTER(C.c_int64))))
        self.kappa = None

    @classmethod
    def from_mesh(cls, mesh, lam=None, opts=None):
        return cls(mesh.dim, mesh.vert, mesh.elem_vert, mesh.orders,
                   mesh.lam if lam is None else lam, opts)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            lib.sip_destroy(h)
            self._h = None

    # ---- info
    def info(self) -> dict:
        i = sip_plan_info()
        check(lib.sip_get_plan_info(self._h, C.byref(i)))
        return i.as_dict()

    def work_model(self, precision=SIP_FP64) -> dict:
        w = sip_work()
        check(lib.sip_work_model(self._h, precision, C.byref(w)))
        return w.as_dict()

    # ---- coefficients
    def set_lambda(self, lam: float):
        check(lib.sip_set_lambda(self._h, float(lam)))
        self.lam = float(lam)

    def set_kappa(self, kappa):
        """kappa: float64 CUDA tensor [nquad] (kept alive by the caller) or None."""
        if kappa is None:
            check(lib.sip_set_kappa(self._h, None, _stream()))
        else:
            self._check(kappa, _torch().float64, self.nquad)
            check(lib.sip_set_kappa(self._h, _ptr(kappa), _stream()))
        self.kappa = kappa

    # ---- operator
    def _check(self, t, dtype, n):
        if not t.is_cuda or t.dtype != dtype or not t.is_contiguous() or t.shape[-1] != n:
            raise SipError(_lib.SIP_ERR_ARG, f"expected contiguous CUDA {dtype} [..., {n}], got {t.dtype} {tuple(t.shape)}")

    def apply(self, x, precision=None, out=None, transpose=False):
        torch = _torch()
        if precision is None:
            precision = SIP_FP32 if x.dtype == torch.float32 else SIP_FP64
        dtype = torch.float32 if precision == SIP_FP32 else torch.float64
        self._check(x, dtype, self.ndof)
        nrhs = 1 if x.dim() == 1 else x.shape[0]
        y = torch.empty_like(x) if out is None else out
        fn = lib.sip_apply_transpose if transpose else lib.sip_apply
        check(fn(self._h, precision, _ptr(x), _ptr(y), nrhs, _stream()))
        return y

    def apply_host(self, x, precision=None, out=None):
        """y = A x for CPU tensors through sip_apply_host, returning when y is
        complete: pinned tensors are read / written in place by the kernels,
        pageable ones are copied through device buffers."""
        torch = _torch()
        if precision is None:
            precision = SIP_FP32 if x.dtype == torch.float32 else SIP_FP64
        dtype = torch.float32 if precision == SIP_FP32 else torch.float64
        if x.is_cuda or x.dtype != dtype or not x.is_contiguous() or x.shape[-1] != self.ndof:
            raise SipError(_lib.SIP_ERR_ARG, f"expected contiguous CPU {dtype} [..., {self.ndof}]")
        nrhs = 1 if x.dim() == 1 else x.shape[0]
        y = torch.empty_like(x) if out is None else out
        check(lib.sip_apply_host(self._h, precision, _ptr(x), _ptr(y), nrhs, _stream()))
        return y

    def apply_transpose(self, x, precision=None, out=None):
        return self.apply(x, precision, out, transpose=True)

    def cg_solve(self, b, mode=SIP_CG_FP64, rtol=1e-10, transpose=False, raise_on_fail=True):
        torch = _torch()
        self._check(b, torch.float64, self.ndof)
        nrhs = 1 if b.dim() == 1 else b.shape[0]
        x = torch.empty_like(b)
        st = sip_stats()
        fn = lib.sip_cg_solve_transpose if transpose else lib.sip_cg_solve
        rc = fn(self._h, mode, _ptr(b), _ptr(x), nrhs, float(rtol), C.byref(st), _stream())
        if raise_on_fail:
            check(rc)
        return x, st.as_dict()

    def grad_kappa(self, ybar, x, out=None, accumulate=False):
        torch = _torch()
        self._check(ybar, torch.float64, self.ndof)
        self._check(x, torch.float64, self.ndof)
        k = torch.zeros(self.nquad, dtype=torch.float64, device=x.device) if out is None else out
        check(lib.sip_grad_kappa(self._h, _ptr(ybar), _ptr(x), _ptr(k), int(accumulate), _stream()))
        return k

    def mass_dot(self, a, b):
        torch = _torch()
        self._check(a, torch.float64, self.ndof)
        self._check(b, torch.float64, self.ndof)
        out = torch.empty((), dtype=torch.float64, device=a.device)
        check(lib.sip_mass_dot(self._h, _ptr(a), _ptr(b), _ptr(out), _stream()))
        return out

    def iproduct(self, f):
        torch = _torch()
        self._check(f, torch.float64, self.nquad)
        b = torch.empty(self.ndof, dtype=torch.float64, device=f.device)
        check(lib.sip_iproduct(self._h, _ptr(f), _ptr(b), _stream()))
        return b

    def quad_points(self):
        torch = _torch()
        xq = torch.empty((self.nquad, self.dim), dtype=torch.float64, device="cuda")
        check(lib.sip_quad_points(self._h, _ptr(xq), _stream()))
        return xq

    # ---- checkpoints of the last solve
    def checkpoint_count(self):
        return int(lib.sip_cg_checkpoint_count(self._h))

    def checkpoint_info(self, slot) -> dict:
        info = _lib.sip_checkpoint_info()
        check(lib.sip_cg_checkpoint_info(self._h, int(slot), C.byref(info)))
        return info.as_dict()

    def _iterate_tensor(self, nrhs):
        torch = _torch()
        shape = (self.ndof,) if nrhs == 1 else (nrhs, self.ndof)
        return torch.empty(shape, dtype=torch.float64, device="cuda")

    def checkpoint_iterate(self, slot):
        x = self._iterate_tensor(self.checkpoint_info(slot)["nrhs"])
        check(lib.sip_cg_checkpoint_iterate(self._h, int(slot), _ptr(x), _stream()))
        return x

    def checkpoint_replay(self, slot, iters):
        x = self._iterate_tensor(self.checkpoint_info(slot)["nrhs"])
        check(lib.sip_cg_checkpoint_replay(self._h, int(slot), int(iters), _ptr(x), _stream()))
        return x

    def checkpoint(self, slot):
        torch = _torch()
        x = torch.empty(self.ndof, dtype=torch.float64, device="cuda")
        r = torch.empty_like(x)
        p = torch.empty_like(x)
        rr = C.c_double()
        it = C.c_int()
        check(lib.sip_cg_checkpoint_get(self._h, slot, _ptr(x), _ptr(r), _ptr(p), C.byref(rr), C.byref(it), _stream()))
        return x, r, p, rr.value, it.value

    def replay(self, x, r, p, rr, iters):
        rrc = C.c_double(rr)
        check(lib.sip_cg_replay(self._h, _ptr(x), _ptr(r), _ptr(p), C.byref(rrc), int(iters), _stream()))
        return rrc.value

    # ---- tile shape
    def autotune(self, precision=SIP_FP64, reps=5):
        check(lib.sip_autotune(self._h, precision, int(reps), _stream()))
        return self.tiling(precision)

    def tiling(self, precision=SIP_FP64):
        t = _lib.sip_tiling()
        check(lib.sip_get_tiling(self._h, precision, C.byref(t)))
        return {"epb_by_order": list(t.epb), "ntiles": t.ntiles, "nctas": t.nctas, "ctas_per_sm": t.ctas_per_sm,
                "persistent": int(t.persistent), "threads": t.threads, "cta_layout": t.cta_layout}

    def set_tiling(self, precision=SIP_FP64, epb_by_order=None, ctas_per_sm=0, persistent=False, threads=256,
                   cta_layout=0):
        """Install elements per tile by order (None or 0 entries: default), the
        CTAs per SM the schedule is balanced for (0: automatic), whether CTAs run
        several tiles each (persistent = 1; 2: the whole apply in one cooperative
        launch), the threads per CTA (32, 64, 128 or 256) and the block order of
        the CTAs (SIP_CTAS_SEQUENTIAL, the default, or SIP_CTAS_SM_MAJOR)."""
        t = _lib.sip_tiling()
        if epb_by_order is not None:
            if len(epb_by_order) != _lib.SIP_MAX_ORDER + 1:
                raise ValueError("epb_by_order needs one entry per order 0..%d" % _lib.SIP_MAX_ORDER)
            for i, v in enumerate(epb_by_order):
                t.epb[i] = int(v)
        t.ctas_per_sm = int(ctas_per_sm)
        t.persistent = int(persistent)  # 0, 1 (persistent CTAs) or 2 (also one launch per apply)
        t.threads = int(threads)
        t.cta_layout = int(cta_layout)
        check(lib.sip_set_tiling(self._h, precision, C.byref(t)))
        return self.tiling(precision)

    # ---- timing of the apply kernels
    def set_timing(self, on: bool):
        check(lib.sip_set_timing(self._h, int(on)))

    def last_kernel_ms(self):
        a, b = C.c_float(), C.c_float()
        check(lib.sip_last_kernel_ms(self._h, C.byref(a), C.byref(b)))
        return a.value, b.value


def _autograd():
    torch = _torch()

    class SipApplyFn(torch.autograd.Function):
        """y = A(lambda, kappa) x with gradients w.r.t. x, lambda and kappa:
        xbar = A^T ybar, lambdabar = ybar^T M x, kappabar = w|J| grad ybar . grad x."""

        @staticmethod
        def forward(ctx, op, x, lam, kappa):
            op.set_lambda(float(lam))
            op.set_kappa(kappa)
            y = op.apply(x)
            ctx.op = op
            ctx.lam = float(lam)
            ctx.save_for_backward(x, kappa if kappa is not None else torch.empty(0))
            ctx.has_kappa = kappa is not None
            return y

        @staticmethod
        def backward(ctx, ybar):
            op = ctx.op
            x, kappa = ctx.saved_tensors
            op.set_lambda(ctx.lam)
            op.set_kappa(kappa if ctx.has_kappa else None)
            ybar = ybar.contiguous()
            xbar = op.apply_transpose(ybar)
            lbar = op.mass_dot(ybar, x)
            kbar = op.grad_kappa(ybar, x) if ctx.needs_input_grad[3] else None
            return None, xbar, lbar, kbar

    class SipSolveFn(torch.autograd.Function):
        """u = A(lambda, kappa)^{-1} b by CG, gradients by the adjoint solve
        psi = A^{-T} ubar: bbar = psi, lambdabar = -psi^T M u,
        kappabar = -w|J| grad psi . grad u."""

        @staticmethod
        def forward(ctx, op, b, lam, kappa, mode, rtol):
            op.set_lambda(float(lam))
            op.set_kappa(kappa)
            u, st = op.cg_solve(b, mode=mode, rtol=rtol)
            ctx.op = op
            ctx.lam = float(lam)
            ctx.mode = mode
            ctx.rtol = rtol
            ctx.has_kappa = kappa is not None
            ctx.save_for_backward(u, kappa if kappa is not None else torch.empty(0))
            ctx.stats = st
            return u

        @staticmethod
        def backward(ctx, ubar):
            op = ctx.op
            u, kappa = ctx.saved_tensors
            op.set_lambda(ctx.lam)
            op.set_kappa(kappa if ctx.has_kappa else None)
            psi, _ = op.cg_solve(ubar.contiguous(), mode=ctx.mode, rtol=ctx.rtol, transpose=True)
            lbar = -op.mass_dot(psi, u)
            kbar = -op.grad_kappa(psi, u) if ctx.needs_input_grad[3] else None
            return None, psi, lbar, kbar, None, None

    return SipApplyFn, SipSolveFn


def __getattr__(name):
    if name in ("SipApplyFn", "SipSolveFn"):
        a, s = _autograd()
        globals()["SipApplyFn"] = a
        globals()["SipSolveFn"] = s
        return globals()[name]
    raise AttributeError(name)
