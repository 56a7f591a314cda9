"""ctypes binding of libsip.so: the C ABI declared in include/sip.h, same names,
argument marshalling only.  Every computation runs in the library's kernels;
if the shared library is missing this module raises at import time."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsip.so")

SIP_OK = 0
SIP_ERR_ARG = 1
SIP_ERR_MESH = 2
SIP_ERR_CUDA = 3
SIP_ERR_OOM = 4
SIP_ERR_NONFINITE = 5
SIP_ERR_NOT_CONVERGED = 6
SIP_ERR_BREAKDOWN = 7
SIP_ERR_NO_DEVICE = 8
SIP_FP64 = 0
SIP_FP32 = 1
SIP_CG_FP64 = 0
SIP_CG_FP32_REFINED = 1
SIP_FACES_SHARED = 0
SIP_FACES_P2P = 1
SIP_RULE_GAUSS = 0
SIP_RULE_GLL = 1
SIP_MAX_ORDER = 10
SIP_CTAS_SM_MAJOR = 1
SIP_CTAS_SEQUENTIAL = 2
SIP_STATIC_TRACE_BYTES = 16 << 20

ERROR_NAMES = {1: "SIP_ERR_ARG", 2: "SIP_ERR_MESH", 3: "SIP_ERR_CUDA", 4: "SIP_ERR_OOM",
               5: "SIP_ERR_NONFINITE", 6: "SIP_ERR_NOT_CONVERGED", 7: "SIP_ERR_BREAKDOWN",
               8: "SIP_ERR_NO_DEVICE"}


class SipError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


class sip_mesh(C.Structure):
    _fields_ = [("dim", C.c_int32), ("n_vert", C.c_int64), ("vert", C.POINTER(C.c_double)),
                ("n_elem", C.c_int64), ("elem_vert", C.POINTER(C.c_int64))]


class sip_options(C.Structure):
    _fields_ = [("tau_scale", C.c_double), ("qvol_extra", C.c_int32), ("boundary", C.c_int32),
                ("inner_rtol", C.c_double), ("max_iter", C.c_int32), ("check_every", C.c_int32),
                ("max_refine", C.c_int32), ("checkpoint_every", C.c_int32),
                ("checkpoint_slots", C.c_int32), ("face_scheme", C.c_int32), ("quad_rule", C.c_int32),
                ("force_interp", C.c_int32), ("qorders", C.POINTER(C.c_int32))]


class sip_stats(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("refinements", C.c_int32), ("applies_fp64", C.c_int32),
                ("applies_fp32", C.c_int32), ("rel_residual", C.c_double), ("seconds", C.c_double),
                ("converged", C.c_int32), ("checkpoints", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class sip_plan_info(C.Structure):
    _fields_ = [("dim", C.c_int32), ("n_elem", C.c_int64), ("ndof", C.c_int64), ("nquad", C.c_int64),
                ("n_faces_interior", C.c_int64), ("n_faces_boundary", C.c_int64),
                ("n_faces_nonconforming", C.c_int64), ("n_elem_affine", C.c_int64),
                ("orient_hist", C.c_int64 * 8), ("order_hist", C.c_int64 * (SIP_MAX_ORDER + 1)),
                ("trace_points", C.c_int64), ("min_h_face", C.c_double), ("max_tau", C.c_double)]

    def as_dict(self):
        d = {}
        for k, _ in self._fields_:
            v = getattr(self, k)
            d[k] = list(v) if not isinstance(v, (int, float)) else v
        return d


class sip_tiling(C.Structure):
    _fields_ = [("epb", C.c_int32 * (SIP_MAX_ORDER + 1)), ("ctas_per_sm", C.c_int32), ("persistent", C.c_int32),
                ("threads", C.c_int32), ("cta_layout", C.c_int32), ("ntiles", C.c_int64), ("nctas", C.c_int64)]


class sip_checkpoint_info(C.Structure):
    _fields_ = [("iteration", C.c_int32), ("refinements", C.c_int32), ("restarts", C.c_int32),
                ("mode", C.c_int32), ("nrhs", C.c_int32), ("transpose", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class sip_work(C.Structure):
    _fields_ = [("flops_trace", C.c_double), ("flops_main", C.c_double), ("bytes_x", C.c_double),
                ("bytes_y", C.c_double), ("bytes_geometry", C.c_double), ("bytes_trace", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_H = C.c_void_p
_P = C.c_void_p
_I = C.c_int
_D = C.c_double

# name -> (restype, argtypes), one line per declaration of include/sip.h
SIGNATURES = {
    "sip_options_default": (None, [C.POINTER(sip_options)]),
    "sip_plan_create": (_I, [C.POINTER(sip_mesh), C.POINTER(C.c_int32), C.POINTER(sip_options), C.POINTER(_H)]),
    "sip_plan_info_get": (_I, [_H, C.POINTER(sip_plan_info)]),
    "sip_plan_destroy": (None, [_H]),
    "sip_create": (_I, [C.POINTER(sip_mesh), C.POINTER(C.c_int32), _D, C.POINTER(sip_options), C.POINTER(_H)]),
    "sip_destroy": (None, [_H]),
    "sip_num_dofs": (C.c_int64, [_H]),
    "sip_num_quad": (C.c_int64, [_H]),
    "sip_dof_offsets": (_I, [_H, C.POINTER(C.c_int64)]),
    "sip_quad_offsets": (_I, [_H, C.POINTER(C.c_int64)]),
    "sip_get_plan_info": (_I, [_H, C.POINTER(sip_plan_info)]),
    "sip_set_lambda": (_I, [_H, _D]),
    "sip_set_kappa": (_I, [_H, _P, _P]),
    "sip_apply": (_I, [_H, _I, _P, _P, _I, _P]),
    "sip_apply_host": (_I, [_H, _I, _P, _P, _I, _P]),
    "sip_apply_transpose": (_I, [_H, _I, _P, _P, _I, _P]),
    "sip_cg_solve": (_I, [_H, _I, _P, _P, _I, _D, C.POINTER(sip_stats), _P]),
    "sip_cg_solve_transpose": (_I, [_H, _I, _P, _P, _I, _D, C.POINTER(sip_stats), _P]),
    "sip_cg_checkpoint_count": (_I, [_H]),
    "sip_cg_checkpoint_get": (_I, [_H, _I, _P, _P, _P, C.POINTER(_D), C.POINTER(_I), _P]),
    "sip_cg_replay": (_I, [_H, _P, _P, _P, C.POINTER(_D), _I, _P]),
    "sip_cg_checkpoint_info": (_I, [_H, _I, C.POINTER(sip_checkpoint_info)]),
    "sip_cg_checkpoint_iterate": (_I, [_H, _I, _P, _P]),
    "sip_cg_checkpoint_replay": (_I, [_H, _I, _I, _P, _P]),
    "sip_grad_kappa": (_I, [_H, _P, _P, _P, _I, _P]),
    "sip_mass_dot": (_I, [_H, _P, _P, _P, _P]),
    "sip_iproduct": (_I, [_H, _P, _P, _P]),
    "sip_quad_points": (_I, [_H, _P, _P]),
    "sip_work_model": (_I, [_H, _I, C.POINTER(sip_work)]),
    "sip_set_timing": (_I, [_H, _I]),
    "sip_last_kernel_ms": (_I, [_H, C.POINTER(C.c_float), C.POINTER(C.c_float)]),
    "sip_autotune": (_I, [_H, _I, _I, _P]),
    "sip_get_tiling": (_I, [_H, _I, C.POINTER(sip_tiling)]),
    "sip_set_tiling": (_I, [_H, _I, C.POINTER(sip_tiling)]),
    "sip_apply_static_scratch": (_I, [_H, _I, _P, _P, _I, _P]),
    "sip_fp_peak": (_I, [_I, _I, _P, C.POINTER(_D)]),
    "sip_last_error": (C.c_char_p, []),
}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_2504_03573_gb300.build.build()")
    lib = C.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()


def check(rc: int):
    if rc != SIP_OK:
        raise SipError(rc, lib.sip_last_error().decode(errors="replace"))
    return rc
