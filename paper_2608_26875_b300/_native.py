"""ctypes binding of libms_b300.so (declarations in include/ms_b300.h and include/ms3_b300.h).

Argument marshalling only: every step of the operator, the solve and the fields runs inside
the CUDA library.  Device buffers are torch tensors (complex128, contiguous, on the CUDA
device); streams are torch CUDA streams.  If the shared library is missing the import fails
loudly -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libms_b300.so")

MS_OK = 0
MS_NOT_CONVERGED = 1
MS_ERR_ARG = -1
MS_ERR_CUDA = -2
MS_ERR_OVERLAP = -3
MS_ERR_NOT_BURIED = -4
MS_ERR_UNSUPPORTED = -5
MS_ERR_RECEIVER_INSIDE = -6
MS_ERR_ALLOC = -7
MS_ERR_NONFINITE = -9
MS_ERR_BREAKDOWN = -10
MS_ERR_TOO_LARGE = -11
MS_ERR_TIMEOUT = -12

MS_PREC_FP64 = 0
MS_PREC_FP32 = 1
MS_PREC_BF16 = 2

MS_PART_T = 1
MS_PART_R = 2
MS_PART_S = 4
MS_PART_T_NEAR = 8
MS_PART_T_FAR = 16

MS3_PART_T = 1
MS3_PART_R = 2
MS3_PART_S = 4

c_int = ctypes.c_int32
c_dp = ctypes.POINTER(ctypes.c_double)
c_ip = ctypes.POINTER(ctypes.c_int32)


class Geometry(ctypes.Structure):
    _fields_ = [("M", c_int), ("centres", c_dp), ("radius", c_dp), ("bc", c_ip), ("proto", c_ip),
                ("rotation", c_dp), ("n_proto", c_int), ("proto_S", c_dp)]


class Geometry3(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int32), ("centres", ctypes.POINTER(ctypes.c_double)),
                ("radius", ctypes.POINTER(ctypes.c_double)), ("bc", ctypes.POINTER(ctypes.c_int32))]


class Options3(ctypes.Structure):
    _fields_ = [("n_r", ctypes.c_int32), ("n_theta", ctypes.c_int32), ("n_panels", ctypes.c_int32),
                ("t_max", ctypes.c_double), ("alpha", ctypes.c_double), ("beta", ctypes.c_double),
                ("restart", ctypes.c_int32), ("max_iters", ctypes.c_int32)]


class Incidence3(ctypes.Structure):
    _fields_ = [("nrhs", ctypes.c_int32), ("kind", ctypes.POINTER(ctypes.c_int32)),
                ("theta", ctypes.POINTER(ctypes.c_double)), ("phi", ctypes.POINTER(ctypes.c_double))]


class Media(ctypes.Structure):
    _fields_ = [("lam_u", ctypes.c_double), ("mu_u", ctypes.c_double),
                ("lam_l", ctypes.c_double), ("mu_l", ctypes.c_double)]


class Options(ctypes.Structure):
    _fields_ = [("n_panels", c_int), ("nodes_per_panel", c_int), ("t_max", ctypes.c_double),
                ("restart", c_int), ("max_iters", c_int), ("check_geometry", c_int),
                ("use_fmm", c_int), ("leaf_target", c_int), ("depth", ctypes.c_double), ("grade", c_int),
                ("tensor_cores", c_int), ("inner_tol", ctypes.c_double), ("block_krylov", c_int),
                ("cuda_graph", c_int), ("tc_wait_test", c_int),
                ("store_near", c_int), ("precond_group", c_int)]


class Incidence(ctypes.Structure):
    _fields_ = [("nrhs", c_int), ("kind", c_ip), ("angle", c_dp)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iterations", c_int), ("refinements", c_int), ("matvecs", c_int),
                ("max_rel_residual", ctypes.c_double), ("seconds", ctypes.c_double)]


# name -> (restype, argtypes); kept in the order of include/ms_b300.h
SIGNATURES = {
    "ms_default_options": (None, [ctypes.POINTER(Options)]),
    "ms_setup": (c_int, [ctypes.POINTER(Geometry), ctypes.POINTER(Media), ctypes.c_double, c_int,
                         ctypes.POINTER(Options), ctypes.POINTER(ctypes.c_void_p)]),
    "ms_apply": (c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, c_int, c_int, ctypes.c_void_p]),
    "ms_apply_adjoint": (c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, c_int, c_int, ctypes.c_void_p]),
    "ms_operator": (c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, c_int, c_int, c_int,
                            ctypes.c_void_p]),
    "ms_rhs": (c_int, [ctypes.c_void_p, ctypes.POINTER(Incidence), ctypes.c_void_p, ctypes.c_void_p]),
    "ms_solve": (c_int, [ctypes.c_void_p, ctypes.POINTER(Incidence), ctypes.c_double, c_int, ctypes.c_void_p,
                         ctypes.POINTER(SolveInfo), ctypes.c_void_p]),
    "ms_rhs_point": (c_int, [ctypes.c_void_p, c_dp, c_dp, c_int, ctypes.c_void_p, ctypes.c_void_p]),
    "ms_solve_rhs": (c_int, [ctypes.c_void_p, ctypes.c_void_p, c_int, ctypes.c_double, c_int, ctypes.c_void_p, c_int,
                             ctypes.POINTER(SolveInfo), ctypes.c_void_p]),
    "ms_fields": (c_int, [ctypes.c_void_p, ctypes.c_void_p, c_int, ctypes.c_void_p, c_int, ctypes.c_void_p,
                          ctypes.c_void_p]),
    "ms_fields_upper": (c_int, [ctypes.c_void_p, ctypes.c_void_p, c_int, ctypes.c_void_p, c_int, ctypes.c_void_p,
                                ctypes.c_void_p]),
    "ms_time_reversal": (c_int, [ctypes.c_void_p, c_dp, c_int, ctypes.c_double, c_int, c_dp, c_dp, c_dp,
                                 ctypes.POINTER(SolveInfo), ctypes.c_void_p]),
    "ms_grad": (c_int, [ctypes.c_void_p, ctypes.POINTER(Incidence), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                        c_int, ctypes.c_double, c_int, ctypes.c_void_p, ctypes.c_void_p,
                        ctypes.POINTER(ctypes.c_double), ctypes.POINTER(SolveInfo), ctypes.c_void_p]),
    "ms_fields_noalloc": (c_int, [ctypes.c_void_p, ctypes.c_void_p, c_int, ctypes.c_void_p, c_int, ctypes.c_void_p,
                                  ctypes.c_void_p]),
    "ms_autotune": (c_int, [ctypes.c_void_p, c_int, c_int, c_ip, c_ip, ctypes.POINTER(ctypes.c_double),
                            ctypes.c_void_p]),
    "ms_work": (c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                        ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "ms_near_stored": (c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)]),
    "ms_tensor_peak": (c_int, [c_int, c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "ms_info": (c_int, [ctypes.c_void_p, c_ip, c_ip, c_ip, c_ip, ctypes.POINTER(ctypes.c_int64)]),
    "ms_destroy": (None, [ctypes.c_void_p]),
    "ms3_default_options": (None, [ctypes.c_void_p]),
    "ms3_setup": (c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, c_int, ctypes.c_void_p, ctypes.c_void_p]),
    "ms3_apply": (c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, c_int, c_int, ctypes.c_void_p]),
    "ms3_operator": (c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, c_int, c_int, c_int,
                             ctypes.c_void_p]),
    "ms3_rhs": (c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "ms3_solve": (c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, c_int, ctypes.c_void_p,
                          ctypes.c_void_p, ctypes.c_void_p]),
    "ms3_info": (c_int, [ctypes.c_void_p, c_ip, c_ip, c_ip, c_ip]),
    "ms3_destroy": (None, [ctypes.c_void_p]),
    "ms_status_string": (ctypes.c_char_p, [c_int]),
    "ms_last_cuda_error": (c_int, [ctypes.c_void_p]),
}

_lib = None


def lib():
    """Load libms_b300.so once; raise if it is missing (build it with paper_2608_26875_b300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run `python -m paper_2608_26875_b300.build` "
                              "(the CUDA library is required; there is no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class MsError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = lib().ms_status_string(status).decode()
        super().__init__(f"{where}: status {status} ({msg})")
        self.status = status


def check(status: int, where: str, allow_warning: bool = False) -> int:
    if status < 0 or (status > 0 and not allow_warning):
        raise MsError(status, where)
    return status
