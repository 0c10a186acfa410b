"""ctypes view of the C ABI in include/wsconv.h (argument marshalling only).

The CUDA library must have been built (``paper_2107_03958_gb300.build.build()``); there is no CPU
fallback, and loading fails loudly when the library is missing.
"""
import ctypes
import os

from . import build as _build

_lib = None


class ConvKernel(ctypes.Structure):
    _fields_ = [("family", ctypes.c_int), ("gamma", ctypes.c_double), ("kappa", ctypes.c_double),
                ("scale", ctypes.c_double)]


class ConvMoments(ctypes.Structure):
    _fields_ = [("method", ctypes.c_int), ("p", ctypes.c_int), ("nodes", ctypes.c_int), ("beta", ctypes.c_double)]


class ConvPlanInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("M", ctypes.c_int), ("period_num", ctypes.c_int),
                ("period_den", ctypes.c_int), ("b", ctypes.c_double), ("a", ctypes.c_double),
                ("precision", ctypes.c_int), ("io", ctypes.c_int), ("family", ctypes.c_int),
                ("batch_max", ctypes.c_int), ("nstages", ctypes.c_int),
                ("radices", ctypes.c_int * 16), ("ghat_bytes", ctypes.c_size_t),
                ("workspace_bytes", ctypes.c_size_t), ("threads_rows", ctypes.c_int),
                ("groups_rows", ctypes.c_int), ("threads_cols", ctypes.c_int),
                ("groups_cols", ctypes.c_int), ("transform_len", ctypes.c_int),
                ("compact", ctypes.c_int), ("elems", ctypes.c_int), ("smem_twiddles", ctypes.c_int),
                ("fused", ctypes.c_int), ("static_log2", ctypes.c_int), ("r2c_split", ctypes.c_int),
                ("static_len", ctypes.c_int), ("long_lines", ctypes.c_int),
                ("cols_pingpong", ctypes.c_int)]


class LsOpts(ctypes.Structure):
    _fields_ = [("restart", ctypes.c_int), ("max_iters", ctypes.c_int), ("tol", ctypes.c_double),
                ("refine", ctypes.c_int), ("inner_tol", ctypes.c_double),
                ("zero_guess", ctypes.c_int)]


class LsInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("restarts", ctypes.c_int),
                ("refinements", ctypes.c_int), ("rel_residual", ctypes.c_double)]


class SrvRequest(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("kernel", ConvKernel), ("n", ctypes.c_int),
                ("period_num", ctypes.c_int), ("period_den", ctypes.c_int),
                ("precision", ctypes.c_int), ("io", ctypes.c_int), ("inp", ctypes.c_void_p),
                ("mask", ctypes.c_void_p), ("m", ctypes.c_void_p), ("out", ctypes.c_void_p),
                ("tol", ctypes.c_double), ("restart", ctypes.c_int), ("max_iters", ctypes.c_int)]


class SrvResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("t_submit", ctypes.c_double), ("t_start", ctypes.c_double),
                ("t_done", ctypes.c_double), ("batched_with", ctypes.c_int), ("iters", ctypes.c_int),
                ("rel_residual", ctypes.c_double)]


class SrvStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_longlong), ("completed", ctypes.c_longlong),
                ("failed", ctypes.c_longlong), ("batches", ctypes.c_longlong),
                ("batched_requests", ctypes.c_longlong), ("plans_built", ctypes.c_longlong),
                ("plans_evicted", ctypes.c_longlong), ("bytes_in_use", ctypes.c_size_t),
                ("plans_cached", ctypes.c_int)]


# every exported symbol of include/wsconv.h with its prototype
PROTOTYPES = {
    "conv_plan": (ctypes.c_int, [ctypes.POINTER(ConvKernel), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                 ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                 ctypes.POINTER(ctypes.c_void_p)]),
    "conv_plan_ex": (ctypes.c_int, [ctypes.POINTER(ConvKernel), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]),
    "conv_plan_moments": (ctypes.c_int, [ctypes.POINTER(ConvKernel), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_int, ctypes.POINTER(ConvMoments), ctypes.POINTER(ctypes.c_void_p)]),
    "conv_workspace_size": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)]),
    "conv_apply": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                  ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]),
    "conv_apply_kernels": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                          ctypes.c_void_p]),
    "conv_apply_multi": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p), ctypes.c_int,
                                        ctypes.c_void_p, ctypes.c_void_p]),
    "conv_multi_workspace_size": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_int,
                                                 ctypes.POINTER(ctypes.c_size_t)]),
    "conv_apply_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "conv_apply_axpby": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_int, ctypes.c_double,
                                        ctypes.c_double, ctypes.c_double, ctypes.c_void_p,
                                        ctypes.c_void_p]),
    "conv_get_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ConvPlanInfo)]),
    "conv_ghat_to_host": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "conv_destroy": (None, [ctypes.c_void_p]),
    "conv_last_error": (ctypes.c_char_p, []),
    "ls_solve": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                ctypes.POINTER(LsOpts), ctypes.POINTER(LsInfo), ctypes.c_void_p]),
    "ls_solve_multi": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.POINTER(LsOpts), ctypes.POINTER(LsInfo),
                                      ctypes.c_void_p]),
    "conv_fs_mask": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_double,
                                    ctypes.c_void_p, ctypes.c_void_p]),
    "conv_device_status": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "conv_apply_host": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_int, ctypes.c_void_p]),
    "conv_timing_enable": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "conv_timing_read": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_longlong)]),
    "srv_create": (ctypes.c_int, [ctypes.c_size_t, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                  ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]),
    "srv_submit": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(SrvRequest),
                                  ctypes.POINTER(ctypes.c_longlong)]),
    "srv_wait": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_longlong, ctypes.c_double,
                                ctypes.POINTER(SrvResult)]),
    "srv_get_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(SrvStats)]),
    "srv_destroy": (None, [ctypes.c_void_p]),
    "srv_cancel": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_longlong]),
    "conv_fault_inject": (ctypes.c_int, [ctypes.c_int, ctypes.c_int]),
    "conv_apply_host_multi": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p,
                                             ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p), ctypes.c_int,
                                             ctypes.c_void_p]),
    "conv_group_create": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_void_p),
                                         ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p),
                                         ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_int),
                                         ctypes.POINTER(ctypes.c_void_p)]),
    "conv_group_launch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "conv_group_destroy": (None, [ctypes.c_void_p]),
    "conv_measure_tc_stage": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                             ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "conv_measure_peaks": (ctypes.c_int, [ctypes.c_size_t, ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(ctypes.c_double)]),
}

STATUS = {0: "CONV_OK", 1: "CONV_EINVAL", 2: "CONV_EUNSUPPORTED", 3: "CONV_ENOMEM", 4: "CONV_ECUDA",
          5: "CONV_ETIMEOUT", 6: "CONV_ENOTCONVERGED", 7: "CONV_ENONFINITE", 8: "CONV_ECANCELLED"}

FAULT = {"alloc": 1, "wait": 2, "drop": 3}


class ConvError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


def lib_path():
    return _build.LIB


def load():
    """Load the CUDA library (no fallback: raises if it has not been built)."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise ImportError("CUDA library %s is missing: run paper_2107_03958_gb300.build.build()" % path)
        L = ctypes.CDLL(path)
        for name, (res, args) in PROTOTYPES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def check(status):
    if status != 0:
        raise ConvError(status, load().conv_last_error().decode(errors="replace"))
