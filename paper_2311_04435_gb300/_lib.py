"""ctypes loader for the in-tree CUDA library ``libsca_gb300.so`` (declared in include/sca.h).

Argument marshalling only.  If the library has not been built the import of the
API fails loudly: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
SO_PATH = os.path.join(HERE, "libsca_gb300.so")

_lock = threading.Lock()
_lib = None

# status codes (include/sca.h)
SCA_OK, SCA_EINVAL, SCA_ENOMEM, SCA_EBUDGET, SCA_ECUDA, SCA_ETIMEOUT, SCA_EPENDING, \
    SCA_ENONFINITE, SCA_ENOTFOUND, SCA_ENOSTATE = range(10)
STATUS_NAMES = ["SCA_OK", "SCA_EINVAL", "SCA_ENOMEM", "SCA_EBUDGET", "SCA_ECUDA", "SCA_ETIMEOUT",
                "SCA_EPENDING", "SCA_ENONFINITE", "SCA_ENOTFOUND", "SCA_ENOSTATE"]
PREC = {"fp64": 0, "fp32": 1, "3xtf32": 2, "bf16x3": 3}
IONIC = {"paper": 0, "half": 1}


class CParams(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int32), ("n_omega", ctypes.c_int32), ("prec", ctypes.c_int32),
                ("ionic", ctypes.c_int32), ("t", ctypes.c_double), ("U", ctypes.c_double),
                ("delta", ctypes.c_double), ("T", ctypes.c_double), ("mu", ctypes.c_double)]


class CAdam(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_double), ("beta1", ctypes.c_double), ("beta2", ctypes.c_double),
                ("eps", ctypes.c_double), ("grad_tol", ctypes.c_double),
                ("max_steps", ctypes.c_int32), ("seed", ctypes.c_uint64)]


# (name, restype, argtypes) for every exported symbol of include/sca.h
_dp = ctypes.POINTER(ctypes.c_double)
_vp = ctypes.c_void_p
_i32p = ctypes.POINTER(ctypes.c_int32)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_PP = ctypes.POINTER(CParams)
_AP = ctypes.POINTER(CAdam)
SIGNATURES = [
    ("sca_create", ctypes.c_int, [_PP, ctypes.POINTER(_vp)]),
    ("sca_destroy", None, [_vp]),
    ("sca_workspace_bytes", ctypes.c_int, [_PP, _u64p]),
    ("sca_set_site_energy", ctypes.c_int, [_vp, _dp]),
    ("sca_potential", ctypes.c_int, [_vp, _dp, _dp]),
    ("sca_grad", ctypes.c_int, [_vp, _dp, _dp, _dp]),
    ("sca_potential_dev", ctypes.c_int, [_vp, _vp, _vp, _vp]),
    ("sca_grad_dev", ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
    ("sca_forward_dev", ctypes.c_int, [_vp, _vp, _vp, _vp]),
    ("sca_backward_dev", ctypes.c_int, [_vp, _vp, _vp, _vp]),
    ("sca_blocks", ctypes.c_int, [_vp, _dp, _dp, _dp]),
    ("sca_debug_assemble", ctypes.c_int, [_vp, _dp, ctypes.c_int32, ctypes.c_int32, _dp]),
    ("sca_adam_init", ctypes.c_int, [_vp, _AP, _dp]),
    ("sca_adam_step", ctypes.c_int, [_vp, ctypes.c_int32, _dp, _dp]),
    ("sca_adam_run", ctypes.c_int, [_vp, ctypes.c_int32, _i32p, _dp, _dp]),
    ("sca_get_phi", ctypes.c_int, [_vp, _dp]),
    ("sca_get_state", ctypes.c_int, [_vp, _dp, _dp, _dp, _i32p]),
    ("sca_set_state", ctypes.c_int, [_vp, _AP, _dp, _dp, _dp, ctypes.c_int32]),
    ("sca_solve", ctypes.c_int, [_PP, _AP, _dp, _dp, _dp, _i32p, _dp]),
    ("sca_server_create", ctypes.c_int, [ctypes.c_uint64, ctypes.c_int32, ctypes.POINTER(_vp)]),
    ("sca_submit", ctypes.c_int, [_vp, _PP, _AP, _u64p]),
    ("sca_poll", ctypes.c_int, [_vp, ctypes.c_uint64, _dp, _dp, _i32p, _dp]),
    ("sca_request_times", ctypes.c_int, [_vp, ctypes.c_uint64, _dp, _dp, _dp, _dp]),
    ("sca_server_destroy", None, [_vp]),
    ("sca_server_create_manual", ctypes.c_int, [ctypes.c_uint64, ctypes.c_int32, ctypes.POINTER(_vp)]),
    ("sca_server_step", ctypes.c_int, [_vp, ctypes.c_double, _i32p, _i32p]),
    ("sca_grad_noalloc_dev", ctypes.c_int, [_PP, _vp, _vp, _vp, _vp]),
    ("sca_set_stream", ctypes.c_int, [_vp, _vp]),
    ("sca_set_wait_limit", ctypes.c_int, [_vp, ctypes.c_int64]),
    ("sca_set_pivoting", ctypes.c_int, [_vp, ctypes.c_int32]),
    ("sca_set_panel_precision", ctypes.c_int, [_vp, ctypes.c_int32]),
    ("sca_set_sm_partition", ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_int32]),
    ("sca_sm_partition", ctypes.c_int, [_vp, _i32p, _i32p]),
    ("sca_dos", ctypes.c_int, [_vp, _dp, _dp, ctypes.c_int32, ctypes.c_double, _dp]),
    ("sca_metropolis_init", ctypes.c_int, [_vp, _dp, ctypes.c_double, ctypes.c_uint64]),
    ("sca_metropolis_step", ctypes.c_int, [_vp, ctypes.c_int32, _dp, ctypes.POINTER(ctypes.c_uint8),
                                           _dp, ctypes.POINTER(ctypes.c_int64)]),
    ("sca_profile_enable", ctypes.c_int, [_vp, ctypes.c_int32]),
    ("sca_profile_read", ctypes.c_int, [_vp, ctypes.c_int32, _dp, _u64p]),
    ("sca_flops_per_grad", ctypes.c_double, [_PP]),
    ("sca_pivoted_blocks", ctypes.c_int32, [_PP]),
    ("sca_last_error", ctypes.c_char_p, []),
    ("sca_version", ctypes.c_char_p, []),
    ("sca_kernel_launches", ctypes.c_uint64, []),
]


class SCAError(RuntimeError):
    def __init__(self, status: int, message: str):
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{name}: {message}")
        self.status = status


def lib(path: str | None = None):
    """The loaded library.  Raises if it has not been built (no fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            so = path or SO_PATH
            if not os.path.exists(so):
                raise RuntimeError(
                    f"CUDA library {so} is missing; build it with "
                    "`python -m paper_2311_04435_gb300.build` (there is no CPU fallback)")
            l = ctypes.CDLL(so)
            for name, res, args in SIGNATURES:
                fn = getattr(l, name)
                fn.restype = res
                fn.argtypes = args
            _lib = l
    return _lib


def check(status: int):
    if status != SCA_OK:
        msg = lib().sca_last_error()
        raise SCAError(status, msg.decode() if msg else "")
    return status
