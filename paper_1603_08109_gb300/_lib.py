"""ctypes binding of libbf_gb300.so (include/bf.h): argument marshalling only.

Every computation runs inside the CUDA library.  If the library is missing
this module raises; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbf_gb300.so")

BF_OK = 0
STATUS = {0: "ok", 1: "invalid argument", 2: "CUDA error", 3: "unsupported parameters",
          4: "device wait timed out", 5: "workspace missing or too small", 6: "non-finite result"}

BOX, GAUSS, GAUSS_RECURSIVE = 0, 1, 2
MAX_ORDER = 1024
MAX_RADIUS = 96


class BFError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        msg = "%s failed: %s (status %d)" % (where, STATUS.get(status, "?"), status)
        if detail:
            msg += ": " + detail
        super().__init__(msg)


class BfParams(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("radius", ctypes.c_int), ("sigma_s", ctypes.c_float),
                ("sigma_r", ctypes.c_float), ("order_N", ctypes.c_int), ("t_c", ctypes.c_float)]


class BfImageDesc(ctypes.Structure):
    _fields_ = [("d_in", ctypes.c_void_p), ("d_out", ctypes.c_void_p), ("d_qaux", ctypes.c_void_p),
                ("height", ctypes.c_int), ("width", ctypes.c_int), ("pitch", ctypes.c_int),
                ("params", BfParams)]


_vp, _i, _f, _d, _sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_float, ctypes.c_double, ctypes.c_size_t
_pp = ctypes.POINTER(BfParams)
_ip = ctypes.POINTER(ctypes.c_int)
_fp = ctypes.POINTER(ctypes.c_float)

# name -> (restype, argtypes)
SIGNATURES = {
    "bf_status_string": (ctypes.c_char_p, [_i]),
    "bf_last_cuda_error": (ctypes.c_char_p, []),
    "bf_version": (_i, []),
    "bf_centre_weight": (_i, [_i, _i, _f, ctypes.POINTER(_d)]),
    "bf_order_from_delta": (_i, [_i, _i, _f, _f, _f, _f, _ip]),
    "bf_volume_order_from_delta": (_i, [_i, _i, _f, _f, _f, _f, _ip]),
    "bf_kernel_error_max": (_i, [_i, _d, _d, _i, _vp, _vp]),
    "bf_order_estimates": (_i, [_d, _d, _d, _ip, _ip, _ip]),
    "bf_fast_forward": (_i, [_vp, _vp, _vp, _i, _i, _i, _pp, _vp]),
    "bf_fast_forward_stored": (_i, [_vp, _vp, _vp, _vp, _sz, _i, _i, _i, _pp, _vp]),
    "bf_fast_forward_workspace": (_i, [_i, _i, _pp, ctypes.POINTER(_sz)]),
    "bf_joint_forward_workspace": (_i, [_i, _i, _pp, ctypes.POINTER(_sz)]),
    "bf_joint_forward_ws": (_i, [_vp, _vp, _vp, _vp, _i, _i, _i, _pp, _vp, _sz, _vp]),
    "bf_fast_forward_ws": (_i, [_vp, _vp, _vp, _i, _i, _i, _pp, _vp, _sz, _vp]),
    "bf_fast_forward_ws_variant": (_i, [_vp, _vp, _vp, _i, _i, _i, _pp, _i, _vp, _sz, _vp]),
    "bf_recursive_workspace": (_i, [_i, _i, _i, ctypes.POINTER(_sz)]),
    "bf_recursive_gauss": (_i, [_vp, _vp, _i, _i, _i, ctypes.c_float, _vp, _sz, _vp]),
    "bf_recursive_forward": (_i, [_vp, _vp, _vp, _i, _i, _i, _pp, _vp, _sz, _vp]),
    "bf_recursive_backward_workspace": (_i, [_i, _i, _i, ctypes.POINTER(_sz)]),
    "bf_recursive_joint_workspace": (_i, [_i, _i, _i, ctypes.POINTER(_sz)]),
    "bf_recursive_joint_forward": (_i, [_vp, _vp, _vp, _vp, _i, _i, _i, _pp, _vp, _sz, _vp]),
    "bf_recursive_backward": (_i, [_vp, _vp, _vp, _vp, _vp, _vp, _i, _i, _i, _pp, _vp, _sz, _vp]),
    "bf_recursive_forward_stored": (_i, [_vp, _vp, _vp, _i, _i, _i, _pp, _vp, _sz, _vp]),
    "bf_fast_forward_many": (_i, [_vp, _vp, _vp, _i, _sz, _i, _i, _i, _pp, _vp]),
    "bf_volume_workspace": (_i, [_i, _i, _i, _pp, ctypes.POINTER(_sz)]),
    "bf_volume_forward": (_i, [_vp, _vp, _vp, _i, _i, _i, _pp, _vp, _sz, _vp]),
    "bf_recursive_backward_stored": (_i, [_vp, _vp, _vp, _vp, _vp, _vp, _i, _i, _i, _pp, _vp, _sz,
                                          _vp]),
    "bf_fast_backward_workspace": (_i, [_i, _i, _pp, ctypes.POINTER(_sz)]),
    "bf_fast_backward": (_i, [_vp, _vp, _vp, _vp, _vp, _vp, _i, _i, _i, _pp, _vp, _sz, _vp]),
    "bf_fast_backward_stored": (_i, [_vp, _vp, _vp, _vp, _sz, _vp, _vp, _vp, _i, _i, _i, _pp,
                                     _vp, _sz, _vp]),
    "bf_fast_backward_noalloc": (_i, [_vp, _vp, _vp, _vp, _vp, _vp, _i, _i, _i, _pp, _vp]),
    "bf_direct": (_i, [_vp, _vp, _i, _i, _i, _pp, _vp]),
    "bf_joint_forward": (_i, [_vp, _vp, _vp, _vp, _i, _i, _i, _pp, _vp]),
    "bf_joint_direct": (_i, [_vp, _vp, _vp, _i, _i, _i, _pp, _vp]),
    "bf_direct_backward_workspace": (_i, [_i, _i, _pp, ctypes.POINTER(_sz)]),
    "bf_direct_backward": (_i, [_vp, _vp, _vp, _vp, _i, _i, _i, _pp, _vp, _sz, _vp]),
    "bf_batch_plan_create": (_i, [ctypes.POINTER(BfImageDesc), _i, ctypes.POINTER(_vp)]),
    "bf_batch_workspace": (_i, [_vp, ctypes.POINTER(_sz)]),
    "bf_batch_info": (_i, [_vp, _ip, _ip]),
    "bf_batch_variants": (_i, [_vp, _ip, _i]),
    "bf_batch_upload": (_i, [_vp, _vp, _sz, _vp]),
    "bf_batch_forward": (_i, [_vp, _vp, _sz, _vp, _vp]),
    "bf_batch_plan_destroy": (None, [_vp]),
    "bf_batch_graph_create": (_i, [_vp, _vp, _sz, _vp, _vp, ctypes.POINTER(_vp)]),
    "bf_graph_launch": (_i, [_vp, _vp]),
    "bf_graph_destroy": (None, [_vp]),
    "bf_variant_count": (_i, [_i]),
    "bf_fast_forward_variant": (_i, [_vp, _vp, _vp, _i, _i, _i, _pp, _i, _vp]),
    "bf_autotune": (_i, [_vp, _vp, _i, _i, _i, _pp, _i, _vp, _ip, _fp]),
    "bf_autotune_ws": (_i, [_vp, _vp, _i, _i, _i, _pp, _vp, _sz, _i, _vp, _ip, _fp]),
    "bf_tuning_radius_bucket": (_i, [_i]),
    "bf_tuning_order_bucket": (_i, [_i]),
    "bf_tuning_get": (_i, [_i, _i, _i, _ip]),
    "bf_tuning_set": (_i, [_i, _i, _i, _i]),
}

_lib = None


def lib() -> ctypes.CDLL:
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libbf_gb300.so is not built (run __graft_entry__.build() or "
                              "python -m paper_1603_08109_gb300.build); there is no CPU fallback")
        handle = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(handle, name)
            fn.restype = res
            fn.argtypes = args
        _lib = handle
    return _lib


def check(status: int, where: str) -> None:
    if status != BF_OK:
        detail = ""
        if status == 2:
            detail = (lib().bf_last_cuda_error() or b"").decode(errors="replace")
        raise BFError(status, where, detail)


def make_params(kind: int, radius: int, sigma_s: float, sigma_r: float, order_N: int,
                t_c: float = 128.0) -> BfParams:
    return BfParams(int(kind), int(radius), float(sigma_s), float(sigma_r), int(order_N),
                    float(t_c))
