"""ctypes loader of libtopomag.so (argument marshalling only).

The library is built in-tree by ``paper_1707_09898_gb300.build``. There is no
fallback: if the shared object is missing or does not load, every call raises.
"""

import ctypes
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtopomag.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "topomag.h")
NET_HEADER = os.path.join(os.path.dirname(HERE), "include", "topomag_net.h")
LBFGSB_HEADER = os.path.join(os.path.dirname(HERE), "include", "topomag_lbfgsb.h")

TM_OK = 0
ERRORS = {-1: "TM_ERR_ARG", -2: "TM_ERR_SIZE", -3: "TM_ERR_STATE", -4: "TM_ERR_CUDA", -5: "TM_ERR_NOMEM",
          -6: "TM_ERR_TIMEOUT", -7: "TM_ERR_INJECTED"}

_lib = None

c_int3 = ctypes.c_int * 3
c_double3 = ctypes.c_double * 3
c_float3 = ctypes.c_float * 3
vp = ctypes.c_void_p

_SIGS = {
    "tm_create": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.c_int]),
    "tm_destroy": (None, [vp]),
    "tm_last_error": (ctypes.c_char_p, [vp]),
    "tm_version": (ctypes.c_char_p, []),
    "tm_set_grid": (ctypes.c_int, [vp, c_int3, ctypes.c_int, c_double3]),
    "tm_set_grid_lengths": (ctypes.c_int, [vp, c_int3, ctypes.c_int, c_double3, c_int3]),
    "tm_default_fft_length": (ctypes.c_int, [ctypes.c_int]),
    "tm_get_fft_lengths": (ctypes.c_int, [vp, c_int3]),
    "tm_set_penalty": (ctypes.c_int, [vp, ctypes.c_double]),
    "tm_set_M0": (ctypes.c_int, [vp, vp, c_double3, vp]),
    "tm_set_tensor": (ctypes.c_int, [vp, vp]),
    "tm_stray_field": (ctypes.c_int, [vp, vp, vp, vp]),
    "tm_stray_field_adjoint": (ctypes.c_int, [vp, vp, vp, vp, vp]),
    "tm_objective_and_gradient": (ctypes.c_int, [vp, vp, vp, vp, c_float3, c_float3, ctypes.POINTER(ctypes.c_double),
                                                 vp, vp, vp]),
    "tm_get_objective": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_double), vp]),
    "tm_copy_objective": (ctypes.c_int, [vp, vp, vp]),
    "tm_set_target": (ctypes.c_int, [vp, vp, vp, c_float3, c_float3, vp]),
    "tm_evaluate": (ctypes.c_int, [vp, vp, ctypes.POINTER(ctypes.c_double), vp, vp]),
    "tm_set_stencil_objective": (ctypes.c_int, [vp, ctypes.c_longlong, vp, vp, vp, vp, vp, vp]),
    "tm_optimize_step": (ctypes.c_int, [vp, vp, vp, ctypes.c_float, ctypes.c_int, vp]),
    "tm_evaluate_step": (ctypes.c_int, [vp, vp, ctypes.c_float, ctypes.c_int, vp, vp, vp]),
    "tm_optimize_step_noalloc": (ctypes.c_int, [vp, vp, ctypes.c_longlong, ctypes.c_float, ctypes.c_int, vp]),
    "tm_check_design": (ctypes.c_int, [vp, vp, ctypes.POINTER(ctypes.c_longlong), vp]),
    "tm_iteration_stats": (ctypes.c_int, [vp, vp, vp, ctypes.c_double * 3, vp]),
    "tm_inject_fault": (ctypes.c_int, [ctypes.c_char_p, ctypes.c_longlong]),
    "tm_selftest_wait_timeout": (ctypes.c_int, [vp, ctypes.c_int, vp]),
    "tm_profile": (ctypes.c_int, [vp, ctypes.c_int]),
    "tm_set_fused": (ctypes.c_int, [vp, ctypes.c_int]),
    "tm_profile_read": (ctypes.c_int, [vp, ctypes.c_double * 9, ctypes.c_int * 9]),
    "tm_debug_tensor_octant": (ctypes.c_int, [vp, vp, vp]),
    "tm_debug_tensor_spectrum": (ctypes.c_int, [vp, vp, vp]),
    # warm-start network kernels (include/topomag_net.h)
    "tmn_conv3d_forward": (ctypes.c_int, [vp, vp, vp, vp] + [ctypes.c_int] * 7 + [vp]),
    "tmn_conv3d_backward_data": (ctypes.c_int, [vp, vp, vp] + [ctypes.c_int] * 7 + [vp]),
    "tmn_conv3d_backward_weight": (ctypes.c_int, [vp, vp, vp, vp, vp, ctypes.c_longlong] + [ctypes.c_int] * 6 + [vp]),
    "tmn_status": (ctypes.c_int, [ctypes.POINTER(ctypes.c_uint)]),
    "tmn_conv3d_backward_weight_work": (ctypes.c_longlong, [ctypes.c_longlong, ctypes.c_int, ctypes.c_int]),
    "tmn_relu_backward": (ctypes.c_int, [vp, vp, ctypes.c_longlong, vp]),
    "tmn_pool": (ctypes.c_int, [vp, vp] + [ctypes.c_int] * 5 + [vp]),
    "tmn_pool_backward": (ctypes.c_int, [vp, vp] + [ctypes.c_int] * 6 + [vp]),
    "tmn_upcat": (ctypes.c_int, [vp, vp, vp] + [ctypes.c_int] * 6 + [vp]),
    "tmn_upcat_backward": (ctypes.c_int, [vp, vp, vp] + [ctypes.c_int] * 6 + [vp]),
    "tmn_head_forward": (ctypes.c_int, [vp, vp, vp, vp, ctypes.c_longlong, ctypes.c_int, vp]),
    "tmn_head_backward": (ctypes.c_int, [vp, vp, vp, vp, ctypes.c_longlong, ctypes.c_int, vp, vp, vp, vp]),
    "tmn_adamw": (ctypes.c_int, [vp, vp, vp, vp, ctypes.c_longlong] + [ctypes.c_float] * 5 + [ctypes.c_int, vp, vp,
                                                                                             ctypes.c_int, ctypes.c_int,
                                                                                             vp]),
    "tmn_pack_conv_weights": (ctypes.c_int, [vp, vp, vp, ctypes.c_int, ctypes.c_int, vp]),
    "tmn_spec_input": (ctypes.c_int, [vp, vp, vp, vp] + [ctypes.c_int] * 5 + [vp]),
    # L-BFGS-B (include/topomag_lbfgsb.h)
    "tm_lbfgsb_create": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.c_int, ctypes.c_longlong, ctypes.c_int,
                                        ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_int]),
    "tm_lbfgsb_destroy": (None, [vp]),
    "tm_lbfgsb_last_error": (ctypes.c_char_p, [vp]),
    "tm_lbfgsb_start": (ctypes.c_int, [vp, vp, vp, vp, vp, ctypes.POINTER(ctypes.c_int), vp]),
    "tm_lbfgsb_iterate": (ctypes.c_int, [vp, ctypes.c_double, vp, vp, vp, vp, ctypes.POINTER(ctypes.c_int), vp]),
    "tm_lbfgsb_info": (ctypes.c_int, [vp, ctypes.c_longlong * 5, ctypes.c_double * 3]),
}


def header_functions():
    """Names of the functions declared in include/topomag.h, topomag_net.h and topomag_lbfgsb.h."""
    names = set()
    for path in (HEADER, NET_HEADER, LBFGSB_HEADER):
        txt = re.sub(r"/\*.*?\*/", "", open(path).read(), flags=re.S)
        names |= set(re.findall(r"\b(tmn?_\w+)\s*\(", txt))
    return sorted(names)


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libtopomag.so not built ({LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class TopomagError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


def check(ctx, code):
    if code != TM_OK:
        msg = lib().tm_last_error(ctx).decode() if ctx else ""
        raise TopomagError(code, msg)
