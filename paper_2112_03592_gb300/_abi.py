"""ctypes declarations of include/apr.h (argument marshalling only; all work runs in libaprconv.so)."""
from __future__ import annotations

import ctypes
import pathlib

_LIB_PATH = pathlib.Path(__file__).resolve().parent / "_build" / "libaprconv.so"
_lib = None

APR_OK = 0
STATUS = {0: "APR_OK", 1: "APR_ERR_INVALID_ARG", 2: "APR_ERR_INVALID_LAYOUT", 3: "APR_ERR_UNSUPPORTED",
          4: "APR_ERR_OOM", 5: "APR_ERR_CUDA", 6: "APR_ERR_TIMEOUT", 7: "APR_ERR_DEVICE"}
(APR_ERR_INVALID_ARG, APR_ERR_INVALID_LAYOUT, APR_ERR_UNSUPPORTED, APR_ERR_OOM, APR_ERR_CUDA, APR_ERR_TIMEOUT,
 APR_ERR_DEVICE) = range(1, 8)
APR_VALIDATE, APR_REQUIRE_BALANCE, APR_HOST_ONLY, APR_SUBDOMAIN = 1, 2, 4, 8
APR_BC_REFLECT, APR_BC_ZERO = 0, 1
APR_STRUCT_ROW_PTR, APR_STRUCT_Y_IDX, APR_STRUCT_TREE_ROW_PTR, APR_STRUCT_TREE_Y_IDX = 0, 1, 2, 3
APR_STRUCT_FWD_ITEMS, APR_STRUCT_TREE_ITEMS, APR_STRUCT_BWD_ITEMS = 4, 5, 6
APR_STRUCT_TREE_NODE_MAP = 7
APR_STRUCT_FWD_PLAN_R1, APR_STRUCT_FWD_PLAN_R2, APR_STRUCT_BWD_PLAN_R1, APR_STRUCT_BWD_PLAN_R2 = 8, 9, 10, 11
APR_TILE_ZX, APR_BLOCK_Y = 8, 64  # work-item geometry, as in include/apr.h

# every function include/apr.h declares, with (restype, argtypes)
_P, _I32, _I64, _U32, _SZ = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_size_t


class AprHostLayout(ctypes.Structure):
    _fields_ = [("l_min", ctypes.c_int32), ("l_max", ctypes.c_int32), ("dims", ctypes.c_int64 * 3),
                ("row_ptr", ctypes.c_void_p), ("y_idx", ctypes.c_void_p), ("n_particles", ctypes.c_int64)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


class AprAllocator(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", ctypes.c_void_p)]


SIGNATURES = {
    "apr_build_device": (_I32, [ctypes.POINTER(AprHostLayout), _U32, _P, ctypes.POINTER(_P)]),
    "apr_build_device_ex": (_I32, [ctypes.POINTER(AprHostLayout), _U32, _P, ctypes.POINTER(AprAllocator),
                                   ctypes.POINTER(_P)]),
    "apr_sobel_stencils": (_I32, [_I32, _P]),
    "apr_convolve_tiles": (_I32, [_P, _P, _P, _P, _I32, _I32, _P, _I64, _I64, _P]),
    "apr_convolve_adjoint_tiles": (_I32, [_P, _P, _I32, _I32, _P, _P, _P, _I64, _I64, _P]),
    "apr_dense_convolve": (_I32, [_P, _I64, _I64, _I64, _P, _I32, _I32, _P, _P]),
    "apr_destroy": (_I32, [_P]),
    "apr_num_particles": (_I64, [_P]),
    "apr_num_tree": (_I64, [_P]),
    "apr_level_range": (_I32, [_P, ctypes.POINTER(_I32), ctypes.POINTER(_I32)]),
    "apr_layout_bytes": (_SZ, [_P]),
    "apr_structure_bytes": (_SZ, [_P, _I32]),
    "apr_export_structure": (_I32, [_P, _I32, _P, _SZ]),
    "apr_tree_restrict": (_I32, [_P, _P, _P, _I32, _P]),
    "apr_convolve": (_I32, [_P, _P, _P, _P, _I32, _I32, _P, _P]),
    "apr_convolve_auto_workspace_bytes": (_SZ, [_P]),
    "apr_convolve_auto": (_I32, [_P, _P, _P, _I32, _I32, _P, _P, _SZ, _P]),
    "apr_gradient_magnitude": (_I32, [_P, _P, _P, _P, _I32, _I32, _P, _P]),
    "apr_backward_workspace_bytes": (_SZ, [_P, _I32]),
    "apr_convolve_backward": (_I32, [_P, _P, _P, _P, _I32, _I32, _P, _P, _P, _P, _SZ, _P]),
    "apr_convolve_backward_noalloc": (_I32, [_P, _P, _P, _P, _I32, _I32, _P, _P, _P, _P]),
    "apr_convolve_adjoint": (_I32, [_P, _P, _I32, _I32, _P, _P, _P, _P]),
    "apr_tree_restrict_adjoint": (_I32, [_P, _P, _P, _P]),
    "apr_tree_restrict_adjoint_levels": (_I32, [_P, _P, _P, _I32, _I32, _P]),
    "apr_stencil_grad_workspace_bytes": (_SZ, [_P, _I32]),
    "apr_convolve_stencil_grad": (_I32, [_P, _P, _P, _I32, _I32, _P, _P, _P, _SZ, _P]),
    "apr_rl_workspace_bytes": (_SZ, [_P]),
    "apr_richardson_lucy": (_I32, [_P, _P, _P, _I32, _I32, _I32, _P, _P, _SZ, _P]),
    "apr_tree_restrict_bf16": (_I32, [_P, _P, _P, _I32, _P]),
    "apr_convolve_mc": (_I32, [_P, _P, _P, _P, _I32, _I32, _I32, _I32, _P, _P]),
    "apr_convolve_mc_relu_bf16": (_I32, [_P, _P, _P, _P, _I32, _I32, _I32, _I32, _P, _P]),
    "apr_mc_backward_workspace_bytes": (_SZ, [_P, _I32, _I32, _I32]),
    "apr_convolve_mc_backward": (_I32, [_P, _P, _P, _P, _I32, _I32, _I32, _I32, _P, _P, _P, _P, _SZ, _P]),
    "apr_mc_embed_bf16": (_I32, [_P, _I64, ctypes.c_float, _P, _P]),
    "apr_mc_relu_bf16": (_I32, [_P, _I64, _P, _P]),
    "apr_mc_relu_backward_bf16": (_I32, [_P, _P, _I64, _P, _P]),
    "apr_mc_readout": (_I32, [_P, _P, _I64, ctypes.c_float, _P, _P]),
    "apr_mc_readout_backward_bf16": (_I32, [_P, _I64, ctypes.c_float, _P, _P]),
    "apr_restrict_stencil": (_I32, [_P, _I32, _I32, _I32, _P]),
    "apr_rescale_stencil": (_I32, [_P, _I32, _I32, _I32, _P]),
    "apr_selftest_bounded_wait": (_I32, [_P, _U32, _P]),
    "apr_sync_status": (_I32, [_P, _P]),
    "apr_status_string": (ctypes.c_char_p, [_I32]),
}
EXTRA = {"apr_last_error_message": (ctypes.c_char_p, [])}


class AprError(RuntimeError):
    def __init__(self, fn, code, detail=""):
        self.code = code
        super().__init__(f"{fn}: {STATUS.get(code, code)}" + (f" ({detail})" if detail else ""))


def lib_path() -> pathlib.Path:
    return _LIB_PATH


def load(build_if_missing: bool = True):
    """Load libaprconv.so (building it first if needed). Fails loudly: there is no fallback."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        from . import _build_lib
        if _build_lib.needs_build():
            _build_lib.build()
    if not _LIB_PATH.exists():
        raise RuntimeError(f"libaprconv.so not built ({_LIB_PATH}); run __graft_entry__.build()")
    lib = ctypes.CDLL(str(_LIB_PATH))
    for name, (res, args) in {**SIGNATURES, **EXTRA}.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def check(fn: str, code: int):
    if code != APR_OK:
        msg = load().apr_last_error_message()
        raise AprError(fn, code, msg.decode() if msg else "")
