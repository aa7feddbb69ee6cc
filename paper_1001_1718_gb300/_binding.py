"""ctypes declarations of the libresample C ABI (include/resample.h).

Argument marshalling only: every computation runs in the CUDA library. If
the library has not been built the first call raises; there is no fallback.
"""
from __future__ import annotations

import ctypes
from pathlib import Path

PKG = Path(__file__).resolve().parent
LIB_PATH = PKG / "_lib" / "libresample.so"

RS_OK, RS_ERR_INVALID_ARG, RS_ERR_UNSUPPORTED, RS_ERR_ALIGNMENT, RS_ERR_WORKSPACE, RS_ERR_CUDA = range(6)
RS_U8, RS_F16, RS_BF16, RS_F32 = range(4)
RS_NEAREST, RS_BILINEAR, RS_BICUBIC = range(3)
RS_COORD_ASYMMETRIC, RS_COORD_HALF_PIXEL, RS_COORD_ALIGN_CORNERS = range(3)
RS_IMPL_AUTO, RS_IMPL_TILED, RS_IMPL_PLAIN, RS_IMPL_STREAM, RS_IMPL_GATHER, RS_IMPL_WINDOW, RS_IMPL_REDUCE = range(7)
RS_FLAG_ANTIALIAS = 1
RS_NOALLOC_MAX_IMAGES = 4096


class RsOptions(ctypes.Structure):
    _fields_ = [("coord", ctypes.c_int32), ("cubic_a", ctypes.c_float), ("impl", ctypes.c_int32),
                ("tile_w", ctypes.c_int32), ("tile_h", ctypes.c_int32), ("threads", ctypes.c_int32),
                ("waves", ctypes.c_int32), ("flags", ctypes.c_int32)]


class RsLayout(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int32), ("C", ctypes.c_int32), ("H", ctypes.c_int32), ("W", ctypes.c_int32),
                ("n_stride", ctypes.c_int64), ("c_stride", ctypes.c_int64),
                ("row_pitch", ctypes.c_int64), ("px_stride", ctypes.c_int64)]


class RsImageDesc(ctypes.Structure):
    _fields_ = [("src", ctypes.c_void_p), ("dst", ctypes.c_void_p),
                ("H", ctypes.c_int32), ("W", ctypes.c_int32), ("C", ctypes.c_int32),
                ("Ho", ctypes.c_int32), ("Wo", ctypes.c_int32), ("method", ctypes.c_int32),
                ("src_pitch", ctypes.c_int64), ("dst_pitch", ctypes.c_int64)]


class RsTileConfig(ctypes.Structure):
    _fields_ = [("impl", ctypes.c_int32), ("tile_w", ctypes.c_int32), ("tile_h", ctypes.c_int32),
                ("threads", ctypes.c_int32), ("waves", ctypes.c_int32),
                ("best_us", ctypes.c_float), ("default_us", ctypes.c_float), ("candidates", ctypes.c_int32)]


P = ctypes.c_void_p
I32 = ctypes.c_int32
SZ = ctypes.c_size_t

# name -> (restype, argtypes); every function include/resample.h declares.
SIGNATURES = {
    "rs_options_init": (None, [ctypes.POINTER(RsOptions)]),
    "rs_layout_hwc": (RsLayout, [I32, I32, I32, I32]),
    "rs_layout_nchw": (RsLayout, [I32, I32, I32, I32]),
    "rs_status_string": (ctypes.c_char_p, [I32]),
    "rs_version": (ctypes.c_char_p, []),
    "rs_last_cuda_error": (ctypes.c_int, []),
    "rs_debug_fault": (I32, [P, ctypes.POINTER(ctypes.c_uint32)]),
    "rs_resize": (I32, [P, I32, I32, I32, I32, P, I32, I32, I32, P]),
    "rs_resize_ex": (I32, [P, ctypes.POINTER(RsLayout), P, ctypes.POINTER(RsLayout), I32, I32,
                           ctypes.POINTER(RsOptions), P]),
    "rs_resize_backward_workspace": (I32, [ctypes.POINTER(RsLayout), ctypes.POINTER(RsLayout), I32,
                                           ctypes.POINTER(RsOptions), ctypes.POINTER(SZ)]),
    "rs_resize_backward": (I32, [P, ctypes.POINTER(RsLayout), P, ctypes.POINTER(RsLayout), I32, I32,
                                 ctypes.POINTER(RsOptions), P, SZ, P]),
    "rs_resize_batched_workspace": (I32, [ctypes.POINTER(RsImageDesc), I32, I32, ctypes.POINTER(SZ)]),
    "rs_resize_batched": (I32, [ctypes.POINTER(RsImageDesc), I32, I32, P, SZ, ctypes.POINTER(RsOptions), P]),
    "rs_resize_batched_noalloc": (I32, [ctypes.POINTER(RsImageDesc), I32, I32, ctypes.POINTER(RsOptions), P]),
    "rs_batched_plan_create": (I32, [ctypes.POINTER(RsImageDesc), I32, I32, P, SZ, ctypes.POINTER(RsOptions),
                                     P, ctypes.POINTER(P)]),
    "rs_batched_plan_launch": (I32, [P, P]),
    "rs_resize_normalize": (I32, [P, ctypes.POINTER(RsLayout), P, ctypes.POINTER(RsLayout), I32, I32,
                                  ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float),
                                  ctypes.POINTER(RsOptions), P]),
    "rs_batched_plan_kernels": (I32, [P, ctypes.POINTER(I32)]),
    "rs_batched_plan_destroy": (I32, [P]),
    "rs_autotune": (I32, [P, ctypes.POINTER(RsLayout), P, ctypes.POINTER(RsLayout), I32, I32,
                          ctypes.POINTER(RsOptions), P, ctypes.POINTER(RsTileConfig)]),
    "rs_autotune_batched": (I32, [ctypes.POINTER(RsImageDesc), I32, I32, P, SZ, ctypes.POINTER(RsOptions), P,
                                  ctypes.POINTER(RsTileConfig)]),
    "rs_tune_cache_save": (I32, [ctypes.c_char_p]),
    "rs_tune_cache_load": (I32, [ctypes.c_char_p]),
    "rs_tune_cache_clear": (None, []),
    "rs_tile_config_for": (I32, [ctypes.POINTER(RsLayout), ctypes.POINTER(RsLayout), I32, I32,
                                 ctypes.POINTER(RsOptions), ctypes.POINTER(RsTileConfig)]),
}

_lib = None


def lib() -> ctypes.CDLL:
    """The loaded CUDA library. Raises if it has not been built."""
    global _lib
    if _lib is None:
        if not LIB_PATH.exists():
            raise RuntimeError(
                f"libresample.so is not built ({LIB_PATH}); run "
                "`python -c 'import __graft_entry__ as g; g.build()'` first")
        L = ctypes.CDLL(str(LIB_PATH))
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class ResampleError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = lib().rs_status_string(status).decode()
        if status == RS_ERR_CUDA:
            msg += f" (cudaError {lib().rs_last_cuda_error()})"
        super().__init__(f"{where}: {msg}")


def check(status: int, where: str) -> None:
    if status != RS_OK:
        raise ResampleError(status, where)


_default_options = None


def options(coord: int = RS_COORD_ASYMMETRIC, cubic_a: float = -0.5, impl: int = RS_IMPL_AUTO,
            tile_w: int = 0, tile_h: int = 0, threads: int = 0, waves: int = 0) -> RsOptions:
    """rs_options with the library's defaults (rs_options_init, called once)
    and the given fields."""
    global _default_options
    if _default_options is None:
        d = RsOptions()
        lib().rs_options_init(ctypes.byref(d))
        _default_options = bytes(d)
    o = RsOptions.from_buffer_copy(_default_options)
    o.coord, o.cubic_a, o.impl = coord, cubic_a, impl
    o.tile_w, o.tile_h, o.threads, o.waves = tile_w, tile_h, threads, waves
    return o
