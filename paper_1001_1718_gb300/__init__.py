"""GB300 image resampling (nearest / bilinear / bicubic) behind a C ABI.

Python front end of libresample.so (include/resample.h). Tensors supply
device memory and the current CUDA stream; every step of the computation runs
in the library's CUDA kernels. Calls on CPU tensors raise: there is no CPU
path.

    resize(x, (Ho, Wo), "bicubic")            # HWC / NHWC, uint8/f16/bf16/f32
    resize(x, (Ho, Wo), "bilinear", layout="nchw")
    ResizeFn.apply(x, (Ho, Wo), "bicubic")    # FP32 NCHW with autograd
    resize_batched(images, sizes, methods)    # ragged batch, one launch
"""
from __future__ import annotations

import ctypes
from typing import Sequence

import torch

from . import _binding as B
from ._binding import ResampleError, lib

METHODS = {"nearest": B.RS_NEAREST, "bilinear": B.RS_BILINEAR, "bicubic": B.RS_BICUBIC}
COORDS = {"asymmetric": B.RS_COORD_ASYMMETRIC, "half_pixel": B.RS_COORD_HALF_PIXEL,
          "align_corners": B.RS_COORD_ALIGN_CORNERS}
IMPLS = {"auto": B.RS_IMPL_AUTO, "tiled": B.RS_IMPL_TILED, "plain": B.RS_IMPL_PLAIN,
         "stream": B.RS_IMPL_STREAM, "gather": B.RS_IMPL_GATHER, "window": B.RS_IMPL_WINDOW,
         "reduce": B.RS_IMPL_REDUCE}
IMPL_NAMES = {v: k for k, v in IMPLS.items()}
DTYPES = {torch.uint8: B.RS_U8, torch.float16: B.RS_F16, torch.bfloat16: B.RS_BF16,
          torch.float32: B.RS_F32}

__all__ = ["resize", "resize_normalize", "resize_backward", "ResizeFn", "resize_batched", "BatchedPlan", "autotune", "autotune_batched",
           "tile_config", "tune_cache_save", "tune_cache_load", "tune_cache_clear", "debug_fault",
           "version", "lib", "ResampleError", "METHODS", "COORDS"]


def _code(table: dict, key, what: str) -> int:
    if isinstance(key, int):
        return key
    try:
        return table[key]
    except KeyError:
        raise ValueError(f"unknown {what} {key!r}; expected one of {sorted(table)}") from None


def _require_cuda(*ts: torch.Tensor) -> None:
    for t in ts:
        if not t.is_cuda:
            raise ValueError("libresample runs on CUDA tensors only (no CPU path)")


def _dtype(t: torch.Tensor) -> int:
    try:
        return DTYPES[t.dtype]
    except KeyError:
        raise ValueError(f"unsupported dtype {t.dtype}") from None


def _layout(t: torch.Tensor, layout: str) -> B.RsLayout:
    """rs_layout of a tensor: 'hwc' accepts (H,W), (H,W,C), (N,H,W,C);
    'nchw' accepts (H,W), (C,H,W), (N,C,H,W). Strides in elements."""
    L = B.RsLayout()
    s = t.stride()
    if layout == "hwc":
        if t.dim() == 2:
            N, H, W, C = 1, *t.shape, 1
            ns, rs_, ps, cs = H * s[0], s[0], s[1], 1
        elif t.dim() == 3:
            N, (H, W, C) = 1, t.shape
            ns, rs_, ps, cs = H * s[0], s[0], s[1], s[2]
        elif t.dim() == 4:
            N, H, W, C = t.shape
            ns, rs_, ps, cs = s
        else:
            raise ValueError("hwc layout wants a 2-, 3- or 4-D tensor")
    elif layout == "nchw":
        if t.dim() == 2:
            N, C, (H, W) = 1, 1, t.shape
            ns, cs, rs_, ps = H * s[0], H * s[0], s[0], s[1]
        elif t.dim() == 3:
            N, (C, H, W) = 1, t.shape
            ns, cs, rs_, ps = C * s[0], s[0], s[1], s[2]
        elif t.dim() == 4:
            N, C, H, W = t.shape
            ns, cs, rs_, ps = s
        else:
            raise ValueError("nchw layout wants a 2-, 3- or 4-D tensor")
    else:
        raise ValueError(f"unknown layout {layout!r}")
    L.N, L.C, L.H, L.W = int(N), int(C), int(H), int(W)
    L.n_stride, L.c_stride, L.row_pitch, L.px_stride = int(ns), int(cs), int(rs_), int(ps)
    return L


def _out_shape(x: torch.Tensor, layout: str, Ho: int, Wo: int) -> tuple:
    sh = list(x.shape)
    if layout == "hwc":
        if x.dim() == 2:
            return (Ho, Wo)
        i = 0 if x.dim() == 3 else 1
        sh[i], sh[i + 1] = Ho, Wo
    else:
        sh[-2], sh[-1] = Ho, Wo
    return tuple(sh)


_raw_stream = getattr(torch._C, "_cuda_getCurrentRawStream", None)


def _stream(t: torch.Tensor) -> int:
    """torch's current stream on t's device, as a raw cudaStream_t."""
    if _raw_stream is not None:
        return _raw_stream(t.device.index)
    return torch.cuda.current_stream(t.device).cuda_stream


class _on_device:
    """Makes t's device current for the library call (the library launches on
    the current device), entering torch's device context only when another
    device is current."""

    def __init__(self, t: torch.Tensor):
        self.ctx = None if t.device.index == torch.cuda.current_device() else torch.cuda.device(t.device)

    def __enter__(self):
        if self.ctx is not None:
            self.ctx.__enter__()

    def __exit__(self, *exc):
        if self.ctx is not None:
            self.ctx.__exit__(*exc)


def _opts(coord, cubic_a, impl, tile, threads, waves=0) -> B.RsOptions:
    tw, th = (tile or (0, 0))
    return B.options(_code(COORDS, coord, "coord"), float(cubic_a), _code(IMPLS, impl, "impl"),
                     int(tw), int(th), int(threads), int(waves))


def resize(x: torch.Tensor, size: Sequence[int], method="bilinear", *, layout: str = "hwc",
           coord="asymmetric", cubic_a: float = -0.5, impl="auto", tile=None, threads: int = 0,
           waves: int = 0, antialias: bool = False, out: torch.Tensor | None = None) -> torch.Tensor:
    """Resample x to size (Ho, Wo). Same dtype out; FP32 arithmetic.

    impl: "auto" (tuned or default kernel), "window", "reduce" (FP32),
    "stream", "tiled", "plain" or "gather" (nearest only);
    tile = (tile_w, tile_h) and threads / waves override the kernel shape.
    antialias: stretch the bilinear / bicubic kernel by the downscale factor
    (see RS_FLAG_ANTIALIAS in include/resample.h)."""
    _require_cuda(x)
    Ho, Wo = int(size[0]), int(size[1])
    if out is None:
        out = torch.empty(_out_shape(x, layout, Ho, Wo), dtype=x.dtype, device=x.device)
    _require_cuda(out)
    if out.dtype != x.dtype:
        raise ValueError("out must have the dtype of x")
    Li, Lo = _layout(x, layout), _layout(out, layout)
    o = _opts(coord, cubic_a, impl, tile, threads, waves)
    if antialias:
        o.flags = B.RS_FLAG_ANTIALIAS
    with _on_device(x):
        B.check(lib().rs_resize_ex(x.data_ptr(), ctypes.byref(Li), out.data_ptr(), ctypes.byref(Lo),
                                   _dtype(x), _code(METHODS, method, "method"), ctypes.byref(o),
                                   _stream(x)), "rs_resize_ex")
    return out


_OUT_DTYPES = {torch.float16: B.RS_F16, torch.bfloat16: B.RS_BF16, torch.float32: B.RS_F32}


def resize_normalize(x: torch.Tensor, size: Sequence[int], method="bilinear", mean=(0.0, 0.0, 0.0),
                     std=(1.0, 1.0, 1.0), *, dtype=torch.float16, coord="asymmetric", cubic_a: float = -0.5,
                     out: torch.Tensor | None = None, impl="auto", chunk: int = 0,
                     antialias: bool = False) -> torch.Tensor:
    """The fused serving pre-process: resample a uint8 (H, W, C) or
    (N, H, W, C) image, normalise every channel, (y - mean[c]) / std[c], and
    return it planar, (C, Ho, Wo) or (N, C, Ho, Wo), as FP16 / BF16 / FP32,
    in one pass (rs_resize_normalize). antialias=True stretches the filter
    by the downscale factor (RS_FLAG_ANTIALIAS, at most 8 taps per axis)."""
    _require_cuda(x)
    if x.dtype != torch.uint8:
        raise ValueError("resize_normalize reads uint8 images")
    try:
        odt = _OUT_DTYPES[dtype]
    except KeyError:
        raise ValueError(f"unsupported output dtype {dtype}") from None
    Ho, Wo = int(size[0]), int(size[1])
    batched = x.dim() == 4
    C = x.shape[-1]
    shape = (x.shape[0], C, Ho, Wo) if batched else (C, Ho, Wo)
    if out is None:
        out = torch.empty(shape, dtype=dtype, device=x.device)
    elif tuple(out.shape) != shape or out.dtype != dtype:
        raise ValueError(f"out must be {shape} of {dtype}")
    Li, Lo = _layout(x, "hwc"), _layout(out, "nchw")
    if len(mean) != C or len(std) != C:
        raise ValueError("mean and std need one value per channel")
    m = (ctypes.c_float * C)(*[float(v) for v in mean])
    s = (ctypes.c_float * C)(*[float(v) for v in std])
    o = _opts(coord, cubic_a, impl, (0, chunk), 0)
    if antialias:
        o.flags = B.RS_FLAG_ANTIALIAS
    with _on_device(x):
        B.check(lib().rs_resize_normalize(x.data_ptr(), ctypes.byref(Li), out.data_ptr(), ctypes.byref(Lo), odt,
                                          _code(METHODS, method, "method"), m, s, ctypes.byref(o), _stream(x)),
                "rs_resize_normalize")
    return out


def backward_workspace_bytes(grad_out: torch.Tensor, in_hw, method, *, layout="nchw",
                             coord="asymmetric", cubic_a=-0.5, antialias: bool = False) -> int:
    H, W = int(in_hw[0]), int(in_hw[1])
    Lo = _layout(grad_out, layout)
    Li = _layout(torch.empty(_out_shape(grad_out, layout, H, W), dtype=grad_out.dtype, device="meta"), layout)
    o = _opts(coord, cubic_a, "auto", None, 0)
    if antialias:
        o.flags = B.RS_FLAG_ANTIALIAS
    n = ctypes.c_size_t(0)
    B.check(lib().rs_resize_backward_workspace(ctypes.byref(Lo), ctypes.byref(Li),
                                               _code(METHODS, method, "method"), ctypes.byref(o),
                                               ctypes.byref(n)), "rs_resize_backward_workspace")
    return n.value


def resize_backward(grad_out: torch.Tensor, in_hw, method="bilinear", *, layout: str = "nchw",
                    coord="asymmetric", cubic_a: float = -0.5, grad_in: torch.Tensor | None = None,
                    workspace: torch.Tensor | None = None, impl="auto",
                    antialias: bool = False) -> torch.Tensor:
    """Adjoint of resize() for FP32: grad_in = A^T grad_out (deterministic).
    impl="auto" picks the kernel ("window", "stream": two passes, "tiled");
    antialias=True is the adjoint of resize(..., antialias=True)."""
    _require_cuda(grad_out)
    H, W = int(in_hw[0]), int(in_hw[1])
    if grad_in is None:
        grad_in = torch.empty(_out_shape(grad_out, layout, H, W), dtype=grad_out.dtype,
                              device=grad_out.device)
    Lo, Li = _layout(grad_out, layout), _layout(grad_in, layout)
    o = _opts(coord, cubic_a, impl, None, 0)
    if antialias:
        o.flags = B.RS_FLAG_ANTIALIAS
    m = _code(METHODS, method, "method")
    n = ctypes.c_size_t(0)
    B.check(lib().rs_resize_backward_workspace(ctypes.byref(Lo), ctypes.byref(Li), m, ctypes.byref(o),
                                               ctypes.byref(n)), "rs_resize_backward_workspace")
    if workspace is None or workspace.numel() * workspace.element_size() < n.value:
        workspace = torch.empty(max(1, n.value), dtype=torch.uint8, device=grad_out.device)
    with _on_device(grad_out):
        B.check(lib().rs_resize_backward(grad_out.data_ptr(), ctypes.byref(Lo), grad_in.data_ptr(),
                                         ctypes.byref(Li), _dtype(grad_out), m, ctypes.byref(o),
                                         workspace.data_ptr(), n.value, _stream(grad_out)),
                "rs_resize_backward")
    return grad_in


class ResizeFn(torch.autograd.Function):
    """Differentiable resize of an FP32 NCHW tensor (forward and adjoint run
    in the library's kernels)."""

    @staticmethod
    def forward(ctx, x, size, method="bilinear", coord="asymmetric", cubic_a=-0.5, antialias=False):
        ctx.in_hw = (x.shape[-2], x.shape[-1])
        ctx.cfg = (method, coord, cubic_a, bool(antialias))
        return resize(x.contiguous(), size, method, layout="nchw", coord=coord, cubic_a=cubic_a,
                      antialias=bool(antialias))

    @staticmethod
    def backward(ctx, g):
        method, coord, cubic_a, antialias = ctx.cfg
        gi = resize_backward(g.contiguous(), ctx.in_hw, method, layout="nchw", coord=coord, cubic_a=cubic_a,
                             antialias=antialias)
        return gi, None, None, None, None, None


def _descs(srcs, dsts, methods) -> tuple:
    n = len(srcs)
    arr = (B.RsImageDesc * n)()
    for k, (s, d) in enumerate(zip(srcs, dsts)):
        if s.dim() != 3 or d.dim() != 3:
            raise ValueError("batched images are (H, W, C) tensors")
        if s.stride(2) != 1 or s.stride(1) != s.shape[2] or d.stride(2) != 1 or d.stride(1) != d.shape[2]:
            raise ValueError("batched images need dense pixels (pitched rows are fine)")
        dd = arr[k]
        dd.src, dd.dst = s.data_ptr(), d.data_ptr()
        dd.H, dd.W, dd.C = s.shape
        dd.Ho, dd.Wo = d.shape[0], d.shape[1]
        dd.method = _code(METHODS, methods[k], "method")
        dd.src_pitch, dd.dst_pitch = s.stride(0), d.stride(0)
    return arr, n


def batched_workspace_bytes(srcs, dsts, methods) -> int:
    arr, n = _descs(srcs, dsts, methods)
    nb = ctypes.c_size_t(0)
    B.check(lib().rs_resize_batched_workspace(arr, n, _dtype(srcs[0]), ctypes.byref(nb)),
            "rs_resize_batched_workspace")
    return nb.value


def resize_batched(srcs: Sequence[torch.Tensor], sizes, methods, *, coord="asymmetric",
                   cubic_a: float = -0.5, outs=None, workspace: torch.Tensor | None = None,
                   impl: str = "auto", tile=None, threads: int = 0, antialias: bool = False):
    """Resample a ragged list of (H, W, C) images in one persistent launch.
    impl="window": tile = (band rows, chunk rows) of the window items;
    impl="tiled": tile = (elements, rows) of every image's tiles.
    antialias=True: every image with the antialias taps (bilinear / bicubic)."""
    _require_cuda(*srcs)
    if outs is None:
        outs = [torch.empty((int(h), int(w), s.shape[2]), dtype=s.dtype, device=s.device)
                for s, (h, w) in zip(srcs, sizes)]
    arr, n = _descs(srcs, outs, methods)
    nb = ctypes.c_size_t(0)
    dt = _dtype(srcs[0])
    B.check(lib().rs_resize_batched_workspace(arr, n, dt, ctypes.byref(nb)), "rs_resize_batched_workspace")
    if workspace is None or workspace.numel() * workspace.element_size() < nb.value:
        workspace = torch.empty(max(1, nb.value), dtype=torch.uint8, device=srcs[0].device)
    o = _opts(coord, cubic_a, impl, tile, threads)
    if antialias:
        o.flags = B.RS_FLAG_ANTIALIAS
    with _on_device(srcs[0]):
        B.check(lib().rs_resize_batched(arr, n, dt, workspace.data_ptr(), nb.value, ctypes.byref(o),
                                        _stream(srcs[0])), "rs_resize_batched")
    return outs


class BatchedPlan:
    """A ragged batch recorded once (work list uploaded, persistent launch
    captured as a CUDA graph) and replayed by launch()."""

    def __init__(self, srcs, outs, methods, *, coord="asymmetric", cubic_a: float = -0.5,
                 impl: str = "auto", tile=None, threads: int = 0, antialias: bool = False):
        _require_cuda(*srcs, *outs)
        self.srcs, self.outs = list(srcs), list(outs)
        arr, n = _descs(self.srcs, self.outs, methods)
        nb = ctypes.c_size_t(0)
        dt = _dtype(srcs[0])
        B.check(lib().rs_resize_batched_workspace(arr, n, dt, ctypes.byref(nb)), "rs_resize_batched_workspace")
        self.workspace = torch.empty(max(1, nb.value), dtype=torch.uint8, device=srcs[0].device)
        o = _opts(coord, cubic_a, impl, tile, threads)
        if antialias:
            o.flags = B.RS_FLAG_ANTIALIAS
        self._plan = ctypes.c_void_p()
        self.device = srcs[0].device
        with torch.cuda.device(self.device):
            B.check(lib().rs_batched_plan_create(arr, n, dt, self.workspace.data_ptr(), nb.value,
                                                 ctypes.byref(o), _stream(srcs[0]), ctypes.byref(self._plan)),
                    "rs_batched_plan_create")

    def kernels(self) -> int:
        """Kernel launches one replay makes (one per non-empty class)."""
        n = ctypes.c_int32(0)
        B.check(lib().rs_batched_plan_kernels(self._plan, ctypes.byref(n)), "rs_batched_plan_kernels")
        return n.value

    def launch(self, stream: int | None = None) -> None:
        with torch.cuda.device(self.device):
            st = torch.cuda.current_stream(self.device).cuda_stream if stream is None else stream
            B.check(lib().rs_batched_plan_launch(self._plan, st), "rs_batched_plan_launch")

    def close(self) -> None:
        if self._plan:
            lib().rs_batched_plan_destroy(self._plan)
            self._plan = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def autotune(x: torch.Tensor, size, method, *, layout="hwc", coord="asymmetric", cubic_a=-0.5,
             out: torch.Tensor | None = None) -> dict:
    """Time every tile configuration for this problem class and cache the best."""
    _require_cuda(x)
    Ho, Wo = int(size[0]), int(size[1])
    if out is None:
        out = torch.empty(_out_shape(x, layout, Ho, Wo), dtype=x.dtype, device=x.device)
    Li, Lo = _layout(x, layout), _layout(out, layout)
    o = _opts(coord, cubic_a, "auto", None, 0)
    best = B.RsTileConfig()
    with _on_device(x):
        B.check(lib().rs_autotune(x.data_ptr(), ctypes.byref(Li), out.data_ptr(), ctypes.byref(Lo), _dtype(x),
                                  _code(METHODS, method, "method"), ctypes.byref(o), _stream(x),
                                  ctypes.byref(best)), "rs_autotune")
    return {"impl": IMPL_NAMES.get(best.impl, best.impl), "tile_w": best.tile_w, "tile_h": best.tile_h,
            "threads": best.threads, "waves": best.waves, "best_us": best.best_us,
            "default_us": best.default_us, "candidates": best.candidates}


def autotune_batched(srcs, outs, methods, *, coord="asymmetric", cubic_a: float = -0.5,
                     workspace: torch.Tensor | None = None, antialias: bool = False) -> dict:
    """Time the batch at each item shape and cache the fastest for later
    batch calls on the same descriptors (the outputs are written)."""
    _require_cuda(*srcs, *outs)
    arr, n = _descs(srcs, outs, methods)
    nb = ctypes.c_size_t(0)
    dt = _dtype(srcs[0])
    B.check(lib().rs_resize_batched_workspace(arr, n, dt, ctypes.byref(nb)), "rs_resize_batched_workspace")
    if workspace is None or workspace.numel() * workspace.element_size() < nb.value:
        workspace = torch.empty(max(1, nb.value), dtype=torch.uint8, device=srcs[0].device)
    o = _opts(coord, cubic_a, "auto", None, 0)
    if antialias:
        o.flags = B.RS_FLAG_ANTIALIAS
    best = B.RsTileConfig()
    with _on_device(srcs[0]):
        B.check(lib().rs_autotune_batched(arr, n, dt, workspace.data_ptr(), nb.value, ctypes.byref(o),
                                          _stream(srcs[0]), ctypes.byref(best)), "rs_autotune_batched")
    return {"impl": IMPL_NAMES.get(best.impl, best.impl), "band": best.tile_w, "chunk": best.tile_h,
            "best_us": best.best_us, "default_us": best.default_us, "candidates": best.candidates}


def tile_config(x: torch.Tensor, size, method, *, layout="hwc", coord="asymmetric", cubic_a=-0.5) -> dict:
    Ho, Wo = int(size[0]), int(size[1])
    Li = _layout(x, layout)
    Lo = _layout(torch.empty(_out_shape(x, layout, Ho, Wo), dtype=x.dtype, device="meta"), layout)
    o = _opts(coord, cubic_a, "auto", None, 0)
    c = B.RsTileConfig()
    B.check(lib().rs_tile_config_for(ctypes.byref(Li), ctypes.byref(Lo), _dtype(x),
                                     _code(METHODS, method, "method"), ctypes.byref(o), ctypes.byref(c)),
            "rs_tile_config_for")
    return {"impl": IMPL_NAMES.get(c.impl, c.impl), "tile_w": c.tile_w, "tile_h": c.tile_h,
            "threads": c.threads, "waves": c.waves}


def tune_cache_save(path: str) -> None:
    B.check(lib().rs_tune_cache_save(str(path).encode()), "rs_tune_cache_save")


def tune_cache_load(path: str) -> None:
    B.check(lib().rs_tune_cache_load(str(path).encode()), "rs_tune_cache_load")


def tune_cache_clear() -> None:
    lib().rs_tune_cache_clear()


def debug_fault(device=None) -> int:
    """Synchronises the current stream and returns (and clears) the device's
    fault word; 0 means no kernel reported a bound violation."""
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    code = ctypes.c_uint32(0)
    with torch.cuda.device(dev):
        B.check(lib().rs_debug_fault(torch.cuda.current_stream(dev).cuda_stream, ctypes.byref(code)),
                "rs_debug_fault")
    return code.value


def version() -> str:
    return lib().rs_version().decode()
