"""ctypes front end of the FP64 CPU oracle (resample_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
benchmark's CPU-baseline leg. It never touches the CUDA library and the CUDA
library never touches it.

Layouts: images are HWC (H, W, C) float64 arrays; planar NCHW tensors are
viewed as one HWC image with N*C interleaved channels (marshalling only: the
arithmetic is identical per channel).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from pathlib import Path

import numpy as np

HERE = Path(__file__).resolve().parent
SRC = HERE / "resample_oracle.c"
BUILD = HERE / "_build"
LIB = BUILD / "liboracle.so"

NEAREST, BILINEAR, BICUBIC = 0, 1, 2
ASYMMETRIC, HALF_PIXEL, ALIGN_CORNERS = 0, 1, 2

_lib = None


def build(force: bool = False) -> Path:
    """Compile the oracle with gcc (OpenMP when available)."""
    if LIB.exists() and not force and LIB.stat().st_mtime >= SRC.stat().st_mtime:
        return LIB
    BUILD.mkdir(exist_ok=True)
    tmp = BUILD / f"liboracle.{os.getpid()}.so"
    base = ["gcc", "-O2", "-ffp-contract=off", "-std=c11", "-shared", "-fPIC",
            str(SRC), "-o", str(tmp), "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True, text=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True, text=True)
    os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        # The mutation tests point this at a deliberately broken build.
        override = os.environ.get("RESAMPLE_ORACLE_LIB")
        if override:
            path = override
        else:
            build()
            path = str(LIB)
        L = ctypes.CDLL(path)
        P, I64, I, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
        L.oracle_resize_f64.argtypes = [P, I64, I64, I64, P, I64, I64, I, I, D]
        L.oracle_resize_points_f64.argtypes = [P, I64, I64, I64, I64, I64, I, I, D,
                                               P, P, I64, P]
        L.oracle_bilinear_eq5_f64.argtypes = [P, I64, I64, P, I64, I64]
        L.oracle_adjoint_f64.argtypes = [P, I64, I64, I64, P, I64, I64, I, I, D]
        L.oracle_axis_matrix.argtypes = [I64, I64, I, I, D, P]
        L.oracle_axis_taps.argtypes = [I64, I64, I, I, D, P, P]
        L.oracle_quantize_u8.argtypes = [P, I64, P]
        L.oracle_to_f16_bits.argtypes = [P, I64, P]
        L.oracle_to_bf16_bits.argtypes = [P, I64, P]
        L.oracle_tile_of_pixel.argtypes = [I64, I64, I64, I64, P, P, P, P]
        L.oracle_num_threads.restype = I
        L.oracle_set_num_threads.argtypes = [I]
        _lib = L
    return _lib


def _p(a: np.ndarray) -> int:
    return a.ctypes.data


def _hwc(src: np.ndarray) -> np.ndarray:
    a = np.ascontiguousarray(src, dtype=np.float64)
    if a.ndim == 2:
        a = a[:, :, None]
    return a


def num_threads() -> int:
    return lib().oracle_num_threads()


def set_num_threads(n: int) -> None:
    lib().oracle_set_num_threads(int(n))


def resize(src, Ho: int, Wo: int, method: int, coord: int = ASYMMETRIC,
           a: float = -0.5) -> np.ndarray:
    """FP64 resampling of an (H, W) or (H, W, C) image; returns (Ho, Wo, C)."""
    x = _hwc(src)
    H, W, C = x.shape
    out = np.empty((Ho, Wo, C), np.float64)
    lib().oracle_resize_f64(_p(x), H, W, C, _p(out), Ho, Wo, method, coord, a)
    return out


def resize_points(src, Ho: int, Wo: int, method: int, coord: int, a: float,
                  ys, xs) -> np.ndarray:
    """FP64 outputs at the points (ys[k], xs[k]); returns (npts, C)."""
    x = _hwc(src)
    H, W, C = x.shape
    ys = np.ascontiguousarray(ys, np.int64)
    xs = np.ascontiguousarray(xs, np.int64)
    out = np.empty((len(ys), C), np.float64)
    lib().oracle_resize_points_f64(_p(x), H, W, C, Ho, Wo, method, coord, a,
                                   _p(ys), _p(xs), len(ys), _p(out))
    return out


def resize_nchw(x, Ho: int, Wo: int, method: int, coord: int = ASYMMETRIC,
                a: float = -0.5) -> np.ndarray:
    N, C, H, W = x.shape
    hwc = np.ascontiguousarray(np.asarray(x, np.float64).reshape(N * C, H, W).transpose(1, 2, 0))
    y = resize(hwc, Ho, Wo, method, coord, a)
    return np.ascontiguousarray(y.transpose(2, 0, 1).reshape(N, C, Ho, Wo))


def resize_normalize(src, Ho: int, Wo: int, method: int, mean, std, coord: int = ASYMMETRIC,
                     a: float = -0.5) -> np.ndarray:
    """The serving pre-process in FP64: resample an (H, W, C) or (N, H, W, C)
    interleaved image (Eqs. 1-5, as resize), then normalise each channel,
    (y - mean[c]) / std[c], and return planar (C, Ho, Wo) or (N, C, Ho, Wo).
    Nothing is rounded in between (the fused pass never stores the resampled
    value); round the result with store() for a storage dtype."""
    x = np.asarray(src, np.float64)
    batched = x.ndim == 4
    if not batched:
        x = x[None]
    N, H, W, C = x.shape
    m = np.asarray(mean, np.float64).reshape(C)
    s = np.asarray(std, np.float64).reshape(C)
    out = np.empty((N, C, Ho, Wo), np.float64)
    for n in range(N):
        y = resize(x[n], Ho, Wo, method, coord, a)          # (Ho, Wo, C)
        out[n] = ((y - m) / s).transpose(2, 0, 1)
    return out if batched else out[0]


def bilinear_eq5(src2d, Ho: int, Wo: int) -> np.ndarray:
    x = np.ascontiguousarray(src2d, np.float64)
    H, W = x.shape
    out = np.empty((Ho, Wo), np.float64)
    lib().oracle_bilinear_eq5_f64(_p(x), H, W, _p(out), Ho, Wo)
    return out


def adjoint(gy, H: int, W: int, method: int, coord: int = ASYMMETRIC,
            a: float = -0.5) -> np.ndarray:
    """Transpose of resize(): (Ho, Wo, C) output gradient -> (H, W, C)."""
    g = _hwc(gy)
    Ho, Wo, C = g.shape
    out = np.empty((H, W, C), np.float64)
    lib().oracle_adjoint_f64(_p(g), Ho, Wo, C, _p(out), H, W, method, coord, a)
    return out


def adjoint_nchw(gy, H: int, W: int, method: int, coord: int = ASYMMETRIC,
                 a: float = -0.5) -> np.ndarray:
    N, C, Ho, Wo = gy.shape
    hwc = np.ascontiguousarray(np.asarray(gy, np.float64).reshape(N * C, Ho, Wo).transpose(1, 2, 0))
    g = adjoint(hwc, H, W, method, coord, a)
    return np.ascontiguousarray(g.transpose(2, 0, 1).reshape(N, C, H, W))


def axis_matrix(n: int, m: int, method: int, coord: int = ASYMMETRIC,
                a: float = -0.5) -> np.ndarray:
    A = np.empty((m, n), np.float64)
    lib().oracle_axis_matrix(n, m, method, coord, a, _p(A))
    return A


def axis_taps(n: int, m: int, method: int, coord: int = ASYMMETRIC, a: float = -0.5):
    idx = np.empty((m, 4), np.int64)
    w = np.empty((m, 4), np.float64)
    lib().oracle_axis_taps(n, m, method, coord, a, _p(idx), _p(w))
    return idx, w


# ---------------------------------------------------------------------------
# Antialiased resampling (an extension: the paper samples point-wise, Eqs.
# 1-5, and says nothing about filtering before a downscale). Reading used:
# the interpolation kernel is stretched by the downscale factor, so every
# output averages the source footprint it covers, and taps that fall outside
# the image are dropped and the rest renormalised.
#   f = max(n / m, 1) (stretch; 1 when upsampling), R = 1 (triangle, the
#   bilinear kernel) or 2 (Keys' cubic with parameter a);
#   centre of output j in source pixel units: c = (j + 1/2) n / m;
#   taps i = floor(c - R f + 1/2) .. floor(c + R f + 1/2) - 1, cut to [0, n);
#   weight of tap i: K((i + 1/2 - c) / f), divided by the sum over the taps.
# Written out in FP64 as dense per-axis matrices; the image is
# Ay X Ax^T per channel (a matrix product).
# ---------------------------------------------------------------------------

def _keys(u: np.ndarray, a: float) -> np.ndarray:
    u = np.abs(u)
    out = np.zeros_like(u)
    m1 = u <= 1
    m2 = (u > 1) & (u < 2)
    out[m1] = ((a + 2) * u[m1] - (a + 3)) * u[m1] ** 2 + 1
    out[m2] = ((a * u[m2] - 5 * a) * u[m2] + 8 * a) * u[m2] - 4 * a
    return out


def aa_axis_matrix(n: int, m: int, method: int, a: float = -0.5) -> np.ndarray:
    """(m, n) FP64 antialias weights of one axis (method BILINEAR or BICUBIC)."""
    if method not in (BILINEAR, BICUBIC):
        raise ValueError("antialias is defined for bilinear and bicubic")
    R = 1.0 if method == BILINEAR else 2.0
    f = max(n / m, 1.0)
    A = np.zeros((m, n), np.float64)
    for j in range(m):
        c = (j + 0.5) * n / m
        lo = max(int(np.floor(c - R * f + 0.5)), 0)
        hi = min(int(np.floor(c + R * f + 0.5)), n)
        i = np.arange(lo, hi, dtype=np.float64)
        u = (i + 0.5 - c) / f
        w = np.maximum(0.0, 1.0 - np.abs(u)) if method == BILINEAR else _keys(u, a)
        tot = w.sum()
        if tot != 0.0:
            w = w / tot
        A[j, lo:hi] = w
    return A


def resize_aa(src, Ho: int, Wo: int, method: int, a: float = -0.5) -> np.ndarray:
    """FP64 antialiased resampling of an (H, W) or (H, W, C) image; (Ho, Wo, C)."""
    x = _hwc(src)
    H, W, C = x.shape
    Ay = aa_axis_matrix(H, Ho, method, a)
    Ax = aa_axis_matrix(W, Wo, method, a)
    out = np.empty((Ho, Wo, C), np.float64)
    for c in range(C):
        out[:, :, c] = Ay @ x[:, :, c] @ Ax.T
    return out


def resize_aa_nchw(x, Ho: int, Wo: int, method: int, a: float = -0.5) -> np.ndarray:
    N, C, H, W = x.shape
    Ay = aa_axis_matrix(H, Ho, method, a)
    Ax = aa_axis_matrix(W, Wo, method, a)
    x = np.asarray(x, np.float64)
    return np.einsum("ih,nchw,jw->ncij", Ay, x, Ax, optimize=True)


def adjoint_aa_nchw(gy, H: int, W: int, method: int, a: float = -0.5) -> np.ndarray:
    """Transpose of resize_aa_nchw(): dX = Ay^T dY Ax per plane, from the same
    FP64 axis matrices; (N, C, H, W)."""
    N, C, Ho, Wo = gy.shape
    Ay = aa_axis_matrix(H, Ho, method, a)
    Ax = aa_axis_matrix(W, Wo, method, a)
    return np.einsum("ih,ncij,jw->nchw", Ay, np.asarray(gy, np.float64), Ax, optimize=True)


def quantize_u8(v) -> np.ndarray:
    x = np.ascontiguousarray(v, np.float64)
    out = np.empty(x.shape, np.uint8)
    lib().oracle_quantize_u8(_p(x), x.size, _p(out))
    return out


def to_f16_bits(v) -> np.ndarray:
    x = np.ascontiguousarray(v, np.float64)
    out = np.empty(x.shape, np.uint16)
    lib().oracle_to_f16_bits(_p(x), x.size, _p(out))
    return out


def to_bf16_bits(v) -> np.ndarray:
    x = np.ascontiguousarray(v, np.float64)
    out = np.empty(x.shape, np.uint16)
    lib().oracle_to_bf16_bits(_p(x), x.size, _p(out))
    return out


def bf16_bits_to_f64(bits) -> np.ndarray:
    b = np.ascontiguousarray(bits, np.uint16).astype(np.uint32) << 16
    return b.view(np.float32).astype(np.float64)


def store(v, dtype: str) -> np.ndarray:
    """Round FP64 values to a storage dtype. Returns uint8, float16, uint16
    (bfloat16 bit patterns) or float32 arrays."""
    if dtype == "u8":
        return quantize_u8(v)
    if dtype == "f16":
        return to_f16_bits(v).view(np.float16)
    if dtype == "bf16":
        return to_bf16_bits(v)
    if dtype == "f32":
        return np.asarray(v, np.float64).astype(np.float32)
    raise ValueError(dtype)


def tile_of_pixel(px: int, py: int, bw: int, bh: int):
    vals = [ctypes.c_int64() for _ in range(4)]
    lib().oracle_tile_of_pixel(px, py, bw, bh, *[ctypes.addressof(v) for v in vals])
    return tuple(v.value for v in vals)  # (bx, by, tx, ty)
