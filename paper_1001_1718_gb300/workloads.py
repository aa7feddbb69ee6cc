"""Seeded synthetic inputs for the resampling workloads.

This module draws the images that both the CUDA path and the FP64 oracle are
fed. It holds none of the resampling arithmetic: it only produces pixels,
target sizes and per-image method choices. Every generator takes an explicit
seed and uses numpy's PCG64, so a given (seed, shape) always yields the same
bytes on any host.

The paper resizes one 800x800 source image by bilinear interpolation at
scales 2..10 (Sec. III.B, Fig. 3); it ships no image. The workloads below stand
in for it with synthetic fields of the shapes and value ranges listed with each
generator.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

NEAREST, BILINEAR, BICUBIC = 0, 1, 2
METHOD_NAMES = {NEAREST: "nearest", BILINEAR: "bilinear", BICUBIC: "bicubic"}


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def out_size(n: int, scale: float) -> int:
    """Output extent for a scale factor: floor(n * scale), at least 1."""
    return max(1, int(math.floor(n * scale)))


def uniform_u8(seed: int, H: int, W: int, C: int = 1) -> np.ndarray:
    """HWC uint8 image, pixels i.i.d. uniform on 0..255."""
    g = rng(seed)
    return g.integers(0, 256, size=(H, W, C), dtype=np.uint8)


def _blob_field(g: np.random.Generator, H: int, W: int, nblobs: int,
                amp: tuple[float, float], sigma: tuple[float, float]) -> np.ndarray:
    """Sum of isotropic Gaussian blobs, float64 (H, W).

    A blob exp(-((y-cy)^2 + (x-cx)^2) / (2 s^2)) factors into a column profile
    times a row profile, so the sum over blobs is one (H x nb) @ (nb x W)
    product.
    """
    a = g.uniform(amp[0], amp[1], size=nblobs)
    s = g.uniform(sigma[0], sigma[1], size=nblobs)
    cy = g.uniform(0.0, H, size=nblobs)
    cx = g.uniform(0.0, W, size=nblobs)
    y = np.arange(H, dtype=np.float64)[:, None]
    x = np.arange(W, dtype=np.float64)[:, None]
    gy = np.exp(-((y - cy[None, :]) ** 2) / (2.0 * s[None, :] ** 2)) * a[None, :]
    gx = np.exp(-((x - cx[None, :]) ** 2) / (2.0 * s[None, :] ** 2))
    return gy @ gx.T


def smooth_field_u8(seed: int, H: int, W: int, C: int = 3, nblobs: int = 64,
                    amp: tuple[float, float] = (-96.0, 96.0),
                    sigma: tuple[float, float] = (32.0, 512.0),
                    noise: float = 8.0) -> np.ndarray:
    """HWC uint8 smooth field: 128 + sum of Gaussian blobs (independent per
    channel) + uniform noise of amplitude `noise`, rounded and clipped to 0..255."""
    g = rng(seed)
    out = np.empty((H, W, C), dtype=np.uint8)
    for c in range(C):
        f = 128.0 + _blob_field(g, H, W, nblobs, amp, sigma)
        f += g.uniform(-noise, noise, size=(H, W))
        out[:, :, c] = np.clip(np.rint(f), 0, 255).astype(np.uint8)
    return out


def float_field(seed: int, H: int, W: int, nblobs: int = 64) -> np.ndarray:
    """Single-channel float64 (H, W): uniform [0,1) plus a smooth blob field
    (amplitudes U(-0.5, 0.5), widths U(64, 1024) px)."""
    g = rng(seed)
    f = g.random((H, W))
    f += _blob_field(g, H, W, nblobs, (-0.5, 0.5), (64.0, 1024.0))
    return f


def normal_nchw(seed: int, N: int, C: int, H: int, W: int) -> np.ndarray:
    """float64 NCHW tensor with i.i.d. N(0, 1) entries."""
    return rng(seed).standard_normal((N, C, H, W))


# --------------------------------------------------------------------------
# Named workloads (sizes, value ranges and seeds of each configuration)
# --------------------------------------------------------------------------

def workload_u8_bilinear_512(seed: int = 1):
    """Single-channel uint8 512x512, uniform 0..255; bilinear x2 to 1024x1024."""
    return uniform_u8(seed, 512, 512, 1), (1024, 1024)


def workload_rgb_4096(seed: int = 2, H: int = 4096, W: int = 4096):
    """RGB uint8 interleaved smooth field (64 blobs + noise 8)."""
    return smooth_field_u8(seed, H, W, 3)


def workload_float_8192(seed: int = 3, H: int = 8192, W: int = 8192):
    """Single-channel float64 field; the caller rounds it to its storage dtype."""
    return float_field(seed, H, W)


@dataclass
class BatchItem:
    H: int
    W: int
    scale: float
    Ho: int
    Wo: int
    method: int
    seed: int


def batch_spec(seed: int = 4, n: int = 256, lo: int = 64, hi: int = 2048,
               smin: float = 0.5, smax: float = 4.0) -> list[BatchItem]:
    """Ragged batch: H and W independently uniform on lo..hi, one scale per
    image uniform on [smin, smax), method alternating bilinear / bicubic."""
    g = rng(seed)
    H = g.integers(lo, hi + 1, size=n)
    W = g.integers(lo, hi + 1, size=n)
    s = g.uniform(smin, smax, size=n)
    items = []
    for k in range(n):
        h, w, sc = int(H[k]), int(W[k]), float(s[k])
        items.append(BatchItem(h, w, sc, out_size(h, sc), out_size(w, sc),
                               BILINEAR if k % 2 == 0 else BICUBIC,
                               seed * 100003 + k))
    return items


def batch_images(items: list[BatchItem], C: int = 3) -> list[np.ndarray]:
    """Pixels for each batch item from the smooth-field generator."""
    return [smooth_field_u8(it.seed, it.H, it.W, C) for it in items]


def workload_nchw_512(seed: int = 5, N: int = 32, C: int = 3, H: int = 512, W: int = 512):
    return normal_nchw(seed, N, C, H, W)


def sample_points(seed: int, Ho: int, Wo: int, n: int) -> tuple[np.ndarray, np.ndarray]:
    """n output coordinates (y, x): the four corners, the edges' midpoints and
    the rest uniform over the image."""
    g = rng(seed)
    ys = [0, 0, Ho - 1, Ho - 1, Ho // 2, 0, Ho - 1, Ho // 2]
    xs = [0, Wo - 1, 0, Wo - 1, 0, Wo // 2, Wo // 2, Wo - 1]
    m = max(0, n - len(ys))
    ys = np.concatenate([np.array(ys[:n], np.int64), g.integers(0, Ho, m)])
    xs = np.concatenate([np.array(xs[:n], np.int64), g.integers(0, Wo, m)])
    return ys.astype(np.int64), xs.astype(np.int64)
