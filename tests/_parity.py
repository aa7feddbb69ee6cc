"""Comparison rules between the CUDA path and the FP64 oracle.

The CUDA path computes in FP32 and rounds once to the storage type. Its FP32
value v is held to the normwise bound |v - exact| <= TOL with
TOL = 1e-5 * max(1, max |src|). For the rounded types this becomes a bracket:
rounding is monotone, so the stored value g must satisfy
    Q(exact - TOL) <= g <= Q(exact + TOL)
where Q is the oracle's rounding to that type (clamp + round half to even for
uint8, round to nearest even for FP16 / BF16). Additionally:
- nearest: bit-exact in every dtype (the source index is exact integer math);
- uint8: |g - Q(exact)| <= 1 step everywhere (the bracket is far narrower
  than a step, so g differs from Q(exact) only next to a rounding tie);
- FP32: |g - exact| <= TOL.
"""
import numpy as np
import torch

TORCH_DT = {"u8": torch.uint8, "f16": torch.float16, "bf16": torch.bfloat16, "f32": torch.float32}
F32_TOL = 1e-5


def to_storage(x64: np.ndarray, dtype: str) -> torch.Tensor:
    """Host float64 values -> CPU tensor of the storage dtype (round to nearest even)."""
    if dtype == "u8":
        return torch.from_numpy(np.clip(np.rint(x64), 0, 255).astype(np.uint8))
    return torch.from_numpy(np.ascontiguousarray(x64)).to(TORCH_DT[dtype])


def as_f64(t: torch.Tensor) -> np.ndarray:
    t = t.detach().cpu()
    if t.dtype == torch.uint8:
        return t.numpy().astype(np.float64)
    return t.to(torch.float64).numpy()


def rounded(v: np.ndarray, dtype: str) -> np.ndarray:
    """The oracle's rounding of v to `dtype`, as float64 values."""
    from oracle import oracle
    r = oracle.store(v, dtype)
    if dtype == "f16":
        return r.view(np.float16).astype(np.float64)
    if dtype == "bf16":
        return oracle.bf16_bits_to_f64(r)
    return r.astype(np.float64)


def tolerance(src_absmax: float) -> float:
    return F32_TOL * max(1.0, src_absmax)


def check(got: torch.Tensor, ref64: np.ndarray, dtype: str, method: int, src_absmax: float,
          what: str = "") -> dict:
    """Asserts the parity rule; returns error statistics."""
    g = as_f64(got).reshape(ref64.shape)
    stats = {"max_abs": float(np.abs(g - ref64).max()) if g.size else 0.0,
             "mean_abs": float(np.abs(g - ref64).mean()) if g.size else 0.0}
    if method == 0:
        bad = g != rounded(ref64, dtype)
        assert not bad.any(), f"{what}: nearest not bit-exact at {int(bad.sum())} elements"
        return stats
    tol = tolerance(src_absmax)
    if dtype == "f32":
        assert stats["max_abs"] <= tol, f"{what}: FP32 error {stats['max_abs']} > {tol}"
        return stats
    lo, hi = rounded(ref64 - tol, dtype), rounded(ref64 + tol, dtype)
    bad = (g < lo) | (g > hi)
    assert not bad.any(), f"{what}: {dtype} outside the rounding bracket at {int(bad.sum())} elements"
    q = rounded(ref64, dtype)
    if dtype == "u8":
        d = np.abs(g - q)
        assert d.max(initial=0) <= 1, f"{what}: uint8 off by {d.max()}"
        stats["u8_off_by_one"] = int((d > 0).sum())
    else:
        stats["differs_from_rounded_oracle"] = int((g != q).sum())
    return stats


def aa_taps(n, m, method):
    """The most antialias taps an output of the axis n -> m has, by the
    header's integer bounds: floor(((2j+1) n -+ 2 R F + m) / (2m)), F = max(n, m),
    cut to [0, n)."""
    R, F = (1 if method == 1 else 2), max(n, m)
    best = 0
    for j in range(m):
        a = (2 * j + 1) * n + m
        lo, hi = max((a - 2 * R * F) // (2 * m), 0), min((a + 2 * R * F) // (2 * m), n)
        best = max(best, hi - lo)
    return best
