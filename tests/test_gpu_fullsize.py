"""Parity at the benchmark workloads' full sizes, in the launch configuration
the benchmark times (AUTO, default options): every output element against
the FP64 oracle's full output, compared in bands of rows. These launches are
the only ones that reach the full-size geometry (32-bit band offsets near
their bound, the occupancy-derived band heights, hundreds of strips)."""
import numpy as np
import pytest
import torch

from _parity import check, to_storage, as_f64

pytestmark = pytest.mark.gpu

NN, BL, BC = 0, 1, 2
MNAME = {NN: "nearest", BL: "bilinear", BC: "bicubic"}


@pytest.fixture(scope="module")
def rs():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1001_1718_gb300 as rs
    return rs


def check_full(y: torch.Tensor, ref: np.ndarray, dtype: str, method: int, absmax: float, what: str,
               band: int = 1024) -> dict:
    """check() on every element, band by band (rows of the leading axis)."""
    stats = {"max_abs": 0.0, "sum_abs": 0.0, "n": 0}
    for r0 in range(0, y.shape[0], band):
        g = y[r0:r0 + band]
        s = check(g, ref[r0:r0 + band], dtype, method, absmax, f"{what} rows {r0}..")
        stats["max_abs"] = max(stats["max_abs"], s["max_abs"])
        stats["sum_abs"] += s["mean_abs"] * g.numel()
        stats["n"] += g.numel()
    assert stats["n"] == ref.size
    return stats


def test_rgb4096_headline_step(rs, oracle):
    """RGB uint8 4096x4096 (the smooth-field recipe): bicubic x2 and x1.7,
    nearest x2, every element. Nearest and the dyadic x2 bicubic are exact;
    x1.7 obeys the uint8 rule."""
    from paper_1001_1718_gb300 import workloads
    img = workloads.workload_rgb_4096(seed=2)
    x = torch.from_numpy(img).cuda()
    x64 = img.astype(np.float64)
    for method, s in ((BC, 2.0), (BC, 1.7), (NN, 2.0)):
        Ho, Wo = workloads.out_size(4096, s), workloads.out_size(4096, s)
        y = rs.resize(x, (Ho, Wo), MNAME[method])
        torch.cuda.synchronize()
        ref = oracle.resize(x64, Ho, Wo, method)
        check_full(y, ref, "u8", method, 255.0, f"rgb4096 {MNAME[method]} x{s}")
        if s == 2.0:   # exact: nearest by index, bicubic by dyadic weights
            for r0 in range(0, Ho, 1024):
                assert np.array_equal(y[r0:r0 + 1024].cpu().numpy(), oracle.quantize_u8(ref[r0:r0 + 1024])), r0
        del y, ref
    assert rs.debug_fault() == 0


@pytest.fixture(scope="module")
def field8192():
    from paper_1001_1718_gb300 import workloads
    return workloads.workload_float_8192(seed=3)


@pytest.mark.parametrize("dtype", ["f32", "f16", "bf16"])
def test_float8192_bicubic_x2(rs, oracle, field8192, dtype):
    """Single-channel 8192x8192 field stored as FP32 / FP16 / BF16, bicubic
    x2 to 16384x16384, every element; the oracle sees the stored values."""
    t = to_storage(field8192, dtype)
    x64 = as_f64(t)
    y = rs.resize(t.cuda(), (16384, 16384), "bicubic")
    torch.cuda.synchronize()
    ref = oracle.resize(x64, 16384, 16384, BC)[:, :, 0]
    check_full(y, ref, dtype, BC, float(np.abs(x64).max()), f"float8192 {dtype}")
    del y, ref
    assert rs.debug_fault() == 0


@pytest.mark.parametrize("method", [BL, BC])
def test_nchw512_forward(rs, oracle, method):
    """NCHW FP32 32x3x512x512, x2 (1024x1024) and x0.5 (256x256, the
    transposed-role window), every element of every plane."""
    from paper_1001_1718_gb300 import workloads
    xn = workloads.workload_nchw_512(seed=5).astype(np.float32)
    x = torch.from_numpy(xn).cuda()
    absmax = float(np.abs(xn).max())
    for S in (1024, 256):
        y = rs.resize(x, (S, S), MNAME[method], layout="nchw")
        torch.cuda.synchronize()
        ref = oracle.resize_nchw(xn.astype(np.float64), S, S, method)
        check_full(y.reshape(-1, S, S), ref.reshape(-1, S, S), "f32", method, absmax,
                   f"nchw512 {MNAME[method]} {S}", band=8)
        del y, ref
    assert rs.debug_fault() == 0
