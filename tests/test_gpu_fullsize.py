"""Parity at the benchmark workloads' full sizes, in the launch configuration
the benchmark times (AUTO, default options): sampled output points (the
corners, the edges' midpoints and uniform points) against the FP64 oracle
evaluated point by point."""
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


def _points(oracle, x64, Ho, Wo, method, seed, n):
    from paper_1001_1718_gb300 import workloads
    ys, xs = workloads.sample_points(seed, Ho, Wo, n)
    ref = oracle.resize_points(x64, Ho, Wo, method, 0, -0.5, ys, xs)
    return ys, xs, ref


def test_rgb4096_headline_step(rs, oracle):
    """RGB uint8 4096x4096 (the smooth-field recipe): bicubic x2 and x1.7,
    nearest x2. Nearest and the dyadic x2 bicubic are exact; x1.7 obeys the
    uint8 rule."""
    from paper_1001_1718_gb300 import workloads
    img = workloads.workload_rgb_4096(seed=2)
    x = torch.from_numpy(img).cuda()
    x64 = img.astype(np.float64)
    for k, (method, s) in enumerate(((BC, 2.0), (BC, 1.7), (NN, 2.0))):
        Ho, Wo = workloads.out_size(4096, s), workloads.out_size(4096, s)
        y = rs.resize(x, (Ho, Wo), MNAME[method])
        torch.cuda.synchronize()
        ys, xs, ref = _points(oracle, x64, Ho, Wo, method, 30 + k, 4096)
        got = y[torch.from_numpy(ys).cuda(), torch.from_numpy(xs).cuda()]
        check(got, ref, "u8", method, 255.0, f"rgb4096 {MNAME[method]} x{s}")
        if s == 2.0:   # exact: nearest by index, bicubic by dyadic weights
            assert np.array_equal(got.cpu().numpy(), oracle.quantize_u8(ref))
    assert rs.debug_fault() == 0


@pytest.fixture(scope="module")
def field8192():
    from paper_1001_1718_gb300 import workloads
    return workloads.workload_float_8192(seed=3)


@pytest.mark.parametrize("dtype", ["f32", "f16", "bf16"])
def test_float8192_bicubic_x2(rs, oracle, field8192, dtype):
    """Single-channel 8192x8192 field stored as FP32 / FP16 / BF16, bicubic
    x2 to 16384x16384; the oracle sees the stored values."""
    t = to_storage(field8192, dtype)
    x64 = as_f64(t)
    y = rs.resize(t.cuda(), (16384, 16384), "bicubic")
    torch.cuda.synchronize()
    ys, xs, ref = _points(oracle, x64, 16384, 16384, BC, 40, 4096)
    got = y[torch.from_numpy(ys).cuda(), torch.from_numpy(xs).cuda()]
    check(got, ref, dtype, BC, float(np.abs(x64).max()), f"float8192 {dtype}")
    del y
    assert rs.debug_fault() == 0


@pytest.mark.parametrize("method", [BL, BC])
def test_nchw512_forward(rs, oracle, method):
    """NCHW FP32 32x3x512x512, x2 (1024x1024) and x0.5 (256x256, the
    transposed-role window), sampled on a first, a middle and a last plane."""
    from paper_1001_1718_gb300 import workloads
    xn = workloads.workload_nchw_512(seed=5).astype(np.float32)
    x = torch.from_numpy(xn).cuda()
    for k, S in enumerate((1024, 256)):
        y = rs.resize(x, (S, S), MNAME[method], layout="nchw")
        torch.cuda.synchronize()
        for n, c in ((0, 0), (15, 1), (31, 2)):
            plane = xn[n, c].astype(np.float64)
            ys, xs, ref = _points(oracle, plane, S, S, method, 50 + 10 * k + n, 2048)
            got = y[n, c][torch.from_numpy(ys).cuda(), torch.from_numpy(xs).cuda()]
            check(got, ref, "f32", method, float(np.abs(plane).max()), f"nchw512 {MNAME[method]} {S} plane {(n, c)}")
    assert rs.debug_fault() == 0
