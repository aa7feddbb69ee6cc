"""GPU backward parity: the gather-form adjoint kernel against the FP64
oracle's adjoint (a scatter over the forward's taps), finite differences of
the oracle forward, autograd plumbing and determinism."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

MN = {0: "nearest", 1: "bilinear", 2: "bicubic"}
CN = {0: "asymmetric", 1: "half_pixel", 2: "align_corners"}


@pytest.fixture(scope="module")
def rs():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1001_1718_gb300 as rs
    return rs


def _tol(oracle, H, W, Ho, Wo, method, coord, gmax):
    """Normwise FP32 bound: 1e-5 * max|dY| * ||Ay^T||_inf * ||Ax^T||_inf."""
    Ay = oracle.axis_matrix(H, Ho, method, coord)
    Ax = oracle.axis_matrix(W, Wo, method, coord)
    return 1e-5 * max(1.0, gmax) * np.abs(Ay.T).sum(1).max() * np.abs(Ax.T).sum(1).max()


SHAPES = [(37, 53, 74, 106), (64, 48, 32, 24), (31, 29, 53, 71), (40, 40, 40, 40), (1, 17, 3, 40),
          (23, 1, 9, 4), (300, 257, 600, 514), (120, 90, 17, 13)]


@pytest.mark.parametrize("method", [0, 1, 2])
@pytest.mark.parametrize("coord", [0, 1, 2])
@pytest.mark.parametrize("impl", ["auto", "tiled"])
def test_adjoint_nchw_matches_oracle(rs, oracle, method, coord, impl):
    for k, (H, W, Ho, Wo) in enumerate(SHAPES):
        g = np.random.default_rng(100 + k).standard_normal((2, 3, Ho, Wo)).astype(np.float32)
        gt = torch.from_numpy(g).cuda()
        gi = rs.resize_backward(gt, (H, W), MN[method], layout="nchw", coord=CN[coord], impl=impl)
        torch.cuda.synchronize()
        ref = oracle.adjoint_nchw(g.astype(np.float64), H, W, method, coord)
        err = np.abs(gi.cpu().numpy().astype(np.float64) - ref).max()
        tol = _tol(oracle, H, W, Ho, Wo, method, coord, np.abs(g).max())
        assert err <= tol, f"{MN[method]} {CN[coord]} {H}x{W}<-{Ho}x{Wo}: {err} > {tol}"
    assert rs.debug_fault() == 0


@pytest.mark.parametrize("C", [1, 3, 4])
@pytest.mark.parametrize("impl", ["auto", "tiled"])
def test_adjoint_hwc_matches_oracle(rs, oracle, C, impl):
    for method in (1, 2):
        H, W, Ho, Wo = 45, 61, 97, 130
        g = np.random.default_rng(7).standard_normal((Ho, Wo, C)).astype(np.float32)
        gi = rs.resize_backward(torch.from_numpy(g).cuda(), (H, W), MN[method], layout="hwc", impl=impl)
        torch.cuda.synchronize()
        ref = oracle.adjoint(g.astype(np.float64), H, W, method)
        tol = _tol(oracle, H, W, Ho, Wo, method, 0, np.abs(g).max())
        assert np.abs(gi.cpu().numpy() - ref).max() <= tol


def test_deterministic(rs):
    g = torch.randn(4, 3, 300, 400, device="cuda")
    a = rs.resize_backward(g, (150, 200), "bicubic")
    b = rs.resize_backward(g, (150, 200), "bicubic")
    c = rs.resize_backward(g, (150, 200), "bicubic")
    assert torch.equal(a, b) and torch.equal(b, c)


@pytest.mark.parametrize("method", [1, 2])
def test_autograd_function(rs, method):
    x = torch.randn(2, 3, 40, 50, device="cuda", requires_grad=True)
    y = rs.ResizeFn.apply(x, (80, 100), MN[method], "half_pixel", -0.5)
    g = torch.randn_like(y)
    y.backward(g)
    ref = rs.resize_backward(g, (40, 50), MN[method], coord="half_pixel")
    assert torch.equal(x.grad, ref)
    # forward through the Function equals resize()
    assert torch.equal(y.detach(), rs.resize(x.detach(), (80, 100), MN[method], layout="nchw", coord="half_pixel"))


@pytest.mark.parametrize("method", [1, 2])
@pytest.mark.parametrize("coord", [0, 1, 2])
@pytest.mark.parametrize("scale", [2.0, 0.5])
def test_against_central_differences(rs, oracle, method, coord, scale):
    """dL/dx of L = <resize(x), g> by FP64 central differences (eps = 1e-6)
    of the oracle forward on a 64x64 crop, at sampled input pixels."""
    H = W = 64
    Ho = Wo = int(64 * scale)
    r = np.random.default_rng(21)
    x = r.standard_normal((H, W))
    g = r.standard_normal((Ho, Wo)).astype(np.float32)
    gi = rs.resize_backward(torch.from_numpy(g).cuda(), (H, W), MN[method], coord=CN[coord])
    gi = gi.cpu().numpy()
    g64 = g.astype(np.float64)
    for (i, j) in [(0, 0), (63, 63), (0, 31), (17, 5), (40, 62), (33, 33)]:
        xp, xm = x.copy(), x.copy()
        xp[i, j] += 1e-6
        xm[i, j] -= 1e-6
        fd = (np.sum(oracle.resize(xp, Ho, Wo, method, coord)[:, :, 0] * g64) -
              np.sum(oracle.resize(xm, Ho, Wo, method, coord)[:, :, 0] * g64)) / 2e-6
        assert abs(gi[i, j] - fd) < 1e-4 * max(1.0, abs(fd))


@pytest.mark.parametrize("method", [1, 2])
@pytest.mark.parametrize("scale", [2.0, 0.5])
def test_full_size_planes(rs, oracle, method, scale):
    """Full size 32x3x512x512 backward; two planes checked against the oracle."""
    H = W = 512
    Ho = Wo = int(512 * scale)
    g = torch.randn(32, 3, Ho, Wo, device="cuda", generator=torch.Generator("cuda").manual_seed(5))
    gi = rs.resize_backward(g, (H, W), MN[method])
    torch.cuda.synchronize()
    for (n, c) in ((0, 0), (31, 2)):
        gp = g[n, c].cpu().numpy().astype(np.float64)
        ref = oracle.adjoint(gp, H, W, method)[:, :, 0]
        tol = _tol(oracle, H, W, Ho, Wo, method, 0, np.abs(gp).max())
        assert np.abs(gi[n, c].cpu().numpy() - ref).max() <= tol
    assert rs.debug_fault() == 0


def test_workspace_errors(rs):
    import ctypes
    from paper_1001_1718_gb300 import _binding as B
    g = torch.randn(1, 1, 20, 20, device="cuda")
    x = torch.empty(1, 1, 10, 10, device="cuda")
    Lo, Li = rs._layout(g, "nchw"), rs._layout(x, "nchw")
    o = B.options()
    st = torch.cuda.current_stream().cuda_stream
    s = B.lib().rs_resize_backward(g.data_ptr(), ctypes.byref(Lo), x.data_ptr(), ctypes.byref(Li), B.RS_F32, 1,
                                   ctypes.byref(o), None, 0, st)
    assert s == B.RS_ERR_WORKSPACE
    s = B.lib().rs_resize_backward(g.data_ptr(), ctypes.byref(Lo), x.data_ptr(), ctypes.byref(Li), B.RS_U8, 1,
                                   ctypes.byref(o), None, 0, st)
    assert s == B.RS_ERR_UNSUPPORTED


def test_plane_groups_and_large_upscale(rs, oracle):
    """More planes than one intermediate group holds, and a x6 upscale
    (wide transposed rows)."""
    # 48 planes whose x-adjoint intermediates (2048 x 768 FP32, 6.3 MB each)
    # exceed one 256 MB group
    g = torch.randn(16, 3, 2048, 1536, device="cuda")
    gi = rs.resize_backward(g, (1024, 768), "bicubic")
    torch.cuda.synchronize()
    for (n, c) in ((0, 0), (15, 2), (13, 1)):
        ref = oracle.adjoint(g[n, c].cpu().numpy().astype(np.float64), 1024, 768, 2)[:, :, 0]
        tol = _tol(oracle, 1024, 768, 2048, 1536, 2, 0, float(g[n, c].abs().max()))
        assert np.abs(gi[n, c].cpu().numpy() - ref).max() <= tol
    del g, gi
    g6 = torch.randn(1, 1, 120, 180, device="cuda")
    gi6 = rs.resize_backward(g6, (20, 30), "bicubic", coord="half_pixel")
    ref = oracle.adjoint(g6[0, 0].cpu().numpy().astype(np.float64), 20, 30, 2, 1)[:, :, 0]
    assert np.abs(gi6[0, 0].cpu().numpy() - ref).max() <= _tol(oracle, 20, 30, 120, 180, 2, 1, float(g6.abs().max()))


# scales up to 2 (at most 8 transposed bicubic taps per axis), dY rows of
# whole 16-byte units
WIN_SHAPES = [(37, 54, 74, 108), (64, 48, 32, 24), (31, 29, 52, 56), (40, 40, 40, 40), (300, 258, 600, 516),
              (120, 90, 20, 12), (1, 17, 3, 32), (200, 150, 400, 300)]
# align-corners steps by (n - 1) / (m - 1): x2 upscales give bicubic 9
# transposed taps, so its shapes stay just below x2 (at most 8)
WIN_SHAPES_ALIGN = [(37, 54, 70, 100), (64, 48, 32, 24), (31, 29, 52, 56), (40, 40, 40, 40), (300, 258, 560, 480),
                    (120, 90, 20, 12), (1, 17, 3, 32), (200, 150, 370, 280)]


@pytest.mark.parametrize("method", [0, 1, 2])
@pytest.mark.parametrize("coord", [0, 1, 2])
def test_window_adjoint(rs, oracle, method, coord):
    """The fused register-window adjoint (dY rows of whole 16-byte units, at
    most 8 transposed taps per axis) against the oracle's adjoint, and equal
    to the two-pass kernels, whose sums it runs in the same order."""
    for k, (H, W, Ho, Wo) in enumerate(WIN_SHAPES_ALIGN if coord == 2 else WIN_SHAPES):
        g = np.random.default_rng(300 + k).standard_normal((2, 3, Ho, Wo)).astype(np.float32)
        gt = torch.from_numpy(g).cuda()
        gi = rs.resize_backward(gt, (H, W), MN[method], layout="nchw", coord=CN[coord], impl="window")
        two = rs.resize_backward(gt, (H, W), MN[method], layout="nchw", coord=CN[coord], impl="stream")
        torch.cuda.synchronize()
        ref = oracle.adjoint_nchw(g.astype(np.float64), H, W, method, coord)
        err = np.abs(gi.cpu().numpy().astype(np.float64) - ref).max()
        tol = _tol(oracle, H, W, Ho, Wo, method, coord, np.abs(g).max())
        assert err <= tol, f"{MN[method]} {CN[coord]} {H}x{W}<-{Ho}x{Wo}: {err} > {tol}"
        assert torch.equal(gi, two), f"window vs two-pass {MN[method]} {CN[coord]} {H}x{W}<-{Ho}x{Wo}"
    # interleaved channels (align-corners: just below x2, as above)
    H, W = (47, 68) if coord == 2 else (45, 66)
    for C in (1, 3, 4):
        g = np.random.default_rng(9).standard_normal((90, 132, C)).astype(np.float32)
        gt = torch.from_numpy(g).cuda()
        gi = rs.resize_backward(gt, (H, W), MN[method], layout="hwc", coord=CN[coord], impl="window")
        two = rs.resize_backward(gt, (H, W), MN[method], layout="hwc", coord=CN[coord], impl="stream")
        torch.cuda.synchronize()
        assert torch.equal(gi, two)
        ref = oracle.adjoint(g.astype(np.float64), H, W, method, coord)
        assert np.abs(gi.cpu().numpy() - ref).max() <= _tol(oracle, H, W, 90, 132, method, coord, np.abs(g).max())
    # not applicable: more than 8 transposed taps along x (bicubic x3), odd dY rows
    with pytest.raises(rs.ResampleError):
        rs.resize_backward(torch.randn(1, 1, 60, 60, device="cuda"), (20, 20), "bicubic", impl="window")
    with pytest.raises(rs.ResampleError):
        rs.resize_backward(torch.randn(1, 1, 40, 41, device="cuda"), (20, 20), "bilinear", impl="window")
    assert rs.debug_fault() == 0


# ---------------------------------------------------------------------------
# The adjoint of the antialiased forward (RS_FLAG_ANTIALIAS)

def _tol_aa(oracle, H, W, Ho, Wo, method, gmax):
    Ay = oracle.aa_axis_matrix(H, Ho, method)
    Ax = oracle.aa_axis_matrix(W, Wo, method)
    return 1e-5 * max(1.0, gmax) * np.abs(Ay.T).sum(1).max() * np.abs(Ax.T).sum(1).max()


AA_SHAPES = [(64, 80, 32, 40), (97, 133, 41, 29), (50, 60, 75, 90), (33, 47, 8, 12), (300, 257, 120, 100),
             (1, 40, 1, 13), (29, 1, 7, 1)]


@pytest.mark.parametrize("method", [1, 2])
@pytest.mark.parametrize("impl", ["auto", "stream", "tiled"])
def test_antialias_adjoint_matches_oracle(rs, oracle, method, impl):
    r = np.random.default_rng(61 + method)
    for (H, W, Ho, Wo) in AA_SHAPES:
        g = r.standard_normal((2, 3, Ho, Wo)).astype(np.float32)
        gi = rs.resize_backward(torch.from_numpy(g).cuda(), (H, W), MN[method], antialias=True, impl=impl)
        torch.cuda.synchronize()
        ref = oracle.adjoint_aa_nchw(g.astype(np.float64), H, W, method)
        err = np.abs(gi.cpu().numpy() - ref).max()
        tol = _tol_aa(oracle, H, W, Ho, Wo, method, np.abs(g).max())
        assert err <= tol, f"{MN[method]} {impl} {H}x{W}<-{Ho}x{Wo}: {err} > {tol}"
    assert rs.debug_fault() == 0


@pytest.mark.parametrize("method", [1, 2])
def test_antialias_autograd_and_central_differences(rs, oracle, method):
    """ResizeFn(antialias=True): the forward equals resize(antialias=True),
    the gradient equals resize_backward(antialias=True) and FP64 central
    differences (eps = 1e-6) of the oracle's antialiased forward."""
    x = torch.randn(2, 3, 64, 64, device="cuda", requires_grad=True)
    y = rs.ResizeFn.apply(x, (26, 32), MN[method], "asymmetric", -0.5, True)
    assert torch.equal(y.detach(), rs.resize(x.detach(), (26, 32), MN[method], layout="nchw", antialias=True))
    g = torch.randn_like(y)
    y.backward(g)
    assert torch.equal(x.grad, rs.resize_backward(g, (64, 64), MN[method], antialias=True))
    r = np.random.default_rng(22)
    x0 = r.standard_normal((64, 64))
    gg = r.standard_normal((26, 32)).astype(np.float32)
    gi = rs.resize_backward(torch.from_numpy(gg).cuda(), (64, 64), MN[method], layout="hwc",
                            antialias=True).cpu().numpy()
    g64 = gg.astype(np.float64)
    for (i, j) in [(0, 0), (63, 63), (0, 31), (17, 5), (40, 62), (33, 33)]:
        xp, xm = x0.copy(), x0.copy()
        xp[i, j] += 1e-6
        xm[i, j] -= 1e-6
        fd = (np.sum(oracle.resize_aa(xp, 26, 32, method)[:, :, 0] * g64) -
              np.sum(oracle.resize_aa(xm, 26, 32, method)[:, :, 0] * g64)) / 2e-6
        assert abs(gi[i, j] - fd) < 1e-4 * max(1.0, abs(fd))


@pytest.mark.parametrize("method", [1, 2])
def test_antialias_adjoint_full_size(rs, oracle, method):
    """FP32 32x3x512x512 at x0.5: every element of the antialiased adjoint."""
    from paper_1001_1718_gb300 import workloads
    g = workloads.normal_nchw(77, 32, 3, 256, 256).astype(np.float32)
    gi = rs.resize_backward(torch.from_numpy(g).cuda(), (512, 512), MN[method], antialias=True)
    torch.cuda.synchronize()
    ref = oracle.adjoint_aa_nchw(g.astype(np.float64), 512, 512, method)
    tol = _tol_aa(oracle, 512, 512, 256, 256, method, np.abs(g).max())
    assert np.abs(gi.cpu().numpy() - ref).max() <= tol
    assert rs.debug_fault() == 0
