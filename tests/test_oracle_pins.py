"""Pins of the FP64 oracle against facts that do not come from the oracle.

Each test checks one function of oracle/resample_oracle.c against a closed
form, an invariant of the definition, the paper's worked example, or an
independent library routine (SciPy, PyTorch, NumPy). The set is chosen so a
plausible slip in the oracle -- a dropped tap, a wrong Keys coefficient, an
off-by-one in the half-pixel map, swapped x / y axes, a missing clamp, a
wrong adjoint index, a wrong rounding rule -- fails at least one of them.
"""
from fractions import Fraction
from pathlib import Path

import numpy as np
import pytest

GOLDEN = Path(__file__).resolve().parent / "golden"
NN, BL, BC = 0, 1, 2
ASYM, HALF, ALIGN = 0, 1, 2
METHODS = (NN, BL, BC)
COORDS = (ASYM, HALF, ALIGN)


def _rng(seed):
    return np.random.default_rng(seed)


def _coord(j, n, m, coord):
    """Source coordinate of output index j (Eq. 1; half-pixel and
    align-corners variants)."""
    j = np.asarray(j, np.float64)
    if coord == ASYM:
        return j * n / m
    if coord == ALIGN:
        return j * (n - 1) / (m - 1) if m > 1 else 0.0 * j
    return (j + 0.5) * n / m - 0.5


# --------------------------------------------------------------------------
# Eq. 6 worked example (Sec. III.A, Fig. 2)

def test_tile_map_worked_example(oracle):
    for line in (GOLDEN / "tile_map_eq6.txt").read_text().splitlines():
        if line.startswith("#") or not line.strip():
            continue
        px, py, bw, bh, bx, by, tx, ty = map(int, line.split())
        assert oracle.tile_of_pixel(px, py, bw, bh) == (bx, by, tx, ty)
        # Eq. 6 forward direction reproduces the pixel.
        assert bx * bw + tx == px and by * bh + ty == py


# --------------------------------------------------------------------------
# Definition-level invariants

@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("coord", COORDS)
def test_identity_is_exact(oracle, method, coord):
    x = _rng(1).standard_normal((13, 17, 3))
    y = oracle.resize(x, 13, 17, method, coord)
    assert np.array_equal(x, y)


@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("coord", COORDS)
@pytest.mark.parametrize("shape", [(5, 7, 23, 11), (19, 12, 8, 30), (1, 9, 4, 2), (6, 1, 6, 5)])
def test_constant_preserved(oracle, method, coord, shape):
    H, W, Ho, Wo = shape
    x = np.full((H, W, 2), 37.25)
    y = oracle.resize(x, Ho, Wo, method, coord)
    tol = 0.0 if method == NN else 1e-13   # (1-t) a + t a rounds in FP64
    assert np.abs(y - 37.25).max() <= tol


@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("coord", COORDS)
@pytest.mark.parametrize("nm", [(7, 16), (16, 7), (10, 17), (31, 9), (5, 5), (1, 6)])
def test_weights_partition_of_unity(oracle, method, coord, nm):
    n, m = nm
    idx, w = oracle.axis_taps(n, m, method, coord)
    assert np.abs(w.sum(axis=1) - 1.0).max() < 1e-14
    k = {NN: 1, BL: 2, BC: 4}[method]
    assert (idx[:, :k] >= 0).all() and (idx[:, :k] <= n - 1).all()


@pytest.mark.parametrize("coord", COORDS)
@pytest.mark.parametrize("a", [-0.5, -0.75, -1.0])
def test_ramps_reproduced_in_interior(oracle, coord, a):
    """Bilinear reproduces a + b*y + c*x wherever no tap is clamped, and so
    does Keys' cubic for a = -1/2 (the only a of first-order consistency:
    other a reproduce constants only). The value is the ramp at the mapped
    coordinate of Eq. 1."""
    H, W, Ho, Wo = 21, 26, 47, 33
    yy, xx = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    img = 3.0 - 0.75 * yy + 1.25 * xx
    yp = _coord(np.arange(Ho), H, Ho, coord)
    xp = _coord(np.arange(Wo), W, Wo, coord)
    ref = 3.0 - 0.75 * yp[:, None] + 1.25 * xp[None, :]
    for method, lo, hi in ((BL, 0, 2), (BC, 1, 3)):
        y = oracle.resize(img, Ho, Wo, method, coord, a)[:, :, 0]
        ok_y = (np.floor(yp) >= lo) & (np.floor(yp) + hi <= H)
        ok_x = (np.floor(xp) >= lo) & (np.floor(xp) + hi <= W)
        sel = ok_y[:, None] & ok_x[None, :]
        assert sel.sum() > 100
        err = np.abs(y - ref)[sel].max()
        if method == BL or a == -0.5:
            assert err < 1e-12
        else:
            assert err > 1e-3


def test_quadratics(oracle):
    """Keys with a = -1/2 reproduces quadratics (it is third-order accurate);
    linear interpolation of x^2 overshoots by exactly t (1 - t)."""
    n, m = 24, 55
    x = np.arange(n, dtype=np.float64)
    f = (x ** 2 - 3.0 * x + 2.0)[None, :].repeat(2, 0)
    xp = _coord(np.arange(m), n, m, ASYM)
    t = xp - np.floor(xp)
    bc = oracle.resize(f, 2, m, BC, ASYM, -0.5)[0, :, 0]
    inter = (np.floor(xp) >= 1) & (np.floor(xp) + 2 <= n - 1)
    assert np.abs(bc - (xp ** 2 - 3 * xp + 2))[inter].max() < 1e-11
    bl = oracle.resize(f, 2, m, BL, ASYM)[0, :, 0]
    inter = np.floor(xp) + 1 <= n - 1
    assert np.abs(bl - (xp ** 2 - 3 * xp + 2 + t * (1 - t)))[inter].max() < 1e-11
    # a = -3/4 does not reproduce quadratics: the oracle must honour `a`.
    bc75 = oracle.resize(f, 2, m, BC, ASYM, -0.75)[0, :, 0]
    assert np.abs(bc75 - (xp ** 2 - 3 * xp + 2))[inter].max() > 1e-3


@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("k", [2, 3, 4])
def test_interpolates_samples_at_integer_scale(oracle, method, k):
    """Asymmetric map at integer scale k: output (k i, k j) lands on source
    sample (i, j) exactly, so every method returns it unchanged."""
    x = _rng(k).standard_normal((9, 11, 3))
    y = oracle.resize(x, 9 * k, 11 * k, method, ASYM)
    assert np.array_equal(y[::k, ::k], x)


def test_catmull_rom_midpoint(oracle):
    rows = [l.split() for l in (GOLDEN / "catmull_rom_midpoint.txt").read_text().splitlines()
            if l.strip() and not l.startswith("#")]
    table = {Fraction(r[0]): [float(Fraction(v)) for v in r[1:]] for r in rows}
    # Asymmetric x2: even outputs have t = 0, odd outputs t = 1/2.
    idx, w = oracle.axis_taps(12, 24, BC, ASYM, -0.5)
    for j in range(2, 20):
        t = Fraction(j * 12, 24) - (j * 12) // 24
        assert list(w[j]) == table[t]
        i0 = (j * 12) // 24
        assert list(idx[j]) == [i0 - 1, i0, i0 + 1, i0 + 2]
    # A unit impulse upsampled x2 shows the weights directly.
    d = np.zeros((1, 12))
    d[0, 6] = 16.0
    y = oracle.resize(d, 1, 24, BC, ASYM)[0, :, 0]
    assert list(y[9:17]) == [-1.0, 0.0, 9.0, 16.0, 9.0, 0.0, -1.0, 0.0]


def test_bilinear_is_convex_combination(oracle):
    x = _rng(3).uniform(-5, 7, (15, 14, 2))
    for coord in COORDS:
        y = oracle.resize(x, 31, 9, BL, coord)
        assert y.min() >= x.min() - 1e-12 and y.max() <= x.max() + 1e-12


# --------------------------------------------------------------------------
# Independent routines

@pytest.mark.parametrize("coord", COORDS)
@pytest.mark.parametrize("shape", [(11, 19, 29, 23), (16, 9, 8, 27), (30, 30, 13, 71), (3, 2, 7, 1)])
def test_bilinear_matches_scipy_linear_interpolation(oracle, coord, shape):
    """scipy.ndimage.map_coordinates(order=1, mode='nearest') is linear
    interpolation with edge replication at arbitrary coordinates."""
    ndi = pytest.importorskip("scipy.ndimage")
    H, W, Ho, Wo = shape
    x = _rng(4).standard_normal((H, W))
    yp = _coord(np.arange(Ho), H, Ho, coord)
    xp = _coord(np.arange(Wo), W, Wo, coord)
    Y, X = np.meshgrid(yp, xp, indexing="ij")
    ref = ndi.map_coordinates(x, [Y, X], order=1, mode="nearest", prefilter=False)
    y = oracle.resize(x, Ho, Wo, BL, coord)[:, :, 0]
    assert np.abs(y - ref).max() < 1e-12


def test_paper_eq5_form_matches(oracle):
    """Eqs. 1-5 in the paper's four-neighbour form (second (1-offsetY) read
    as (1-offsetX)) agree with the separable bilinear definition."""
    x = _rng(5).standard_normal((17, 23))
    for Ho, Wo in ((34, 46), (51, 29), (8, 11), (17, 23)):
        a = oracle.bilinear_eq5(x, Ho, Wo)
        b = oracle.resize(x, Ho, Wo, BL, ASYM)[:, :, 0]
        assert np.abs(a - b).max() < 1e-13


@pytest.mark.parametrize("nm", [(10, 20), (20, 10), (16, 64), (64, 16), (12, 48)])
def test_nearest_matches_torch_nearest(oracle, nm):
    """torch 'nearest' picks floor(j * n / m), Eq. 2's x1. Its float scale
    is exact when n / m is a power of two, as on these sizes, on both axes
    (different ratios on x and y)."""
    torch = pytest.importorskip("torch")
    n, m = nm
    x = _rng(6).standard_normal((n, 2 * n))
    t = torch.nn.functional.interpolate(torch.from_numpy(x)[None, None], size=(m, m),
                                        mode="nearest")[0, 0].numpy()
    y = oracle.resize(x, m, m, NN, ASYM)[:, :, 0]
    assert np.array_equal(y, t)


def test_nearest_brute_force_exact_integer(oracle):
    """The exact integer index floor(j n / m) against a float formula with an
    exactness guard, on every size pair up to 40."""
    for n in range(1, 41):
        for m in range(1, 41):
            idx, _ = oracle.axis_taps(n, m, NN, ASYM)
            for j in range(m):
                f = j * n / m
                i = int(np.floor(f))
                if abs(f - round(f)) > 1e-9 or abs(f - round(f)) == 0:
                    assert idx[j, 0] == i
            idx, _ = oracle.axis_taps(n, m, NN, HALF)
            for j in range(m):
                f = (j + 0.5) * n / m
                if abs(f - round(f)) > 1e-9:
                    assert idx[j, 0] == min(int(np.floor(f)), n - 1)


@pytest.mark.parametrize("shape", [(7, 9, 13, 20), (7, 9, 4, 5), (16, 12, 8, 6), (5, 40, 11, 17)])
def test_half_pixel_matches_torch(oracle, shape):
    """torch bilinear / bicubic with align_corners=False use the half-pixel
    map, edge clamping and (for bicubic) Keys' kernel with a = -3/4."""
    torch = pytest.importorskip("torch")
    F = torch.nn.functional
    H, W, Ho, Wo = shape
    x = _rng(7).standard_normal((2, 3, H, W))
    tx = torch.from_numpy(x)
    tb = F.interpolate(tx, size=(Ho, Wo), mode="bilinear", align_corners=False).numpy()
    tc = F.interpolate(tx, size=(Ho, Wo), mode="bicubic", align_corners=False).numpy()
    assert np.abs(oracle.resize_nchw(x, Ho, Wo, BL, HALF) - tb).max() < 1e-12
    assert np.abs(oracle.resize_nchw(x, Ho, Wo, BC, HALF, -0.75) - tc).max() < 1e-12


@pytest.mark.parametrize("shape", [(7, 9, 13, 20), (9, 7, 4, 5), (16, 12, 8, 6), (5, 40, 11, 17), (6, 5, 1, 9)])
def test_align_corners_matches_torch(oracle, shape):
    """torch bilinear / bicubic with align_corners=True use the map
    x = j (n - 1) / (m - 1) (x = 0 for one output), edge clamping and (for
    bicubic) Keys' kernel with a = -3/4."""
    torch = pytest.importorskip("torch")
    F = torch.nn.functional
    H, W, Ho, Wo = shape
    x = _rng(17).standard_normal((2, 3, H, W))
    tx = torch.from_numpy(x)
    tb = F.interpolate(tx, size=(Ho, Wo), mode="bilinear", align_corners=True).numpy()
    tc = F.interpolate(tx, size=(Ho, Wo), mode="bicubic", align_corners=True).numpy()
    assert np.abs(oracle.resize_nchw(x, Ho, Wo, BL, ALIGN) - tb).max() < 1e-12
    assert np.abs(oracle.resize_nchw(x, Ho, Wo, BC, ALIGN, -0.75) - tc).max() < 1e-12


@pytest.mark.parametrize("method", METHODS)
def test_align_corners_keeps_corners(oracle, method):
    """Under align-corners the four corner samples land exactly on the four
    corner outputs, at any scale, for every method."""
    x = _rng(18).standard_normal((11, 14, 2))
    for Ho, Wo in ((23, 5), (4, 31), (11, 14), (2, 2)):
        y = oracle.resize(x, Ho, Wo, method, ALIGN)
        for (a, b), (c, d) in (((0, 0), (0, 0)), ((0, -1), (0, -1)), ((-1, 0), (-1, 0)), ((-1, -1), (-1, -1))):
            assert np.array_equal(y[a, b], x[c, d])


def test_align_corners_nearest_rounds(oracle):
    """Align-corners nearest takes the sample nearest to j (n - 1) / (m - 1)
    (ties upward), by exact rational arithmetic."""
    for n, m in ((7, 16), (16, 7), (10, 17), (31, 9), (5, 5), (9, 1), (2, 40)):
        idx, _ = oracle.axis_taps(n, m, NN, ALIGN)
        for j in range(m):
            x = Fraction(j * (n - 1), m - 1) if m > 1 else Fraction(0)
            assert idx[j, 0] == int(np.floor(x + Fraction(1, 2)))


@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("coord", COORDS)
def test_matrix_form(oracle, method, coord):
    """Direct 2-D loops equal Ay X Ax^T with the one-axis matrices, per
    channel, on a non-square image with different x and y ratios."""
    H, W, Ho, Wo = 9, 14, 22, 5
    x = _rng(8).standard_normal((H, W, 2))
    Ay = oracle.axis_matrix(H, Ho, method, coord)
    Ax = oracle.axis_matrix(W, Wo, method, coord)
    y = oracle.resize(x, Ho, Wo, method, coord)
    for c in range(2):
        assert np.abs(y[:, :, c] - Ay @ x[:, :, c] @ Ax.T).max() < 1e-13


def test_points_match_full(oracle):
    x = _rng(9).standard_normal((20, 30, 3))
    for method in METHODS:
        full = oracle.resize(x, 37, 55, method, HALF)
        ys = np.array([0, 36, 5, 20, 36])
        xs = np.array([0, 54, 17, 0, 1])
        pts = oracle.resize_points(x, 37, 55, method, HALF, -0.5, ys, xs)
        assert np.array_equal(pts, full[ys, xs])


def test_nchw_view_is_per_plane(oracle):
    x = _rng(10).standard_normal((2, 3, 8, 6))
    y = oracle.resize_nchw(x, 5, 13, BC, HALF)
    for n in range(2):
        for c in range(3):
            assert np.array_equal(y[n, c], oracle.resize(x[n, c], 5, 13, BC, HALF)[:, :, 0])


# --------------------------------------------------------------------------
# Adjoint

@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("coord", COORDS)
@pytest.mark.parametrize("shape", [(9, 12, 20, 25), (16, 16, 8, 8), (10, 7, 10, 7), (5, 13, 11, 4)])
def test_adjoint_dot_product(oracle, method, coord, shape):
    H, W, Ho, Wo = shape
    r = _rng(11)
    x = r.standard_normal((H, W, 2))
    g = r.standard_normal((Ho, Wo, 2))
    lhs = np.sum(oracle.resize(x, Ho, Wo, method, coord) * g)
    rhs = np.sum(x * oracle.adjoint(g, H, W, method, coord))
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))


@pytest.mark.parametrize("method", METHODS)
def test_adjoint_is_matrix_transpose(oracle, method):
    H, W, Ho, Wo = 8, 11, 17, 6
    g = _rng(12).standard_normal((Ho, Wo))
    Ay = oracle.axis_matrix(H, Ho, method, HALF)
    Ax = oracle.axis_matrix(W, Wo, method, HALF)
    ref = Ay.T @ g @ Ax
    assert np.abs(oracle.adjoint(g, H, W, method, HALF)[:, :, 0] - ref).max() < 1e-13


@pytest.mark.parametrize("method", (BL, BC))
@pytest.mark.parametrize("coord", COORDS)
@pytest.mark.parametrize("scale", (2.0, 0.5))
def test_adjoint_matches_central_differences(oracle, method, coord, scale):
    """The gradient of <resize(x), g> with respect to x, by FP64 central
    differences (eps = 1e-6) of the forward, equals the adjoint applied to g.
    64x64 crop; a random subset of input pixels plus all four corners."""
    H = W = 64
    Ho = Wo = int(H * scale)
    r = _rng(13)
    x = r.standard_normal((H, W))
    g = r.standard_normal((Ho, Wo))
    adj = oracle.adjoint(g, H, W, method, coord)[:, :, 0]
    pts = [(0, 0), (0, W - 1), (H - 1, 0), (H - 1, W - 1)] + \
          [tuple(p) for p in r.integers(0, H, (28, 2))]
    eps = 1e-6
    for (i, j) in pts:
        xp = x.copy()
        xm = x.copy()
        xp[i, j] += eps
        xm[i, j] -= eps
        fp = np.sum(oracle.resize(xp, Ho, Wo, method, coord)[:, :, 0] * g)
        fm = np.sum(oracle.resize(xm, Ho, Wo, method, coord)[:, :, 0] * g)
        fd = (fp - fm) / (2 * eps)
        assert abs(fd - adj[i, j]) < 1e-6 * max(1.0, abs(adj[i, j]))


# --------------------------------------------------------------------------
# Storage rounding

def test_quantize_u8_against_numpy(oracle):
    r = _rng(14)
    v = np.concatenate([r.uniform(-20, 280, 20000), np.arange(-3, 260) + 0.5,
                        np.array([-0.0, 0.0, 254.5, 255.5, 1e9, -1e9, 0.49999999999, 2.5000000001])])
    ref = np.clip(np.rint(v), 0, 255).astype(np.uint8)   # rint: half to even
    assert np.array_equal(oracle.quantize_u8(v), ref)


def test_f16_rounding_against_numpy(oracle):
    r = _rng(15)
    v = np.concatenate([
        r.standard_normal(20000) * 10.0 ** r.integers(-9, 6, 20000),
        np.array([65504.0, 65519.99, 65520.0, 70000.0, -65520.0, 2.0 ** -24, 2.0 ** -25,
                  2.0 ** -25 * 1.0000001, 3 * 2.0 ** -26, 0.0, -0.0, 1.0 + 2.0 ** -11,
                  1.0 + 3 * 2.0 ** -11, np.inf, -np.inf]),
    ])
    bits = oracle.to_f16_bits(v)
    assert np.array_equal(bits, v.astype(np.float16).view(np.uint16))


def _bf16_value(bits):
    b = np.uint32(bits) << np.uint32(16)
    return float(np.array([b], np.uint32).view(np.float32)[0])


def test_bf16_rounding_is_nearest_even(oracle):
    """Against torch's float32->bfloat16 conversion for doubles that are
    float32 values, and against the nearest-ties-to-even property in exact
    rational arithmetic for doubles that are not."""
    torch = pytest.importorskip("torch")
    r = _rng(16)
    f32 = (r.standard_normal(20000) * 10.0 ** r.integers(-30, 30, 20000)).astype(np.float32)
    f32 = np.concatenate([f32, np.array([1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 3.3895314e38], np.float32)])
    ref = torch.from_numpy(f32).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    assert np.array_equal(oracle.to_bf16_bits(f32.astype(np.float64)), ref)
    # Doubles between float32 values: the decision is beyond float32 precision.
    d = 1.0 + 2.0 ** -8 + np.array([2.0 ** -40, -2.0 ** -40, 2.0 ** -30])
    d = np.concatenate([d, r.uniform(-3, 3, 2000)])
    for v, bits in zip(d, oracle.to_bf16_bits(d)):
        fv = Fraction(float(v))
        err = abs(fv - Fraction(_bf16_value(bits)))
        for nb in (int(bits) - 1, int(bits) + 1):       # neighbouring bf16 codes
            e2 = abs(fv - Fraction(_bf16_value(nb & 0xFFFF)))
            assert err < e2 or (err == e2 and (int(bits) & 1) == 0)


# ---------------------------------------------------------------------------
# Antialiased resampling (extension; the reading is written in the oracle).

@pytest.mark.parametrize("method", [1, 2])
@pytest.mark.parametrize("shape", [(64, 80, 32, 40), (64, 80, 21, 33), (40, 30, 45, 17), (17, 23, 60, 70)])
def test_aa_matches_torch_antialias(oracle, method, shape):
    """torch's antialiased interpolate (PIL's filters, Keys a = -0.5 for
    bicubic) is an independent implementation of the same definition."""
    torch = pytest.importorskip("torch")
    H, W, Ho, Wo = shape
    x = np.random.default_rng(H * W).standard_normal((1, 2, H, W))
    ref = oracle.resize_aa_nchw(x, Ho, Wo, method, -0.5)
    t = torch.nn.functional.interpolate(torch.from_numpy(x), size=(Ho, Wo), mode={1: "bilinear", 2: "bicubic"}[method],
                                        antialias=True, align_corners=False).numpy()
    assert np.abs(ref - t).max() < 1e-12


@pytest.mark.parametrize("method", [1, 2])
@pytest.mark.parametrize("shape", [(64, 80, 32, 40), (50, 70, 19, 31), (20, 30, 45, 41)])
def test_aa_adjoint_matches_torch_autograd(oracle, method, shape):
    """The adjoint of the antialiased resampling against torch's own
    backward of its antialiased interpolate (FP64 autograd)."""
    torch = pytest.importorskip("torch")
    H, W, Ho, Wo = shape
    r = np.random.default_rng(H + 7 * W)
    x = torch.from_numpy(r.standard_normal((2, 3, H, W))).requires_grad_(True)
    gy = r.standard_normal((2, 3, Ho, Wo))
    y = torch.nn.functional.interpolate(x, size=(Ho, Wo), mode={1: "bilinear", 2: "bicubic"}[method],
                                        antialias=True, align_corners=False)
    (y * torch.from_numpy(gy)).sum().backward()
    ref = oracle.adjoint_aa_nchw(gy, H, W, method, -0.5)
    assert np.abs(ref - x.grad.numpy()).max() < 1e-12


def test_aa_adjoint_inner_product(oracle):
    """<A x, g> = <x, A^T g> for a non-square downscale (A and A^T from the
    forward and the adjoint separately)."""
    r = np.random.default_rng(5)
    x = r.standard_normal((1, 2, 41, 67))
    g = r.standard_normal((1, 2, 13, 29))
    for method in (1, 2):
        lhs = np.sum(oracle.resize_aa_nchw(x, 13, 29, method) * g)
        rhs = np.sum(x * oracle.adjoint_aa_nchw(g, 41, 67, method))
        assert abs(lhs - rhs) < 1e-10 * max(1.0, abs(lhs))


def test_aa_rows_sum_to_one_and_closed_form(oracle):
    for n, m in ((100, 50), (97, 31), (30, 90), (64, 63)):
        for method in (1, 2):
            A = oracle.aa_axis_matrix(n, m, method)
            assert np.abs(A.sum(1) - 1.0).max() < 1e-14
    # triangle at x0.5: an interior output averages 4 samples with 1/8, 3/8, 3/8, 1/8
    A = oracle.aa_axis_matrix(100, 50, 1)
    j = 20
    nz = np.nonzero(A[j])[0]
    assert list(nz) == [2 * j - 1, 2 * j, 2 * j + 1, 2 * j + 2]
    assert np.allclose(A[j, nz], [1 / 8, 3 / 8, 3 / 8, 1 / 8], atol=1e-15)


@pytest.mark.parametrize("method", [1, 2])
def test_aa_upscale_is_half_pixel_interpolation_inside(oracle, method):
    """Without a downscale the filter is not stretched: away from the
    borders (no taps cut) antialiased resampling is half-pixel
    interpolation."""
    x = np.random.default_rng(3).standard_normal((40, 50, 1))
    a = oracle.resize_aa(x, 100, 110, method)
    b = oracle.resize(x, 100, 110, method, 1)
    assert np.abs(a[10:-10, 10:-10] - b[10:-10, 10:-10]).max() < 1e-13


# ---------------------------------------------------------------------------
# The fused serving pre-process: resample, then (y - mean) / std per channel,
# laid out planar. Pinned against torch's FP64 interpolate (half-pixel map,
# Keys a = -3/4 for bicubic, its own implementation) followed by torch's own
# normalise and permute.

@pytest.mark.parametrize("method", [1, 2])
@pytest.mark.parametrize("shape", [(2, 13, 17, 3), (1, 9, 31, 4), (3, 20, 11, 1)])
def test_resize_normalize_matches_torch(oracle, method, shape):
    torch = pytest.importorskip("torch")
    F = torch.nn.functional
    r = np.random.default_rng(77)
    x = r.integers(0, 256, shape).astype(np.float64)
    N, H, W, C = shape
    mean = r.uniform(0, 255, C)
    std = r.uniform(20, 90, C)
    for Ho, Wo in ((2 * H + 1, W + 7), (max(1, H // 2), max(1, W // 3))):
        got = oracle.resize_normalize(x, Ho, Wo, method, mean, std, coord=1, a=-0.75)
        mode = "bilinear" if method == 1 else "bicubic"
        t = F.interpolate(torch.from_numpy(x).permute(0, 3, 1, 2), size=(Ho, Wo), mode=mode, align_corners=False)
        ref = ((t - torch.from_numpy(mean)[None, :, None, None]) / torch.from_numpy(std)[None, :, None, None]).numpy()
        assert got.shape == (N, C, Ho, Wo)
        assert np.abs(got - ref).max() < 1e-11, (method, shape, Ho, Wo)


def test_resize_normalize_single_image_and_identity(oracle):
    """An (H, W, C) image gives (C, Ho, Wo); at identity size with mean 0 and
    std 1 the output is the input, transposed to planar, exactly."""
    r = np.random.default_rng(78)
    x = r.integers(0, 256, (7, 9, 3)).astype(np.float64)
    y = oracle.resize_normalize(x, 7, 9, 2, [0, 0, 0], [1, 1, 1])
    assert y.shape == (3, 7, 9)
    assert np.array_equal(y, x.transpose(2, 0, 1))
    # a constant channel maps to (value - mean) / std exactly (partition of unity)
    c = np.full((5, 6, 2), 200.0)
    y = oracle.resize_normalize(c, 11, 13, 2, [100.0, 50.0], [50.0, 25.0])
    assert np.allclose(y[0], 2.0, atol=1e-13) and np.allclose(y[1], 6.0, atol=1e-13)
