"""GPU forward parity: the CUDA path (through the C ABI) against the FP64
oracle, element by element, on seeded inputs at sizes that span several
tiles with ragged tails, plus degenerate shapes and guard-band checks."""
import numpy as np
import pytest
import torch

from _parity import check, to_storage, as_f64, aa_taps as _aa_taps

pytestmark = pytest.mark.gpu

NN, BL, BC = 0, 1, 2
MNAME = {NN: "nearest", BL: "bilinear", BC: "bicubic"}
CNAME = {0: "asymmetric", 1: "half_pixel", 2: "align_corners"}


@pytest.fixture(scope="module")
def rs():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1001_1718_gb300 as rs
    return rs


def _src(seed, shape, dtype):
    r = np.random.default_rng(seed)
    if dtype == "u8":
        x = r.integers(0, 256, size=shape).astype(np.float64)
    else:
        x = r.standard_normal(shape) * 3.0
    t = to_storage(x, dtype)
    return t, as_f64(t)     # the oracle sees exactly the stored values


SIZES = [
    (37, 53, 91, 117),       # non-integer upscale, ragged
    (300, 200, 600, 400),    # x2, several tiles
    (257, 311, 128, 155),    # downscale
    (64, 64, 64, 64),        # identity
    (1, 50, 3, 77),          # one source row
    (40, 1, 80, 5),          # one source column
    (5, 7, 1, 1),            # single output pixel
    (129, 517, 333, 1290),   # wide, many tiles
]


@pytest.mark.parametrize("method", [NN, BL, BC])
@pytest.mark.parametrize("coord", [0, 1, 2])
@pytest.mark.parametrize("dtype", ["u8", "f16", "bf16", "f32"])
@pytest.mark.parametrize("C", [1, 3, 4])
def test_hwc_all_sizes(rs, oracle, method, coord, dtype, C):
    for k, (H, W, Ho, Wo) in enumerate(SIZES):
        t, x64 = _src(1000 + k, (H, W, C), dtype)
        y = rs.resize(t.cuda(), (Ho, Wo), MNAME[method], coord=CNAME[coord])
        torch.cuda.synchronize()
        ref = oracle.resize(x64, Ho, Wo, method, coord)
        check(y, ref, dtype, method, np.abs(x64).max(), f"{MNAME[method]} {CNAME[coord]} {dtype} C={C} {H}x{W}->{Ho}x{Wo}")
    assert rs.debug_fault() == 0


@pytest.mark.parametrize("method", [NN, BL, BC])
@pytest.mark.parametrize("impl", ["plain", "tiled"])
def test_plain_and_tiled_nchw(rs, oracle, method, impl):
    N, C, H, W = 2, 3, 75, 131
    for (Ho, Wo), coord in (((150, 262), 0), ((37, 65), 1), ((201, 97), 0)):
        t, x64 = _src(7, (N, C, H, W), "f32")
        y = rs.resize(t.cuda(), (Ho, Wo), MNAME[method], layout="nchw", coord=CNAME[coord], impl=impl)
        torch.cuda.synchronize()
        ref = oracle.resize_nchw(x64, Ho, Wo, method, coord)
        check(y, ref, "f32", method, np.abs(x64).max(), f"nchw {impl} {MNAME[method]}")


@pytest.mark.parametrize("tile", [(128, 4, 128), (256, 8, 256), (512, 32, 256), (1024, 64, 256), (128, 1, 128)])
def test_explicit_tile_configs(rs, oracle, tile):
    tw, th, nt = tile
    t, x64 = _src(11, (203, 301, 3), "u8")
    for method in (BL, BC):
        for (Ho, Wo) in ((406, 602), (345, 511), (101, 150)):
            try:
                y = rs.resize(t.cuda(), (Ho, Wo), MNAME[method], tile=(tw, th), threads=nt)
            except rs.ResampleError as e:
                # A tall, wide tile at a downscale needs more shared memory
                # than a block has: the call is refused before any launch.
                assert e.status == 1 and tw * th >= 512 * 32
                continue
            torch.cuda.synchronize()
            check(y, oracle.resize(x64, Ho, Wo, method), "u8", method, 255.0, f"tile {tile}")


def test_plain_kernel_block_shapes(rs, oracle):
    """The paper's tile-dimension sweep (Sec. III.B): every block shape gives
    the same result."""
    t, x64 = _src(12, (80, 80, 1), "u8")
    ref = oracle.resize(x64, 160, 160, BL)
    for bw, bh in ((32, 4), (8, 8), (4, 8), (8, 4), (32, 16), (16, 16), (64, 2), (1, 1)):
        y = rs.resize(t.cuda(), (160, 160), "bilinear", impl="plain", tile=(bw, bh))
        torch.cuda.synchronize()
        check(y, ref, "u8", BL, 255.0, f"plain {bw}x{bh}")


@pytest.mark.parametrize("method", [BL, BC])
def test_x2_uint8_is_bit_exact(rs, oracle, method):
    """Asymmetric x2: weights are dyadic (1/2; -1/16, 9/16), every FP32
    product and sum of uint8 data is exact, so the GPU equals the FP64
    oracle bit for bit."""
    t, x64 = _src(13, (150, 173, 3), "u8")
    y = rs.resize(t.cuda(), (300, 346), MNAME[method])
    torch.cuda.synchronize()
    q = oracle.quantize_u8(oracle.resize(x64, 300, 346, method))
    assert np.array_equal(y.cpu().numpy(), q)


@pytest.mark.parametrize("dtype", ["u8", "f16", "bf16", "f32"])
@pytest.mark.parametrize("method", [NN, BL, BC])
def test_identity_is_exact(rs, method, dtype):
    t, _ = _src(14, (33, 47, 3), dtype)
    for coord in ("asymmetric", "half_pixel"):
        y = rs.resize(t.cuda(), (33, 47), MNAME[method], coord=coord)
        assert torch.equal(y.cpu(), t)


def test_guard_bands_and_pitched_rows(rs, oracle):
    """Writes stay inside the output: guard bands around dst and the gaps of
    pitched rows keep their canary values."""
    H, W, C, Ho, Wo = 45, 61, 3, 97, 130
    t, x64 = _src(15, (H, W, C), "u8")
    src_pitch, dst_pitch = W * C + 13, Wo * C + 29
    sbuf = torch.zeros(H * src_pitch + 64, dtype=torch.uint8)
    sbuf[:H * src_pitch].view(H, src_pitch)[:, :W * C] = t.reshape(H, W * C)
    guard = 4096
    dbuf = torch.full((guard + Ho * dst_pitch + guard,), 0xA5, dtype=torch.uint8, device="cuda")
    s = sbuf.cuda()
    src = s[:H * src_pitch].view(H, src_pitch)[:, :W * C].view(H, W, C)
    dst = dbuf[guard:guard + Ho * dst_pitch].view(Ho, dst_pitch)[:, :Wo * C].view(Ho, Wo, C)
    for method in (NN, BL, BC):
        dbuf.fill_(0xA5)
        rs.resize(src, (Ho, Wo), MNAME[method], out=dst)
        torch.cuda.synchronize()
        d = dbuf.cpu().numpy()
        assert (d[:guard] == 0xA5).all() and (d[guard + Ho * dst_pitch:] == 0xA5).all()
        rows = d[guard:guard + Ho * dst_pitch].reshape(Ho, dst_pitch)
        assert (rows[:, Wo * C:] == 0xA5).all()
        check(dst, oracle.resize(x64, Ho, Wo, method), "u8", method, 255.0, "pitched")


def test_invalid_call_writes_nothing(rs):
    """A call that fails validation launches nothing: dst keeps its contents."""
    x = torch.zeros(64, 64, 3, dtype=torch.uint8, device="cuda")
    y = torch.full((128, 128, 3), 7, dtype=torch.uint8, device="cuda")
    with pytest.raises(rs.ResampleError):
        rs.resize(x, (128, 128), "bicubic", coord=5)
    with pytest.raises(rs.ResampleError):
        rs.resize(x, (128, 128), "bicubic", out=y, tile=(100, 8))   # tile width not a multiple of 4
    torch.cuda.synchronize()
    assert (y == 7).all()


def test_half_pixel_bicubic_matches_torch(rs):
    """Secondary cross-check: torch's bicubic (align_corners=False) is the
    half-pixel map with a = -3/4."""
    x = torch.randn(2, 3, 50, 70, device="cuda")
    for size in ((100, 140), (33, 41), (77, 200)):
        y = rs.resize(x, size, "bicubic", layout="nchw", coord="half_pixel", cubic_a=-0.75)
        r = torch.nn.functional.interpolate(x, size=size, mode="bicubic", align_corners=False)
        assert (y - r).abs().max().item() < 1e-4


@pytest.mark.parametrize("cfg", [(512, 16, 4), (128, 4, 2), (256, 8, 8), (1024, 32, 1), (512, 1, 4), (128, 32, 16)])
@pytest.mark.parametrize("dtype", ["u8", "f32", "bf16"])
def test_stream_kernel_configs(rs, oracle, cfg, dtype):
    """The streaming kernel at explicit strip widths, chunk heights and band
    counts (several chunks and bands per image, ragged last strip / chunk /
    band), on rows that allow 16-byte loads and rows that do not."""
    tw, ch, waves = cfg
    for k, (H, W, C, Ho, Wo, method, coord) in enumerate([
            (160, 256, 4, 320, 512, BC, 0),     # 16-byte rows (vector loads)
            (157, 203, 3, 301, 391, BC, 1),     # odd rows (element loads)
            (96, 128, 1, 173, 250, BL, 0),
            (200, 160, 3, 99, 81, BC, 0),       # downscale
            (64, 64, 3, 64, 64, NN, 1)]):
        t, x64 = _src(300 + k, (H, W, C), dtype)
        try:
            y = rs.resize(t.cuda(), (Ho, Wo), MNAME[method], coord=CNAME[coord], impl="stream",
                          tile=(tw, ch), waves=waves)
        except rs.ResampleError as e:
            # footprint too large for a block's shared memory: refused before any launch
            assert e.status == 1 and (Ho < H or tw * ch >= 1024 * 32)
            continue
        torch.cuda.synchronize()
        check(y, oracle.resize(x64, Ho, Wo, method, coord), dtype, method, np.abs(x64).max(),
              f"stream {cfg} {dtype} {H}x{W}x{C}->{Ho}x{Wo}")
    assert rs.debug_fault() == 0


@pytest.mark.parametrize("impl", ["stream", "tiled", "plain", "window", "gather"])
def test_kernels_agree_bitwise(rs, impl):
    """Every kernel computes each output element with the same FP32
    operations in the same order (horizontal taps, then vertical), so they
    agree bit for bit (the gather kernel only does nearest, the register
    window kernel only bilinear / bicubic)."""
    x = torch.randint(0, 256, (333, 517, 3), dtype=torch.uint8, device="cuda")
    xf = torch.randn(2, 3, 190, 260, device="cuda")
    methods = {"gather": ("nearest",), "window": ("bilinear", "bicubic")}.get(
        impl, ("bilinear", "bicubic", "nearest"))
    for method in methods:
        ref = rs.resize(x, (701, 911), method, impl="tiled")
        assert torch.equal(rs.resize(x, (701, 911), method, impl=impl), ref)
        reff = rs.resize(xf, (97, 555), method, layout="nchw", impl="tiled")
        got = rs.resize(xf, (97, 555), method, layout="nchw", impl=impl)
        assert torch.equal(got, reff)


@pytest.mark.parametrize("dtype", ["u8", "f16", "f32"])
@pytest.mark.parametrize("cfg", [(None, 0), ((16, 1), 0), ((64, 4), 0), ((1024, 2), 0), ((256, 16), 0)])
def test_gather_kernel_nearest(rs, oracle, dtype, cfg):
    """The nearest-neighbour gather kernel is bit-exact against the oracle at
    several strip widths / rows per thread (strip widths are in elements and
    are rounded to the kernel's 16-byte unit by the caller)."""
    tile, _ = cfg
    ev = {"u8": 16, "f16": 8, "f32": 4}[dtype]
    if tile is not None:
        tile = (max(ev, (tile[0] // ev) * ev), tile[1])
    for k, (H, W, C, Ho, Wo, coord) in enumerate([(100, 130, 3, 200, 260, 0), (77, 91, 1, 160, 33, 1),
                                                   (256, 256, 4, 128, 512, 0), (9, 1000, 3, 31, 1999, 1)]):
        t, x64 = _src(500 + k, (H, W, C), dtype)
        y = rs.resize(t.cuda(), (Ho, Wo), "nearest", coord=CNAME[coord], impl="gather", tile=tile)
        torch.cuda.synchronize()
        check(y, oracle.resize(x64, Ho, Wo, NN, coord), dtype, NN, 1.0, f"gather {cfg} {dtype}")
        assert torch.equal(y, rs.resize(t.cuda(), (Ho, Wo), "nearest", coord=CNAME[coord], impl="tiled"))


@pytest.mark.parametrize("cfg", [(8, 2), (4, 1), (16, 4), (4, 8)])
@pytest.mark.parametrize("dtype", ["u8", "f32", "f16"])
def test_window_kernel_configs(rs, oracle, cfg, dtype):
    """The register-window kernel at several chunk heights and band counts,
    on 16-byte rows and odd rows, up- and downscale, both coordinate maps."""
    chunk, waves = cfg
    for k, (H, W, C, Ho, Wo, method, coord) in enumerate([
            (160, 512, 4, 321, 1024, BC, 0),
            (157, 203, 3, 301, 391, BC, 1),
            (96, 128, 1, 173, 250, BL, 0),
            (200, 160, 3, 99, 81, BC, 0),
            (31, 700, 1, 62, 1399, BL, 1),
            (2, 3, 3, 7, 5, BC, 0)]):
        t, x64 = _src(700 + k, (H, W, C), dtype)
        try:
            y = rs.resize(t.cuda(), (Ho, Wo), MNAME[method], coord=CNAME[coord], impl="window",
                          tile=(1024, chunk), waves=waves)
        except rs.ResampleError as e:
            assert e.status == 1 and Ho < H          # downscale footprint too large for the chunk
            continue
        torch.cuda.synchronize()
        check(y, oracle.resize(x64, Ho, Wo, method, coord), dtype, method, np.abs(x64).max(),
              f"window {cfg} {dtype} {H}x{W}x{C}->{Ho}x{Wo}")
    assert rs.debug_fault() == 0


@pytest.mark.parametrize("dtype", ["u8", "f16", "f32"])
@pytest.mark.parametrize("band", [None, 1, 7, 100])
def test_gather_staged_rows(rs, oracle, dtype, band):
    """The staged-rows nearest kernel (4096-byte strips, source rows of whole
    16-byte units, upsampled columns): several strips with a ragged last one,
    strips that start inside an output pixel, rows up- and downsampled, both
    coordinate maps, bit-exact against the oracle and the tiled kernel."""
    es = {"u8": 1, "f16": 2, "f32": 4}[dtype]
    tile = (4096 // es, band) if band else None
    for k, (H, W, C, Ho, Wo, coord) in enumerate([(64, 1024, 3, 150, 2048, 0), (33, 512, 1, 20, 3001, 1),
                                                   (40, 256, 4, 97, 700, 0), (7, 96, 2, 300, 129, 1),
                                                   (120, 48, 3, 37, 4097, 0)]):
        if (W * C * es) % 16:
            W += (16 // np.gcd(16, C * es)) - W % (16 // np.gcd(16, C * es))
        t, x64 = _src(900 + k, (H, W, C), dtype)
        y = rs.resize(t.cuda(), (Ho, Wo), "nearest", coord=CNAME[coord], impl="gather", tile=tile)
        torch.cuda.synchronize()
        check(y, oracle.resize(x64, Ho, Wo, NN, coord), dtype, NN, 1.0, f"staged {dtype} {band} {H}x{W}x{C}->{Ho}x{Wo}")
        assert torch.equal(y, rs.resize(t.cuda(), (Ho, Wo), "nearest", coord=CNAME[coord], impl="tiled"))
    assert rs.debug_fault() == 0


@pytest.mark.parametrize("dtype", ["u8", "f16", "bf16", "f32"])
def test_window_exact_x2(rs, oracle, dtype):
    """The register window at exactly x2 vertically under the asymmetric map
    with 16-byte source rows (the kernels that emit two rows per source
    position without the per-position table): several bands and strips,
    both methods, chunks of 4 and 8 rows; against the oracle and bit for bit
    against the tiled kernel. Near misses (2H + 1 rows, the half-pixel map)
    take the general kernels and must agree the same way."""
    cases = [((1, 3, 300, 256), (600, 512), 0), ((2, 1, 37, 64), (74, 100), 0), ((1, 4, 130, 48), (260, 96), 0),
             ((1, 3, 300, 256), (601, 512), 0), ((1, 3, 300, 256), (600, 512), 1)]
    for k, ((N, C, H, W), (Ho, Wo), coord) in enumerate(cases):
        t, x64 = _src(2000 + k, (N, C, H, W), dtype)
        for method in (BL, BC):
            ref = rs.resize(t.cuda(), (Ho, Wo), MNAME[method], layout="nchw", coord=CNAME[coord], impl="tiled")
            for chunk in (4, 8):
                y = rs.resize(t.cuda(), (Ho, Wo), MNAME[method], layout="nchw", coord=CNAME[coord], impl="window",
                              tile=(1024, chunk))
                torch.cuda.synchronize()
                assert torch.equal(y, ref), (dtype, (N, C, H, W), (Ho, Wo), coord, MNAME[method], chunk)
            check(y, oracle.resize_nchw(x64, Ho, Wo, method, coord), dtype, method, np.abs(x64).max(),
                  f"window x2 {dtype} {MNAME[method]} {(N, C, H, W)}->{Ho}x{Wo}")
    # interleaved RGB, 16-byte rows, several strips
    t, x64 = _src(2100, (120, 448, 3), dtype)
    y = rs.resize(t.cuda(), (240, 1000), "bicubic", impl="window", tile=(1024, 8))
    torch.cuda.synchronize()
    assert torch.equal(y, rs.resize(t.cuda(), (240, 1000), "bicubic", impl="tiled"))
    check(y, oracle.resize(x64, 240, 1000, BC, 0), dtype, BC, np.abs(x64).max(), f"window x2 hwc {dtype}")
    assert rs.debug_fault() == 0


@pytest.mark.parametrize("dtype", ["u8", "f16", "bf16", "f32"])
def test_window_shifted_staging(rs, oracle, dtype):
    """The register-window kernel on source rows that are not whole 16-byte
    units (odd widths, NCHW planes starting mid-unit, a pitched view whose
    first row starts mid-unit): the shifted copies and their element-wise
    fill at the plane's first and last rows, against the oracle and the
    tiled kernel, bit for bit."""
    for k, (N, C, H, W, Ho, Wo, method, coord) in enumerate([(2, 3, 75, 131, 150, 262, BC, 0),
                                                              (1, 2, 41, 67, 123, 201, BL, 1),
                                                              (3, 1, 33, 19, 70, 45, BC, 1)]):
        t, x64 = _src(1200 + k, (N, C, H, W), dtype)
        y = rs.resize(t.cuda(), (Ho, Wo), MNAME[method], layout="nchw", coord=CNAME[coord], impl="window",
                      tile=(1024, 4))
        torch.cuda.synchronize()
        check(y, oracle.resize_nchw(x64, Ho, Wo, method, coord), dtype, method, np.abs(x64).max(),
              f"shifted nchw {dtype} {(N, C, H, W)}->{Ho}x{Wo}")
        ref = rs.resize(t.cuda(), (Ho, Wo), MNAME[method], layout="nchw", coord=CNAME[coord], impl="tiled")
        assert torch.equal(y, ref)
    # an interleaved view whose rows start one element into a wider buffer
    t, x64 = _src(1300, (97, 211, 3), dtype)
    big = torch.zeros((97, 215, 3), dtype=t.dtype)
    big[:, 1:212] = t
    view = big.cuda()[:, 1:212]
    y = rs.resize(view, (190, 400), "bicubic", impl="window", tile=(1024, 8))
    torch.cuda.synchronize()
    check(y, oracle.resize(x64, 190, 400, BC, 0), dtype, BC, np.abs(x64).max(), f"shifted view {dtype}")
    assert rs.debug_fault() == 0


def _unclamped_columns(n, m, method, coord):
    """Output columns none of whose taps leave [0, n) (exact integer map)."""
    K = 2 if method == BL else 4
    keep = []
    for j in range(m):
        i0 = (j * n) // m if coord == 0 else ((2 * j + 1) * n - m) // (2 * m)
        f = i0 - 1 if K == 4 else i0
        if f >= 0 and f + K - 1 <= n - 1:
            keep.append(j)
    return keep


@pytest.mark.parametrize("method", [NN, BL, BC])
def test_align_corners_every_kernel(rs, oracle, method):
    """The align-corners map through every forward kernel that takes the
    method (explicit impl), against the oracle, and bit for bit against the
    tiled kernel (same FP32 operations in the same order)."""
    impls = ["plain", "tiled", "stream"] + (["gather"] if method == NN else ["window", "reduce"])
    ran = {i: 0 for i in impls}
    for k, (N, C, H, W, Ho, Wo) in enumerate([(2, 3, 75, 132, 150, 262), (1, 2, 96, 128, 37, 50),
                                              (1, 1, 300, 516, 700, 1200), (1, 4, 9, 12, 1, 7)]):
        for dtype in ("u8", "f32"):
            t, x64 = _src(1900 + k, (N, C, H, W), dtype)
            ref64 = oracle.resize_nchw(x64, Ho, Wo, method, 2)
            tiled = rs.resize(t.cuda(), (Ho, Wo), MNAME[method], layout="nchw", coord="align_corners", impl="tiled")
            for impl in impls:
                if impl == "reduce" and dtype != "f32":
                    continue
                try:
                    y = rs.resize(t.cuda(), (Ho, Wo), MNAME[method], layout="nchw", coord="align_corners", impl=impl)
                except rs.ResampleError:
                    # the window kernel bounds the footprint of a whole 1024-element
                    # strip, so it refuses strong downscales under any map
                    assert impl == "window" and Ho < H, (impl, dtype, (H, W, Ho, Wo))
                    continue
                ran[impl] += 1
                torch.cuda.synchronize()
                check(y, ref64, dtype, method, np.abs(x64).max(),
                      f"align {impl} {MNAME[method]} {dtype} {(N, C, H, W)}->{Ho}x{Wo}")
                if impl != "reduce":
                    assert torch.equal(y, tiled), (impl, dtype, (N, C, H, W, Ho, Wo))
    assert all(v > 0 for v in ran.values()), ran
    assert rs.debug_fault() == 0


REDUCE_CASES = [
    # (N, C, H, W, Ho, Wo, coord); NCHW, W a multiple of 4
    (2, 3, 64, 80, 32, 40, 0),         # x0.5
    (1, 2, 100, 124, 37, 51, 1),       # ragged downscale, half-pixel
    (1, 1, 700, 1200, 300, 600, 0),    # two strips, bands of 256 rows and a tail
    (1, 1, 33, 20, 9, 5, 1),           # near 1/4: edge taps clamp on both sides
    (2, 4, 40, 36, 90, 72, 1),         # an upscale (any scale applies)
    (1, 1, 4, 4, 1, 1, 0),             # one output pixel
    (1, 3, 512, 512, 256, 256, 1),     # the NCHW x0.5 workload's plane shape
]


@pytest.mark.parametrize("method", [BL, BC])
def test_reduce_matches_oracle(rs, oracle, method):
    """RS_IMPL_REDUCE (the fused window pass in its transposed roles, point
    taps of Eqs. 1-5 computed in the kernel, clamped edge taps merged)
    against the FP64 oracle: NCHW and interleaved, both coordinate maps,
    ragged strips and bands."""
    for k, (N, C, H, W, Ho, Wo, coord) in enumerate(REDUCE_CASES):
        t, x64 = _src(1600 + k, (N, C, H, W), "f32")
        y = rs.resize(t.cuda(), (Ho, Wo), MNAME[method], layout="nchw", coord=CNAME[coord], impl="reduce")
        torch.cuda.synchronize()
        check(y, oracle.resize_nchw(x64, Ho, Wo, method, coord), "f32", method, np.abs(x64).max(),
              f"reduce nchw {MNAME[method]} {CNAME[coord]} {(N, C, H, W)}->{Ho}x{Wo}")
        # Same FP32 operations in the same order as the tiled kernel (x taps,
        # then y taps, ascending), except in columns whose x taps clamp onto
        # an edge column, where REDUCE merges them: bit-equal elsewhere.
        ref = rs.resize(t.cuda(), (Ho, Wo), MNAME[method], layout="nchw", coord=CNAME[coord], impl="tiled")
        cols = _unclamped_columns(W, Wo, method, coord)
        assert torch.equal(y[..., cols], ref[..., cols])
    for k, (H, W, C, Ho, Wo) in enumerate([(90, 128, 3, 45, 50), (256, 200, 3, 64, 52), (61, 77, 4, 30, 20)]):
        t, x64 = _src(1700 + k, (H, W, C), "f32")
        for coord in (0, 1):
            y = rs.resize(t.cuda(), (Ho, Wo), MNAME[method], coord=CNAME[coord], impl="reduce")
            torch.cuda.synchronize()
            check(y, oracle.resize(x64, Ho, Wo, method, coord), "f32", method, np.abs(x64).max(),
                  f"reduce hwc {MNAME[method]} {CNAME[coord]} {H}x{W}x{C}->{Ho}x{Wo}")
    if method == BC:   # another Keys parameter
        t, x64 = _src(1800, (1, 2, 96, 64), "f32")
        y = rs.resize(t.cuda(), (40, 30), "bicubic", layout="nchw", cubic_a=-0.75, impl="reduce")
        torch.cuda.synchronize()
        check(y, oracle.resize_nchw(x64, 40, 30, BC, 0, a=-0.75), "f32", BC, np.abs(x64).max(), "reduce a=-0.75")
    assert rs.debug_fault() == 0


def test_reduce_auto_and_refusals(rs, oracle):
    """AUTO takes REDUCE for a large FP32 vertical downscale, and the result
    matches the oracle; REDUCE refuses what it does not cover."""
    x = torch.randn(8, 3, 512, 512, device="cuda")
    assert rs.tile_config(x, (256, 256), "bilinear", layout="nchw")["impl"] == "reduce"
    y = rs.resize(x, (256, 256), "bicubic", layout="nchw")
    ref = oracle.resize_nchw(x[1:2].double().cpu().numpy(), 256, 256, BC, 0)
    check(y[1:2], ref, "f32", BC, float(x.abs().max()), "auto reduce x0.5")
    with pytest.raises(rs.ResampleError):          # FP32 only
        rs.resize(torch.zeros(64, 64, dtype=torch.uint8, device="cuda"), (32, 32), "bilinear", impl="reduce")
    with pytest.raises(rs.ResampleError):          # nearest has its own gather
        rs.resize(torch.zeros(64, 64, device="cuda"), (32, 32), "nearest", impl="reduce")
    with pytest.raises(rs.ResampleError):          # rows of 63 FP32 elements are not whole 16-byte units
        rs.resize(torch.zeros(64, 63, device="cuda"), (32, 32), "bilinear", impl="reduce")
    with pytest.raises(rs.ResampleError):          # no shape parameters
        rs.resize(torch.zeros(64, 64, device="cuda"), (32, 32), "bilinear", impl="reduce", tile=(512, 4))
    assert rs.debug_fault() == 0


@pytest.mark.parametrize("method", [BL, BC])
def test_antialias_matches_oracle(rs, oracle, method):
    """RS_FLAG_ANTIALIAS (the kernel stretched by the downscale factor, taps
    cut to the image and renormalised) against the FP64 oracle: FP32 NCHW
    and interleaved, down- and upscales, ragged strips."""
    for k, (N, C, H, W, Ho, Wo) in enumerate([(2, 3, 64, 80, 32, 40), (1, 2, 97, 132, 49, 67),
                                               (1, 1, 300, 520, 170, 300), (2, 1, 40, 36, 90, 72)]):
        if method == BC and (H / Ho > 2 or W / Wo > 2):
            continue
        x = np.random.default_rng(1400 + k).standard_normal((N, C, H, W)).astype(np.float32)
        y = rs.resize(torch.from_numpy(x).cuda(), (Ho, Wo), MNAME[method], layout="nchw", antialias=True)
        torch.cuda.synchronize()
        ref = oracle.resize_aa_nchw(x.astype(np.float64), Ho, Wo, method)
        check(y, ref, "f32", method, float(np.abs(x).max()), f"antialias nchw {MNAME[method]} {(N, C, H, W)}->{Ho}x{Wo}")
    # interleaved channels; bilinear down to 1/4
    x = np.random.default_rng(1500).standard_normal((256, 200, 3)).astype(np.float32)
    for (Ho, Wo) in ((128, 100), (64, 52), (130, 101)):
        if method == BC and (256 / Ho > 2 or 200 / Wo > 2):
            continue
        y = rs.resize(torch.from_numpy(x).cuda(), (Ho, Wo), MNAME[method], antialias=True)
        torch.cuda.synchronize()
        check(y, oracle.resize_aa(x.astype(np.float64), Ho, Wo, method), "f32", method, float(np.abs(x).max()),
              f"antialias hwc {MNAME[method]} -> {Ho}x{Wo}")
    assert rs.debug_fault() == 0


@pytest.mark.parametrize("method", [BL, BC])
@pytest.mark.parametrize("dtype", ["u8", "f16", "bf16", "f32"])
def test_antialias_window_every_dtype(rs, oracle, method, dtype):
    """RS_FLAG_ANTIALIAS on the general window form (antialias taps, at most 8
    per axis) for every storage dtype: uint8 / FP16 / BF16 sources (and FP32
    through impl='window'), interleaved and planar, down- and upscales,
    ragged strips, against the FP64 definition under the storage rule."""
    impl = "window" if dtype == "f32" else "auto"
    cases = [((180, 240, 3), (90, 120)), ((97, 133, 3), (49, 67)), ((300, 520, 1), (170, 300)),
             ((40, 36, 4), (90, 72)), ((256, 200, 3), (64, 52)), ((77, 91, 2), (77, 91)),
             ((3, 200, 3), (1, 100)), ((200, 3, 1), (100, 1))]
    for k, (shape, (Ho, Wo)) in enumerate(cases):
        H, W = shape[0], shape[1]
        taps = max(_aa_taps(n, m, method) for n, m in ((H, Ho), (W, Wo)))
        t, x64 = _src(1600 + k, shape, dtype)
        if taps > 8 and impl == "window":   # the window forms hold at most 8 taps per axis
            with pytest.raises(rs.ResampleError):
                rs.resize(t.cuda(), (Ho, Wo), MNAME[method], antialias=True, impl=impl)
            continue
        y = rs.resize(t.cuda(), (Ho, Wo), MNAME[method], antialias=True, impl=impl)
        torch.cuda.synchronize()
        check(y, oracle.resize_aa(x64, Ho, Wo, method), dtype, method, float(np.abs(x64).max()),
              f"antialias window {dtype} {MNAME[method]} {shape}->{Ho}x{Wo}")
    # planar (NCHW) planes
    t, x64 = _src(1700, (2, 3, 120, 150), dtype)
    y = rs.resize(t.cuda(), (60, 75), MNAME[method], layout="nchw", antialias=True, impl=impl)
    torch.cuda.synchronize()
    check(y, oracle.resize_aa_nchw(x64, 60, 75, method), dtype, method, float(np.abs(x64).max()),
          f"antialias window nchw {dtype} {MNAME[method]}")
    assert rs.debug_fault() == 0


def test_antialias_refusals(rs):
    xf = torch.randn(64, 64, device="cuda")
    with pytest.raises(rs.ResampleError):          # nearest has no filter to stretch
        rs.resize(xf, (32, 32), "nearest", antialias=True)
    with pytest.raises(rs.ResampleError):          # more than 8 taps: not on the window form
        rs.resize(xf, (20, 20), "bicubic", antialias=True, impl="window")


@pytest.mark.parametrize("method", [BL, BC])
@pytest.mark.parametrize("dtype", ["u8", "f16", "bf16", "f32"])
def test_antialias_many_taps(rs, oracle, method, dtype):
    """More than 8 antialias taps per axis (the many-tap tiled kernel):
    downscales by 3 to 40 on one or both axes, ragged tiles (outputs not
    multiples of 32 columns or of the tile height), 1-4 interleaved
    channels and planar planes, against the FP64 definition under the
    storage rule; impl="tiled" runs the same kernel on a few-tap case."""
    cases = [((300, 420, 3), (37, 41)), ((97, 1200, 1), (90, 29)), ((640, 90, 4), (16, 88)),
             ((1000, 1000, 2), (25, 33)), ((129, 257, 3), (3, 5)), ((64, 64, 1), (1, 1))]
    for k, (shape, (Ho, Wo)) in enumerate(cases):
        t, x64 = _src(1800 + k, shape, dtype)
        y = rs.resize(t.cuda(), (Ho, Wo), MNAME[method], antialias=True)
        torch.cuda.synchronize()
        check(y, oracle.resize_aa(x64, Ho, Wo, method), dtype, method, float(np.abs(x64).max()),
              f"antialias many taps {dtype} {MNAME[method]} {shape}->{Ho}x{Wo}")
    t, x64 = _src(1900, (2, 3, 200, 150), dtype)
    y = rs.resize(t.cuda(), (20, 15), MNAME[method], layout="nchw", antialias=True)
    torch.cuda.synchronize()
    check(y, oracle.resize_aa_nchw(x64, 20, 15, method), dtype, method, float(np.abs(x64).max()),
          f"antialias many taps nchw {dtype} {MNAME[method]}")
    t, x64 = _src(1901, (90, 120, 3), dtype)
    y = rs.resize(t.cuda(), (60, 70), MNAME[method], antialias=True, impl="tiled")
    torch.cuda.synchronize()
    check(y, oracle.resize_aa(x64, 60, 70, method), dtype, method, float(np.abs(x64).max()),
          f"antialias tiled {dtype} {MNAME[method]}")
    # the vertical-first streaming kernel on request, few and many taps,
    # tiles of several widths, a ragged last band, planar planes
    for k, (shape, (Ho, Wo)) in enumerate([((90, 120, 3), (45, 150)), ((333, 1900, 3), (70, 400)),
                                            ((200, 64, 4), (200, 30)), ((1000, 41, 1), (37, 41))]):
        t, x64 = _src(1950 + k, shape, dtype)
        y = rs.resize(t.cuda(), (Ho, Wo), MNAME[method], antialias=True, impl="stream")
        torch.cuda.synchronize()
        check(y, oracle.resize_aa(x64, Ho, Wo, method), dtype, method, float(np.abs(x64).max()),
              f"antialias stream {dtype} {MNAME[method]} {shape}->{Ho}x{Wo}")
    t, x64 = _src(1960, (2, 3, 300, 150), dtype)
    y = rs.resize(t.cuda(), (61, 70), MNAME[method], layout="nchw", antialias=True, impl="stream")
    torch.cuda.synchronize()
    check(y, oracle.resize_aa_nchw(x64, 61, 70, method), dtype, method, float(np.abs(x64).max()),
          f"antialias stream nchw {dtype} {MNAME[method]}")
    with pytest.raises(rs.ResampleError):   # a vertical upscale: not the streaming form
        rs.resize(t[0, 0].cuda(), (400, 20), MNAME[method], antialias=True, impl="stream")
    assert rs.debug_fault() == 0
