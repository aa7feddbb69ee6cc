"""C ABI checks that need no GPU: the library builds for sm_103a, loads,
exports every function include/resample.h declares, and its host-side
argument validation rejects bad calls before touching CUDA."""
import ctypes
import re
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]
HEADER = ROOT / "include" / "resample.h"


@pytest.fixture(scope="module")
def L():
    from paper_1001_1718_gb300 import build as b
    b.build()
    from paper_1001_1718_gb300 import _binding
    return _binding.lib()


def declared_functions():
    text = HEADER.read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = set(re.findall(r"\b(rs_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("rs_resize", "rs_resize_ex", "rs_resize_backward", "rs_resize_batched",
                     "rs_autotune", "rs_status_string"):
        assert required in names


def test_every_declared_symbol_is_exported(L):
    from paper_1001_1718_gb300 import _binding
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing
    # and the binding declares a signature for each
    assert set(declared_functions()) <= set(_binding.SIGNATURES)


def test_status_strings_and_defaults(L):
    from paper_1001_1718_gb300 import _binding as B
    assert L.rs_status_string(0) == b"ok"
    assert L.rs_status_string(4).startswith(b"workspace")
    o = B.options()
    assert (o.coord, o.cubic_a, o.impl, o.tile_w, o.tile_h, o.threads, o.waves) == (0, -0.5, 0, 0, 0, 0, 0)
    lay = L.rs_layout_hwc(2, 5, 7, 3)
    assert (lay.N, lay.C, lay.H, lay.W, lay.px_stride, lay.c_stride, lay.row_pitch, lay.n_stride) == \
        (2, 3, 5, 7, 3, 1, 21, 105)
    lay = L.rs_layout_nchw(2, 3, 5, 7)
    assert (lay.px_stride, lay.row_pitch, lay.c_stride, lay.n_stride) == (1, 7, 35, 105)


def test_validation_rejects_before_any_launch(L):
    """Each call below fails host validation, so no CUDA call is made."""
    from paper_1001_1718_gb300 import _binding as B
    P = 0x10000  # never dereferenced: validation fails first
    Q = 0x90000000
    # null pointers
    assert L.rs_resize(None, 4, 4, 1, B.RS_U8, Q, 8, 8, B.RS_BILINEAR, None) == B.RS_ERR_INVALID_ARG
    assert L.rs_resize(P, 4, 4, 1, B.RS_U8, None, 8, 8, B.RS_BILINEAR, None) == B.RS_ERR_INVALID_ARG
    # sizes out of range
    for H, W, Ho, Wo in ((0, 4, 8, 8), (4, 4, 0, 8), (70000, 4, 8, 8), (4, 4, 8, 65536), (-3, 4, 8, 8)):
        assert L.rs_resize(P, H, W, 1, B.RS_U8, Q, Ho, Wo, B.RS_BILINEAR, None) == B.RS_ERR_INVALID_ARG
    # channels, dtype, method
    assert L.rs_resize(P, 4, 4, 5, B.RS_U8, Q, 8, 8, B.RS_BILINEAR, None) == B.RS_ERR_INVALID_ARG
    assert L.rs_resize(P, 4, 4, 1, 7, Q, 8, 8, B.RS_BILINEAR, None) == B.RS_ERR_INVALID_ARG
    assert L.rs_resize(P, 4, 4, 1, B.RS_U8, Q, 8, 8, 9, None) == B.RS_ERR_INVALID_ARG
    # misaligned FP32 pointer
    assert L.rs_resize(P + 2, 4, 4, 1, B.RS_F32, Q, 8, 8, B.RS_BILINEAR, None) == B.RS_ERR_ALIGNMENT
    # overlapping source and destination
    assert L.rs_resize(P, 16, 16, 1, B.RS_U8, P + 100, 8, 8, B.RS_BILINEAR, None) == B.RS_ERR_INVALID_ARG


def test_coordinate_map_and_impl_options(L):
    """The three coordinate maps are accepted and others refused; RS_IMPL_REDUCE
    is refused for what it does not cover (host logic: no buffers needed)."""
    import ctypes
    from paper_1001_1718_gb300 import _binding as B
    Li, Lo = L.rs_layout_nchw(2, 3, 64, 80), L.rs_layout_nchw(2, 3, 32, 40)
    c = B.RsTileConfig()
    for coord in (B.RS_COORD_ASYMMETRIC, B.RS_COORD_HALF_PIXEL, B.RS_COORD_ALIGN_CORNERS):
        o = B.options(coord=coord)
        assert L.rs_tile_config_for(ctypes.byref(Li), ctypes.byref(Lo), B.RS_F32, B.RS_BICUBIC, ctypes.byref(o),
                                    ctypes.byref(c)) == 0
    for coord in (-1, 3):
        o = B.options(coord=coord)
        assert L.rs_tile_config_for(ctypes.byref(Li), ctypes.byref(Lo), B.RS_F32, B.RS_BICUBIC, ctypes.byref(o),
                                    ctypes.byref(c)) == B.RS_ERR_INVALID_ARG
    o = B.options(impl=B.RS_IMPL_REDUCE + 1)
    assert L.rs_tile_config_for(ctypes.byref(Li), ctypes.byref(Lo), B.RS_F32, B.RS_BILINEAR, ctypes.byref(o),
                                ctypes.byref(c)) == B.RS_ERR_INVALID_ARG
    o = B.options(impl=B.RS_IMPL_REDUCE)
    assert L.rs_tile_config_for(ctypes.byref(Li), ctypes.byref(Lo), B.RS_F32, B.RS_BILINEAR, ctypes.byref(o),
                                ctypes.byref(c)) == 0 and c.impl == B.RS_IMPL_REDUCE
    for dt, m in ((B.RS_U8, B.RS_BILINEAR), (B.RS_F16, B.RS_BICUBIC), (B.RS_F32, B.RS_NEAREST)):
        assert L.rs_tile_config_for(ctypes.byref(Li), ctypes.byref(Lo), dt, m, ctypes.byref(o),
                                    ctypes.byref(c)) == B.RS_ERR_INVALID_ARG
    # rows of 63 FP32 elements are not whole 16-byte units
    Lr, Lro = L.rs_layout_nchw(1, 1, 64, 63), L.rs_layout_nchw(1, 1, 32, 32)
    assert L.rs_tile_config_for(ctypes.byref(Lr), ctypes.byref(Lro), B.RS_F32, B.RS_BILINEAR, ctypes.byref(o),
                                ctypes.byref(c)) == B.RS_ERR_INVALID_ARG


def test_layout_validation(L):
    from paper_1001_1718_gb300 import _binding as B
    P, Q = 0x10000, 0x90000000
    good_in = L.rs_layout_nchw(2, 3, 8, 8)
    good_out = L.rs_layout_nchw(2, 3, 16, 16)
    o = B.options(coord=5)
    assert L.rs_resize_ex(P, ctypes.byref(good_in), Q, ctypes.byref(good_out), B.RS_F32, 1,
                          ctypes.byref(o), None) == B.RS_ERR_INVALID_ARG
    o = B.options(cubic_a=float("nan"))
    assert L.rs_resize_ex(P, ctypes.byref(good_in), Q, ctypes.byref(good_out), B.RS_F32, 2,
                          ctypes.byref(o), None) == B.RS_ERR_INVALID_ARG
    bad = L.rs_layout_nchw(2, 3, 8, 8)
    bad.row_pitch = 4                 # shorter than a row
    assert L.rs_resize_ex(P, ctypes.byref(bad), Q, ctypes.byref(good_out), B.RS_F32, 1,
                          None, None) == B.RS_ERR_INVALID_ARG
    bad = L.rs_layout_nchw(2, 3, 8, 8)
    bad.c_stride = 10                 # planes overlap
    assert L.rs_resize_ex(P, ctypes.byref(bad), Q, ctypes.byref(good_out), B.RS_F32, 1,
                          None, None) == B.RS_ERR_INVALID_ARG
    mismatch = L.rs_layout_nchw(1, 3, 16, 16)   # N differs
    assert L.rs_resize_ex(P, ctypes.byref(good_in), Q, ctypes.byref(mismatch), B.RS_F32, 1,
                          None, None) == B.RS_ERR_INVALID_ARG
    hwc5 = L.rs_layout_hwc(1, 8, 8, 5)
    assert L.rs_resize_ex(P, ctypes.byref(hwc5), Q, ctypes.byref(L.rs_layout_hwc(1, 4, 4, 5)),
                          B.RS_U8, 1, None, None) == B.RS_ERR_UNSUPPORTED
    # unknown option flags; antialias has no nearest form
    o = B.options()
    o.flags = 2
    assert L.rs_resize_ex(P, ctypes.byref(good_in), Q, ctypes.byref(good_out), B.RS_F32, B.RS_BILINEAR,
                          ctypes.byref(o), None) == B.RS_ERR_INVALID_ARG
    o.flags = B.RS_FLAG_ANTIALIAS
    assert L.rs_resize_ex(P, ctypes.byref(good_in), Q, ctypes.byref(good_out), B.RS_F32, B.RS_NEAREST,
                          ctypes.byref(o), None) == B.RS_ERR_INVALID_ARG
    # window chunks must hold whole groups of taps (4 for bicubic)
    o = B.options(impl=B.RS_IMPL_WINDOW, tile_w=1024, tile_h=6)
    assert L.rs_resize_ex(P, ctypes.byref(good_in), Q, ctypes.byref(good_out), B.RS_F32, B.RS_BICUBIC,
                          ctypes.byref(o), None) == B.RS_ERR_INVALID_ARG
    # plain kernel block too large
    o = B.options(impl=B.RS_IMPL_PLAIN, tile_w=64, tile_h=32)
    assert L.rs_resize_ex(P, ctypes.byref(good_in), Q, ctypes.byref(good_out), B.RS_F32, 1,
                          ctypes.byref(o), None) == B.RS_ERR_INVALID_ARG


def test_batched_options_validation(L):
    """Batch calls reject kernels with no batched form and window shapes
    out of range on the host, before the work list is uploaded."""
    from paper_1001_1718_gb300 import _binding as B
    arr = (B.RsImageDesc * 1)()
    d = arr[0]
    d.src, d.dst = 0x10000, 0x90000000      # never dereferenced: validation fails first
    d.H, d.W, d.C, d.Ho, d.Wo, d.method = 8, 8, 3, 16, 16, B.RS_BICUBIC
    d.src_pitch, d.dst_pitch = 24, 48
    ws = 0x20000000
    for o in (B.options(impl=B.RS_IMPL_STREAM), B.options(impl=B.RS_IMPL_GATHER), B.options(impl=B.RS_IMPL_PLAIN),
              B.options(impl=B.RS_IMPL_WINDOW, tile_w=257), B.options(impl=B.RS_IMPL_WINDOW, tile_h=2),
              B.options(impl=B.RS_IMPL_WINDOW, tile_h=33)):
        assert L.rs_resize_batched(arr, 1, B.RS_U8, ws, 1 << 20, ctypes.byref(o), None) == B.RS_ERR_INVALID_ARG
        assert L.rs_resize_batched_noalloc(arr, 1, B.RS_U8, ctypes.byref(o), None) == B.RS_ERR_INVALID_ARG
    assert L.rs_autotune_batched(arr, 1, B.RS_U8, ws, 1 << 20, None, None, None) == B.RS_ERR_INVALID_ARG


def test_tune_cache_file_roundtrip(L, tmp_path):
    p = tmp_path / "tune.txt"
    key = "sms=152;dt=0;m=2;C=3;coord=0;sy=4;sx=4;sz=27"
    p.write_text(f"# resample-tune v2\n{key} 3 512 16 256 4\nbogus line\nk2 1 512 16 100 0\n")
    assert L.rs_tune_cache_load(str(p).encode()) == 0
    q = tmp_path / "out.txt"
    assert L.rs_tune_cache_save(str(q).encode()) == 0
    text = q.read_text()
    assert f"{key} 3 512 16 256 4" in text
    assert "k2" not in text            # invalid thread count: dropped
    stale = tmp_path / "stale.txt"
    stale.write_text("# resample-tune v1\nkey 512 16 256\n")   # old format: ignored
    assert L.rs_tune_cache_load(str(stale).encode()) != 0
    L.rs_tune_cache_clear()
    assert L.rs_tune_cache_save(str(q).encode()) == 0
    assert q.read_text().strip().startswith("# resample-tune v2")
    assert len(q.read_text().strip().splitlines()) == 1


def test_tile_config_query_without_buffers(L):
    """The kernel AUTO would pick for a problem, from layouts alone."""
    import paper_1001_1718_gb300 as rs
    from paper_1001_1718_gb300 import _binding as B
    Li, Lo = L.rs_layout_hwc(1, 4096, 4096, 3), L.rs_layout_hwc(1, 8192, 8192, 3)
    c = B.RsTileConfig()
    # Without a GPU, num_sms() falls back to 1 and the shared-memory limit to
    # 48 KB; the choice itself is host logic: a large upscale runs the
    # register-window kernel (chunks of 8 staged rows on a GB300, 4 within
    # the 48 KB fallback).
    assert L.rs_tile_config_for(ctypes.byref(Li), ctypes.byref(Lo), B.RS_U8, B.RS_BICUBIC, None,
                                ctypes.byref(c)) == 0
    assert c.impl == B.RS_IMPL_WINDOW and c.tile_w == 1024 and c.tile_h in (4, 8)
    # an FP32 x0.5 downscale runs the window pass in its transposed roles;
    # uint8 does not (it stores bytes; REDUCE is FP32 only)
    Li, Lo = L.rs_layout_nchw(32, 3, 512, 512), L.rs_layout_nchw(32, 3, 256, 256)
    for m in (B.RS_BILINEAR, B.RS_BICUBIC):
        assert L.rs_tile_config_for(ctypes.byref(Li), ctypes.byref(Lo), B.RS_F32, m, None, ctypes.byref(c)) == 0
        assert c.impl == B.RS_IMPL_REDUCE
    assert L.rs_tile_config_for(ctypes.byref(Li), ctypes.byref(Lo), B.RS_U8, B.RS_BICUBIC, None, ctypes.byref(c)) == 0
    assert c.impl != B.RS_IMPL_REDUCE
    # an explicit REDUCE takes no shape parameters
    o = B.options(impl=B.RS_IMPL_REDUCE, tile_w=512)
    assert L.rs_tile_config_for(ctypes.byref(Li), ctypes.byref(Lo), B.RS_F32, B.RS_BILINEAR, ctypes.byref(o),
                                ctypes.byref(c)) != 0
    del rs


def test_product_path_refuses_cpu_tensors():
    import torch
    import paper_1001_1718_gb300 as rs
    with pytest.raises(ValueError):
        rs.resize(torch.zeros(4, 4, 3, dtype=torch.uint8), (8, 8), "bilinear")


def test_resize_normalize_validation(L):
    """rs_resize_normalize checks its arguments on the host before anything
    is launched (no GPU needed for these refusals)."""
    from paper_1001_1718_gb300 import _binding as B
    P, Q = 0x10000, 0x90000000      # never dereferenced
    li, lo = L.rs_layout_hwc(2, 16, 16, 3), L.rs_layout_nchw(2, 3, 32, 32)
    m = (ctypes.c_float * 3)(120.0, 110.0, 100.0)
    sd = (ctypes.c_float * 3)(58.0, 57.0, 57.0)
    bad_sd = (ctypes.c_float * 3)(58.0, 0.0, 57.0)

    def call(src=P, inl=li, dst=Q, outl=lo, dt=B.RS_F16, meth=B.RS_BILINEAR, mean=m, std=sd, opt=None):
        return L.rs_resize_normalize(src, ctypes.byref(inl), dst, ctypes.byref(outl), dt, meth, mean, std,
                                     ctypes.byref(opt) if opt is not None else None, None)
    assert call(src=0) == B.RS_ERR_INVALID_ARG
    assert call(mean=None) == B.RS_ERR_INVALID_ARG
    assert call(dt=B.RS_U8) == B.RS_ERR_INVALID_ARG               # outputs are FP16 / BF16 / FP32
    assert call(meth=B.RS_NEAREST) == B.RS_ERR_UNSUPPORTED
    assert call(std=bad_sd) == B.RS_ERR_INVALID_ARG               # a zero std
    assert call(outl=L.rs_layout_hwc(2, 32, 32, 3)) == B.RS_ERR_INVALID_ARG   # the output must be planar
    assert call(inl=L.rs_layout_nchw(2, 3, 16, 16)) == B.RS_ERR_INVALID_ARG   # the source must be interleaved
    assert call(outl=L.rs_layout_nchw(1, 3, 32, 32)) == B.RS_ERR_INVALID_ARG  # N differs
    assert call(opt=B.options(impl=B.RS_IMPL_TILED)) == B.RS_ERR_INVALID_ARG
    o = B.options()
    o.flags = 2                                                   # an unknown flag
    assert call(opt=o) == B.RS_ERR_INVALID_ARG
    o = B.options(tile_h=8)
    o.flags = B.RS_FLAG_ANTIALIAS                                 # the antialiased form takes no chunk height
    assert call(opt=o) == B.RS_ERR_INVALID_ARG
    assert call(dst=Q + 1) == B.RS_ERR_ALIGNMENT                  # FP16 output on an odd address


def test_backward_workspace_flags(L):
    """rs_resize_backward_workspace on the host: RS_FLAG_ANTIALIAS sizes the
    transposed antialias tables (at a x0.25 downscale the stretched ranges
    put every input in more outputs than the point taps do, so the tables
    are wider), nearest has no antialiased form, and unknown flags are
    refused."""
    from paper_1001_1718_gb300 import _binding as B
    dy = L.rs_layout_nchw(1, 1, 16, 16)    # forward output (grad_out)
    dx = L.rs_layout_nchw(1, 1, 64, 64)    # forward input (grad_in)
    n = ctypes.c_size_t(0)

    def ws(method, flags):
        o = B.options()
        o.flags = flags
        st = L.rs_resize_backward_workspace(ctypes.byref(dy), ctypes.byref(dx), method, ctypes.byref(o), ctypes.byref(n))
        return st, n.value

    st0, plain = ws(B.RS_BILINEAR, 0)
    st1, aa = ws(B.RS_BILINEAR, B.RS_FLAG_ANTIALIAS)
    assert st0 == B.RS_OK and st1 == B.RS_OK
    # tables: H (8 + 4 K_y) + W (8 + 4 K_x), each section 256-byte aligned, plus the FP32 intermediate
    assert aa > plain
    assert ws(B.RS_NEAREST, B.RS_FLAG_ANTIALIAS)[0] == B.RS_ERR_INVALID_ARG
    assert ws(B.RS_BILINEAR, 2)[0] == B.RS_ERR_INVALID_ARG
    assert ws(B.RS_BICUBIC, B.RS_FLAG_ANTIALIAS)[0] == B.RS_OK
