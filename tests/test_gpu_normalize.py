"""The fused serving pre-process (rs_resize_normalize) on the GPU: uint8
interleaved images resampled, normalised per channel and stored planar as
FP16 / BF16 / FP32 in one pass, element by element against the FP64 oracle
(resample, then (y - mean) / std, then round to the output dtype), under the
usual bracket rule with the FP32 bound taken in normalised units."""
import numpy as np
import pytest
import torch

from _parity import check

pytestmark = pytest.mark.gpu
BL, BC = 1, 2
MNAME = {BL: "bilinear", BC: "bicubic"}
TDT = {"f16": torch.float16, "bf16": torch.bfloat16, "f32": torch.float32}
MEAN = (123.675, 116.28, 103.53, 60.0)
STD = (58.395, 57.12, 57.375, 33.0)


@pytest.fixture(scope="module")
def rs():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1001_1718_gb300 as rs
    return rs


def _img(seed, shape):
    from paper_1001_1718_gb300 import workloads
    if len(shape) == 3:
        return workloads.smooth_field_u8(seed, *shape)
    return np.stack([workloads.smooth_field_u8(seed + k, *shape[1:]) for k in range(shape[0])])


CASES = [  # (shape (N,)H,W,C, (Ho, Wo), coord)
    ((300, 256, 3), (600, 512), 0),            # exact x2: the X2 form
    ((257, 411, 3), (517, 701), 0),            # general upscale, ragged strips
    ((3, 120, 200, 3), (240, 400), 0),         # batched exact x2
    ((2, 333, 180, 3), (97, 310), 1),          # batched, mixed up / down, half-pixel
    ((1000, 1500, 3), (256, 384), 0),          # downscale by ~3.9
    ((64, 96, 1), (128, 192), 0),              # one channel, exact x2
    ((77, 53, 4), (150, 101), 2),              # four channels, align-corners
]


@pytest.mark.parametrize("dtype", ["f16", "bf16", "f32"])
@pytest.mark.parametrize("method", [BL, BC])
def test_resize_normalize_matches_oracle(rs, oracle, dtype, method):
    for k, (shape, (Ho, Wo), coord) in enumerate(CASES):
        img = _img(300 + k, shape)
        C = shape[-1]
        x = torch.from_numpy(img).cuda()
        y = rs.resize_normalize(x, (Ho, Wo), MNAME[method], MEAN[:C], STD[:C], dtype=TDT[dtype],
                                coord=["asymmetric", "half_pixel", "align_corners"][coord])
        torch.cuda.synchronize()
        ref = oracle.resize_normalize(img.astype(np.float64), Ho, Wo, method, MEAN[:C], STD[:C], coord=coord)
        assert tuple(y.shape) == ref.shape
        check(y, ref, dtype, method, 255.0 / min(STD[:C]), f"normalize {dtype} {MNAME[method]} {shape}->{Ho}x{Wo}")
    assert rs.debug_fault() == 0


def test_resize_normalize_pitched_views_and_out(rs, oracle):
    """A source view with a row pitch wider than its pixels, and an output
    written into a pitched planar view of a larger buffer: the guard bands
    around the written planes stay untouched."""
    img = _img(400, (90, 140, 3))
    big = torch.zeros((90, 150, 3), dtype=torch.uint8)
    big[:, 3:143] = torch.from_numpy(img)
    view = big.cuda()[:, 3:143]
    guard = torch.full((3, 181, 281), 7.0, dtype=torch.float16, device="cuda")
    out = guard[:, :180, :280]
    assert not out.is_contiguous()
    rs.resize_normalize(view, (180, 280), "bicubic", MEAN[:3], STD[:3], out=out)
    torch.cuda.synchronize()
    ref = oracle.resize_normalize(img.astype(np.float64), 180, 280, BC, MEAN[:3], STD[:3])
    check(out, ref, "f16", BC, 255.0 / min(STD[:3]), "normalize pitched view")
    assert (guard[:, 180:] == 7.0).all() and (guard[:, :, 280:] == 7.0).all()
    with pytest.raises(ValueError):   # the binding wants the output's shape
        rs.resize_normalize(view, (180, 280), "bicubic", MEAN[:3], STD[:3], out=guard)


def test_resize_normalize_refusals(rs):
    x = torch.zeros((8, 8, 3), dtype=torch.uint8, device="cuda")
    with pytest.raises(rs.ResampleError) as e:
        rs.resize_normalize(x, (16, 16), "nearest", MEAN[:3], STD[:3])
    assert e.value.status == 2
    with pytest.raises(rs.ResampleError):
        rs.resize_normalize(x, (16, 16), "bilinear", MEAN[:3], (1.0, 0.0, 1.0))
    with pytest.raises(ValueError):
        rs.resize_normalize(x.float(), (16, 16), "bilinear", MEAN[:3], STD[:3])
    with pytest.raises(ValueError):
        rs.resize_normalize(x, (16, 16), "bilinear", MEAN[:2], STD[:2])


@pytest.mark.parametrize("method", [BL, BC])
def test_resize_normalize_antialias(rs, oracle, method):
    """The fused pre-process with RS_FLAG_ANTIALIAS: serving-style
    downscales of uint8 frames (the antialiased window form up to 8 taps per
    axis, the many-tap tiled kernel beyond: a 1280x720 frame to 160x90),
    against the FP64 antialias definition followed by the normalisation."""
    cases = [((2, 240, 320, 3), (120, 160), torch.float16), ((1, 300, 410, 3), (96, 131), torch.bfloat16),
             ((3, 100, 90, 1), (100, 90), torch.float32), ((1, 720, 1280, 3), (90, 160), torch.float16),
             ((2, 333, 250, 4), (41, 29), torch.float32), ((1, 500, 40, 1), (20, 2), torch.bfloat16),
             ((3, 4, 300, 3), (1, 150), torch.float16)]
    names = {torch.float16: "f16", torch.bfloat16: "bf16", torch.float32: "f32"}
    for k, (shape, (Ho, Wo), dt) in enumerate(cases):
        img = _img(500 + k, shape)
        x = torch.from_numpy(img).cuda()
        C = shape[-1]
        y = rs.resize_normalize(x, (Ho, Wo), MNAME[method], MEAN[:C], STD[:C], dtype=dt, antialias=True)
        torch.cuda.synchronize()
        ref = np.stack([((oracle.resize_aa(im.astype(np.float64), Ho, Wo, method) - np.array(MEAN[:C])) /
                         np.array(STD[:C])).transpose(2, 0, 1) for im in img])
        check(y, ref, names[dt], method, 255.0 / min(STD[:C]),
              f"normalize antialias {MNAME[method]} {shape}->{Ho}x{Wo}")
    assert rs.debug_fault() == 0
