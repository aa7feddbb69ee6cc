"""GPU batched path: one persistent launch over ragged images of different
sizes, scales, channel counts and methods, against the FP64 oracle and
against per-image launches (bit for bit: the per-element arithmetic does
not depend on the tiling); the replayable graph plan; the full 256-image
workload, every element."""
import numpy as np
import pytest
import torch

from _parity import check, aa_taps

pytestmark = pytest.mark.gpu
MN = {0: "nearest", 1: "bilinear", 2: "bicubic"}


@pytest.fixture(scope="module")
def rs():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1001_1718_gb300 as rs
    return rs


def _batch(seed, n, dtype=torch.uint8):
    r = np.random.default_rng(seed)
    srcs, sizes, methods, host = [], [], [], []
    for k in range(n):
        H, W = int(r.integers(5, 300)), int(r.integers(5, 300))
        C = int(r.choice([1, 3, 4]))
        s = float(r.uniform(0.5, 4.0))
        Ho, Wo = max(1, int(H * s)), max(1, int(W * s * r.uniform(0.8, 1.25)))
        if dtype == torch.uint8:
            x = r.integers(0, 256, (H, W, C)).astype(np.uint8)
        else:
            x = r.standard_normal((H, W, C)).astype(np.float32)
        host.append(x)
        srcs.append(torch.from_numpy(x).cuda())
        sizes.append((Ho, Wo))
        methods.append(MN[k % 3])
    return srcs, sizes, methods, host


@pytest.mark.parametrize("dtype", [torch.uint8, torch.float32])
def test_batched_matches_oracle_and_single(rs, oracle, dtype):
    srcs, sizes, methods, host = _batch(3, 24, dtype)
    outs = rs.resize_batched(srcs, sizes, methods)
    torch.cuda.synchronize()
    dn = "u8" if dtype == torch.uint8 else "f32"
    for x, s, m, y, h in zip(srcs, sizes, methods, outs, host):
        single = rs.resize(x, s, m)
        assert torch.equal(single, y)
        code = rs.METHODS[m]
        check(y, oracle.resize(h.astype(np.float64), s[0], s[1], code), dn, code,
              float(np.abs(h).max()), f"batched {m} {h.shape}->{s}")
    assert rs.debug_fault() == 0


@pytest.mark.parametrize("coord", ["half_pixel", "align_corners"])
def test_batched_coordinate_maps(rs, oracle, coord):
    """The batch under the other coordinate maps: each image equals the
    single-image call with the same map and matches the oracle."""
    srcs, sizes, methods, host = _batch(5, 12)
    outs = rs.resize_batched(srcs, sizes, methods, coord=coord)
    torch.cuda.synchronize()
    code = {"half_pixel": 1, "align_corners": 2}[coord]
    for x, s, m, y, h in zip(srcs, sizes, methods, outs, host):
        assert torch.equal(rs.resize(x, s, m, coord=coord), y)
        check(y, oracle.resize(h.astype(np.float64), s[0], s[1], rs.METHODS[m], code), "u8", rs.METHODS[m],
              float(np.abs(h).max()), f"batched {coord} {m} {h.shape}->{s}")
    assert rs.debug_fault() == 0


def test_plan_replay(rs):
    srcs, sizes, methods, _ = _batch(4, 16)
    outs = [torch.zeros((h, w, x.shape[2]), dtype=torch.uint8, device="cuda") for x, (h, w) in zip(srcs, sizes)]
    plan = rs.BatchedPlan(srcs, outs, methods)
    plan.launch()
    torch.cuda.synchronize()
    ref = [rs.resize(x, s, m) for x, s, m in zip(srcs, sizes, methods)]
    assert all(torch.equal(a, b) for a, b in zip(outs, ref))
    # the graph reads the same buffers: new input pixels give new outputs
    for x in srcs:
        x.copy_(255 - x)
    for o in outs:
        o.zero_()
    plan.launch()
    plan.launch()
    torch.cuda.synchronize()
    ref = [rs.resize(x, s, m) for x, s, m in zip(srcs, sizes, methods)]
    assert all(torch.equal(a, b) for a, b in zip(outs, ref))
    plan.close()


def test_pitched_images_and_invalid(rs):
    x = torch.randint(0, 256, (50, 70 * 3 + 5), dtype=torch.uint8, device="cuda")
    src = x[:, :210].view(50, 70, 3)
    yb = torch.zeros(100, 140 * 3 + 7, dtype=torch.uint8, device="cuda")
    dst = yb[:, :420].view(100, 140, 3)
    rs.resize_batched([src], [(100, 140)], ["bicubic"], outs=[dst])
    assert torch.equal(dst, rs.resize(src, (100, 140), "bicubic"))
    assert (yb[:, 420:] == 0).all()
    # overlapping destination and source is rejected
    with pytest.raises(rs.ResampleError):
        rs.resize_batched([src, src], [(100, 140), (20, 20)], ["bilinear", "bilinear"], outs=[dst, src[:20, :20]])


def test_full_batch_workload(rs, oracle):
    """256 RGB images, H and W uniform on 64..2048, scale uniform on [0.5, 4),
    methods alternating bilinear / bicubic, launched as the benchmark times
    them (the replayable plan, AUTO item shapes): every element of every image
    against the oracle's full output; every 16th image against a per-image
    launch."""
    from paper_1001_1718_gb300 import workloads
    items = workloads.batch_spec(seed=4)
    imgs = workloads.batch_images(items)
    srcs = [torch.from_numpy(im).cuda() for im in imgs]
    sizes = [(it.Ho, it.Wo) for it in items]
    methods = [MN[it.method] for it in items]
    outs = [torch.full((h, w, 3), 77, dtype=torch.uint8, device="cuda") for h, w in sizes]
    plan = rs.BatchedPlan(srcs, outs, methods)
    plan.launch()
    torch.cuda.synchronize()
    off_by_one = 0
    for k, (it, im, y) in enumerate(zip(items, imgs, outs)):
        ref = oracle.resize(im.astype(np.float64), it.Ho, it.Wo, it.method)
        st = check(y, ref, "u8", it.method, 255.0, f"batch image {k}")
        off_by_one += st.get("u8_off_by_one", 0)
        if k % 16 == 0:
            assert torch.equal(y, rs.resize(srcs[k], sizes[k], methods[k]))
        del ref
    plan.close()
    assert rs.debug_fault() == 0


def test_batch_item_shapes_agree(rs):
    """Window items of any band / chunk height and plain tiles compute each
    output element with the same operations: every shape gives the same
    bytes as the default; tuning picks one of them and changes nothing."""
    srcs, sizes, methods, _ = _batch(9, 20)
    ref = rs.resize_batched(srcs, sizes, methods)
    for impl, tile in (("window", (1, 0)), ("window", (32, 4)), ("window", (256, 8)), ("window", (77, 16)),
                       ("tiled", None), ("tiled", (256, 8))):
        got = rs.resize_batched(srcs, sizes, methods, impl=impl, tile=tile)
        assert all(torch.equal(a, b) for a, b in zip(got, ref)), (impl, tile)
    outs = [torch.empty_like(y) for y in ref]
    best = rs.autotune_batched(srcs, outs, methods)
    assert best["impl"] in ("window", "tiled") and best["candidates"] >= 2
    assert best["best_us"] > 0 and best["best_us"] <= best["default_us"]
    assert all(torch.equal(a, b) for a, b in zip(outs, ref))
    plan = rs.BatchedPlan(srcs, [torch.zeros_like(y) for y in ref], methods)   # uses the tuned shape
    plan.launch()
    torch.cuda.synchronize()
    assert all(torch.equal(a, b) for a, b in zip(plan.outs, ref))
    plan.close()
    with pytest.raises(rs.ResampleError):
        rs.resize_batched(srcs, sizes, methods, impl="stream")
    with pytest.raises(rs.ResampleError):
        rs.resize_batched(srcs, sizes, methods, impl="window", tile=(300, 8))
    rs.tune_cache_clear()
    assert rs.debug_fault() == 0


def _aa_batch(seed, n, dtype):
    """Ragged batch of mostly downscales (x0.08 to x1.6): items within the
    window forms' 8 taps per axis and items beyond them (many-tap tiles)."""
    from _parity import to_storage, as_f64
    r = np.random.default_rng(seed)
    srcs, sizes, methods, host = [], [], [], []
    for k in range(n):
        H, W = int(r.integers(20, 400)), int(r.integers(20, 400))
        C = int(r.choice([1, 3, 4]))
        s = float(r.uniform(0.08, 1.6))
        Ho, Wo = max(1, int(H * s)), max(1, int(W * s * r.uniform(0.8, 1.25)))
        x = r.integers(0, 256, (H, W, C)).astype(np.float64) if dtype == "u8" else r.standard_normal((H, W, C)) * 3
        t = to_storage(x, dtype)
        host.append(as_f64(t))
        srcs.append(t.cuda())
        sizes.append((Ho, Wo))
        methods.append(MN[1 + k % 2])
    return srcs, sizes, methods, host


@pytest.mark.parametrize("dtype", ["u8", "f16", "f32"])
def test_batched_antialias(rs, oracle, dtype):
    """RS_FLAG_ANTIALIAS on the batch (window items and many-tap tiles in one
    call), the replayable plan and the all-tiles shape, against the FP64
    antialias definition under the storage rule; uint8 / FP16 items within
    the window forms' 8 taps per axis equal the single-image antialiased call
    (the same kernel's arithmetic; beyond 8 taps the single-image call sums
    y first on vertical downscales, the batch's tiles x first)."""
    srcs, sizes, methods, host = _aa_batch(31, 20, dtype)
    outs = rs.resize_batched(srcs, sizes, methods, antialias=True)
    torch.cuda.synchronize()
    for x, s, m, y, h in zip(srcs, sizes, methods, outs, host):
        code = rs.METHODS[m]
        check(y, oracle.resize_aa(h, s[0], s[1], code), dtype, code, float(np.abs(h).max()),
              f"batched antialias {m} {h.shape}->{s}")
        taps = max(aa_taps(h.shape[0], s[0], code), aa_taps(h.shape[1], s[1], code))
        if dtype != "f32" and taps <= 8:
            assert torch.equal(rs.resize(x, s, m, antialias=True), y), (m, h.shape, s)
    plan_outs = [torch.zeros_like(y) for y in outs]
    plan = rs.BatchedPlan(srcs, plan_outs, methods, antialias=True)
    plan.launch()
    torch.cuda.synchronize()
    assert all(torch.equal(a, b) for a, b in zip(plan_outs, outs))
    tiled = rs.resize_batched(srcs, sizes, methods, antialias=True, impl="tiled")
    torch.cuda.synchronize()
    for s, m, y, h in zip(sizes, methods, tiled, host):
        code = rs.METHODS[m]
        check(y, oracle.resize_aa(h, s[0], s[1], code), dtype, code, float(np.abs(h).max()),
              f"batched antialias tiled {m} {h.shape}->{s}")
    with pytest.raises(rs.ResampleError):   # nearest has no antialias filter
        rs.resize_batched(srcs[:2], sizes[:2], ["nearest", "bilinear"], antialias=True)
    assert rs.debug_fault() == 0
