"""The single-image autotuner on the GPU (rs_autotune).

rs_autotune times candidate kernels and shapes on the caller's buffers and
caches the fastest under the problem's key; later RS_IMPL_AUTO calls use it.
Every kernel computes each output element with the same FP32 operations in
the same order, so the tuned configuration's output must equal the default
configuration's byte for byte; AUTO must then report the tuned
configuration; and a save / clear / load round trip of the cache file must
restore it.
"""
import pytest
import torch

from paper_1001_1718_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rs():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1001_1718_gb300 as rs
    return rs


def _cfg(d):
    return {k: d[k] for k in ("impl", "tile_w", "tile_h", "threads", "waves")}


@pytest.mark.parametrize("method, size", [("bicubic", (1020, 1360)), ("bilinear", (333, 500))])
def test_autotune_single_image(rs, tmp_path, method, size):
    img = workloads.smooth_field_u8(41, 600, 800, 3)
    x = torch.from_numpy(img).cuda()
    rs.tune_cache_clear()
    default_cfg = rs.tile_config(x, size, method)
    y_default = rs.resize(x, size, method)
    best = rs.autotune(x, size, method)
    assert best["candidates"] >= 2 and best["best_us"] > 0 and best["best_us"] <= best["default_us"] * 1.0001
    tuned_cfg = rs.tile_config(x, size, method)
    assert tuned_cfg == _cfg(best), (tuned_cfg, best)
    y_tuned = rs.resize(x, size, method)
    torch.cuda.synchronize()
    assert torch.equal(y_tuned, y_default), (default_cfg, tuned_cfg)
    # cache file round trip
    path = tmp_path / "tune.txt"
    rs.tune_cache_save(str(path))
    assert path.read_text().startswith("# resample-tune v2")
    assert "gpu=" in path.read_text()
    rs.tune_cache_clear()
    assert rs.tile_config(x, size, method) == default_cfg
    rs.tune_cache_load(str(path))
    assert rs.tile_config(x, size, method) == tuned_cfg
    assert torch.equal(rs.resize(x, size, method), y_default)
    rs.tune_cache_clear()
    assert rs.debug_fault() == 0
