"""The batched entry point that allocates nothing.

rs_resize_batched_noalloc serves callers that cannot obtain device memory
for a workspace (a framework's allocator owns the device memory, a serving
path forbids allocation after start-up, a plugin host only hands out its
input and output buffers): its work list lives in a fixed array inside the
library. This test calls it through the C ABI twice in a row, on two
different ragged batches, and checks each result against the workspace
entry point rs_resize_batched on the same inputs (the same kernel, so the
outputs must agree bit for bit). It also checks the over-capacity refusal.

This file sorts last so that a run stopping at the first failure has run
every other test first; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu
METHODS = ("nearest", "bilinear", "bicubic")


@pytest.fixture(scope="module")
def rs():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1001_1718_gb300 as rs
    return rs


def _batch(seed, n):
    r = np.random.default_rng(seed)
    srcs, sizes, methods = [], [], []
    for k in range(n):
        H, W, C = int(r.integers(8, 400)), int(r.integers(8, 400)), int(r.choice([1, 3, 4]))
        s = float(r.uniform(0.5, 4.0))
        srcs.append(torch.from_numpy(r.integers(0, 256, (H, W, C)).astype(np.uint8)).cuda())
        sizes.append((max(1, int(H * s)), max(1, int(W * s))))
        methods.append(METHODS[k % 3])
    return srcs, sizes, methods


def _noalloc(rs, srcs, outs, methods):
    from paper_1001_1718_gb300 import _binding as B
    arr, n = rs._descs(srcs, outs, methods)
    o = B.options()
    st = torch.cuda.current_stream().cuda_stream
    return B.lib().rs_resize_batched_noalloc(arr, n, B.RS_U8, ctypes.byref(o), st)


def test_noalloc_matches_workspace_entry_point(rs):
    for seed, n in ((11, 40), (12, 17)):            # two calls in a row, different batches
        srcs, sizes, methods = _batch(seed, n)
        ref = rs.resize_batched(srcs, sizes, methods)
        outs = [torch.full_like(y, 7) for y in ref]
        assert _noalloc(rs, srcs, outs, methods) == 0
        torch.cuda.synchronize()
        for k, (a, b) in enumerate(zip(outs, ref)):
            assert torch.equal(a, b), f"batch {seed} image {k} differs"
    assert rs.debug_fault() == 0


def test_noalloc_rejects_more_images_than_it_holds(rs):
    from paper_1001_1718_gb300 import _binding as B
    x = torch.zeros(4, 4, 1, dtype=torch.uint8, device="cuda")
    n = B.RS_NOALLOC_MAX_IMAGES + 1
    outs = [torch.full((8, 8, 1), 3, dtype=torch.uint8, device="cuda") for _ in range(n)]
    assert _noalloc(rs, [x] * n, outs, ["bilinear"] * n) == B.RS_ERR_WORKSPACE
    torch.cuda.synchronize()
    assert all((y == 3).all() for y in outs[:4])   # nothing was launched
