"""The batched entry point that allocates nothing.

rs_resize_batched_noalloc serves callers that cannot obtain device memory
for a workspace (a framework's allocator owns the device memory, a serving
path forbids allocation after start-up, a plugin host only hands out its
input and output buffers): its work list lives in a fixed array inside the
library. These tests call it through the C ABI twice in a row, on two
different ragged batches (with a synchronisation between the calls, and
without one on the same stream), in uint8 and FP32, and check each result
against the workspace entry point rs_resize_batched on the same inputs (the
same kernels, so the outputs must agree bit for bit). They also check the
over-capacity refusal and the refusal while the stream is being captured.

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


def _batch(seed, n, dtype=torch.uint8):
    r = np.random.default_rng(seed)
    srcs, sizes, methods = [], [], []
    for k in range(n):
        H, W, C = int(r.integers(8, 400)), int(r.integers(8, 400)), int(r.choice([1, 3, 4]))
        s = float(r.uniform(0.5, 4.0))
        if dtype == torch.uint8:
            x = torch.from_numpy(r.integers(0, 256, (H, W, C)).astype(np.uint8))
        else:
            x = torch.from_numpy(r.standard_normal((H, W, C))).to(dtype)
        srcs.append(x.cuda())
        sizes.append((max(1, int(H * s)), max(1, int(W * s))))
        methods.append(METHODS[k % 3])
    return srcs, sizes, methods


def _noalloc(rs, srcs, outs, methods):
    from paper_1001_1718_gb300 import _binding as B
    arr, n = rs._descs(srcs, outs, methods)
    o = B.options()
    st = torch.cuda.current_stream().cuda_stream
    return B.lib().rs_resize_batched_noalloc(arr, n, rs._dtype(srcs[0]), ctypes.byref(o), st)


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


@pytest.mark.parametrize("dtype", [torch.uint8, torch.float32])
def test_noalloc_back_to_back_on_one_stream(rs, dtype):
    """Two calls queued on one stream with no synchronisation between them:
    the second call refills the shared array only after the first call's
    kernels (same stream), so both batches come out right."""
    batches = [_batch(seed, n, dtype) for seed, n in ((21, 33), (22, 26))]
    refs = [rs.resize_batched(*b) for b in batches]
    torch.cuda.synchronize()
    outs = [[torch.full_like(y, 5) for y in ref] for ref in refs]
    for (srcs, _, methods), o in zip(batches, outs):
        assert _noalloc(rs, srcs, o, methods) == 0
    torch.cuda.synchronize()
    for b, (o, ref) in enumerate(zip(outs, refs)):
        for k, (a, r) in enumerate(zip(o, ref)):
            assert torch.equal(a, r), f"{dtype} batch {b} image {k} differs"
    assert rs.debug_fault() == 0


def test_noalloc_refuses_a_capturing_stream(rs):
    """The descriptors are copied from host staging memory that the next call
    refills, so a call on a stream under capture is refused and does nothing."""
    from paper_1001_1718_gb300 import _binding as B
    srcs, sizes, methods = _batch(31, 3)
    outs = [torch.full((h, w, s.shape[2]), 9, dtype=torch.uint8, device="cuda") for s, (h, w) in zip(srcs, sizes)]
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        probe = torch.zeros(1, device="cuda") + 1
        status = _noalloc(rs, srcs, outs, methods)
    assert status == B.RS_ERR_UNSUPPORTED
    del graph, probe
    torch.cuda.synchronize()
    assert all((y == 9).all() for y in outs)


def test_noalloc_rejects_more_images_than_it_holds(rs):
    from paper_1001_1718_gb300 import _binding as B
    x = torch.zeros(4, 4, 1, dtype=torch.uint8, device="cuda")
    n = B.RS_NOALLOC_MAX_IMAGES + 1
    outs = [torch.full((8, 8, 1), 3, dtype=torch.uint8, device="cuda") for _ in range(n)]
    assert _noalloc(rs, [x] * n, outs, ["bilinear"] * n) == B.RS_ERR_WORKSPACE
    torch.cuda.synchronize()
    assert all((y == 3).all() for y in outs[:4])   # nothing was launched
