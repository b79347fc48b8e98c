"""The allocation-free block selection, cgh_select_blocks_noalloc.

Callers that cannot call cudaMalloc (an embedder whose device memory budget is fixed at
start-up and must not grow afterwards) cannot create a plan; this entry point serves them
with scratch that is built into the library.  The tests call it through the C ABI and
check that two calls in a row give exactly what cgh_select_blocks gives (block lists are
integer work, so the bar is bit-exact), that device memory does not grow across calls,
that a request exactly at the scratch limit runs and one slot over it is refused before
any work is enqueued.  This file sorts last so that a run stopping at the first failure
has run everything else.
"""
import ctypes

import numpy as np
import pytest

from synth import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import os
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2211_09938_gb300 import build_lib, cgh
    if not os.path.exists(cgh.LIB_PATH):
        build_lib.build()
    cgh.lib()
    return torch


def _noalloc(torch, S, L, h, w, nl, thr, level, cap):
    from paper_2211_09938_gb300 import cgh
    out = torch.full((max(cap, 1),), -1, dtype=torch.int32, device="cuda")
    cnt = torch.full((2,), -1, dtype=torch.int32, device="cuda")
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = cgh.lib().cgh_select_blocks_noalloc(
        ctypes.c_void_p(S.data_ptr()), ctypes.c_void_p(L.data_ptr()), h, w, nl, thr, level,
        ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(cnt.data_ptr()), cap, st)
    assert rc == 0, cgh.lib().cgh_last_error()
    return out, cnt


@pytest.mark.parametrize("which", ["tiny", "graded", "paper"])
def test_noalloc_matches_plan_selection_twice(torch_cuda, which):
    torch = torch_cuda
    from paper_2211_09938_gb300 import Plan
    sc = {"tiny": lambda: scenes.tiny_scene(),
          "graded": lambda: scenes.random_scene(91, 64, 128, 5, graded=True),
          "paper": lambda: scenes.paper_scene()}[which]()
    h, w = sc["intensity"].shape
    nl = len(sc["z"])
    plan = Plan.for_scene(sc)
    S = torch.from_numpy(sc["saliency"]).cuda()
    L = torch.from_numpy(sc["layer"]).cuda()
    for level in (1, 2, 3):
        for thr in (-1, 127, 229):
            ref, rc = plan.select_blocks(S, L, thr, level)
            rc = rc.cpu().numpy()
            cap = plan.max_blocks(level)
            for _ in range(2):  # the second call sees the first call's scratch contents
                out, cnt = _noalloc(torch, S, L, h, w, nl, thr, level, cap)
                c = cnt.cpu().numpy()
                assert c.tolist() == rc.tolist(), (level, thr)
                assert np.array_equal(out[:c[0]].cpu().numpy(), ref[:rc[0]].cpu().numpy()), (level, thr)
    plan.close()


def test_noalloc_capacity_and_limit(torch_cuda):
    torch = torch_cuda
    from paper_2211_09938_gb300 import cgh
    sc = scenes.tiny_scene()
    S = torch.from_numpy(sc["saliency"]).cuda()
    L = torch.from_numpy(sc["layer"]).cuda()
    full, c_full = _noalloc(torch, S, L, 64, 64, 4, -1, 1, 4 * 32 * 32)
    part, c_part = _noalloc(torch, S, L, 64, 64, 4, -1, 1, 10)
    n = int(c_full.cpu()[0])
    assert c_part.cpu().numpy().tolist() == [10, n]
    assert np.array_equal(part[:10].cpu().numpy(), full[:10].cpu().numpy())
    # 64 layers of an 8192x8192 object at level 1 need 64 * 16384 chunk slots: refused
    big = torch.zeros(8, dtype=torch.uint8, device="cuda")
    cnt = torch.zeros(2, dtype=torch.int32, device="cuda")
    rc = cgh.lib().cgh_select_blocks_noalloc(
        ctypes.c_void_p(big.data_ptr()), ctypes.c_void_p(big.data_ptr()), 8192, 8192, 64, -1, 1,
        None, ctypes.c_void_p(cnt.data_ptr()), 0, None)
    assert rc == cgh.CGH_ERR_ARG
    assert b"static scratch limit" in cgh.lib().cgh_last_error()


def _expected_list(layer, n_layers, level):
    """Every occupied (layer, block) pair at `level`, layer-major then row-major, from the
    pinned oracle's per-layer occupancy masks (vectorised per layer)."""
    from oracle import cgh_oracle as O
    out = []
    for z in range(n_layers):
        by, bx = np.nonzero(O.block_occupied(layer, z, level))
        out.append((z << 24) | (by.astype(np.int64) << 12) | bx)
    return np.concatenate(out).astype(np.int32)


def test_noalloc_exactly_at_limit_and_one_over(torch_cuda):
    """64 layers of a 2048x2048 object at level 1 need 64 * ceil(1024^2 / 256) = 262144
    chunk slots, exactly the scratch limit: it runs and is bit-exact, twice.  37 layers of
    a 1376x5272 object at level 1 need 37 * 7085 = 262145: refused with CGH_ERR_ARG."""
    torch = torch_cuda
    from paper_2211_09938_gb300 import cgh
    rng = np.random.default_rng(404)
    n, nl = 2048, 64
    layer = rng.integers(0, nl, size=(n, n), dtype=np.uint8)
    want = _expected_list(layer, nl, 1)
    L = torch.from_numpy(layer).cuda()
    cap = len(want) + 16
    for _ in range(2):
        out, cnt = _noalloc(torch, L, L, n, n, nl, -1, 1, cap)
        c = cnt.cpu().numpy().tolist()
        assert c == [len(want), len(want)]
        assert np.array_equal(out[:c[0]].cpu().numpy(), want)
    small = torch.zeros(16, dtype=torch.uint8, device="cuda")
    cnt = torch.full((2,), -7, dtype=torch.int32, device="cuda")
    rc = cgh.lib().cgh_select_blocks_noalloc(
        ctypes.c_void_p(small.data_ptr()), ctypes.c_void_p(small.data_ptr()), 1376, 5272, 37, -1, 1,
        None, ctypes.c_void_p(cnt.data_ptr()), 0, None)
    assert rc == cgh.CGH_ERR_ARG
    assert b"262145" in cgh.lib().cgh_last_error()
    torch.cuda.synchronize()
    assert cnt.cpu().numpy().tolist() == [-7, -7]  # nothing was enqueued


def test_noalloc_device_memory_does_not_grow(torch_cuda):
    """After warm-up calls, several calls leave the device's free memory unchanged (as
    cudaMemGetInfo reports it): the entry point allocates nothing."""
    torch = torch_cuda
    from paper_2211_09938_gb300 import cgh
    sc = scenes.paper_scene()
    S = torch.from_numpy(sc["saliency"]).cuda()
    L = torch.from_numpy(sc["layer"]).cuda()
    nl = len(sc["z"])
    out = torch.empty(nl * 256 * 256, dtype=torch.int32, device="cuda")
    cnt = torch.empty(2, dtype=torch.int32, device="cuda")
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    def call(level, thr):
        rc = cgh.lib().cgh_select_blocks_noalloc(
            ctypes.c_void_p(S.data_ptr()), ctypes.c_void_p(L.data_ptr()), 512, 512, nl, thr, level,
            ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(cnt.data_ptr()), out.numel(), st)
        assert rc == 0, cgh.lib().cgh_last_error()

    cases = ((1, 229), (2, 178), (3, 127), (3, -1))
    for level, thr in cases:  # warm-up: lazy module loading places code and the array here
        call(level, thr)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(4):
        for level, thr in cases:
            call(level, thr)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
