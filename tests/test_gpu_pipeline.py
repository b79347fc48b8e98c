"""The streaming pipeline: scenes submitted back to back through two device slots (copies
overlapping compute; with concurrent slots, one plan and compute stream each, so that
consecutive scenes' steps overlap) give exactly the holograms of the plain library calls,
scene by scene, for both superposition forms."""
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


@pytest.mark.parametrize("form,graphs,concurrent,depth", [("tc_bf16x3", True, False, 2), ("direct_lut", False, False, 2),
                                                           ("tc_bf16x3", True, True, 3), ("tc_fp16x3", False, True, 2)])
def test_pipeline_matches_direct_calls(torch_cuda, form, graphs, concurrent, depth):
    torch = torch_cuda
    from paper_2211_09938_gb300 import Plan
    from paper_2211_09938_gb300.pipeline import ProgressivePipeline
    base = scenes.random_scene(120, 64, 128, 3, graded=True)
    plan = Plan.for_scene(base, flags=Plan.DETERMINISTIC)
    seeds = [121, 122, 123, 124, 125]
    scs = [scenes.random_scene(sd, 64, 128, 3, graded=True) for sd in seeds]
    pipe = ProgressivePipeline(plan, scenes.THRESHOLDS_U8, form=form, depth=depth, graphs=graphs,
                               concurrent=concurrent)
    outs = [torch.empty((128, 128), dtype=torch.complex64).pin_memory() for _ in scs]
    for sc, hH in zip(scs, outs):
        pipe.submit(torch.from_numpy(sc["intensity"]).pin_memory(), torch.from_numpy(sc["layer"]).pin_memory(),
                    torch.from_numpy(sc["saliency"]).pin_memory(), hH)
    pipe.synchronize()
    assert pipe.status() == 0
    for sc, hH in zip(scs, outs):
        I = torch.from_numpy(sc["intensity"]).cuda()
        L = torch.from_numpy(sc["layer"]).cuda()
        S = torch.from_numpy(sc["saliency"]).cuda()
        coeffs = plan.haar_decompose(I, L)
        lists, counts = plan.progressive_lists(S, L, scenes.THRESHOLDS_U8)
        H = plan.progressive_hologram(coeffs, lists, counts, form=form).cpu()
        torch.cuda.synchronize()
        assert torch.equal(H, hH), (form, np.abs((H - hH).numpy()).max())


def test_pipeline_concurrent_paper_scale(torch_cuda):
    """Four concurrent slots at paper scale (512x512 objects, 16 layers, 1024x1024 holograms):
    the slots' single-launch selections (352 CTAs each, cooperative) and GEMMs overlap on the
    GPU; every bounded wait completes (status 0) and each hologram equals the plain calls'."""
    torch = torch_cuda
    from paper_2211_09938_gb300 import Plan
    from paper_2211_09938_gb300.pipeline import ProgressivePipeline
    base = scenes.paper_scene(seed=2100)
    plan = Plan.for_scene(base, flags=Plan.DETERMINISTIC)
    scs = [scenes.paper_scene(seed=2101 + k) for k in range(8)]
    pipe = ProgressivePipeline(plan, scenes.THRESHOLDS_U8, form="tc_bf16x3", depth=4, concurrent=True)
    outs = [torch.empty((1024, 1024), dtype=torch.complex64).pin_memory() for _ in scs]
    for rep in range(3):  # the later passes overlap slots that are already warm
        for sc, hH in zip(scs, outs):
            pipe.submit(torch.from_numpy(sc["intensity"]).pin_memory(), torch.from_numpy(sc["layer"]).pin_memory(),
                        torch.from_numpy(sc["saliency"]).pin_memory(), hH)
    assert pipe.status() == 0
    for sc, hH in zip(scs[:3], outs[:3]):
        I = torch.from_numpy(sc["intensity"]).cuda()
        L = torch.from_numpy(sc["layer"]).cuda()
        S = torch.from_numpy(sc["saliency"]).cuda()
        coeffs = plan.haar_decompose(I, L)
        lists, counts = plan.progressive_lists(S, L, scenes.THRESHOLDS_U8)
        H = plan.progressive_hologram(coeffs, lists, counts, form="tc_bf16x3").cpu()
        torch.cuda.synchronize()
        assert torch.equal(H, hH)
