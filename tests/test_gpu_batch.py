"""Batches of uneven scenes through one persistent launch per GEMM stage: every scene's
hologram equals its single-scene result and the FP64 oracle, also under CUDA-graph replay."""
import numpy as np
import pytest

from oracle import cgh_oracle as O
from synth import scenes

pytestmark = pytest.mark.gpu


def make_scenes():
    return [scenes.random_scene(501, 32, 64, 2, sal_fraction=0.3),
            scenes.random_scene(502, 64, 128, 5, graded=True),
            scenes.random_scene(503, 128, 256, 7, sal_fraction=0.1),
            scenes.random_scene(504, 64, 256, 3, sal_fraction=0.5),
            scenes.tiny_scene(seed=505),
            scenes.random_scene(506, 96, 192, 4, graded=True)]


@pytest.mark.parametrize("form", ["tc_bf16x3", "tc_fp16x3"])
def test_batch_matches_single_scene_and_oracle(form):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2211_09938_gb300 import Plan
    from paper_2211_09938_gb300.cgh import Batch
    scs = make_scenes()
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        plans = [Plan.for_scene(sc, stream=st) for sc in scs]
        I = [torch.from_numpy(sc["intensity"]).cuda() for sc in scs]
        L = [torch.from_numpy(sc["layer"]).cuda() for sc in scs]
        S = [torch.from_numpy(sc["saliency"]).cuda() for sc in scs]
        Hs = [torch.empty(sc["holo"], dtype=torch.complex64, device="cuda") for sc in scs]
        batch = Batch(plans, I, L, S, scenes.THRESHOLDS_U8, Hs, form=form, stream=st)
        batch.run(stream=st)
    st.synchronize()
    got = [h.cpu().numpy().copy() for h in Hs]
    for k, sc in enumerate(scs):
        g = O.geometry_of(sc)
        ref_lists = O.progressive_lists(sc["saliency"], sc["layer"], g.n_layers, scenes.THRESHOLDS_U8)
        Href = O.progressive_hologram(sc["intensity"], sc["layer"], ref_lists, g)
        err = O.rel_l2(got[k], Href)
        print(f"batch {form} scene {k} ({sc['intensity'].shape[0]}->{sc['holo'][0]}, Z={g.n_layers}): {err:.2e}")
        assert err <= 1e-5
        with torch.cuda.stream(st):
            coeffs = plans[k].haar_decompose(I[k], L[k], stream=st)
            lists, counts = plans[k].progressive_lists(S[k], L[k], scenes.THRESHOLDS_U8, stream=st)
            H1 = plans[k].progressive_hologram(coeffs, lists, counts, form=form, stream=st)
        st.synchronize()
        # different K splits sum in a different FP32 order: both are within 1e-5 of FP64
        assert O.rel_l2(got[k], H1.cpu().numpy()) <= 1e-5
    # retuned split and CUDA-graph replay give the same holograms
    batch.set_tuning(8)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=st):
        batch.run(stream=st)
    for h in Hs:
        h.zero_()
    with torch.cuda.stream(st):
        g.replay()
    st.synchronize()
    for k in range(len(scs)):
        assert O.rel_l2(Hs[k].cpu().numpy(), got[k]) <= 1e-5
    batch.close()
