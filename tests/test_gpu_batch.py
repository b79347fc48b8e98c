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
        # measured max: bf16x3 4.4e-6, fp16x3 2.3e-6 (the benchmark spec bars 1e-3 / 1e-5)
        assert err <= (1.5e-5 if form == "tc_bf16x3" else 7e-6)
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
    # stage 2 on CTA pairs (256x128 tiles), twice in a row
    batch.set_stage2_tiles(Plan.TILES_PAIR)
    for _ in range(2):
        for h in Hs:
            h.fill_(float("nan"))
        with torch.cuda.stream(st):
            batch.run(stream=st)
        st.synchronize()
        for k in range(len(scs)):
            assert O.rel_l2(Hs[k].cpu().numpy(), got[k]) <= 1e-5, k
    assert all(p.status() == 0 for p in plans)
    batch.close()


def _oracle_progressive_separable(sc):
    """The FP64 progressive hologram as the point-wise hologram of the progressively
    reconstructed object (pinned equal to the residual-map form), computed separably:
    fast enough for 1024x1024 objects at 2048x2048 holograms."""
    g = O.geometry_of(sc)
    lists = O.progressive_lists(sc["saliency"], sc["layer"], g.n_layers, scenes.THRESHOLDS_U8)
    A = O.progressive_object(sc["intensity"], sc["layer"], lists, g.n_layers)
    return O.pointwise_hologram_separable(A / 64.0, g)


@pytest.mark.parametrize("form,bar", [("tc_fp16x3", 1e-5), ("tc_bf16x3", 5e-5)])
def test_batch_at_bench_sizes(form, bar):
    """The sizes the 64-scene batch benchmark runs: a 512->1024 scene with 16 layers and a
    1024->2048 scene with 28 layers, beside small and mid scenes of very different K, in one
    batch with the autotuned stage-2 split.  Stage-2 work units then span scenes of very
    different K.  Every hologram is checked against the FP64 oracle."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2211_09938_gb300 import Plan, autotune
    from paper_2211_09938_gb300.cgh import Batch
    scs = [scenes.random_scene(611, 512, 1024, 16, sal_fraction=0.3),
           scenes.random_scene(612, 1024, 2048, 28, sal_fraction=0.45),
           scenes.random_scene(613, 128, 256, 4, sal_fraction=0.05),
           scenes.random_scene(614, 256, 512, 32, sal_fraction=0.6)]
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        plans = [Plan.for_scene(sc, stream=st) for sc in scs]
        I = [torch.from_numpy(sc["intensity"]).cuda() for sc in scs]
        L = [torch.from_numpy(sc["layer"]).cuda() for sc in scs]
        S = [torch.from_numpy(sc["saliency"]).cuda() for sc in scs]
        Hs = [torch.empty(sc["holo"], dtype=torch.complex64, device="cuda") for sc in scs]
        batch = Batch(plans, I, L, S, scenes.THRESHOLDS_U8, Hs, form=form, stream=st)
    tuned = autotune.tune_batch(batch, plans, form, st)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=st):
        batch.run(stream=st)
    for h in Hs:
        h.fill_(float("nan"))
    with torch.cuda.stream(st):
        g.replay()
    st.synchronize()
    for k, sc in enumerate(scs):
        err = O.rel_l2(Hs[k].cpu().numpy(), _oracle_progressive_separable(sc))
        print(f"batch {form} ({tuned}) scene {k} ({sc['intensity'].shape[0]}->{sc['holo'][0]}, "
              f"Z={len(sc['z'])}): rel-L2 {err:.2e}")
        assert err <= bar, (k, err)
    assert all(p.status() == 0 for p in plans)
    batch.close()
    for p in plans:
        p.close()
