"""The whole hot path (tables, DWT, selection, superposition) captured as one CUDA graph
and replayed gives the eager result (up to the order of the atomic additions)."""
import numpy as np
import pytest

from oracle import cgh_oracle as O
from synth import scenes

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("form", ["direct_lut", "tc_bf16x3"])
def test_graph_replay_matches_eager(form):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2211_09938_gb300 import Plan
    sc = scenes.tiny_scene()
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        plan = Plan.for_scene(sc, stream=st)
        I = torch.from_numpy(sc["intensity"]).cuda()
        L = torch.from_numpy(sc["layer"]).cuda()
        S = torch.from_numpy(sc["saliency"]).cuda()
        coeffs = torch.empty((plan.n_layers, 64, 64), dtype=torch.int32, device="cuda")
        counts = torch.zeros((4, 2), dtype=torch.int32, device="cuda")
        lists = [torch.empty(plan.max_blocks(3 if k == 0 else k), dtype=torch.int32, device="cuda")
                 for k in range(4)]
        H = torch.empty((256, 256), dtype=torch.complex64, device="cuda")

    def step():
        plan.build_tables(stream=st)
        plan.haar_decompose(I, L, coeffs, stream=st)
        plan.progressive_lists(S, L, scenes.THRESHOLDS_U8, counts=counts, lists=lists, stream=st)
        plan.progressive_hologram(coeffs, lists, counts, holo=H, form=form, stream=st)

    with torch.cuda.stream(st):
        step()
    st.synchronize()
    eager = H.cpu().numpy().copy()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=st):
        step()
    for _ in range(2):
        H.zero_()
        with torch.cuda.stream(st):
            g.replay()
        st.synchronize()
        assert O.rel_l2(H.cpu().numpy(), eager) < 1e-6
    ref_lists = O.progressive_lists(sc["saliency"], sc["layer"], 4, scenes.THRESHOLDS_U8)
    Href = O.progressive_hologram(sc["intensity"], sc["layer"], ref_lists, O.geometry_of(sc))
    assert O.rel_l2(H.cpu().numpy(), Href) < 1e-5
