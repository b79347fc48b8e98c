"""Precision workload: the paper-scale scene (512x512 object) at a 2048x2048 hologram with
32 layers.  Every form against the FP64 oracle, for the full hologram and layer by layer
(each layer's own work lists), with rel-L2 and max-abs error printed.
Bars: direct FP32 <= 1e-5 rel-L2; per layer every form <= 1e-5 (fp16/bf16 hi+lo: 1e-5 /
1e-3); the full 32-layer hologram with the default chains <= 1e-5 for fp16 hi+lo (chains of
at most 32 K steps; measured 6.7e-6) and <= 7e-5 for bf16 hi+lo (chains up to 128; measured
2.2e-5, the benchmark spec bar 1e-3); with 8-step chains <= 1e-5 for both."""
import numpy as np
import pytest

from oracle import cgh_oracle as O
from synth import scenes

pytestmark = pytest.mark.gpu

BARS = {"direct_lut": 3e-6, "tc_fp16x3": 8e-6, "tc_bf16x3": 1.6e-5}  # per layer, ~3x achieved


@pytest.fixture(scope="module")
def setup():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2211_09938_gb300 import Plan
    sc = scenes.paper_scene(n_layers=32, holo=2048)
    g = O.geometry_of(sc)
    ref_lists = O.progressive_lists(sc["saliency"], sc["layer"], 32, scenes.THRESHOLDS_U8)
    plan = Plan.for_scene(sc)
    I = torch.from_numpy(sc["intensity"]).cuda()
    L = torch.from_numpy(sc["layer"]).cuda()
    coeffs = plan.haar_decompose(I, L)
    return sc, g, ref_lists, plan, coeffs


def _lists_for_layer(ref_lists, z):
    return [x[(x >> 24) == z] for x in ref_lists]


def _dev_lists(torch, lists):
    dl = [torch.from_numpy(np.concatenate([x, np.zeros(1, np.int32)]).astype(np.int32)).cuda() for x in lists]
    cnt = torch.from_numpy(np.array([[len(x), len(x)] for x in lists], np.int32)).cuda()
    return dl, cnt


def test_precision_full_and_per_layer(setup):
    import torch
    sc, g, ref_lists, plan, coeffs = setup
    Href = O.progressive_hologram(sc["intensity"], sc["layer"], ref_lists, g)
    dl, cnt = _dev_lists(torch, ref_lists)
    full, worst = {}, {f: 0.0 for f in BARS}
    for form in BARS:
        H = plan.progressive_hologram(coeffs, dl, cnt, form=form).cpu().numpy()
        full[form] = O.rel_l2(H, Href)
        mx = float(np.max(np.abs(H - Href)))
        print(f"{form} 512->2048 Z32 full: rel-L2 {full[form]:.3e} max-abs {mx:.3e} "
              f"(|H|max {np.abs(Href).max():.3e})")
    rng = np.random.default_rng(0)
    for z in sorted(rng.choice(32, size=8, replace=False).tolist()):
        lz = _lists_for_layer(ref_lists, z)
        if len(lz[0]) == 0:
            continue
        Hz_ref = O.progressive_hologram(sc["intensity"], sc["layer"], lz, g)
        dlz, cz = _dev_lists(torch, lz)
        for form in BARS:
            Hz = plan.progressive_hologram(coeffs, dlz, cz, form=form).cpu().numpy()
            err = O.rel_l2(Hz, Hz_ref)
            print(f"{form} layer {z:2d}: rel-L2 {err:.3e} max-abs {float(np.max(np.abs(Hz - Hz_ref))):.3e}")
            worst[form] = max(worst[form], err)
    print("full rel-L2:", full, "worst per-layer rel-L2:", worst)
    # Short accumulation chains: the tensor pipe's FP32 accumulation error grows with the
    # number of MMAs summed in one TMEM accumulator; capping a chain at 8 K steps (256 K
    # elements) and adding the partial sums in L2 (round-to-nearest atomics) brings both
    # split forms under the FP32 bar.
    plan.set_tuning(8)
    short = {}
    for form in ("tc_fp16x3", "tc_bf16x3"):
        H = plan.progressive_hologram(coeffs, dl, cnt, form=form).cpu().numpy()
        short[form] = O.rel_l2(H, Href)
    plan.set_tuning(0)
    print("full rel-L2 with 8-step chains:", short)
    for form, bar in BARS.items():
        assert worst[form] <= bar, (form, worst[form])
    assert full["direct_lut"] <= 1e-5
    # default chains: fp16 hi+lo caps them at 32 K steps and meets the FP32 bar; bf16 hi+lo
    # runs up to 128 K steps (bar 1e-3, regression margin 3x)
    assert full["tc_fp16x3"] <= 1e-5 and full["tc_bf16x3"] <= 7e-5
    assert short["tc_fp16x3"] <= 1e-5 and short["tc_bf16x3"] <= 1e-5
