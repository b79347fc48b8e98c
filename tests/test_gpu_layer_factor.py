"""The plan's layer factor (Eq. 1's exp(jkz)/z per layer, dropped by default): every form
of the hologram, the point-wise kernels and the reconstruction against the FP64 oracle
with the factor kept.  Bars: each form's own (FP32 1e-5, bf16 hi+lo 1e-3, fp16 hi+lo 1e-5,
reconstruction 1e-4)."""
import numpy as np
import pytest

from oracle import cgh_oracle as O
from synth import scenes

pytestmark = pytest.mark.gpu

BARS = {"direct_lut": 1e-5, "tc_bf16x3": 1e-3, "tc_fp16x3": 1e-5}


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


def _scene(name):
    sc = dict(scenes.tiny_scene() if name == "tiny" else scenes.paper_scene())
    sc["layer_factor"] = True
    return sc


@pytest.mark.parametrize("name", ["tiny", "paper"])
def test_layer_factor_forms(torch_cuda, name):
    torch = torch_cuda
    from paper_2211_09938_gb300 import Plan
    sc = _scene(name)
    g = O.geometry_of(sc)
    plan = Plan.for_scene(sc)
    I = torch.from_numpy(sc["intensity"]).cuda()
    L = torch.from_numpy(sc["layer"]).cuda()
    S = torch.from_numpy(sc["saliency"]).cuda()
    coeffs = plan.haar_decompose(I, L)
    lists, counts = plan.progressive_lists(S, L, scenes.THRESHOLDS_U8)
    ref_lists = O.progressive_lists(sc["saliency"], sc["layer"], g.n_layers, scenes.THRESHOLDS_U8)
    Href = O.progressive_hologram(sc["intensity"], sc["layer"], ref_lists, g)
    for form, bar in BARS.items():
        H = plan.progressive_hologram(coeffs, lists, counts, form=form).cpu().numpy()
        err = O.rel_l2(H, Href)
        print(f"layer factor {name} {form}: rel-L2 {err:.2e}")
        assert err <= bar, form
    # reconstruction: the adjoint, conj(c_z) per layer
    if name == "tiny":
        Hd = torch.from_numpy(Href.astype(np.complex64)).cuda()
        F, A = plan.reconstruct(Hd, L)
        torch.cuda.synchronize()
        R = O.reconstruct_fields(Href, g)
        err = O.rel_l2(F.cpu().numpy(), R)
        print(f"layer factor reconstruction: {err:.2e}")
        assert err <= 1e-4


def test_layer_factor_pointwise_kernels(torch_cuda):
    torch = torch_cuda
    from paper_2211_09938_gb300 import Plan
    sc = _scene("tiny")
    g = O.geometry_of(sc)
    plan = Plan.for_scene(sc)
    I = torch.from_numpy(sc["intensity"]).cuda()
    L = torch.from_numpy(sc["layer"]).cuda()
    H = plan.plain_direct(I, L).cpu().numpy()
    err = O.rel_l2(H, O.plain_pointwise_hologram(sc["intensity"], sc["layer"], g))
    print(f"layer factor plain direct: {err:.2e}")
    assert err <= 1e-5
    depth = scenes.depth_map(130, 64, 0.10, 0.13, holes=0.05)
    Hc = plan.pointcloud_direct(I, torch.from_numpy(depth).cuda()).cpu().numpy()
    err = O.rel_l2(Hc, O.pointcloud_hologram(sc["intensity"], depth, g))
    print(f"layer factor point cloud: {err:.2e}")
    assert err <= 1e-5
