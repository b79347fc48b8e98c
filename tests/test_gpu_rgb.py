"""Colour holograms on the GPU: three channels at their own wavelengths as one batch,
each channel against the FP64 oracle at that wavelength.

Bars: the tensor forms' own (bf16 hi+lo rel-L2 1e-3, fp16 hi+lo 1e-5), the batched and
single-scene paths agree to 1e-5 (same products, different split-K summation order), and
the reconstructed amplitudes to the reconstruction bar 1e-4."""
import numpy as np
import pytest

from oracle import cgh_oracle as O
from synth import scenes

pytestmark = pytest.mark.gpu

TOL = {"tc_bf16x3": 1e-3, "tc_fp16x3": 1e-5}


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


@pytest.mark.parametrize("form", ["tc_fp16x3", "tc_bf16x3"])
def test_rgb_channels_match_oracle(torch_cuda, form):
    torch = torch_cuda
    from paper_2211_09938_gb300.rgb import RGBHologram, WAVELENGTHS_RGB
    sc = scenes.rgb_scene(111, 128, 256, 4)
    n, hh = 128, 256
    Ic = [torch.from_numpy(np.ascontiguousarray(sc["intensity"][c])).cuda() for c in range(3)]
    L = torch.from_numpy(sc["layer"]).cuda()
    S = torch.from_numpy(sc["saliency"]).cuda()
    holos = [torch.empty((hh, hh), dtype=torch.complex64, device="cuda") for _ in range(3)]
    rgb = RGBHologram((n, n), (hh, hh), sc["pitch"], sc["z"], Ic, L, S, scenes.THRESHOLDS_U8, holos, form=form)
    rgb.run()
    amps = rgb.reconstruct(L)
    torch.cuda.synchronize()
    lists = O.progressive_lists(sc["saliency"], sc["layer"], 4, scenes.THRESHOLDS_U8)
    for c, lam in enumerate(WAVELENGTHS_RGB):
        g = O.Geometry((n, n), (hh, hh), sc["pitch"], lam, sc["z"])
        Href = O.progressive_hologram(sc["intensity"][c], sc["layer"], lists, g)
        err = O.rel_l2(holos[c].cpu().numpy(), Href)
        # the single-scene path of the same plan
        plan = rgb.plans[c]
        coeffs = plan.haar_decompose(Ic[c], L)
        li, cn = plan.progressive_lists(S, L, scenes.THRESHOLDS_U8)
        Hs = plan.progressive_hologram(coeffs, li, cn, form=form)
        torch.cuda.synchronize()
        err_s = O.rel_l2(holos[c].cpu().numpy(), Hs.cpu().numpy())
        Aref = O.composite_amplitude(O.reconstruct_fields(holos[c].cpu().numpy().astype(np.complex128), g),
                                     sc["layer"])
        err_a = O.rel_l2(amps[c].cpu().numpy(), Aref)
        print(f"rgb {form} channel {c} ({lam * 1e9:.0f} nm): vs oracle {err:.2e}, vs single scene {err_s:.2e}, "
              f"amplitude {err_a:.2e}")
        assert err <= TOL[form] and err_s <= 1e-5 and err_a <= 1e-4
    # the channels differ (different wavelengths and intensities)
    assert O.rel_l2(holos[0].cpu().numpy(), holos[2].cpu().numpy()) > 0.1
    rgb.close()
