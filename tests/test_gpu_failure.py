"""Failure detection without a GPU fault: a bounded device wait that runs out reports
CGH_ERR_TIMEOUT through the plan's status word, the kernel returns, and the context keeps
working.  Host-side failures (bad arguments, NULL pointers) are covered in test_abi.py."""
import numpy as np
import pytest

from oracle import cgh_oracle as O
from synth import scenes

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_survives():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2211_09938_gb300 import Plan, cgh
    sc = scenes.tiny_scene()
    plan = Plan.for_scene(sc)
    assert plan.status() == cgh.CGH_OK
    plan.selftest_timeout(20000)  # 20 ms
    assert plan.status() == cgh.CGH_ERR_TIMEOUT
    assert plan.status() == cgh.CGH_OK  # read-and-clear
    # the context is still usable: a full progressive hologram afterwards is correct
    I = torch.from_numpy(sc["intensity"]).cuda()
    L = torch.from_numpy(sc["layer"]).cuda()
    S = torch.from_numpy(sc["saliency"]).cuda()
    coeffs = plan.haar_decompose(I, L)
    lists, counts = plan.progressive_lists(S, L, scenes.THRESHOLDS_U8)
    H = plan.progressive_hologram(coeffs, lists, counts, form="tc_bf16x3")
    torch.cuda.synchronize()
    ref_lists = O.progressive_lists(sc["saliency"], sc["layer"], 4, scenes.THRESHOLDS_U8)
    Href = O.progressive_hologram(sc["intensity"], sc["layer"], ref_lists, O.geometry_of(sc))
    assert O.rel_l2(H.cpu().numpy(), Href) <= 1e-5
    assert plan.status() == cgh.CGH_OK
    with pytest.raises(cgh.CghError):
        plan.selftest_timeout(0)
