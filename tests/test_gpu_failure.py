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


@pytest.mark.parametrize("form", ["direct_lut", "tc_bf16x3"])
def test_inflated_list_count_is_clamped_and_reported(form):
    """A device count larger than any list the plan can produce is clamped to the plan's
    largest list (layers x blocks at that level) and reported as CGH_ERR_ARG through the
    status word.  The list buffer is allocated past the inflated count, so nothing is read
    out of bounds even without the clamp: entries between the real count and the clamp
    are out-of-plan (add nothing), and entries past the clamp are valid but unselected
    blocks, which would change the hologram if they were walked."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2211_09938_gb300 import Plan, cgh
    sc = scenes.tiny_scene()
    g = O.geometry_of(sc)
    plan = Plan.for_scene(sc)
    I = torch.from_numpy(sc["intensity"]).cuda()
    L = torch.from_numpy(sc["layer"]).cuda()
    S = torch.from_numpy(sc["saliency"]).cuda()
    coeffs = plan.haar_decompose(I, L)
    lists, counts = plan.progressive_lists(S, L, scenes.THRESHOLDS_U8)
    c = counts.cpu().numpy()
    real = [lists[k][:int(c[k, 0])].cpu().numpy() for k in range(4)]
    cmax = plan.max_blocks(1)
    extra = 4096
    occupied = O.select_blocks(sc["saliency"], sc["layer"], g.n_layers, -1, 1)
    unselected = np.setdiff1d(occupied, real[1])
    assert len(unselected) >= 16
    buf = np.empty(cmax + extra, np.int32)
    buf[:len(real[1])] = real[1]
    buf[len(real[1]):cmax] = O.pack_entry(127, 0, 0)  # layer 127: outside the plan
    buf[cmax:] = np.resize(unselected, extra)
    bad_lists = list(lists)
    bad_lists[1] = torch.from_numpy(buf).cuda()
    bad_counts = counts.clone()
    bad_counts[1, 0] = cmax + extra
    assert plan.status() == cgh.CGH_OK
    H = plan.progressive_hologram(coeffs, bad_lists, bad_counts, form=form)
    torch.cuda.synchronize()
    assert plan.status() == cgh.CGH_ERR_ARG
    Href = O.progressive_hologram(sc["intensity"], sc["layer"], real, g)
    tol = 1e-5 if form == "direct_lut" else 3e-5
    assert O.rel_l2(H.cpu().numpy(), Href) <= tol
    # a negative count reads as an empty list, also reported
    neg = counts.clone()
    neg[2, 0] = -5
    H2 = plan.progressive_hologram(coeffs, lists, neg, form=form)
    torch.cuda.synchronize()
    assert plan.status() == cgh.CGH_ERR_ARG
    no2 = [real[0], real[1], np.zeros(0, np.int32), real[3]]
    assert O.rel_l2(H2.cpu().numpy(), O.progressive_hologram(sc["intensity"], sc["layer"], no2, g)) <= tol
    # a clean call afterwards records nothing
    plan.progressive_hologram(coeffs, lists, counts, form=form)
    torch.cuda.synchronize()
    assert plan.status() == cgh.CGH_OK
    plan.close()


def test_grid_barrier_wait_times_out_and_context_survives():
    """The single-launch selection's grid barrier: with every CTA present all of them cross
    and nothing is recorded; with one CTA that never arrives (a flag nothing sets) every
    waiting CTA gives up after the limit, CGH_ERR_TIMEOUT is recorded, and the kernel
    returns.  The selection then still works on the same plan (its own barrier word is
    separate)."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2211_09938_gb300 import Plan, cgh
    sc = scenes.tiny_scene()
    plan = Plan.for_scene(sc)
    crossed = torch.zeros(1, dtype=torch.int32, device="cuda")
    plan.selftest_grid_barrier(64, -1, 200000, crossed)
    torch.cuda.synchronize()
    assert int(crossed.item()) == 64 and plan.status() == cgh.CGH_OK
    crossed.zero_()
    plan.selftest_grid_barrier(64, 17, 20000, crossed)  # 20 ms
    torch.cuda.synchronize()
    assert int(crossed.item()) == 0
    assert plan.status() == cgh.CGH_ERR_TIMEOUT
    assert plan.status() == cgh.CGH_OK
    S = torch.from_numpy(sc["saliency"]).cuda()
    L = torch.from_numpy(sc["layer"]).cuda()
    I = torch.from_numpy(sc["intensity"]).cuda()
    coeffs = plan.haar_decompose(I, L)
    H, lists, counts = plan.progressive_step(S, L, coeffs, scenes.THRESHOLDS_U8, form="tc_bf16x3")
    torch.cuda.synchronize()
    ref = O.progressive_lists(sc["saliency"], sc["layer"], 4, scenes.THRESHOLDS_U8)
    c = counts.cpu().numpy()
    for k in range(4):
        assert np.array_equal(lists[k][:c[k, 0]].cpu().numpy(), ref[k])
    assert plan.status() == cgh.CGH_OK
    with pytest.raises(cgh.CghError):
        plan.selftest_grid_barrier(1, -1, 1000, crossed)
    plan.close()
