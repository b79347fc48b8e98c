"""cgh_progressive_step: selection and superposition in one call.

The step's lists and counts are the oracle's bit for bit; its hologram meets the tensor
forms' rel-L2 bars against the FP64 oracle and, on a deterministic plan (no split-K
atomics), equals the two-call path (cgh_select_progressive + cgh_progressive_hologram)
bit for bit, whether the selection ran as the single cooperative launch (small count
tables) or as three passes with the flags taken from the lists (large tables)."""
import numpy as np
import pytest

from oracle import cgh_oracle as O
from synth import scenes

pytestmark = pytest.mark.gpu

# the benchmark spec bars: 1e-5 (fp16 hi+lo, the FP32 bar) and 1e-3 (bf16 hi+lo); the per-scene
# regression bars sit at about 3x what each form achieves (never above its benchmark spec bar).
BF16X3_TOL = 1e-3
FP16X3_TOL = 1e-5
SCENE_TOL = {  # scene: (bf16x3, fp16x3, fp16x2); achieved bf16x3 1.07e-5 / 2.1e-6 / 2.2e-6 / 2.35e-5
    "paper_512_z16": (3.5e-5, 1e-5, 1e-3),
    "graded_64_s2_z5": (7e-6, 2e-6, 5e-4),
    "single_layer_32_s2": (7e-6, 2e-6, 6e-4),
    "large_table_512_z40": (7e-5, 1e-5, 8e-4),
}


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


def _inputs(torch, sc, flags=0):
    from paper_2211_09938_gb300 import Plan
    plan = Plan.for_scene(sc, flags=flags)
    I = torch.from_numpy(sc["intensity"]).cuda()
    L = torch.from_numpy(sc["layer"]).cuda()
    S = torch.from_numpy(sc["saliency"]).cuda()
    return plan, I, L, S, plan.haar_decompose(I, L)


def _two_calls(plan, S, L, coeffs, form, thr=scenes.THRESHOLDS_U8, lists=None):
    lists, counts = plan.progressive_lists(S, L, thr, lists=lists)
    H = plan.progressive_hologram(coeffs, lists, counts, form=form)
    return H, lists, counts


SCENES = {
    # level-1 table 16 layers x 256 chunks: the cooperative selection
    "paper_512_z16": lambda: scenes.paper_scene(),
    "graded_64_s2_z5": lambda: scenes.random_scene(79, 64, 128, 5, graded=True),
    "single_layer_32_s2": lambda: scenes.random_scene(78, 32, 64, 1, graded=True),
    # level-1 table 40 layers x 256 chunks > 8192: three passes, flags from the lists
    "large_table_512_z40": lambda: scenes.random_scene(99, 512, 1024, 40, graded=True),
}


@pytest.mark.parametrize("name", list(SCENES))
@pytest.mark.parametrize("form,tol", [("tc_bf16x3", BF16X3_TOL), ("tc_fp16x3", FP16X3_TOL), ("tc_fp16x2", 1e-3)])
def test_step_matches_oracle_and_two_calls(torch_cuda, name, form, tol):
    """Default plan: lists bit-exact and hologram within the form's bar against the oracle.
    Deterministic plan: the step's hologram equals the two calls' bit for bit."""
    torch = torch_cuda
    from paper_2211_09938_gb300 import Plan
    sc = SCENES[name]()
    ref_lists = O.progressive_lists(sc["saliency"], sc["layer"], len(sc["z"]), scenes.THRESHOLDS_U8)
    plan, I, L, S, coeffs = _inputs(torch, sc)
    H, lists, counts = plan.progressive_step(S, L, coeffs, scenes.THRESHOLDS_U8, form=form)
    torch.cuda.synchronize()
    assert plan.status() == 0
    c = counts.cpu().numpy()
    for k in range(4):
        assert c[k, 0] == c[k, 1] == len(ref_lists[k]), k
        assert np.array_equal(lists[k][:c[k, 0]].cpu().numpy(), ref_lists[k]), k
    Href = O.progressive_hologram(sc["intensity"], sc["layer"], ref_lists, O.geometry_of(sc))
    err = O.rel_l2(H.cpu().numpy(), Href)
    print(f"{form} {name}: rel-L2 {err:.3e}")
    assert err <= min(tol, SCENE_TOL[name][("tc_bf16x3", "tc_fp16x3", "tc_fp16x2").index(form)])

    dplan, I, L, S, coeffs = _inputs(torch, sc, flags=Plan.DETERMINISTIC)
    H, lists, counts = dplan.progressive_step(S, L, coeffs, scenes.THRESHOLDS_U8, form=form)
    H2, lists2, counts2 = _two_calls(dplan, S, L, coeffs, form)
    torch.cuda.synchronize()
    assert dplan.status() == 0
    assert np.array_equal(counts.cpu().numpy(), counts2.cpu().numpy())
    for k in range(4):
        n = int(c[k, 0])
        assert np.array_equal(lists[k][:n].cpu().numpy(), lists2[k][:n].cpu().numpy()), k
    assert np.array_equal(H.cpu().numpy(), H2.cpu().numpy())


def test_step_repeated_and_captured(torch_cuda):
    """The grid barrier needs no reset: repeated calls, then the step captured in a CUDA
    graph (with the DWT on a side stream that the step waits for through coeffs_ready) and
    replayed, give the same lists and hologram (split-K plan: compared within FP32
    summation-order noise) and leave the status word clear."""
    torch = torch_cuda
    sc = scenes.paper_scene()
    plan, I, L, S, coeffs = _inputs(torch, sc)
    counts = torch.zeros((4, 2), dtype=torch.int32, device="cuda")
    lists = [torch.empty(plan.max_blocks(3 if k == 0 else k), dtype=torch.int32, device="cuda") for k in range(4)]
    holo = torch.empty((plan.holo_h, plan.holo_w), dtype=torch.complex64, device="cuda")
    outs = []
    for _ in range(3):
        plan.progressive_step(S, L, coeffs, scenes.THRESHOLDS_U8, counts=counts, lists=lists, holo=holo)
        outs.append((holo.cpu().numpy(), [l.cpu().numpy() for l in lists], counts.cpu().numpy()))
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    with torch.cuda.graph(g, stream=stream):
        fork = torch.cuda.Event()
        fork.record(stream)
        side.wait_event(fork)
        plan.haar_decompose(I, L, coeffs, stream=side)
        ready = torch.cuda.Event()
        ready.record(side)
        plan.progressive_step(S, L, coeffs, scenes.THRESHOLDS_U8, counts=counts, lists=lists, holo=holo,
                              coeffs_ready=ready, stream=stream)
    for _ in range(3):
        with torch.cuda.stream(stream):
            holo.zero_()
            counts.zero_()
            coeffs.zero_()
            g.replay()
        stream.synchronize()
        outs.append((holo.cpu().numpy(), [l.cpu().numpy() for l in lists], counts.cpu().numpy()))
    assert plan.status() == 0
    H0, l0, c0 = outs[0]
    for Hk, lk, ck in outs[1:]:
        assert np.array_equal(ck, c0)
        for k in range(4):
            assert np.array_equal(lk[k][:c0[k, 0]], l0[k][:c0[k, 0]])
        assert O.rel_l2(Hk, H0) <= 1e-6


def test_step_capacity_overflow(torch_cuda):
    """Lists shorter than the selection: the step writes the first entries, reports the
    totals, and its hologram is that of the written entries only (the flags the fused
    selection marks follow the written entries)."""
    torch = torch_cuda
    sc = scenes.paper_scene()
    plan, I, L, S, coeffs = _inputs(torch, sc)
    ref_lists = O.progressive_lists(sc["saliency"], sc["layer"], plan.n_layers, scenes.THRESHOLDS_U8)
    caps = [len(ref_lists[0]) // 2, len(ref_lists[1]) // 3, len(ref_lists[2]), 1]
    mk = lambda: [torch.empty(c, dtype=torch.int32, device="cuda") for c in caps]
    lists = mk()
    H, lists, counts = plan.progressive_step(S, L, coeffs, scenes.THRESHOLDS_U8, lists=lists, form="tc_fp16x3")
    c = counts.cpu().numpy()
    for k in range(4):
        assert c[k, 1] == len(ref_lists[k]) and c[k, 0] == min(caps[k], len(ref_lists[k])), k
        assert np.array_equal(lists[k][:c[k, 0]].cpu().numpy(), ref_lists[k][:c[k, 0]]), k
    H2, _, _ = _two_calls(plan, S, L, coeffs, "tc_fp16x3", lists=mk())
    torch.cuda.synchronize()
    assert O.rel_l2(H.cpu().numpy(), H2.cpu().numpy()) <= 1e-6  # split-K: summation order only
    trunc = [ref_lists[k][:c[k, 0]] for k in range(4)]
    Href = O.progressive_hologram(sc["intensity"], sc["layer"], trunc, O.geometry_of(sc))
    assert O.rel_l2(H.cpu().numpy(), Href) <= FP16X3_TOL


def test_step_direct_lut(torch_cuda):
    """The CUDA-core form through the step: the two calls in sequence."""
    torch = torch_cuda
    from paper_2211_09938_gb300 import Plan
    sc = scenes.random_scene(79, 64, 128, 5, graded=True)
    plan, I, L, S, coeffs = _inputs(torch, sc, flags=Plan.DETERMINISTIC)
    H, lists, counts = plan.progressive_step(S, L, coeffs, scenes.THRESHOLDS_U8, form="direct_lut")
    H2, _, counts2 = _two_calls(plan, S, L, coeffs, "direct_lut")
    torch.cuda.synchronize()
    assert np.array_equal(counts.cpu().numpy(), counts2.cpu().numpy())
    assert np.array_equal(H.cpu().numpy(), H2.cpu().numpy())
