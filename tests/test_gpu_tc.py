"""Tensor-core (tcgen05) separable form: the GEMM machinery against torch, then the
progressive hologram against the FP64 oracle.

Bars: the diagnostic GEMM is exact up to FP32 accumulation order (operands are exact
bf16/fp16 values); the progressive hologram meets the benchmark spec bars (rel-L2 <= 1e-3 for
the bf16 hi+lo path, <= 1e-5 for the fp16 hi+lo path) with regression margins of about 3x
what each form achieves."""
import numpy as np
import pytest

from oracle import cgh_oracle as O
from synth import scenes

pytestmark = pytest.mark.gpu

# The benchmark spec bars are 1e-5 rel-L2 (FP32) and 1e-3 (bf16 split); the regression bars
# below sit at about 3x what each form achieves (never above its benchmark spec bar), so a loss
# of accuracy fails a test long before a bar is crossed.  Paper scale: bf16x3 1.07e-5,
# fp16x3 6.5e-6, fp16x2 2.9e-4; small scenes: bf16x3 <= 4.5e-6, fp16x3 <= 5.6e-7.
BF16X3_TOL = 3.5e-5
FP16X3_TOL = 1e-5
FP16X2_TOL = 1e-3  # fringe rounded once to fp16 (unit roundoff 2^-11), data hi+lo
SMALL_TOL = {"tc_bf16x3": 1.5e-5, "tc_fp16x3": 2e-6, "tc_fp16x2": 8e-4}


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


@pytest.mark.parametrize("M,N,K", [(128, 128, 32), (200, 136, 96), (1024, 512, 512), (384, 640, 1024)])
@pytest.mark.parametrize("fp16", [False, True])
def test_selftest_gemm_matches_torch(torch_cuda, M, N, K, fp16):
    torch = torch_cuda
    from paper_2211_09938_gb300.cgh import tc_selftest_gemm
    g = torch.Generator(device="cpu").manual_seed(M * 7 + N * 3 + K)
    dt = torch.float16 if fp16 else torch.bfloat16
    A = torch.randn(M, K, generator=g).to(dt)
    B = torch.randn(N, K, generator=g).to(dt)
    ref = A.double() @ B.double().T
    ref_abs = A.double().abs() @ B.double().abs().T
    C = tc_selftest_gemm(A.cuda().view(torch.int16), B.cuda().view(torch.int16), fp16=fp16)
    torch.cuda.synchronize()
    # products of 16-bit values are exact in FP32; only the FP32 summation rounds
    bound = K * 2.0 ** -24 * ref_abs + 1e-6
    assert bool(((C.cpu().double() - ref).abs() <= bound).all()), (C.cpu().double() - ref).abs().max()


SCENES = {
    "tiny_64_to_256_z4": lambda: scenes.tiny_scene(),
    "graded_64_s2_z5": lambda: scenes.random_scene(79, 64, 128, 5, graded=True),
    "single_layer_32_s2": lambda: scenes.random_scene(78, 32, 64, 1, graded=True),
    "s3_48_z3": lambda: scenes.random_scene(80, 48, 144, 3, graded=True),
}


def run(torch, sc, form, thresholds=None, order=None, dims=False):
    from paper_2211_09938_gb300 import Plan
    plan = Plan.for_scene(sc)
    if order is not None:
        plan.set_contraction(order)
    I = torch.from_numpy(sc["intensity"]).cuda()
    L = torch.from_numpy(sc["layer"]).cuda()
    S = torch.from_numpy(sc["saliency"]).cuda()
    coeffs = plan.haar_decompose(I, L)
    thr = thresholds or scenes.THRESHOLDS_U8
    lists, counts = plan.progressive_lists(S, L, thr)
    H = plan.progressive_hologram(coeffs, lists, counts, form=form)
    torch.cuda.synchronize()
    assert plan.status() == 0
    ref_lists = O.progressive_lists(sc["saliency"], sc["layer"], plan.n_layers, thr)
    if dims:
        kr, kc = plan.tc_layer_dims()
        return H.cpu().numpy(), ref_lists, (sum(kr), sum(kc))
    return H.cpu().numpy(), ref_lists


@pytest.mark.parametrize("name", list(SCENES))
@pytest.mark.parametrize("form,tol", [("tc_bf16x3", BF16X3_TOL), ("tc_fp16x3", FP16X3_TOL),
                                      ("tc_fp16x2", FP16X2_TOL)])
def test_progressive_tc(torch_cuda, name, form, tol):
    sc = SCENES[name]()
    H, ref_lists = run(torch_cuda, sc, form)
    Href = O.progressive_hologram(sc["intensity"], sc["layer"], ref_lists, O.geometry_of(sc))
    err = O.rel_l2(H, Href)
    print(f"{form} {name}: rel-L2 {err:.3e}")
    assert err <= min(tol, SMALL_TOL[form])


@pytest.mark.parametrize("form,tol", [("tc_bf16x3", BF16X3_TOL), ("tc_fp16x3", FP16X3_TOL),
                                      ("tc_fp16x2", FP16X2_TOL)])
def test_progressive_tc_paper_scale(torch_cuda, form, tol):
    sc = scenes.paper_scene()
    H, ref_lists = run(torch_cuda, sc, form)
    Href = O.progressive_hologram(sc["intensity"], sc["layer"], ref_lists, O.geometry_of(sc))
    err = O.rel_l2(H, Href)
    print(f"{form} 512->1024 Z16: rel-L2 {err:.3e}")
    assert err <= tol


def _transposed(sc):
    t = dict(sc)
    for k in ("intensity", "layer", "saliency"):
        t[k] = np.ascontiguousarray(sc[k].T)
    return t


def test_contraction_orders(torch_cuda):
    """H = sum_z E_z A^_z E_z^T contracted over the layers' object rows, or (square object)
    over their columns with H written transposed: both orders match the oracle; the
    automatic choice takes the smaller contraction; transposing the scene transposes the
    hologram and flips the automatic choice; a non-square object keeps rows."""
    from paper_2211_09938_gb300 import Plan
    torch = torch_cuda
    sc = scenes.paper_scene()
    Href = O.progressive_hologram(sc["intensity"], sc["layer"],
                                  O.progressive_lists(sc["saliency"], sc["layer"], 16, scenes.THRESHOLDS_U8),
                                  O.geometry_of(sc))
    got = {}
    for order in (Plan.CONTRACT_ROWS, Plan.CONTRACT_COLS, Plan.CONTRACT_AUTO):
        H, _, (sr, sc_) = run(torch, sc, "tc_fp16x3", order=order, dims=True)
        err = O.rel_l2(H, Href)
        print(f"order {order}: contraction K {sr} (other axis {sc_}), rel-L2 {err:.3e}")
        assert err <= FP16X3_TOL
        got[order] = (H, sr, sc_)
    r_rows, r_cols = got[Plan.CONTRACT_ROWS][1], got[Plan.CONTRACT_COLS][1]
    assert r_rows != r_cols and got[Plan.CONTRACT_AUTO][1] == min(r_rows, r_cols)
    # the transposed scene: same hologram transposed, the other order chosen
    st = _transposed(sc)
    Ht, _, (srt, _) = run(torch, st, "tc_fp16x3", dims=True)
    assert O.rel_l2(Ht, got[Plan.CONTRACT_AUTO][0].T) <= 2 * FP16X3_TOL
    assert srt == min(r_rows, r_cols)
    # non-square object: the column order is not available and rows are used
    rect = dict(scenes.random_scene(83, 64, 128, 3, graded=True))
    rect["intensity"] = np.ascontiguousarray(rect["intensity"][:, :40])
    rect["layer"] = np.ascontiguousarray(rect["layer"][:, :40])
    rect["saliency"] = np.ascontiguousarray(rect["saliency"][:, :40])
    rect["holo"] = (128, 80)
    H, ref_lists = run(torch, rect, "tc_fp16x3", order=Plan.CONTRACT_COLS)
    Hr = O.progressive_hologram(rect["intensity"], rect["layer"], ref_lists, O.geometry_of(rect))
    assert O.rel_l2(H, Hr) <= FP16X3_TOL


PAIR_SCENES = {
    "paper_512_to_1024_z16": lambda: scenes.paper_scene(),
    "tiny_64_to_256_z4": lambda: scenes.tiny_scene(),
    # 3 row tiles (the last CTA pair has one CTA past the hologram) and ragged columns
    "s3_48_z3": lambda: scenes.random_scene(80, 48, 144, 3, graded=True),
    "odd_tiles_96_to_384_z5": lambda: scenes.random_scene(84, 96, 384, 5, graded=True),
}


@pytest.mark.parametrize("name", list(PAIR_SCENES))
@pytest.mark.parametrize("form", ["tc_fp16x3", "tc_bf16x3", "tc_fp16x2"])
def test_stage2_cta_pairs_match_single_cta_and_oracle(torch_cuda, name, form):
    """Stage 2 on CTA pairs (256 x 128 tiles, tcgen05 cta_group::2) against one CTA per
    128 x 128 tile and the FP64 oracle: both within the form's bar, and close to each other
    (they sum the same products in a different order)."""
    torch = torch_cuda
    from paper_2211_09938_gb300 import Plan
    sc = PAIR_SCENES[name]()
    plan = Plan.for_scene(sc)
    I = torch.from_numpy(sc["intensity"]).cuda()
    L = torch.from_numpy(sc["layer"]).cuda()
    S = torch.from_numpy(sc["saliency"]).cuda()
    coeffs = plan.haar_decompose(I, L)
    lists, counts = plan.progressive_lists(S, L, scenes.THRESHOLDS_U8)
    assert plan.stage2_tiles_used() == Plan.TILES_AUTO  # no separable call yet
    plan.progressive_hologram(coeffs, lists, counts, form=form)
    # the default: CTA pairs from 64 tiles of 128 x 128 (1024 x 1024 holograms and larger)
    tiles_default = Plan.TILES_PAIR if -(-sc["holo"][0] // 128) * -(-sc["holo"][1] // 128) >= 64 else Plan.TILES_CTA
    assert plan.stage2_tiles_used() == tiles_default
    got = {}
    for tiles in (Plan.TILES_CTA, Plan.TILES_PAIR):
        plan.set_stage2_tiles(tiles)
        H = plan.progressive_hologram(coeffs, lists, counts, form=form)
        H2 = plan.progressive_hologram(coeffs, lists, counts, form=form)  # a second call, same plan
        torch.cuda.synchronize()
        assert plan.status() == 0
        assert plan.stage2_tiles_used() == tiles  # the shape asked for is the one that ran
        got[tiles] = (H.cpu().numpy(), H2.cpu().numpy())
    ref_lists = O.progressive_lists(sc["saliency"], sc["layer"], plan.n_layers, scenes.THRESHOLDS_U8)
    Href = O.progressive_hologram(sc["intensity"], sc["layer"], ref_lists, O.geometry_of(sc))
    bar = {"tc_fp16x3": FP16X3_TOL, "tc_bf16x3": BF16X3_TOL, "tc_fp16x2": FP16X2_TOL}[form]
    e_cta = O.rel_l2(got[Plan.TILES_CTA][0], Href)
    e_pair = O.rel_l2(got[Plan.TILES_PAIR][0], Href)
    d = O.rel_l2(got[Plan.TILES_PAIR][0], got[Plan.TILES_CTA][0])
    print(f"{form} {name}: one CTA {e_cta:.3e}, CTA pairs {e_pair:.3e}, pairs vs one CTA {d:.3e}")
    assert e_cta <= bar and e_pair <= bar
    assert e_pair <= 1.5 * e_cta + 1e-7
    assert O.rel_l2(got[Plan.TILES_PAIR][1], got[Plan.TILES_PAIR][0]) <= 2 * e_pair + 1e-7
    plan.close()


@pytest.mark.parametrize("name", list(PAIR_SCENES))
@pytest.mark.parametrize("form", ["tc_fp16x3", "tc_bf16x3", "tc_fp16x2"])
def test_fused_stages_match_two_launches_and_oracle(torch_cuda, name, form):
    """Both GEMM stages in one cooperative launch (stage 2 waiting per layer for stage 1's
    stored tiles) against two launches and the FP64 oracle, over two calls in a row (the
    per-layer counters are reset by the compaction of the next call)."""
    torch = torch_cuda
    from paper_2211_09938_gb300 import Plan
    sc = PAIR_SCENES[name]()
    plan = Plan.for_scene(sc)
    I = torch.from_numpy(sc["intensity"]).cuda()
    L = torch.from_numpy(sc["layer"]).cuda()
    S = torch.from_numpy(sc["saliency"]).cuda()
    coeffs = plan.haar_decompose(I, L)
    lists, counts = plan.progressive_lists(S, L, scenes.THRESHOLDS_U8)
    got = {}
    for fused in (False, True):
        plan.set_fusion(fused)
        plan.set_stage2_tiles(Plan.TILES_CTA)
        plan.profile(True)
        H = plan.progressive_hologram(coeffs, lists, counts, form=form)
        prof = plan.profile_read()
        plan.profile(False)
        H2 = plan.progressive_hologram(coeffs, lists, counts, form=form)
        torch.cuda.synchronize()
        assert plan.status() == 0
        # the fused path ran as one launch, the other as two
        assert (prof["tc_fused"] > 0) == fused and (prof["tc_stage2"] > 0) == (not fused)
        got[fused] = (H.cpu().numpy(), H2.cpu().numpy())
    ref_lists = O.progressive_lists(sc["saliency"], sc["layer"], plan.n_layers, scenes.THRESHOLDS_U8)
    Href = O.progressive_hologram(sc["intensity"], sc["layer"], ref_lists, O.geometry_of(sc))
    bar = {"tc_fp16x3": FP16X3_TOL, "tc_bf16x3": BF16X3_TOL, "tc_fp16x2": FP16X2_TOL}[form]
    e2 = O.rel_l2(got[False][0], Href)
    e1 = O.rel_l2(got[True][0], Href)
    print(f"{form} {name}: two launches {e2:.3e}, fused {e1:.3e}, "
          f"fused vs two {O.rel_l2(got[True][0], got[False][0]):.3e}")
    assert e2 <= bar and e1 <= bar
    # same chains, same order of products: only the split of the partial sums may differ
    assert O.rel_l2(got[True][0], got[False][0]) <= 1e-6
    assert O.rel_l2(got[True][1], got[True][0]) <= 1e-6
    plan.close()
