"""GPU parity of the DWT, block selection, direct superposition and plain point-wise
kernels against the FP64 oracle, through the C ABI (ctypes binding).

Bars: bit-exact for DWT coefficients and work lists; relative L2 error <= 1e-5 for
the FP32 holograms against FP64."""
import numpy as np
import pytest

from oracle import cgh_oracle as O
from synth import scenes

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2211_09938_gb300 import build_lib, cgh
    import os
    if not os.path.exists(cgh.LIB_PATH):
        build_lib.build()
    cgh.lib()
    return torch


def dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def plan_for(sc):
    from paper_2211_09938_gb300 import Plan
    return Plan.for_scene(sc)


SCENES = {
    "tiny_64_to_256_z4": lambda: scenes.tiny_scene(),
    "ragged_40x24_s3_z3": lambda: _rect_scene(40, 24, 3, 3, seed=77),
    "single_layer_32_s2": lambda: scenes.random_scene(78, 32, 64, 1, graded=True),
    "graded_64_s2_z5": lambda: scenes.random_scene(79, 64, 128, 5, graded=True),
}


def _rect_scene(h, w, s, nl, seed):
    rng = np.random.default_rng(seed)
    sc = scenes.random_scene(seed, max(h, w), s * max(h, w), nl, graded=True)
    sc["intensity"] = np.ascontiguousarray(sc["intensity"][:h, :w])
    sc["layer"] = np.ascontiguousarray(rng.integers(0, nl, size=(h, w)).astype(np.uint8))
    sc["saliency"] = np.ascontiguousarray(sc["saliency"][:h, :w])
    sc["holo"] = (s * h, s * w)
    return sc


def _geom(sc):
    return O.geometry_of(sc)


@pytest.mark.parametrize("name", list(SCENES))
def test_haar_bit_exact(torch_cuda, name):
    torch = torch_cuda
    sc = SCENES[name]()
    plan = plan_for(sc)
    C = plan.haar_decompose(dev(torch, sc["intensity"]), dev(torch, sc["layer"])).cpu().numpy()
    planes = O.object_planes(sc["intensity"], sc["layer"], plan.n_layers)
    for z in range(plan.n_layers):
        assert np.array_equal(C[z], O.haar_forward(planes[z], 3)), z


def test_haar_bit_exact_paper_scale(torch_cuda):
    torch = torch_cuda
    sc = scenes.paper_scene()
    plan = plan_for(sc)
    C = plan.haar_decompose(dev(torch, sc["intensity"]), dev(torch, sc["layer"])).cpu().numpy()
    planes = O.object_planes(sc["intensity"], sc["layer"], plan.n_layers)
    for z in range(plan.n_layers):
        assert np.array_equal(C[z], O.haar_forward(planes[z], 3)), z


@pytest.mark.parametrize("name", list(SCENES))
def test_select_bit_exact(torch_cuda, name):
    torch = torch_cuda
    sc = SCENES[name]()
    plan = plan_for(sc)
    S, L = dev(torch, sc["saliency"]), dev(torch, sc["layer"])
    for level in (1, 2, 3):
        for t in (-1, 0, 127, 178, 229, 255):
            lst, cnt = plan.select_blocks(S, L, t, level)
            c = cnt.cpu().numpy()
            ref = O.select_blocks(sc["saliency"], sc["layer"], plan.n_layers, t, level)
            assert c[0] == c[1] == len(ref), (level, t, c, len(ref))
            assert np.array_equal(lst[:c[0]].cpu().numpy(), ref), (level, t)


def test_select_paper_scale_and_capacity(torch_cuda):
    torch = torch_cuda
    sc = scenes.paper_scene()
    plan = plan_for(sc)
    S, L = dev(torch, sc["saliency"]), dev(torch, sc["layer"])
    ref_lists = O.progressive_lists(sc["saliency"], sc["layer"], plan.n_layers, scenes.THRESHOLDS_U8)
    lists, counts = plan.progressive_lists(S, L, scenes.THRESHOLDS_U8)
    c = counts.cpu().numpy()
    for k in range(4):
        assert c[k, 0] == c[k, 1] == len(ref_lists[k])
        assert np.array_equal(lists[k][:c[k, 0]].cpu().numpy(), ref_lists[k])
    # capacity overflow: the first `capacity` entries, the true total reported
    cap = len(ref_lists[1]) // 3
    out = torch.full((cap + 4,), -7, dtype=torch.int32, device="cuda")
    lst, cnt = plan.select_blocks(S, L, scenes.THRESHOLDS_U8[1], 1, out=out, capacity=cap)
    c = cnt.cpu().numpy()
    assert c[0] == cap and c[1] == len(ref_lists[1])
    got = lst.cpu().numpy()
    assert np.array_equal(got[:cap], ref_lists[1][:cap])
    assert np.all(got[cap:] == -7)  # nothing written past the capacity


def test_select_empty_and_zero_capacity(torch_cuda):
    torch = torch_cuda
    sc = scenes.tiny_scene()
    plan = plan_for(sc)
    S = torch.zeros(sc["saliency"].shape, dtype=torch.uint8, device="cuda")
    L = dev(torch, sc["layer"])
    lst, cnt = plan.select_blocks(S, L, 0, 1)
    assert cnt.cpu().numpy().tolist() == [0, 0]
    out = torch.empty(1, dtype=torch.int32, device="cuda")
    lst, cnt = plan.select_blocks(dev(torch, sc["saliency"]), L, -1, 2, out=out, capacity=0)
    c = cnt.cpu().numpy()
    assert c[0] == 0 and c[1] == len(O.select_blocks(sc["saliency"], sc["layer"], 4, -1, 2))


def run_progressive(torch, sc, form="direct_lut", thresholds=None, lists_override=None):
    plan = plan_for(sc)
    I, L, S = dev(torch, sc["intensity"]), dev(torch, sc["layer"]), dev(torch, sc["saliency"])
    coeffs = plan.haar_decompose(I, L)
    thr = thresholds or scenes.THRESHOLDS_U8
    if lists_override is None:
        lists, counts = plan.progressive_lists(S, L, thr)
        ref_lists = O.progressive_lists(sc["saliency"], sc["layer"], plan.n_layers, thr)
    else:
        ref_lists = lists_override
        lists = [dev(torch, np.concatenate([x, np.zeros(1, np.int32)]).astype(np.int32)) for x in ref_lists]
        counts = dev(torch, np.array([[len(x), len(x)] for x in ref_lists], np.int32))
    H = plan.progressive_hologram(coeffs, lists, counts, form=form)
    torch.cuda.synchronize()
    return plan, H.cpu().numpy(), ref_lists


@pytest.mark.parametrize("name", list(SCENES))
def test_progressive_direct_lut(torch_cuda, name):
    sc = SCENES[name]()
    _, H, ref_lists = run_progressive(torch_cuda, sc)
    Href = O.progressive_hologram(sc["intensity"], sc["layer"], ref_lists, _geom(sc))
    assert O.rel_l2(H, Href) <= FP32_TOL


def test_progressive_direct_lut_mask_extremes(torch_cuda):
    torch = torch_cuda
    sc = scenes.random_scene(90, 32, 128, 3)
    g = _geom(sc)
    zero = np.zeros_like(sc["layer"])
    all_lists = [O.select_blocks(zero, sc["layer"], 3, -1, 3)] + [
        O.select_blocks(zero, sc["layer"], 3, -1, l) for l in (1, 2, 3)]
    _, H, _ = run_progressive(torch, sc, lists_override=all_lists)
    Hpw = O.plain_pointwise_hologram(sc["intensity"], sc["layer"], g)
    assert O.rel_l2(H, Hpw) <= FP32_TOL
    e = np.zeros(0, np.int32)
    lll = [all_lists[0], e, e, e]
    _, H0, _ = run_progressive(torch, sc, lists_override=lll)
    assert O.rel_l2(H0, O.progressive_hologram(sc["intensity"], sc["layer"], lll, g)) <= FP32_TOL
    none = [e, e, e, e]
    _, Hn, _ = run_progressive(torch, sc, lists_override=none)
    assert np.all(Hn == 0)


def test_progressive_accumulate(torch_cuda):
    torch = torch_cuda
    sc = scenes.tiny_scene()
    plan = plan_for(sc)
    I, L, S = dev(torch, sc["intensity"]), dev(torch, sc["layer"]), dev(torch, sc["saliency"])
    coeffs = plan.haar_decompose(I, L)
    lists, counts = plan.progressive_lists(S, L, scenes.THRESHOLDS_U8)
    H1 = plan.progressive_hologram(coeffs, lists, counts).clone()
    H2 = plan.progressive_hologram(coeffs, lists, counts, holo=H1.clone(), accumulate=True)
    torch.cuda.synchronize()
    assert O.rel_l2(H2.cpu().numpy(), 2 * H1.cpu().numpy()) < 1e-6


def test_progressive_direct_lut_paper_scale(torch_cuda):
    sc = scenes.paper_scene()
    _, H, ref_lists = run_progressive(torch_cuda, sc)
    Href = O.progressive_hologram(sc["intensity"], sc["layer"], ref_lists, _geom(sc))
    err = O.rel_l2(H, Href)
    print(f"direct_lut 512->1024 Z16 rel-L2 {err:.3e}")
    assert err <= FP32_TOL


@pytest.mark.parametrize("name", ["tiny_64_to_256_z4", "ragged_40x24_s3_z3"])
def test_plain_direct(torch_cuda, name):
    torch = torch_cuda
    sc = SCENES[name]()
    plan = plan_for(sc)
    H = plan.plain_direct(dev(torch, sc["intensity"]), dev(torch, sc["layer"]))
    torch.cuda.synchronize()
    Href = O.plain_pointwise_hologram(sc["intensity"], sc["layer"], _geom(sc))
    assert O.rel_l2(H.cpu().numpy(), Href) <= FP32_TOL


def test_plain_direct_paper_scale_sampled(torch_cuda):
    """512->1024, 16 layers: 192 sampled pixels (corners, edges, random) against the
    brute-force FP64 sum over all 262144 points."""
    torch = torch_cuda
    sc = scenes.paper_scene()
    plan = plan_for(sc)
    H = plan.plain_direct(dev(torch, sc["intensity"]), dev(torch, sc["layer"])).cpu().numpy()
    rng = np.random.default_rng(5)
    mm = np.concatenate([[0, 0, 1023, 1023, 511], rng.integers(0, 1024, 187)])
    nn = np.concatenate([[0, 1023, 0, 1023, 512], rng.integers(0, 1024, 187)])
    ref = O.plain_pointwise_hologram(sc["intensity"], sc["layer"], _geom(sc), pixels=(mm, nn))
    err = O.rel_l2(H[mm, nn], ref)
    print(f"plain direct sampled rel-L2 {err:.3e}")
    assert err <= FP32_TOL


def test_plain_direct_exact_reduction_large_offsets(torch_cuda):
    """P8 on the GPU: a_z = 1/4 makes every fringe value 1 or j; one point in the
    corner of a 512 -> 2048 geometry probes offsets up to 2047 (d^2 ~ 4.2e6)."""
    torch = torch_cuda
    from paper_2211_09938_gb300 import Plan
    z = 8e-6 ** 2 / (2 * 532e-9 * 0.25)
    plan = Plan((512, 512), (2048, 2048), 8e-6, 532e-9, [z])
    I = np.zeros((512, 512), np.uint8)
    I[0, 0] = 200
    H = plan.plain_direct(dev(torch, I), dev(torch, np.zeros((512, 512), np.uint8))).cpu().numpy()
    m = np.arange(2048)
    exp = 200 * (1j ** ((m[:, None] % 2) + (m[None, :] % 2)))
    assert np.max(np.abs(H - exp)) < 200 * 2e-6


def test_selection_rejects_misaligned_inputs(torch_cuda):
    """Blocks are read a row at a time as 8-byte vectors: saliency and layer maps that do
    not start on an 8-byte boundary are refused on the host, before anything runs."""
    torch = torch_cuda
    from paper_2211_09938_gb300.cgh import CghError
    sc = scenes.tiny_scene()
    plan = plan_for(sc)
    buf = torch.zeros(64 * 64 + 8, dtype=torch.uint8, device="cuda")
    L = buf[1:1 + 64 * 64].view(64, 64)  # one byte off
    S = dev(torch, sc["saliency"])
    with pytest.raises(CghError):
        plan.select_blocks(S, L, 127, 1)
    with pytest.raises(CghError):
        plan.progressive_lists(S, L, scenes.THRESHOLDS_U8)


def test_select_large_count_table(torch_cuda):
    """A 512x512 object with 40 layers (a level-1 count table of 40 layers x 256 chunks):
    the oracle's lists bit for bit, capacity overflow included."""
    torch = torch_cuda
    sc = scenes.random_scene(99, 512, 1024, 40, graded=True)
    plan = plan_for(sc)
    S, L = dev(torch, sc["saliency"]), dev(torch, sc["layer"])
    ref_lists = O.progressive_lists(sc["saliency"], sc["layer"], 40, scenes.THRESHOLDS_U8)
    lists, counts = plan.progressive_lists(S, L, scenes.THRESHOLDS_U8)
    c = counts.cpu().numpy()
    for k in range(4):
        assert c[k, 0] == c[k, 1] == len(ref_lists[k]), k
        assert np.array_equal(lists[k][:c[k, 0]].cpu().numpy(), ref_lists[k]), k
    cap = len(ref_lists[1]) // 3
    out = torch.empty(cap, dtype=torch.int32, device="cuda")
    lst, cnt = plan.select_blocks(S, L, scenes.THRESHOLDS_U8[1], 1, out=out, capacity=cap)
    cc = cnt.cpu().numpy()
    assert cc[0] == cap and cc[1] == len(ref_lists[1])
    assert np.array_equal(lst.cpu().numpy(), ref_lists[1][:cap])


def test_select_many_scan_blocks(torch_cuda):
    """A 1024x1024 object with 64 layers: the level-1 count table (64 layers x 1024 chunks)
    spans 16 scan blocks, so list offsets cross block boundaries in every layer."""
    torch = torch_cuda
    sc = scenes.random_scene(98, 1024, 1024, 64, graded=True)
    plan = plan_for(sc)
    S, L = dev(torch, sc["saliency"]), dev(torch, sc["layer"])
    ref_lists = O.progressive_lists(sc["saliency"], sc["layer"], 64, scenes.THRESHOLDS_U8)
    for _ in range(2):  # the scan's CTA counter restarts on every call
        lists, counts = plan.progressive_lists(S, L, scenes.THRESHOLDS_U8)
        c = counts.cpu().numpy()
        for k in range(4):
            assert c[k, 0] == c[k, 1] == len(ref_lists[k]), k
            assert np.array_equal(lists[k][:c[k, 0]].cpu().numpy(), ref_lists[k]), k


@pytest.mark.parametrize("n_layers", [32, 33])
def test_select_fused_table_limit(torch_cuda, n_layers):
    """512x512 object: 32 layers give a level-1 count table of exactly 8192 entries (the
    single-launch selection), 33 layers one chunk column more (the three passes).  Both give
    the oracle's lists bit for bit, through cgh_select_progressive and cgh_select_blocks."""
    torch = torch_cuda
    sc = scenes.random_scene(300 + n_layers, 512, 1024, n_layers, graded=True)
    plan = plan_for(sc)
    S, L = dev(torch, sc["saliency"]), dev(torch, sc["layer"])
    ref_lists = O.progressive_lists(sc["saliency"], sc["layer"], n_layers, scenes.THRESHOLDS_U8)
    lists, counts = plan.progressive_lists(S, L, scenes.THRESHOLDS_U8)
    c = counts.cpu().numpy()
    for k in range(4):
        assert c[k, 0] == c[k, 1] == len(ref_lists[k]), k
        assert np.array_equal(lists[k][:c[k, 0]].cpu().numpy(), ref_lists[k]), k
    lst, cnt = plan.select_blocks(S, L, scenes.THRESHOLDS_U8[1], 1)
    cc = cnt.cpu().numpy()
    assert cc[0] == cc[1] == len(ref_lists[1])
    assert np.array_equal(lst[:cc[0]].cpu().numpy(), ref_lists[1])
    assert plan.status() == 0


def test_select_max_object(torch_cuda):
    """The largest object the plan accepts (8192 x 8192, 4 layers plus unassigned pixels):
    the four lists (up to 5.8 million entries, block coordinates up to 4095) equal the
    oracle's bit for bit; the count table takes the three-pass selection."""
    torch = torch_cuda
    from paper_2211_09938_gb300 import Plan
    n, Z = 8192, 4
    rng = np.random.default_rng(8192)
    layer = np.repeat(np.arange(Z, dtype=np.uint8), n // Z)[:, None].repeat(n, 1)
    layer[rng.random((n, n)) < 0.01] = 255  # pixels owned by no layer
    sal = rng.integers(0, 256, size=(n, n), dtype=np.uint8)
    plan = Plan((n, n), (n, n), 8e-6, 532e-9, [0.10, 0.11, 0.12, 0.13])
    lists, counts = plan.progressive_lists(dev(torch, sal), dev(torch, layer), scenes.THRESHOLDS_U8)
    c = counts.cpu().numpy()
    ref = O.progressive_lists(sal, layer, Z, scenes.THRESHOLDS_U8)
    for k in range(4):
        assert c[k, 0] == c[k, 1] == len(ref[k]), k
        assert np.array_equal(lists[k][:c[k, 0]].cpu().numpy(), ref[k]), k
    assert plan.status() == 0


def _lists_vectorised(sal, layer, n_layers, thresholds):
    """The four work lists from the pinned oracle's per-layer selection masks, vectorised
    per layer (the oracle's own list builder loops in Python, too slow at 8192^2)."""
    out = []
    for k, level in enumerate((3, 1, 2, 3)):
        thr = -1 if k == 0 else thresholds[level]
        parts = []
        for z in range(n_layers):
            by, bx = np.nonzero(O.selected_mask(sal, layer, z, thr, level))
            parts.append((z << 24) | (by.astype(np.int64) << 12) | bx)
        out.append(np.concatenate(parts).astype(np.int32))
    return out


def _ml_inputs(rng, n, n_layers, pattern):
    """Saliency and layer maps for the multi-level selection.  smooth: a noisy saliency
    bump over sinusoidal layer bands with a few pixels on no layer (blocks of one, two and
    rarely more layers); noise: every pixel's layer and saliency at random, 5% on no layer
    (most blocks hold three or more layers); flat: saliency and layer constant on 8x8 and
    16x16 tiles, saliency values at and just above each threshold (the one-value paths)."""
    if pattern == "smooth":
        yy, xx = np.mgrid[0:n, 0:n] / n
        sal = np.clip(255 * np.exp(-((yy - 0.4) ** 2 + (xx - 0.6) ** 2) / 0.05) + rng.normal(0, 8, (n, n)),
                      0, 255).astype(np.uint8)
        layer = (np.floor((0.5 + 0.5 * np.sin(6 * yy + 3 * xx)) * n_layers).clip(0, n_layers - 1)).astype(np.uint8)
        layer[rng.random((n, n)) < 0.002] = 255  # a few pixels on no layer
    elif pattern == "noise":
        sal = rng.integers(0, 256, (n, n), dtype=np.uint8)
        layer = rng.integers(0, n_layers, (n, n), dtype=np.uint8)
        layer[rng.random((n, n)) < 0.05] = 255
    else:
        t = list(scenes.THRESHOLDS_U8.values())
        vals = np.array(sorted({0, 255} | set(t) | {x + 1 for x in t}), np.uint8)
        sal = np.kron(rng.choice(vals, (n // 8, n // 8)), np.ones((8, 8), np.uint8))
        tiles = rng.integers(0, n_layers + 1, (n // 16, n // 16)).astype(np.uint8)
        tiles[tiles == n_layers] = 255  # tiles with no point
        layer = np.kron(tiles, np.ones((16, 16), np.uint8))
    return sal, layer


@pytest.mark.parametrize("n,n_layers,pattern", [(2048, 6, "smooth"), (4096, 3, "smooth"), (8192, 4, "smooth"),
                                                (2048, 5, "noise"), (2048, 7, "flat")])
def test_select_multilevel_large_objects(torch_cuda, n, n_layers, pattern):
    """Objects whose width is a multiple of 2048 take the multi-level selection (one read
    of the inputs for all four lists, then per-block records): bit-exact against the
    oracle's selection masks, with a truncating capacity on the level-1 list, and through
    the tensor-form step (which marks the operand flags in the same pass) equal to the
    two-call path bit for bit on a deterministic plan."""
    torch = torch_cuda
    from paper_2211_09938_gb300 import Plan
    rng = np.random.default_rng(n + n_layers)
    sal, layer = _ml_inputs(rng, n, n_layers, pattern)
    want = _lists_vectorised(sal, layer, n_layers, scenes.THRESHOLDS_U8)
    sc = dict(intensity=np.zeros((n, n), np.uint8), layer=layer, saliency=sal,
              z=np.linspace(0.08, 0.2, n_layers), holo=(n, n), pitch=8e-6, wavelength=532e-9)
    plan = Plan.for_scene(sc)
    S = torch.from_numpy(sal).cuda()
    L = torch.from_numpy(layer).cuda()
    lists, counts = plan.progressive_lists(S, L, scenes.THRESHOLDS_U8)
    c = counts.cpu().numpy()
    for k in range(4):
        assert c[k, 0] == c[k, 1] == len(want[k]), (k, c[k], len(want[k]))
        assert np.array_equal(lists[k][:c[k, 0]].cpu().numpy(), want[k]), k
    cap = len(want[1]) // 3
    short = [l.clone() for l in lists]
    short[1] = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
    l2, c2 = plan.progressive_lists(S, L, scenes.THRESHOLDS_U8, lists=short)
    c2 = c2.cpu().numpy()
    assert c2[1].tolist() == [cap, len(want[1])]
    assert np.array_equal(l2[1].cpu().numpy(), want[1][:cap])
    plan.close()
    if n == 2048:
        I = torch.from_numpy(rng.integers(0, 256, (n, n), dtype=np.uint8)).cuda()
        dplan = Plan.for_scene(sc, flags=Plan.DETERMINISTIC)
        coeffs = dplan.haar_decompose(I, L)
        H1, ls, cs = dplan.progressive_step(S, L, coeffs, scenes.THRESHOLDS_U8, form="tc_fp16x3")
        lo, co = dplan.progressive_lists(S, L, scenes.THRESHOLDS_U8)
        H2 = dplan.progressive_hologram(coeffs, lo, co, form="tc_fp16x3")
        torch.cuda.synchronize()
        assert dplan.status() == 0
        assert torch.equal(H1, H2)
        dplan.close()
