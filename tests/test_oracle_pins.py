"""Pins of the FP64 oracle against things other than itself: closed forms, exact
roots of unity, brute force, invariants and the numbers Section 3 prints.

Each test names the oracle function it pins and the mistake it would catch."""
import os

import numpy as np
import pytest

from oracle import cgh_oracle as O
from synth import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
PITCH, LAM = 8e-6, 532e-9


def z_for_rate(a):
    """Distance at which the Fresnel rate p^2/(2 lambda z) equals a."""
    return PITCH * PITCH / (2.0 * LAM * a)


def all_salient_lists(layer, n_layers, levels=3):
    """LLL + every occupied detail block (threshold -1 at every level)."""
    return [O.select_blocks(np.zeros_like(layer), layer, n_layers, -1, levels)] + [
        O.select_blocks(np.zeros_like(layer), layer, n_layers, -1, l) for l in range(1, levels + 1)]


def lll_only_lists(layer, n_layers, levels=3):
    e = np.zeros(0, np.int32)
    return [O.select_blocks(np.zeros_like(layer), layer, n_layers, -1, levels), e, e, e]


def read_haar_examples():
    out = []
    lines = [l.strip() for l in open(os.path.join(GOLDEN, "haar_worked_examples.txt"))
             if l.strip() and not l.startswith("#")]
    k = 0
    while k < len(lines):
        levels = int(lines[k].split()[1])
        k += 1
        inp = []
        while lines[k] != "->":
            inp.append([int(v) for v in lines[k].split()])
            k += 1
        k += 1
        n = len(inp)
        exp = [[int(v) for v in lines[k + r].split()] for r in range(n)]
        k += n
        out.append((levels, np.array(inp), np.array(exp)))
    return out


# ---------------------------------------------------------------- fringe (P8)

def test_fringe_quarter_rate_is_exact_roots_of_unity():
    """P8: a_z = 1/4 gives f(d) = 1 for even d and +j for odd d (d^2 = 0 or 1 mod 4).
    Catches a wrong sign of the phase (would give -j), a missing square, and a lossy
    range reduction at large offsets."""
    a = O.fresnel_rate(PITCH, LAM, z_for_rate(0.25))
    d = np.arange(-4096, 4097)
    f = O.point_fringe_1d(d, a)
    exp = np.where(d % 2 == 0, 1.0 + 0j, 1j)
    assert np.max(np.abs(f - exp)) < 1e-8


def test_fringe_eighth_rate():
    """P8: a_z = 1/8: d = 0 mod 4 -> 1, d = 2 mod 4 -> -1, d odd -> exp(j pi/4)."""
    a = O.fresnel_rate(PITCH, LAM, z_for_rate(0.125))
    d = np.arange(-4096, 4097)
    f = O.point_fringe_1d(d, a)
    exp = np.where(d % 4 == 0, 1.0 + 0j, np.where(d % 4 == 2, -1.0 + 0j, np.exp(1j * np.pi / 4)))
    assert np.max(np.abs(f - exp)) < 1e-8


def test_fringe_unit_modulus_and_even():
    a = O.fresnel_rate(PITCH, LAM, 0.1)
    d = np.arange(0, 3000)
    f = O.point_fringe_1d(d, a)
    assert np.allclose(np.abs(f), 1.0, atol=1e-14)
    assert np.allclose(f, O.point_fringe_1d(-d, a), atol=0)


def test_fresnel_rate_value():
    """a_z = p^2 / (2 lambda z): at p = 8 um, lambda = 532 nm, z = 0.1 m the
    paraxial phase pi (d p)^2/(lambda z) is 2 pi * 6.0150e-4 * d^2."""
    a = O.fresnel_rate(PITCH, LAM, 0.1)
    assert abs(a - 6.4e-11 / (2 * 532e-9 * 0.1)) < 1e-18
    assert abs(a - 6.015037593984962e-4) < 1e-15


# ---------------------------------------------------------------- Haar (P3)

def test_haar_worked_examples():
    """Hand-derived examples (tests/golden): catches swapped X/Y bands, a wrong
    sign in D and a wrong Mallat quadrant."""
    for levels, inp, exp in read_haar_examples():
        got = O.haar_forward(inp, levels)
        assert np.array_equal(got, exp), (levels, got, exp)


def test_haar_perfect_reconstruction_all_binary_cells():
    """P3 brute force: every 2x2 cell with values in {0, 255} (16 cells) and every
    4x4 ... 8x8 tiling of them inverts exactly."""
    for bits in range(16):
        v = [(bits >> k) & 1 for k in range(4)]
        A = 255 * np.array([[v[0], v[1]], [v[2], v[3]]])
        C = O.haar_forward(A, 1)
        assert np.array_equal(O.haar_inverse(C, 1), A)
    rng = np.random.default_rng(3)
    for _ in range(20):
        A = 255 * rng.integers(0, 2, size=(8, 8))
        assert np.array_equal(O.haar_inverse(O.haar_forward(A, 3), 3), A)


def test_haar_perfect_reconstruction_random_and_scaled():
    rng = np.random.default_rng(0)
    A = rng.integers(0, 256, size=(32, 48))
    C = O.haar_forward(A, 3)
    assert np.array_equal(O.haar_inverse(C, 3), A)
    keep = {l: np.ones((32 >> l, 48 >> l), bool) for l in (1, 2, 3)}
    assert np.array_equal(O.haar_synthesis_scaled(C, keep, 3), 64 * A)
    assert np.allclose(O.haar_synthesis_real(O.haar_forward_real(A, 3), keep, 3), A)


def test_haar_ranges():
    """LL3 of an 8x8 block is at most 64*255 = 16320; |detail| at level 3 at most 32*255."""
    A = np.full((8, 8), 255)
    C = O.haar_forward(A, 3)
    assert C[0, 0] == 16320
    A = np.zeros((8, 8), int)
    A[:, :4] = 255
    C = O.haar_forward(A, 3)
    assert C[0, 1] == 8160  # X3 = (left half) - (right half) = 32 * 255


def test_haar_lowpass_only_gives_block_means():
    """Dropping every detail gives the 8x8 block means (times 64 exactly)."""
    rng = np.random.default_rng(1)
    A = rng.integers(0, 256, size=(16, 24))
    C = O.haar_forward(A, 3)
    keep = {l: np.zeros((16 >> l, 24 >> l), bool) for l in (1, 2, 3)}
    V = O.haar_synthesis_scaled(C, keep, 3)
    means = A.reshape(2, 8, 3, 8).sum(axis=(1, 3))
    assert np.array_equal(V, np.kron(means, np.ones((8, 8), int)))


# ---------------------------------------------------------------- selection

def brute_select(sal, layer, n_layers, threshold, level):
    """Pixel-by-pixel scan (no reshapes): independent of the oracle's block max."""
    k = 1 << level
    h, w = sal.shape
    out = []
    for z in range(n_layers):
        for by in range(h // k):
            for bx in range(w // k):
                occ = False
                mx = -1
                for y in range(by * k, by * k + k):
                    for x in range(bx * k, bx * k + k):
                        occ = occ or layer[y, x] == z
                        mx = max(mx, int(sal[y, x]))
                if occ and (threshold < 0 or mx > threshold):
                    out.append(z * (1 << 24) + by * 4096 + bx)
    return out


def test_select_blocks_brute_force():
    rng = np.random.default_rng(5)
    sal = rng.integers(0, 256, size=(16, 24)).astype(np.uint8)
    layer = rng.integers(0, 3, size=(16, 24)).astype(np.uint8)
    layer[:8, :8] = 0  # a block owned by a single layer
    for level in (1, 2, 3):
        for t in (-1, 0, 127, 200, 255):
            got = O.select_blocks(sal, layer, 3, t, level).tolist()
            assert got == brute_select(sal, layer, 3, t, level), (level, t)


def test_select_threshold_is_strict():
    sal = np.full((8, 8), 127, np.uint8)
    layer = np.zeros((8, 8), np.uint8)
    assert O.select_blocks(sal, layer, 1, 127, 3).size == 0
    assert O.select_blocks(sal, layer, 1, 126, 3).size == 1


def test_pack_roundtrip():
    for z, by, bx in ((0, 0, 0), (31, 4095, 4095), (7, 12, 345)):
        assert O.unpack_entry(O.pack_entry(z, by, bx)) == (z, by, bx)


def test_operator_counts_of_section_3():
    """P6: at 256x256 the LLL needs 1024 operators and the point-wise hologram
    65536 (values printed in Section 3, tests/golden/operator_counts.txt); with every
    detail block selected the detail-basis term count equals the pixel count."""
    vals = {}
    for l in open(os.path.join(GOLDEN, "operator_counts.txt")):
        if l.strip() and not l.startswith("#"):
            k, v = l.split()
            vals[k] = int(v)
    n = vals["object_edge"]
    layer = np.zeros((n, n), np.uint8)
    lists = all_salient_lists(layer, 1)
    assert len(lists[0]) == vals["lll_operators"]
    assert n * n == vals["pointwise_operators"]
    assert O.detail_term_count(lists) == vals["pointwise_operators"]


def _hand_scene_16():
    layer = np.zeros((16, 16), np.uint8)
    layer[:, 6:] = 1
    sal = np.zeros((16, 16), np.uint8)
    sal[5, 5] = 240
    return layer, sal


def test_operator_count_hand_counted_16x16():
    """operator_count (reading R20: 1 per LLL block, 1 per residual-map cell) against a
    count done by hand on a 16x16 two-layer object with one salient pixel
    (tests/golden/operator_counts_16x16.txt).  Also pins the four lists entry by entry.
    A weight of 3 per detail block (the detail-coefficient count) gives 21, not 26."""
    want, vals = {0: [], 1: [], 2: [], 3: []}, {}
    for line in open(os.path.join(GOLDEN, "operator_counts_16x16.txt")):
        f = line.split()
        if not f or f[0].startswith("#"):
            continue
        if f[0] == "entry":
            want[int(f[1])].append(O.pack_entry(int(f[2]), int(f[3]), int(f[4])))
        else:
            vals[f[0]] = int(f[1])
    layer, sal = _hand_scene_16()
    lists = O.progressive_lists(sal, layer, 2, scenes.THRESHOLDS_U8)
    for k in range(4):
        assert lists[k].tolist() == want[k], k
    assert O.operator_count(lists) == vals["operators"]
    assert layer.size == vals["pointwise_operators"]


def _residual_cells_superposed(lists, n_layers, obj_shape, levels=3):
    """Walks the loop of the residual-map form (Section 2 steps 2-5) and counts the cells
    it superposes with a LUT block: one per listed LLL block, and at each level every
    cell of the residual grid that the strided 2x2 synthesis of a selected block
    writes to.  No weight is written down: the cells are counted where they land."""
    masks = O.masks_from_lists(lists, n_layers, obj_shape, levels)
    Ho, Wo = obj_shape
    total = 0
    for z in range(n_layers):
        total += int(masks[0][z].sum())
        for l in range(levels, 0, -1):
            h, w = Ho >> l, Wo >> l
            cells = np.zeros((2 * h, 2 * w), dtype=bool)
            for r in (0, 1):
                for c in (0, 1):
                    cells[r::2, c::2] |= masks[l][z]
            total += int(cells.sum())
    return total


@pytest.mark.parametrize("seed,n,n_layers", [(51, 32, 3), (52, 64, 5), (53, 16, 1)])
def test_operator_count_equals_superposed_residual_cells(seed, n, n_layers):
    """operator_count equals the number of LUT-block superpositions the residual-map
    loop performs, on graded scenes where every level selects a different subset."""
    sc = scenes.random_scene(seed, n, 2 * n, n_layers, graded=True)
    lists = O.progressive_lists(sc["saliency"], sc["layer"], n_layers, scenes.THRESHOLDS_U8)
    assert all(len(x) > 0 for x in lists)
    assert O.operator_count(lists) == _residual_cells_superposed(lists, n_layers, (n, n))
    # each cumulative stage of the level sweep as well
    e = np.zeros(0, np.int32)
    for keep in ((0,), (0, 3), (0, 3, 2)):
        st = [lists[k] if k in keep else e for k in range(4)]
        assert O.operator_count(st) == _residual_cells_superposed(st, n_layers, (n, n))


# ---------------------------------------------------------------- the comparator


def test_rel_l2_hand_values():
    """rel_l2 = ||x - ref||_2 / ||ref||_2 over all elements (Frobenius for 2-D), complex
    moduli, ||x|| when ref is zero.  Each value is worked out by hand; the comment names
    the plausible slip each one catches."""
    # ||[3,-4]|| / ||[0,4]|| = 5/4; dividing by the squared norm gives 5/16, squaring both 25/16
    assert O.rel_l2(np.array([3.0, 0.0]), np.array([0.0, 4.0])) == pytest.approx(1.25, rel=1e-15)
    # orthogonal perturbation of [3,4] by 0.1*[-4,3]: |d| = 0.5, |ref| = 5
    assert O.rel_l2(np.array([3.0 - 0.4, 4.0 + 0.3]), np.array([3.0, 4.0])) == pytest.approx(0.1, rel=1e-14)
    # conj(j) - j = -2j: a comparator that drops imaginary parts reads 0
    assert O.rel_l2(np.array([-1j]), np.array([1j])) == pytest.approx(2.0, rel=1e-15)
    # purely imaginary error on a real reference: |0.25j| / |2| = 0.125
    assert O.rel_l2(np.array([2.0 + 0.25j]), np.array([2.0])) == pytest.approx(0.125, rel=1e-15)
    # 2-D: difference = identity (Frobenius sqrt 2, spectral 1) over ref = diag(2, 0) (both 2)
    ref = np.array([[2.0, 0.0], [0.0, 0.0]])
    assert O.rel_l2(ref + np.eye(2), ref) == pytest.approx(np.sqrt(2.0) / 2.0, rel=1e-15)
    # zero reference: the absolute norm, |[3, 4j]| = 5
    assert O.rel_l2(np.array([3.0, 4j]), np.zeros(2)) == pytest.approx(5.0, rel=1e-15)
    assert O.rel_l2(np.zeros(3), np.zeros(3)) == 0.0


def test_rel_l2_scaling_and_symmetry_of_scale():
    """rel_l2(ref (1 + e), ref) = |e| for any complex ref and complex e, and the result
    does not change when both arrays are scaled by the same complex factor."""
    rng = np.random.default_rng(7)
    ref = rng.standard_normal((5, 7)) + 1j * rng.standard_normal((5, 7))
    for e in (1e-6, -3e-3, 0.5j, 0.2 - 0.1j):
        assert O.rel_l2(ref * (1 + e), ref) == pytest.approx(abs(e), rel=1e-9)
    x = ref + 1e-3 * rng.standard_normal(ref.shape)
    assert O.rel_l2(x * (3 - 4j), ref * (3 - 4j)) == pytest.approx(O.rel_l2(x, ref), rel=1e-12)


# ---------------------------------------------------------------- holograms

def tiny_geom(n=8, s=4, n_layers=1, a=None, z=None):
    if z is None:
        z = [z_for_rate(a)] * n_layers if a is not None else np.linspace(0.001, 0.0015, n_layers)
    return O.Geometry((n, n), (n * s, n * s), PITCH, LAM, z)


def test_single_point_closed_form_quarter_rate():
    """P1: one pixel of value v, everything salient, a = 1/4: H(m, n) = v * j^(odd(dm)
    + odd(dn)) with dm = m - s i, dn = n - s j.  Catches a wrong stride, a transposed
    offset, a dropped residual level and a wrong Haar scale."""
    n, s = 16, 4
    g = tiny_geom(n, s, 1, a=0.25)
    for (i, j, v) in ((0, 0, 255), (5, 11, 17), (15, 3, 200)):
        I = np.zeros((n, n), np.int64)
        I[i, j] = v
        layer = np.zeros((n, n), np.uint8)
        H = O.progressive_hologram(I, layer, all_salient_lists(layer, 1), g)
        m = np.arange(n * s)[:, None] - s * i
        q = np.arange(n * s)[None, :] - s * j
        exp = v * (1j ** ((m % 2) + (q % 2)))
        assert np.max(np.abs(H - exp)) < 1e-7 * v


def test_single_point_closed_form_general_rate():
    """P1 at a generic rate: H(s i + dm, s j + dn) = v exp(j pi p^2 (dm^2+dn^2)/(lambda z))
    checked at a few offsets from the physical formula in radians."""
    n, s = 16, 2
    z = 0.0123
    g = O.Geometry((n, n), (n * s, n * s), PITCH, LAM, [z])
    I = np.zeros((n, n), np.int64)
    I[6, 9] = 100
    layer = np.zeros((n, n), np.uint8)
    H = O.progressive_hologram(I, layer, all_salient_lists(layer, 1), g)
    for (dm, dn) in ((0, 0), (1, 0), (0, 3), (-7, 5), (13, -11)):
        phase = np.pi * ((dm * PITCH) ** 2 + (dn * PITCH) ** 2) / (LAM * z)
        assert abs(H[12 + dm, 18 + dn] - 100 * np.exp(1j * phase)) < 1e-9


def test_linearity():
    """P2: H(alpha A + beta B) = alpha H(A) + beta H(B) with the same masks."""
    n = 16
    rng = np.random.default_rng(7)
    g = tiny_geom(n, 2, 2)
    layer = rng.integers(0, 2, size=(n, n)).astype(np.uint8)
    sal = rng.integers(0, 256, size=(n, n)).astype(np.uint8)
    lists = O.progressive_lists(sal, layer, 2, scenes.THRESHOLDS_U8)
    A = rng.integers(0, 100, size=(n, n))
    B = rng.integers(0, 100, size=(n, n))
    HA = O.progressive_hologram(A, layer, lists, g)
    HB = O.progressive_hologram(B, layer, lists, g)
    HAB = O.progressive_hologram(2 * A + 3 * B, layer, lists, g)
    assert O.rel_l2(HAB, 2 * HA + 3 * HB) < 1e-12


def test_all_salient_equals_pointwise():
    """P4a: with every detail block kept the progressive hologram equals the plain
    point-wise hologram of the object (the basis is complete)."""
    n = 16
    sc = scenes.random_scene(11, n, 2 * n, 3)
    g = O.geometry_of(sc)
    lists = all_salient_lists(sc["layer"], 3)
    H = O.progressive_hologram(sc["intensity"], sc["layer"], lists, g)
    planes = O.object_planes(sc["intensity"], sc["layer"], 3)
    Href = O.pointwise_hologram_direct(planes, g)
    assert O.rel_l2(H, Href) < 1e-11


def test_empty_mask_equals_block_mean_image():
    """P4b: with no detail block selected the hologram equals the point-wise hologram
    of the per-layer 8x8 block-mean image."""
    n = 16
    sc = scenes.random_scene(12, n, 2 * n, 2)
    g = O.geometry_of(sc)
    lists = lll_only_lists(sc["layer"], 2)
    H = O.progressive_hologram(sc["intensity"], sc["layer"], lists, g)
    planes = O.object_planes(sc["intensity"], sc["layer"], 2).astype(np.float64)
    means = planes.reshape(2, 2, 8, 2, 8).mean(axis=(2, 4))
    blocky = np.stack([np.kron(means[z], np.ones((8, 8))) for z in range(2)])
    Href = O.pointwise_hologram_direct(blocky, g)
    assert O.rel_l2(H, Href) < 1e-11


def test_arbitrary_mask_residual_form_equals_pointwise_of_progressive_object():
    """P5: the residual-map form (block fringes per level) equals the point-wise
    hologram of the progressively reconstructed object (two independent paths)."""
    n = 32
    sc = scenes.random_scene(13, n, 2 * n, 3, graded=True)
    g = O.geometry_of(sc)
    lists = O.progressive_lists(sc["saliency"], sc["layer"], 3, scenes.THRESHOLDS_U8)
    assert all(len(x) for x in lists)  # every level has work
    H = O.progressive_hologram(sc["intensity"], sc["layer"], lists, g)
    Ahat = O.progressive_object(sc["intensity"], sc["layer"], lists, 3) / 64.0
    Href = O.pointwise_hologram_separable(Ahat, g)
    assert O.rel_l2(H, Href) < 1e-11


def test_lists_that_are_not_nested():
    """P5 for lists that are not nested (detail blocks without their LLL block, e.g. a
    truncated LLL list): the residual-map form still equals the point-wise hologram of the
    progressive object, and the hologram is additive over any split of the entries.
    Catches a superposition that drops (or needs) the LLL block under a detail block."""
    n = 32
    sc = scenes.random_scene(14, n, 2 * n, 3, graded=True)
    g = O.geometry_of(sc)
    full = O.progressive_lists(sc["saliency"], sc["layer"], 3, scenes.THRESHOLDS_U8)
    assert all(len(x) for x in full)
    part_a = [full[0][: len(full[0]) // 3], full[1][::2], full[2][1::2], full[3]]
    part_b = [full[0][len(full[0]) // 3:], full[1][1::2], full[2][::2], np.zeros(0, np.int32)]
    Ha = O.progressive_hologram(sc["intensity"], sc["layer"], part_a, g)
    Ahat = O.progressive_object(sc["intensity"], sc["layer"], part_a, 3) / 64.0
    assert O.rel_l2(Ha, O.pointwise_hologram_separable(Ahat, g)) < 1e-11
    Hb = O.progressive_hologram(sc["intensity"], sc["layer"], part_b, g)
    H = O.progressive_hologram(sc["intensity"], sc["layer"], full, g)
    assert O.rel_l2(Ha + Hb, H) < 1e-12
    # detail blocks alone: the object is their residual only (zero block mean)
    details = [np.zeros(0, np.int32), full[1], full[2], full[3]]
    Ad = O.progressive_object(sc["intensity"], sc["layer"], details, 3)
    assert np.all(Ad.reshape(3, n // 8, 8, n // 8, 8).sum(axis=(2, 4)) == 0)


def test_progressive_object_extremes():
    rng = np.random.default_rng(2)
    I = rng.integers(0, 256, size=(16, 16))
    layer = np.zeros((16, 16), np.uint8)
    full = O.progressive_object(I, layer, all_salient_lists(layer, 1), 1)
    assert np.array_equal(full[0], 64 * I)
    none = O.progressive_object(I, layer, lll_only_lists(layer, 1), 1)
    means = I.reshape(2, 8, 2, 8).sum(axis=(1, 3))
    assert np.array_equal(none[0], np.kron(means, np.ones((8, 8), int)))


def test_direct_equals_separable():
    """P7: brute-force 2-D sum (full squared distance) equals E A E^T (factorised)."""
    rng = np.random.default_rng(8)
    g = tiny_geom(12, 3, 2)
    planes = rng.uniform(-1, 1, size=(2, 12, 12))
    Hd = O.pointwise_hologram_direct(planes, g)
    Hs = O.pointwise_hologram_separable(planes, g)
    assert O.rel_l2(Hs, Hd) < 1e-12


def test_direct_sampled_pixels():
    rng = np.random.default_rng(9)
    g = tiny_geom(8, 4, 1)
    planes = rng.uniform(0, 1, size=(1, 8, 8))
    Hs = O.pointwise_hologram_separable(planes, g)
    mm = np.array([0, 5, 31, 17])
    nn = np.array([3, 0, 31, 22])
    Hp = O.pointwise_hologram_direct(planes, g, (mm, nn))
    assert np.allclose(Hp, Hs[mm, nn], atol=1e-12)


# ---------------------------------------------------------------- reconstruction / adjoint

def test_backprop_of_single_point_peaks_at_point():
    """The back-propagated field of one point's own hologram equals v * Nh^2 at that
    point (every hologram pixel adds |f|^2 = 1)."""
    n, s = 8, 4
    g = tiny_geom(n, s, 1)
    planes = np.zeros((1, n, n))
    planes[0, 3, 5] = 2.0
    H = O.pointwise_hologram_separable(planes, g)
    R = O.reconstruct_fields(H, g)
    assert abs(R[0, 3, 5] - 2.0 * (n * s) ** 2) < 1e-8


def test_adjoint_dot_product():
    """P9: <F(I), G> = <I, F^*(G)> for the real-input progressive operator."""
    n = 16
    rng = np.random.default_rng(21)
    sc = scenes.random_scene(21, n, 2 * n, 2, graded=True)
    g = O.geometry_of(sc)
    lists = O.progressive_lists(sc["saliency"], sc["layer"], 2, scenes.THRESHOLDS_U8)
    I = rng.integers(0, 256, size=(n, n))
    G = rng.normal(size=(2 * n, 2 * n)) + 1j * rng.normal(size=(2 * n, 2 * n))
    FI = O.progressive_hologram(I, sc["layer"], lists, g)
    lhs = np.real(np.vdot(FI, G))
    rhs = float(np.sum(I * O.progressive_adjoint(G, sc["layer"], lists, g)))
    assert abs(lhs - rhs) <= 1e-10 * max(1.0, abs(lhs))


def test_progressive_hologram_real_integer_case_linearity_and_adjoint():
    """progressive_hologram_real: on an integer object it equals the residual-map form
    (progressive_hologram, pinned by P1-P5); it is linear over real objects; and
    <F(x), G> = <x, F^*(G)> with progressive_adjoint for a real, non-integer x."""
    n = 16
    rng = np.random.default_rng(23)
    sc = scenes.random_scene(23, n, 2 * n, 3, graded=True)
    g = O.geometry_of(sc)
    lists = O.progressive_lists(sc["saliency"], sc["layer"], 3, scenes.THRESHOLDS_U8)
    Hi = O.progressive_hologram(sc["intensity"], sc["layer"], lists, g)
    assert O.rel_l2(O.progressive_hologram_real(sc["intensity"].astype(np.float64), sc["layer"], lists, g),
                    Hi) < 1e-12
    x = rng.normal(size=(n, n)) * 50.0
    y = rng.normal(size=(n, n)) * 50.0
    Fx = O.progressive_hologram_real(x, sc["layer"], lists, g)
    Fy = O.progressive_hologram_real(y, sc["layer"], lists, g)
    assert O.rel_l2(O.progressive_hologram_real(2.0 * x - 0.5 * y, sc["layer"], lists, g), 2.0 * Fx - 0.5 * Fy) < 1e-12
    G = rng.normal(size=(2 * n, 2 * n)) + 1j * rng.normal(size=(2 * n, 2 * n))
    lhs = np.real(np.vdot(Fx, G))
    rhs = float(np.sum(x * O.progressive_adjoint(G, sc["layer"], lists, g)))
    assert abs(lhs - rhs) <= 1e-10 * max(1.0, abs(lhs))


def test_reconstruct_is_adjoint_of_pointwise():
    rng = np.random.default_rng(22)
    g = tiny_geom(8, 2, 2)
    planes = rng.normal(size=(2, 8, 8))
    G = rng.normal(size=(16, 16)) + 1j * rng.normal(size=(16, 16))
    lhs = np.real(np.vdot(O.pointwise_hologram_separable(planes, g), G))
    R = O.reconstruct_fields(G, g)
    rhs = float(np.sum(planes * np.real(R)))
    assert abs(lhs - rhs) <= 1e-10 * abs(lhs)


# ---------------------------------------------------------------- SSIM (P10)

def brute_ssim(x, y, win=11, sigma=1.5, c1=1e-4, c2=9e-4):
    t = np.arange(win) - (win - 1) / 2.0
    w = np.exp(-(t[:, None] ** 2 + t[None, :] ** 2) / (2 * sigma * sigma))
    w /= w.sum()
    vals = []
    for r in range(x.shape[0] - win + 1):
        for c in range(x.shape[1] - win + 1):
            px, py = x[r:r + win, c:c + win], y[r:r + win, c:c + win]
            mx, my = np.sum(w * px), np.sum(w * py)
            vx = np.sum(w * (px - mx) ** 2)
            vy = np.sum(w * (py - my) ** 2)
            cxy = np.sum(w * (px - mx) * (py - my))
            vals.append((2 * mx * my + c1) * (2 * cxy + c2) / ((mx * mx + my * my + c1) * (vx + vy + c2)))
    return float(np.mean(vals))


def test_ssim_identity_and_brute_force():
    rng = np.random.default_rng(4)
    x = rng.uniform(0, 1, size=(20, 18))
    y = np.clip(x + rng.normal(0, 0.1, size=x.shape), 0, 1)
    assert abs(O.ssim(x, x) - 1.0) < 1e-12
    assert abs(O.ssim(x, y) - brute_ssim(x, y)) < 1e-10
    assert O.ssim(x, y) < 0.99


def test_all_salient_reconstruction_ssim_is_one():
    """P10: all-salient progressive reconstruction has SSIM 1 against the point-wise one."""
    n = 32
    sc = scenes.random_scene(31, n, 2 * n, 2)
    g = O.geometry_of(sc)
    Hp = O.progressive_hologram(sc["intensity"], sc["layer"], all_salient_lists(sc["layer"], 2), g)
    Hf = O.plain_pointwise_hologram(sc["intensity"], sc["layer"], g)
    a1 = O.composite_amplitude(O.reconstruct_fields(Hp, g), sc["layer"])
    a2 = O.composite_amplitude(O.reconstruct_fields(Hf, g), sc["layer"])
    assert abs(O.ssim(a1 / a2.max(), a2 / a2.max()) - 1.0) < 1e-9


def test_progressive_levels_improve_quality():
    """Section 3 (Table 3 trend): the LLL-only reconstruction has lower SSIM against the
    point-wise reference than the progressive one, which is lower than all-salient."""
    n = 32
    sc = scenes.random_scene(32, n, 2 * n, 1, graded=True)
    g = O.geometry_of(sc)
    Hf = O.plain_pointwise_hologram(sc["intensity"], sc["layer"], g)
    ref = O.composite_amplitude(O.reconstruct_fields(Hf, g), sc["layer"])
    ref = ref / ref.max()

    def q(lists):
        H = O.progressive_hologram(sc["intensity"], sc["layer"], lists, g)
        a = O.composite_amplitude(O.reconstruct_fields(H, g), sc["layer"])
        return O.ssim(a / ref.max() / (a.max() / ref.max()), ref)

    s_lll = q(lll_only_lists(sc["layer"], 1))
    s_prog = q(O.progressive_lists(sc["saliency"], sc["layer"], 1, {3: 0, 2: 100, 1: 200}))
    s_all = q(all_salient_lists(sc["layer"], 1))
    assert s_lll < s_prog < s_all


# ---------------------------------------------------------------- propagation / phase optimisation

def test_propagate_is_adjoint_of_reconstruct():
    """<reconstruct(H), F> = <H, propagate(F)> for complex H and F (real inner product)."""
    rng = np.random.default_rng(41)
    g = tiny_geom(8, 2, 3)
    H = rng.normal(size=(16, 16)) + 1j * rng.normal(size=(16, 16))
    F = rng.normal(size=(3, 8, 8)) + 1j * rng.normal(size=(3, 8, 8))
    lhs = np.real(np.vdot(O.reconstruct_fields(H, g), F))
    rhs = np.real(np.vdot(H, O.propagate_fields(F, g)))
    assert abs(lhs - rhs) <= 1e-10 * abs(lhs)


def test_propagate_real_fields_is_pointwise_and_single_point():
    rng = np.random.default_rng(42)
    g = tiny_geom(8, 4, 2)
    planes = rng.uniform(0, 1, size=(2, 8, 8))
    assert O.rel_l2(O.propagate_fields(planes, g), O.pointwise_hologram_direct(planes, g)) < 1e-12
    # one complex point of value 2j at a = 1/4: H = 2j * j^(odd(dm) + odd(dn))
    g4 = tiny_geom(8, 4, 1, a=0.25)
    F = np.zeros((1, 8, 8), complex)
    F[0, 2, 5] = 2j
    m = np.arange(32)[:, None] - 8
    n = np.arange(32)[None, :] - 20
    assert np.max(np.abs(O.propagate_fields(F, g4) - 2j * 1j ** ((m % 2) + (n % 2)))) < 1e-7


def test_phase_opt_gradient_matches_finite_differences():
    """O7: the analytic phase gradient against central differences of the FP64 loss."""
    rng = np.random.default_rng(43)
    g = tiny_geom(8, 2, 2)
    layer = rng.integers(0, 2, size=(8, 8)).astype(np.uint8)
    target = rng.uniform(0, 1, size=(8, 8))
    weight = np.where(rng.uniform(size=(8, 8)) > 0.5, 4.0, 1.0)
    phase = rng.uniform(-np.pi, np.pi, size=(16, 16))
    kappa = 20.0
    grad = O.phase_opt_grad(phase, target, weight, layer, g, kappa)
    h = 1e-6
    for (m, n) in ((0, 0), (3, 7), (15, 15), (8, 2), (11, 13)):
        e = np.zeros_like(phase)
        e[m, n] = h
        fd = (O.phase_opt_loss(phase + e, target, weight, layer, g, kappa)
              - O.phase_opt_loss(phase - e, target, weight, layer, g, kappa)) / (2 * h)
        assert abs(fd - grad[m, n]) <= 1e-6 * max(1.0, abs(fd)), (m, n, fd, grad[m, n])


# ---------------------------------------------------------------- angular spectrum (A1-A5)

def _signed(k, P):
    return k if k < P // 2 else k - P


def test_asm_brute_force_tiny():
    """A1: the ASM reconstruction against its definition written as explicit sums: the
    forward DFT of the zero-padded hologram, the plane-wave phase advance through the
    direction cosine gamma = sqrt(1 - (lambda fx)^2 - (lambda fy)^2), the inverse DFT at
    the object pixels (s i, s j), and the p^2/(lambda z) scale.  Catches a DFT sign or
    normalisation slip, frequency ordering, the sampling stride and a transposed axis."""
    rng = np.random.default_rng(51)
    n, s = 4, 2
    g = O.Geometry((n, n), (n * s, n * s), PITCH, LAM, [0.004, 0.0065])
    N = n * s
    H = rng.normal(size=(N, N)) + 1j * rng.normal(size=(N, N))
    H[0, 1] += 3.0  # break any symmetry between the axes
    for pad in (1, 2):
        P = pad * N
        X = np.zeros((P, P), complex)
        for k in range(P):
            for l in range(P):
                acc = 0j
                for m in range(N):
                    for q in range(N):
                        acc += H[m, q] * np.exp(-2j * np.pi * (k * m + l * q) / P)
                X[k, l] = acc
        R = O.asm_reconstruct_fields(H, g, pad=pad)
        for zi in range(2):
            z = g.z[zi]
            for i in range(n):
                for j in range(n):
                    acc = 0j
                    for k in range(P):
                        for l in range(P):
                            sy, sx = LAM * _signed(k, P) / (P * PITCH), LAM * _signed(l, P) / (P * PITCH)
                            gamma = np.sqrt(1.0 - sx * sx - sy * sy)
                            T = np.exp(-2j * np.pi * z * (gamma - 1.0) / LAM)
                            acc += X[k, l] * T * np.exp(2j * np.pi * (k * s * i + l * s * j) / P)
                    want = acc / P ** 2 * PITCH ** 2 / (LAM * z)
                    assert abs(R[zi, i, j] - want) <= 1e-12 * max(1.0, abs(want)), (pad, zi, i, j)


def test_asm_is_unitary():
    """A2: |T| = 1 on propagating waves, so with no padding and s = 1 the back-propagated
    field has the hologram's energy (Parseval), up to the p^2/(lambda z) scale."""
    rng = np.random.default_rng(52)
    g = O.Geometry((32, 32), (32, 32), PITCH, LAM, [0.05, 0.12])
    H = rng.normal(size=(32, 32)) + 1j * rng.normal(size=(32, 32))
    R = O.asm_reconstruct_fields(H, g, pad=1)
    for zi in range(2):
        scale = PITCH ** 2 / (LAM * g.z[zi])
        assert abs(np.linalg.norm(R[zi]) / scale / np.linalg.norm(H) - 1.0) < 1e-12


def test_asm_plane_wave_phase():
    """A3: a grid plane wave exp(j 2 pi (ky m + kx n) / N) comes back as itself times
    exp(-j k z (cos(theta) - 1)), cos(theta) the direction cosine along the axis."""
    N = 64
    g = O.Geometry((N, N), (N, N), PITCH, LAM, [0.1])
    m = np.arange(N)
    for ky, kx in ((0, 0), (5, -3), (-31, 17), (32, 32)):
        H = np.exp(2j * np.pi * (ky * m[:, None] + kx * m[None, :]) / N)
        R = O.asm_reconstruct_fields(H, g, pad=1)[0] / (PITCH ** 2 / (LAM * 0.1))
        sin2 = (LAM * ky / (N * PITCH)) ** 2 + (LAM * kx / (N * PITCH)) ** 2
        cos_t = np.sqrt(1.0 - sin2)
        want = H * np.exp(-2j * np.pi / LAM * 0.1 * (cos_t - 1.0))
        assert np.max(np.abs(R - want)) < 1e-9


def test_asm_transfer_fresnel_limit():
    """A4: for lambda f << 1 the transfer function tends to the Fresnel one,
    exp(+j pi lambda z f^2) (the sign that back-propagates the point fringes of Eq. 1),
    with the next term (z / lambda) (lambda f)^4 / 8 cycles bounding the difference."""
    g = O.Geometry((64, 64), (64, 64), PITCH, LAM, [0.2])
    P = 64
    T = O.asm_transfer(g, 0, P)
    f = np.fft.fftfreq(P, d=PITCH)
    f2 = f[None, :] ** 2 + f[:, None] ** 2
    fres = np.exp(1j * np.pi * LAM * 0.2 * f2)
    err_cycles = np.abs(np.angle(T * np.conj(fres))) / (2 * np.pi)
    bound = 1.05 * (0.2 / LAM) * (LAM * LAM * f2) ** 2 / 8.0 + 1e-12
    assert np.all(err_cycles <= bound)
    assert np.all(np.abs(np.abs(T) - 1.0) < 1e-12)


def test_asm_refocuses_a_point_fringe():
    """A5: the Fresnel point fringe of one object pixel (Eq. 1) reconstructs with its
    amplitude maximum at that pixel, for both paddings and several layers."""
    n, s = 16, 4
    g = O.Geometry((n, n), (n * s, n * s), PITCH, LAM, [0.02, 0.03])
    for zi in range(2):
        for (i, j) in ((3, 4), (8, 8), (12, 2)):
            F = np.zeros((2, n, n), complex)
            F[zi, i, j] = 1.0
            H = O.propagate_fields(F, g)
            for pad in (1, 2):
                A = np.abs(O.asm_reconstruct_fields(H, g, pad=pad)[zi])
                assert np.unravel_index(np.argmax(A), A.shape) == (i, j), (zi, i, j, pad)


def test_asm_band_limit():
    """A6: the band limit zeroes exactly the frequencies with |fx| or |fy| above
    1 / (lambda sqrt((2 df z)^2 + 1)), and changes nothing when that exceeds Nyquist."""
    g = O.Geometry((64, 64), (64, 64), PITCH, LAM, [0.2, 0.001])
    P = 64
    T0, T1 = O.asm_transfer(g, 0, P), O.asm_transfer(g, 0, P, band_limit=True)
    df = 1.0 / (P * PITCH)
    k = np.array([_signed(x, P) for x in range(P)])
    lim = 1.0 / (LAM * np.sqrt((2 * df * 0.2) ** 2 + 1.0))
    keep = (np.abs(k)[None, :] * df <= lim) & (np.abs(k)[:, None] * df <= lim)
    assert 0 < keep.sum() < P * P
    assert np.array_equal(T1 != 0, keep) and np.allclose(T1[keep], T0[keep], rtol=0, atol=0)
    assert np.array_equal(O.asm_transfer(g, 1, P, band_limit=True), O.asm_transfer(g, 1, P))


# ---------------------------------------------------------------- per-point depth (D1-D3)

def test_pointcloud_reduces_to_layers():
    """D1: with every pixel's depth set to its layer's distance, the per-point sum is the
    layered point-wise hologram (separable evaluation, pinned above).  The distances are
    float32 values, so the float32 depth map holds them exactly."""
    sc = scenes.random_scene(61, 16, 32, 3)
    zs = [float(np.float32(z)) for z in (0.05, 0.0625, 0.09)]
    g = O.Geometry((16, 16), (32, 32), PITCH, LAM, zs)
    lay = sc["layer"].copy()
    lay[0, :4] = 7  # pixels of no layer are no point
    depth = np.where(lay < 3, np.asarray(zs)[np.minimum(lay, 2)], np.nan).astype(np.float32)
    H1 = O.pointcloud_hologram(sc["intensity"], depth, g)
    H2 = O.plain_pointwise_hologram(sc["intensity"], lay, g)
    assert O.rel_l2(H1, H2) < 1e-12


def test_pointcloud_single_point_closed_form():
    """D2: one point at rate exactly 1/4 (wavelength chosen so that z = 2 p^2 / lambda is
    a power of two): H(m, n) = v * j^(odd(dm) + odd(dn)); every other pixel's depth is 0,
    negative, NaN or infinite (no point)."""
    n, s = 8, 4
    z = 2.0 ** -12
    lam = 2 * PITCH * PITCH / z
    g = O.Geometry((n, n), (n * s, n * s), PITCH, lam, [1.0])
    depth = np.full((n, n), np.nan, np.float32)
    depth[1, 1], depth[2, 2], depth[3, 3] = 0.0, -0.1, np.inf
    depth[5, 2] = z
    I = np.full((n, n), 200, np.uint8)
    I[5, 2] = 17
    H = O.pointcloud_hologram(I, depth, g)
    m = np.arange(n * s)[:, None] - 5 * s
    q = np.arange(n * s)[None, :] - 2 * s
    assert np.max(np.abs(H - 17 * 1j ** ((m % 2) + (q % 2)))) < 1e-10


def test_pointcloud_brute_force_two_depths():
    """D3: two points at different depths against Eq. 1's paraxial phase written out,
    pi (d p)^2 / (lambda z), summed by hand (no reduction needed at these offsets)."""
    g = O.Geometry((4, 4), (8, 8), PITCH, LAM, [1.0])
    depth = np.full((4, 4), np.nan, np.float32)
    depth[0, 3], depth[2, 1] = 0.013, 0.021
    I = np.zeros((4, 4), np.uint8)
    I[0, 3], I[2, 1] = 50, 90
    H = O.pointcloud_hologram(I, depth, g)
    for m in range(8):
        for n in range(8):
            want = 0j
            for (i, j) in ((0, 3), (2, 1)):
                r2 = ((m - 2 * i) * PITCH) ** 2 + ((n - 2 * j) * PITCH) ** 2
                want += I[i, j] * np.exp(1j * np.pi * r2 / (LAM * float(depth[i, j])))
            assert abs(H[m, n] - want) < 1e-9


# ---------------------------------------------------------------- colour channels (C1)

def test_wavelength_enters_only_through_the_rate():
    """C1: lambda appears only in a_z = p^2 / (2 lambda z): a channel at wavelength l1 and
    distances z equals a channel at l2 and distances z l1 / l2, for the progressive
    hologram, the point-wise one and the Fresnel reconstruction."""
    sc = scenes.rgb_scene(71, 16, 32, 2)
    lam_r, lam_b = 638e-9, 450e-9
    z = np.array([0.05, 0.07])
    gr = O.Geometry((16, 16), (32, 32), PITCH, lam_r, z)
    gb = O.Geometry((16, 16), (32, 32), PITCH, lam_b, z * lam_r / lam_b)
    I = sc["intensity"][0]
    lists = O.progressive_lists(sc["saliency"], sc["layer"], 2, scenes.THRESHOLDS_U8)
    Hr = O.progressive_hologram(I, sc["layer"], lists, gr)
    Hb = O.progressive_hologram(I, sc["layer"], lists, gb)
    assert O.rel_l2(Hb, Hr) < 1e-12
    assert O.rel_l2(O.plain_pointwise_hologram(I, sc["layer"], gb), O.plain_pointwise_hologram(I, sc["layer"], gr)) < 1e-12
    assert O.rel_l2(O.reconstruct_fields(Hr, gb), O.reconstruct_fields(Hr, gr)) < 1e-12
    # and a different wavelength at the same distances gives a different hologram
    g2 = O.Geometry((16, 16), (32, 32), PITCH, lam_b, z)
    assert O.rel_l2(O.progressive_hologram(I, sc["layer"], lists, g2), Hr) > 0.1


# ---------------------------------------------------------------- the layer factor (F1-F3)

def test_layer_factor_single_point_is_eq1():
    """F1: with the layer factor kept, one salient point of value v at (i, j) on the layer at
    z gives Eq. 1 in its paraxial form written out, v/z exp(j 2 pi z / lambda)
    exp(j pi (d p)^2 / (lambda z)), for the progressive, point-wise and propagated forms."""
    n, s = 8, 2
    z = 0.0123
    g = O.Geometry((n, n), (n * s, n * s), PITCH, LAM, [z], layer_factor=True)
    I = np.zeros((n, n), np.uint8)
    I[3, 5] = 91
    lay = np.zeros((n, n), np.uint8)
    m = np.arange(n * s)[:, None] - s * 3
    q = np.arange(n * s)[None, :] - s * 5
    r2 = (m * PITCH) ** 2 + (q * PITCH) ** 2
    want = 91 / z * np.exp(2j * np.pi * z / LAM) * np.exp(1j * np.pi * r2 / (LAM * z))
    Hp = O.progressive_hologram(I, lay, all_salient_lists(lay, 1), g)
    assert np.max(np.abs(Hp - want)) <= 1e-9 * np.max(np.abs(want))
    Hd = O.plain_pointwise_hologram(I, lay, g, pixels=np.nonzero(np.ones((n * s, n * s))))
    assert np.max(np.abs(Hd.reshape(n * s, n * s) - want)) <= 1e-9 * np.max(np.abs(want))
    F = np.zeros((1, n, n), complex)
    F[0, 3, 5] = 91
    assert np.max(np.abs(O.propagate_fields(F, g) - want)) <= 1e-9 * np.max(np.abs(want))


def test_layer_factor_adjoint_and_scaling():
    """F2: reconstruction stays the adjoint of propagation with the factor, and every
    layer's hologram is the factorless one times exp(j 2 pi frac(z/lambda)) / z."""
    rng = np.random.default_rng(44)
    g = O.Geometry((8, 8), (16, 16), PITCH, LAM, [0.05, 0.07, 0.11], layer_factor=True)
    g0 = O.Geometry((8, 8), (16, 16), PITCH, LAM, [0.05, 0.07, 0.11])
    H = rng.normal(size=(16, 16)) + 1j * rng.normal(size=(16, 16))
    F = rng.normal(size=(3, 8, 8)) + 1j * rng.normal(size=(3, 8, 8))
    lhs = np.vdot(O.reconstruct_fields(H, g), F)
    rhs = np.vdot(H, O.propagate_fields(F, g))
    assert abs(lhs - rhs) <= 1e-10 * abs(lhs)
    for k, z in enumerate(g.z):
        Fk = np.zeros_like(F)
        Fk[k] = F[k]
        c = np.exp(2j * np.pi * z / LAM) / z  # unreduced: ~1e-10 rad of FP64 rounding
        assert O.rel_l2(O.propagate_fields(Fk, g), c * O.propagate_fields(Fk, g0)) < 1e-9


def test_layer_factor_pointcloud_reduces_to_layers():
    """F3: with the factor, a depth map holding the layer distances gives the layered
    point-wise hologram (each point's factor is its own depth's)."""
    sc = scenes.random_scene(62, 16, 32, 3)
    zs = [float(np.float32(z)) for z in (0.05, 0.0625, 0.09)]
    g = O.Geometry((16, 16), (32, 32), PITCH, LAM, zs, layer_factor=True)
    depth = np.asarray(zs, np.float32)[sc["layer"]]
    assert O.rel_l2(O.pointcloud_hologram(sc["intensity"], depth, g),
                    O.plain_pointwise_hologram(sc["intensity"], sc["layer"], g)) < 1e-12
