"""Inverse angular-spectrum reconstruction on the GPU (hand-written FFTs) against the FP64
oracle (numpy FFTs, transfer function from its definition).

Bar, derived from the arithmetic: every 1-D FP32 FFT of length <= 4096 carries ~1.2e-7
rel-L2 rounding (measured against an FP64 DFT), four of them sit on the path (forward rows
and columns, inverse columns and rows), and the transfer function's phase is formed to
< 1e-6 rad (64-bit fixed-point Fresnel term plus an FP32 correction below a quarter cycle):
about 1e-6 in all, held to rel-L2 1e-5."""
import numpy as np
import pytest

from oracle import cgh_oracle as O
from synth import scenes

pytestmark = pytest.mark.gpu

TOL = 1e-5


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


def _holo(sc, g):
    lists = O.progressive_lists(sc["saliency"], sc["layer"], g.n_layers, scenes.THRESHOLDS_U8)
    return O.progressive_hologram(sc["intensity"], sc["layer"], lists, g)


@pytest.mark.parametrize("name,make,pad,band", [
    ("64_to_128_z3_s2", lambda: scenes.random_scene(95, 64, 128, 3, graded=True), 1, False),
    ("64_to_128_z3_s2", lambda: scenes.random_scene(95, 64, 128, 3, graded=True), 2, False),
    ("tiny_64_to_256_z4_s4", lambda: scenes.tiny_scene(), 1, False),
    ("tiny_64_to_256_z4_s4", lambda: scenes.tiny_scene(), 2, True),
    ("128_to_128_z2_s1", lambda: scenes.random_scene(96, 128, 128, 2), 2, False),
    ("paper_512_to_1024_z16", lambda: scenes.paper_scene(), 2, False),
])
def test_asm_matches_oracle(torch_cuda, name, make, pad, band):
    torch = torch_cuda
    from paper_2211_09938_gb300 import Plan
    sc = make()
    g = O.geometry_of(sc)
    H = _holo(sc, g)
    plan = Plan.for_scene(sc)
    L = torch.from_numpy(sc["layer"]).cuda()
    F, A = plan.reconstruct_asm(torch.from_numpy(H.astype(np.complex64)).cuda(), L, pad=pad, band_limit=band)
    torch.cuda.synchronize()
    R = O.asm_reconstruct_fields(H.astype(np.complex64).astype(np.complex128), g, pad=pad, band_limit=band)
    errF = O.rel_l2(F.cpu().numpy(), R)
    errA = O.rel_l2(A.cpu().numpy(), O.composite_amplitude(R, sc["layer"]))
    print(f"asm {name} pad {pad} band {band}: fields {errF:.2e} amplitude {errA:.2e}")
    assert errF <= TOL and errA <= TOL
    # each layer on its own, so that no layer hides behind a larger one
    for z in range(g.n_layers):
        assert O.rel_l2(F[z].cpu().numpy(), R[z]) <= TOL, z


def test_asm_outputs_edge_cases(torch_cuda):
    """amplitude only, fields only, pixels whose layer index is >= Z (amplitude 0), and a
    repeated call with the other padding (buffers re-planned)."""
    torch = torch_cuda
    from paper_2211_09938_gb300 import Plan
    sc = scenes.random_scene(97, 64, 128, 2)
    g = O.geometry_of(sc)
    lay = sc["layer"].copy()
    lay[:5, :7] = 200
    H = _holo(sc, g).astype(np.complex64)
    plan = Plan.for_scene(sc)
    Hd = torch.from_numpy(H).cuda()
    Ld = torch.from_numpy(lay).cuda()
    _, A = plan.reconstruct_asm(Hd, Ld, fields=False, pad=2)
    F, none = plan.reconstruct_asm(Hd, None, amplitude=False, pad=1)
    F2, A2 = plan.reconstruct_asm(Hd, Ld, pad=2)
    torch.cuda.synchronize()
    assert none is None
    R2 = O.asm_reconstruct_fields(H.astype(np.complex128), g, pad=2)
    R1 = O.asm_reconstruct_fields(H.astype(np.complex128), g, pad=1)
    a = A.cpu().numpy()
    assert np.all(a[:5, :7] == 0)
    keep = lay < 2
    ref = np.abs(R2[np.where(keep, lay, 0), np.arange(64)[:, None], np.arange(64)[None, :]]) * keep
    assert O.rel_l2(a, ref) <= TOL
    assert torch.equal(A, A2)
    assert O.rel_l2(F.cpu().numpy(), R1) <= TOL and O.rel_l2(F2.cpu().numpy(), R2) <= TOL


def test_asm_refocuses_points(torch_cuda):
    """A single point hologram reconstructs with its maximum at that point (pin A5 on the GPU)."""
    torch = torch_cuda
    from paper_2211_09938_gb300 import Plan
    n, s = 64, 2
    z = [0.02, 0.035]
    g = O.Geometry((n, n), (n * s, n * s), 8e-6, 532e-9, z)
    plan = Plan((n, n), (n * s, n * s), 8e-6, 532e-9, z)
    for zi in range(2):
        for (i, j) in ((10, 50), (33, 33)):
            F = np.zeros((2, n, n), complex)
            F[zi, i, j] = 1.0
            H = torch.from_numpy(O.propagate_fields(F, g).astype(np.complex64)).cuda()
            R, _ = plan.reconstruct_asm(H, amplitude=False, pad=2)
            A = R[zi].abs().cpu().numpy()
            assert np.unravel_index(np.argmax(A), A.shape) == (i, j)


def test_asm_rejects_bad_arguments(torch_cuda):
    torch = torch_cuda
    from paper_2211_09938_gb300 import Plan
    from paper_2211_09938_gb300.cgh import CghError
    sc = scenes.random_scene(98, 64, 128, 2)
    plan = Plan.for_scene(sc)
    H = torch.zeros((128, 128), dtype=torch.complex64, device="cuda")
    with pytest.raises(CghError):
        plan.reconstruct_asm(H, None, pad=3)
    with pytest.raises(CghError):
        plan.reconstruct_asm(H, None, fields=False)  # amplitude without layers
    with pytest.raises(CghError):
        plan.reconstruct_asm(H, None, fields=False, amplitude=False)
    # P / s below 64: 32x32 object on a 64x64 hologram without padding
    small = Plan((32, 32), (64, 64), 8e-6, 532e-9, [0.01])
    with pytest.raises(CghError):
        small.reconstruct_asm(torch.zeros((64, 64), dtype=torch.complex64, device="cuda"), None, pad=1)
    # non-power-of-two hologram
    odd = Plan((96, 96), (192, 192), 8e-6, 532e-9, [0.01])
    with pytest.raises(CghError):
        odd.reconstruct_asm(torch.zeros((192, 192), dtype=torch.complex64, device="cuda"), None)


def test_asm_stride_8_and_single_layer(torch_cuda):
    """s = 8 (folded edge P/8) and a single layer, both paddings."""
    torch = torch_cuda
    from paper_2211_09938_gb300 import Plan
    sc = scenes.random_scene(126, 64, 512, 1)
    g = O.geometry_of(sc)
    H = _holo(sc, g).astype(np.complex64)
    plan = Plan.for_scene(sc)
    for pad in (1, 2):
        F, _ = plan.reconstruct_asm(torch.from_numpy(H).cuda(), amplitude=False, pad=pad)
        torch.cuda.synchronize()
        err = O.rel_l2(F.cpu().numpy(), O.asm_reconstruct_fields(H.astype(np.complex128), g, pad=pad))
        print(f"asm s=8 pad {pad}: {err:.2e}")
        assert err <= TOL
