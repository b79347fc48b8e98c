"""Per-point depth (3-D objects without depth layers) on the GPU against the FP64 oracle.

The kernel is the exact-reduction direct sum (64-bit fixed-point phase, SFU sine/cosine,
FP32 accumulation in two levels), so the bar is the direct kernels' FP32 bar, rel-L2 1e-5;
a depth map holding the layer distances must reproduce the layered kernel bit for bit."""
import numpy as np
import pytest

from oracle import cgh_oracle as O
from synth import scenes

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5


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


def dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("n,holo,shape", [(32, 128, None), (40, 120, (40, 24))])
def test_pointcloud_matches_oracle(torch_cuda, n, holo, shape):
    """Every hologram pixel; continuous depths in [0.08, 0.20] m with 10% holes (NaN, 0,
    negative); a ragged 40x24 object at stride 3."""
    torch = torch_cuda
    from paper_2211_09938_gb300 import Plan
    sc = scenes.random_scene(101, n, holo, 1)
    I = sc["intensity"]
    depth = scenes.depth_map(102, n, holes=0.1)
    if shape is not None:
        I, depth = I[:shape[0], :shape[1]].copy(), depth[:shape[0], :shape[1]].copy()
    s = holo // n
    hh, hw = s * I.shape[0], s * I.shape[1]
    plan = Plan(I.shape, (hh, hw), sc["pitch"], sc["wavelength"], [0.1])
    H = plan.pointcloud_direct(dev(torch, I), dev(torch, depth))
    torch.cuda.synchronize()
    g = O.Geometry(I.shape, (hh, hw), sc["pitch"], sc["wavelength"], [0.1])
    ref = O.pointcloud_hologram(I, depth, g)
    err = O.rel_l2(H.cpu().numpy(), ref)
    print(f"pointcloud {I.shape} -> {(hh, hw)}: rel-L2 {err:.2e}")
    assert err <= FP32_TOL


def test_pointcloud_paper_scale_sampled(torch_cuda):
    """512 -> 1024 with a continuous depth per point: 128 sampled pixels (corners and
    random) against the FP64 sum over all 262144 points."""
    torch = torch_cuda
    from paper_2211_09938_gb300 import Plan
    sc = scenes.paper_scene()
    depth = scenes.depth_map(103, 512)
    plan = Plan.for_scene(sc)
    H = plan.pointcloud_direct(dev(torch, sc["intensity"]), dev(torch, depth)).cpu().numpy()
    rng = np.random.default_rng(7)
    mm = np.concatenate([[0, 0, 1023, 1023], rng.integers(0, 1024, 124)])
    nn = np.concatenate([[0, 1023, 0, 1023], rng.integers(0, 1024, 124)])
    ref = O.pointcloud_hologram(sc["intensity"], depth, O.geometry_of(sc), pixels=(mm, nn))
    err = O.rel_l2(H[mm, nn], ref)
    print(f"pointcloud paper scale sampled rel-L2 {err:.2e}")
    assert err <= FP32_TOL


def test_pointcloud_equals_layered_kernel_bitwise(torch_cuda):
    """Depths equal to the layer distances (float32 values) give cgh_plain_direct's
    result bit for bit; accumulate adds onto the buffer."""
    torch = torch_cuda
    from paper_2211_09938_gb300 import Plan
    sc = scenes.random_scene(104, 64, 128, 4)
    zs = [float(np.float32(z)) for z in sc["z"]]
    lay = sc["layer"].copy()
    lay[:3, :5] = 9  # no layer: no point in either form
    plan = Plan((64, 64), (128, 128), sc["pitch"], sc["wavelength"], zs)
    depth = np.where(lay < 4, np.asarray(zs, np.float32)[np.minimum(lay, 3)], np.nan).astype(np.float32)
    I, L, D = dev(torch, sc["intensity"]), dev(torch, lay), dev(torch, depth)
    Hp = plan.plain_direct(I, L)
    Hc = plan.pointcloud_direct(I, D)
    Ha = plan.pointcloud_direct(I, D, holo=Hc.clone(), accumulate=True)
    torch.cuda.synchronize()
    assert torch.equal(Hp, Hc)
    assert torch.equal(Ha, Hc + Hc)


def test_pointcloud_exact_reduction_large_offsets(torch_cuda):
    """One point at rate exactly 1/4 in the corner of a 512 -> 2048 geometry: offsets up to
    2047 (squared distance ~8.4e6) give fringe values 1 or j exactly."""
    torch = torch_cuda
    from paper_2211_09938_gb300 import Plan
    z = 2.0 ** -12
    lam = 2 * 8e-6 * 8e-6 / z
    plan = Plan((512, 512), (2048, 2048), 8e-6, lam, [0.1])
    I = np.zeros((512, 512), np.uint8)
    I[0, 0] = 200
    depth = np.full((512, 512), np.nan, np.float32)
    depth[0, 0] = z
    H = plan.pointcloud_direct(dev(torch, I), dev(torch, depth)).cpu().numpy()
    m = np.arange(2048)
    exp = 200 * (1j ** ((m[:, None] % 2) + (m[None, :] % 2)))
    assert np.max(np.abs(H - exp)) < 200 * 2e-6


def test_pointcloud_rejects_bad_arguments(torch_cuda):
    torch = torch_cuda
    from paper_2211_09938_gb300 import Plan, lib
    from paper_2211_09938_gb300.cgh import CghError, check
    plan = Plan((32, 32), (64, 64), 8e-6, 532e-9, [0.1])
    I = torch.zeros((32, 32), dtype=torch.uint8, device="cuda")
    with pytest.raises(CghError):
        plan.pointcloud_direct(I, None)
    with pytest.raises(CghError):
        check(lib().cgh_pointcloud_direct(plan.handle, I.data_ptr(), I.data_ptr(),
                                          torch.zeros(64, 64, dtype=torch.complex64, device="cuda").data_ptr(), 2, None))


def test_pointcloud_no_points(torch_cuda):
    """A depth map without a single valid depth gives a zero hologram, and accumulating it
    leaves the buffer as it was."""
    torch = torch_cuda
    from paper_2211_09938_gb300 import Plan
    plan = Plan((32, 32), (64, 64), 8e-6, 532e-9, [0.1])
    I = torch.full((32, 32), 255, dtype=torch.uint8, device="cuda")
    D = torch.full((32, 32), float("nan"), dtype=torch.float32, device="cuda")
    D[0, :8] = 0.0
    D[1, :8] = -1.0
    D[2, :8] = float("inf")
    H = plan.pointcloud_direct(I, D)
    prev = torch.randn(64, 64, dtype=torch.complex64, device="cuda")
    H2 = plan.pointcloud_direct(I, D, holo=prev.clone(), accumulate=True)
    torch.cuda.synchronize()
    assert torch.count_nonzero(H).item() == 0
    assert torch.equal(H2, prev)
