"""Reconstruction, propagation, the progressive-operator adjoint and the phase-only
optimisation on the GPU against the FP64 oracle.

Bars: the bf16 hi+lo tensor-core products with FP32 accumulation stay within rel-L2
1e-4 of FP64 (typically ~1e-5); adjoint identities hold to the same order; the phase
gradient matches the FP64 analytic gradient to rel-L2 1e-3 and central finite
differences (h = 1e-3) on 64 entries."""
import numpy as np
import pytest

from oracle import cgh_oracle as O
from synth import scenes

pytestmark = pytest.mark.gpu

TOL = 1e-4


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


def cplx(rng, *shape):
    return (rng.normal(size=shape) + 1j * rng.normal(size=shape)).astype(np.complex64)


@pytest.mark.parametrize("name,make", [
    ("tiny_64_to_256_z4", lambda: scenes.tiny_scene()),
    ("single_layer_32_s2", lambda: scenes.random_scene(78, 32, 64, 1, graded=True)),
    ("paper_512_to_1024_z16", lambda: scenes.paper_scene()),
])
def test_reconstruct_matches_oracle(torch_cuda, name, make):
    torch = torch_cuda
    from paper_2211_09938_gb300 import Plan
    sc = make()
    g = O.geometry_of(sc)
    plan = Plan.for_scene(sc)
    lists = O.progressive_lists(sc["saliency"], sc["layer"], g.n_layers, scenes.THRESHOLDS_U8)
    H = O.progressive_hologram(sc["intensity"], sc["layer"], lists, g)
    Hd = torch.from_numpy(H.astype(np.complex64)).cuda()
    L = torch.from_numpy(sc["layer"]).cuda()
    F, A = plan.reconstruct(Hd, L)
    torch.cuda.synchronize()
    R = O.reconstruct_fields(H, g)
    errF = O.rel_l2(F.cpu().numpy(), R)
    errA = O.rel_l2(A.cpu().numpy(), O.composite_amplitude(R, sc["layer"]))
    print(f"reconstruct {name}: fields {errF:.2e} amplitude {errA:.2e}")
    assert errF <= TOL and errA <= TOL


def test_propagate_matches_oracle_and_is_adjoint(torch_cuda):
    torch = torch_cuda
    from paper_2211_09938_gb300 import Plan
    rng = np.random.default_rng(12)
    sc = scenes.tiny_scene()
    g = O.geometry_of(sc)
    plan = Plan.for_scene(sc)
    F = cplx(rng, 4, 64, 64)
    Hg = plan.propagate(torch.from_numpy(F).cuda())
    torch.cuda.synchronize()
    Href = O.propagate_fields(F, g)
    err = O.rel_l2(Hg.cpu().numpy(), Href)
    print(f"propagate tiny: {err:.2e}")
    assert err <= TOL
    # accumulate adds onto what is there
    H2 = plan.propagate(torch.from_numpy(F).cuda(), holo=Hg.clone(), accumulate=True)
    torch.cuda.synchronize()
    assert O.rel_l2(H2.cpu().numpy(), 2 * Href) <= TOL
    # <reconstruct(H), F> = <H, propagate(F)> on the GPU
    Hx = cplx(rng, 256, 256)
    Rx, _ = plan.reconstruct(torch.from_numpy(Hx).cuda(), amplitude=False)
    lhs = np.real(np.vdot(Rx.cpu().numpy().astype(np.complex128), F.astype(np.complex128)))
    rhs = np.real(np.vdot(Hx.astype(np.complex128), Hg.cpu().numpy().astype(np.complex128)))
    assert abs(lhs - rhs) <= 1e-4 * abs(lhs)


def test_adjoint_matches_oracle(torch_cuda):
    torch = torch_cuda
    from paper_2211_09938_gb300 import Plan
    rng = np.random.default_rng(13)
    sc = scenes.random_scene(81, 64, 128, 3, graded=True)
    g = O.geometry_of(sc)
    plan = Plan.for_scene(sc)
    L = torch.from_numpy(sc["layer"]).cuda()
    S = torch.from_numpy(sc["saliency"]).cuda()
    lists, counts = plan.progressive_lists(S, L, scenes.THRESHOLDS_U8)
    G = cplx(rng, 128, 128)
    grad = plan.adjoint(torch.from_numpy(G).cuda(), lists, counts, L)
    torch.cuda.synchronize()
    ref_lists = O.progressive_lists(sc["saliency"], sc["layer"], 3, scenes.THRESHOLDS_U8)
    ref = O.progressive_adjoint(G, sc["layer"], ref_lists, g)
    err = O.rel_l2(grad.cpu().numpy(), ref)
    print(f"adjoint: {err:.2e}")
    assert err <= TOL
    # dot-product identity against the GPU forward (direct form, FP32)
    I = rng.integers(0, 256, size=(64, 64)).astype(np.uint8)
    coeffs = plan.haar_decompose(torch.from_numpy(I).cuda(), L)
    FI = plan.progressive_hologram(coeffs, lists, counts)
    torch.cuda.synchronize()
    lhs = np.real(np.vdot(FI.cpu().numpy().astype(np.complex128), G.astype(np.complex128)))
    rhs = float(np.sum(I.astype(np.float64) * grad.cpu().numpy()))
    assert abs(lhs - rhs) <= 1e-4 * abs(lhs)


def test_amplitude_backward_and_phase_kernels(torch_cuda):
    torch = torch_cuda
    from paper_2211_09938_gb300 import Plan
    from paper_2211_09938_gb300.cgh import phase_grad, phase_to_field
    rng = np.random.default_rng(14)
    sc = scenes.tiny_scene()
    plan = Plan.for_scene(sc)
    F = cplx(rng, 4, 64, 64)
    F[0, 0, 0] = 0
    gA = rng.normal(size=(64, 64)).astype(np.float32)
    gF = plan.amplitude_backward(torch.from_numpy(F).cuda(), torch.from_numpy(sc["layer"]).cuda(),
                                 torch.from_numpy(gA).cuda()).cpu().numpy()
    ref = np.zeros_like(F)
    lay = sc["layer"].astype(int)
    ii, jj = np.indices(lay.shape)
    v = F[lay, ii, jj]
    a = np.abs(v)
    ref[lay, ii, jj] = np.where(a > 0, gA * v / np.where(a > 0, a, 1), 0)
    assert np.allclose(gF, ref, atol=1e-5)
    phi = rng.uniform(-10, 10, size=(300,)).astype(np.float32)
    H = phase_to_field(torch.from_numpy(phi).cuda()).cpu().numpy()
    assert np.allclose(H, np.exp(1j * phi.astype(np.float64)), atol=2e-6)
    g = cplx(rng, 300)
    gp = phase_grad(torch.from_numpy(H).cuda(), torch.from_numpy(g).cuda()).cpu().numpy()
    assert np.allclose(gp, np.imag(g * np.conj(H)), atol=1e-5)


@pytest.mark.parametrize("n,holo,nl", [(64, 128, 4), (512, 1024, 8)])
def test_batched_reconstruction_and_propagation_equal_single_calls(torch_cuda, n, holo, nl):
    """cgh_reconstruct_batch / cgh_propagate_batch / cgh_amplitude_backward_batch run each
    GEMM stage once over the (hologram, layer) pairs: on a deterministic plan the results
    equal one call per hologram bit for bit, through batch sizes that grow the plan's scratch
    and one that fits it."""
    torch = torch_cuda
    from paper_2211_09938_gb300 import Plan
    sc = scenes.random_scene(77 + n, n, holo, nl)
    plan = Plan.for_scene(sc, flags=Plan.DETERMINISTIC)
    L = torch.from_numpy(sc["layer"]).cuda()
    rng = np.random.default_rng(n)
    for nb in (3, 2, 5):
        H = torch.from_numpy(cplx(rng, nb, holo, holo).astype(np.complex64)).cuda()
        F, A = plan.reconstruct_batch(H, L)
        g = torch.from_numpy(rng.standard_normal((nb, n, n)).astype(np.float32)).cuda()
        gF = plan.amplitude_backward_batch(F, L, g)
        Hp = plan.propagate_batch(gF)
        torch.cuda.synchronize()
        for b in range(nb):
            f1, a1 = plan.reconstruct(H[b], L)
            gf1 = plan.amplitude_backward(f1, L, g[b])
            h1 = plan.propagate(gf1)
            torch.cuda.synchronize()
            assert torch.equal(F[b], f1) and torch.equal(A[b], a1), (nb, b)
            assert torch.equal(gF[b], gf1), (nb, b)
            assert torch.equal(Hp[b], h1), (nb, b)
    plan.close()


def _opt_case(torch, n=64, holo=128, nl=4, seed=15, flags=0):
    from paper_2211_09938_gb300 import Plan
    sc = scenes.random_scene(seed, n, holo, nl)
    rng = np.random.default_rng(seed)
    plan = Plan.for_scene(sc, flags=flags)
    target = (sc["intensity"].astype(np.float32) / 255.0)
    weight = np.where(sc["saliency"] > 0, 4.0, 1.0).astype(np.float32)
    phase = rng.uniform(-np.pi, np.pi, size=(holo, holo)).astype(np.float32)
    return sc, plan, target, weight, phase


def test_phase_gradient_vs_oracle_and_finite_differences(torch_cuda):
    torch = torch_cuda
    from paper_2211_09938_gb300 import optim
    sc, plan, target, weight, phase = _opt_case(torch)
    g = O.geometry_of(sc)
    L = torch.from_numpy(sc["layer"]).cuda()
    T = torch.from_numpy(target).cuda()
    W = torch.from_numpy(weight).cuda()
    with torch.no_grad():
        kappa = optim.fit_kappa(optim.reconstruct_amplitude(torch.from_numpy(phase).cuda(), plan, L), T)
    ph = torch.from_numpy(phase).cuda().requires_grad_(True)
    loss = optim.weighted_loss(optim.reconstruct_amplitude(ph, plan, L, True), T, W, kappa)
    loss.backward()
    grad = ph.grad.cpu().numpy().astype(np.float64)
    ref = O.phase_opt_grad(phase.astype(np.float64), target, weight, sc["layer"], g, kappa)
    err = O.rel_l2(grad, ref)
    print(f"phase gradient vs FP64 oracle: {err:.2e}")
    assert err <= 1e-3
    # checkpointed and stored-field backward agree exactly
    ph2 = torch.from_numpy(phase).cuda().requires_grad_(True)
    optim.weighted_loss(optim.reconstruct_amplitude(ph2, plan, L, False), T, W, kappa).backward()
    assert torch.equal(ph2.grad, ph.grad)
    # central finite differences of the FP64 oracle loss, h = 1e-3, 64 random entries
    rng = np.random.default_rng(16)
    idx = rng.integers(0, phase.size, size=64)
    h = 1e-3
    fd = []
    for k in idx:
        e = np.zeros(phase.size)
        e[k] = h
        e = e.reshape(phase.shape)
        fd.append((O.phase_opt_loss(phase + e, target, weight, sc["layer"], g, kappa)
                   - O.phase_opt_loss(phase - e, target, weight, sc["layer"], g, kappa)) / (2 * h))
    fd = np.array(fd)
    gk = grad.reshape(-1)[idx]
    err_fd = np.linalg.norm(gk - fd) / np.linalg.norm(fd)
    print(f"phase gradient vs central differences (64 entries): {err_fd:.2e}")
    assert err_fd <= 1e-2


def test_phase_gradient_at_bench_size(torch_cuda):
    """The phase-optimisation benchmark's size: 512x512 object, 1024x1024 hologram, 8 layers.
    The autograd gradient (checkpointed reconstruction, propagation backward) against the
    FP64 oracle's analytic gradient over every entry, and against central differences
    (h = 1e-3) of the FP64 oracle loss on 64 random entries."""
    torch = torch_cuda
    from paper_2211_09938_gb300 import optim
    sc, plan, target, weight, phase = _opt_case(torch, n=512, holo=1024, nl=8, seed=5000)
    g = O.geometry_of(sc)
    L = torch.from_numpy(sc["layer"]).cuda()
    T = torch.from_numpy(target).cuda()
    W = torch.from_numpy(weight).cuda()
    with torch.no_grad():
        kappa = optim.fit_kappa(optim.reconstruct_amplitude(torch.from_numpy(phase).cuda(), plan, L), T)
    ph = torch.from_numpy(phase).cuda().requires_grad_(True)
    optim.weighted_loss(optim.reconstruct_amplitude(ph, plan, L, True), T, W, kappa).backward()
    grad = ph.grad.cpu().numpy().astype(np.float64)
    ref = O.phase_opt_grad(phase.astype(np.float64), target, weight, sc["layer"], g, kappa)
    err = O.rel_l2(grad, ref)
    rng = np.random.default_rng(5001)
    idx = rng.choice(phase.size, size=64, replace=False)
    h = 1e-3
    fd = []
    for k in idx:
        e = np.zeros(phase.size)
        e[k] = h
        e = e.reshape(phase.shape)
        fd.append((O.phase_opt_loss(phase + e, target, weight, sc["layer"], g, kappa)
                   - O.phase_opt_loss(phase - e, target, weight, sc["layer"], g, kappa)) / (2 * h))
    fd = np.array(fd)
    err_fd = float(np.linalg.norm(grad.reshape(-1)[idx] - fd) / np.linalg.norm(fd))
    print(f"bench-size phase gradient: vs FP64 oracle {err:.2e}, vs central differences (64 entries) {err_fd:.2e}")
    assert err <= 1e-3 and err_fd <= 1e-2


def test_phase_optimisation_decreases_and_resumes_bit_identically(torch_cuda, tmp_path):
    torch = torch_cuda
    from paper_2211_09938_gb300 import Plan, optim
    sc, plan, target, weight, phase = _opt_case(torch, flags=Plan.DETERMINISTIC)
    L = torch.from_numpy(sc["layer"]).cuda()
    T = torch.from_numpy(np.stack([target, target[::-1].copy()])).cuda()
    W = torch.from_numpy(weight).cuda()
    ph0 = torch.from_numpy(np.stack([phase, -phase])).cuda()
    a = optim.PhaseOptimiser(plan, L, T, W, ph0, lr=0.05)
    losses = [a.step() for _ in range(6)]
    assert losses[-1] < losses[0]
    b = optim.PhaseOptimiser(plan, L, T, W, ph0, lr=0.05)
    for _ in range(3):
        b.step()
    path = tmp_path / "phase.pt"
    torch.save(b.state_dict(), path)
    c = optim.PhaseOptimiser(plan, L, T, W, torch.zeros_like(ph0), lr=0.05)
    c.load_state_dict(torch.load(path))
    for _ in range(3):
        c.step()
    assert c.step_count == 6
    assert torch.equal(c.phase.detach(), a.phase.detach())
    # the holograms on their own streams and plans give the same phases bit for bit
    d = optim.PhaseOptimiser(plan, L, T, W, ph0, lr=0.05, concurrent=True)
    for _ in range(6):
        d.step()
    assert torch.equal(d.phase.detach(), a.phase.detach())
    # one captured step replayed: the same run (the capture's warm-up steps are undone), to
    # the rounding of the capturable Adam update
    e = optim.PhaseOptimiser(plan, L, T, W, ph0, lr=0.05, graph=True)
    lg = [e.step() for _ in range(6)]
    assert e.step_count == 6
    np.testing.assert_allclose(lg, losses, rtol=1e-5)
    err = float((e.phase.detach() - a.phase.detach()).abs().max())
    print(f"graph-captured optimiser: max phase difference after 6 steps {err:.2e}")
    assert err <= 1e-4
    # save after 3 replayed steps, load into a fresh graph optimiser (which captures again
    # around the loaded state) and finish: the uninterrupted replayed run, bit for bit
    f = optim.PhaseOptimiser(plan, L, T, W, ph0, lr=0.05, graph=True)
    for _ in range(3):
        f.step()
    torch.save(f.state_dict(), tmp_path / "phase_graph.pt")
    g2 = optim.PhaseOptimiser(plan, L, T, W, torch.zeros_like(ph0), lr=0.05, graph=True)
    g2.load_state_dict(torch.load(tmp_path / "phase_graph.pt"))
    for _ in range(3):
        g2.step()
    assert g2.step_count == 6
    assert torch.equal(g2.phase.detach(), e.phase.detach())


@pytest.mark.parametrize("name,make", [
    ("graded_64_to_128_z4", lambda: scenes.random_scene(171, 64, 128, 4, graded=True)),
    ("paper_512_to_1024_z16", lambda: scenes.paper_scene()),
])
def test_progressive_apply_matches_oracle_and_integer_path(torch_cuda, name, make):
    """cgh_progressive_apply on a real object against the FP64 oracle's real-object
    operator; on the integer intensity it is the hologram cgh_progressive_hologram gives."""
    torch = torch_cuda
    from paper_2211_09938_gb300 import Plan
    sc = make()
    g = O.geometry_of(sc)
    plan = Plan.for_scene(sc)
    L = torch.from_numpy(sc["layer"]).cuda()
    S = torch.from_numpy(sc["saliency"]).cuda()
    I = torch.from_numpy(sc["intensity"]).cuda()
    lists, counts = plan.progressive_lists(S, L, scenes.THRESHOLDS_U8)
    ref_lists = O.progressive_lists(sc["saliency"], sc["layer"], g.n_layers, scenes.THRESHOLDS_U8)
    rng = np.random.default_rng(172)
    x = (sc["intensity"].astype(np.float64) + rng.normal(size=sc["intensity"].shape) * 7.3).astype(np.float32)
    H = plan.progressive_apply(torch.from_numpy(x).cuda(), lists, counts, L)
    Hi = plan.progressive_apply(I.float(), lists, counts, L)
    Hp = plan.progressive_hologram(plan.haar_decompose(I, L), lists, counts, form="tc_fp16x3")
    torch.cuda.synchronize()
    err = O.rel_l2(H.cpu().numpy(), O.progressive_hologram_real(x.astype(np.float64), sc["layer"], ref_lists, g))
    Href = O.progressive_hologram(sc["intensity"], sc["layer"], ref_lists, g)
    erri = O.rel_l2(Hi.cpu().numpy(), Href)
    print(f"progressive_apply {name}: real object {err:.2e}, integer object {erri:.2e}, "
          f"vs progressive_hologram {O.rel_l2(Hi.cpu().numpy(), Hp.cpu().numpy()):.2e}")
    assert err <= TOL and erri <= TOL
    assert O.rel_l2(Hi.cpu().numpy(), Hp.cpu().numpy()) <= TOL
    assert plan.status() == 0


def test_progressive_autograd_vs_oracle_adjoint_and_finite_differences(torch_cuda):
    """torch.autograd through ProgressiveOperator (forward cgh_progressive_apply, backward
    cgh_adjoint): the object gradient of a nonlinear loss of the hologram matches the FP64
    oracle's adjoint applied to the same cotangent, and central finite differences
    (h = 1e-3) of the loss evaluated with the FP64 oracle's forward on 64 random entries."""
    torch = torch_cuda
    from paper_2211_09938_gb300 import Plan, optim
    sc = scenes.random_scene(181, 32, 64, 3, graded=True)
    g = O.geometry_of(sc)
    plan = Plan.for_scene(sc)
    L = torch.from_numpy(sc["layer"]).cuda()
    S = torch.from_numpy(sc["saliency"]).cuda()
    lists, counts = plan.progressive_lists(S, L, scenes.THRESHOLDS_U8)
    ref_lists = O.progressive_lists(sc["saliency"], sc["layer"], g.n_layers, scenes.THRESHOLDS_U8)
    rng = np.random.default_rng(182)
    x0 = sc["intensity"].astype(np.float64) / 255.0 + 0.1 * rng.normal(size=sc["intensity"].shape)
    W = rng.uniform(0.5, 2.0, size=sc["holo"])
    T = cplx(rng, *sc["holo"]).astype(np.complex128) * 20.0

    def loss_np(x):
        H = O.progressive_hologram_real(x, sc["layer"], ref_lists, g)
        return float(np.sum(W * np.abs(H - T) ** 2))

    x = torch.from_numpy(x0.astype(np.float32)).cuda().requires_grad_(True)
    H = optim.progressive_hologram(x, plan, lists, counts, L)
    Wd = torch.from_numpy(W).cuda()
    Td = torch.from_numpy(T).cuda()
    loss = (Wd * (H.to(torch.complex128) - Td).abs() ** 2).sum()
    loss.backward()
    grad = x.grad.double().cpu().numpy()
    # the oracle adjoint of the cotangent dL/dH = 2 W (H - T) at the FP64 forward
    Hn = O.progressive_hologram_real(x0, sc["layer"], ref_lists, g)
    want = O.progressive_adjoint(2.0 * W * (Hn - T), sc["layer"], ref_lists, g)
    err = O.rel_l2(grad, want)
    idx = rng.choice(x0.size, size=64, replace=False)
    h = 1e-3
    fd = []
    for k in idx:
        e = np.zeros(x0.size)
        e[k] = h
        e = e.reshape(x0.shape)
        fd.append((loss_np(x0 + e) - loss_np(x0 - e)) / (2 * h))
    fd = np.array(fd)
    err_fd = float(np.linalg.norm(grad.reshape(-1)[idx] - fd) / np.linalg.norm(fd))
    print(f"object gradient: vs oracle adjoint {err:.2e}, vs central differences {err_fd:.2e}")
    assert err <= 1e-3 and err_fd <= 1e-3
