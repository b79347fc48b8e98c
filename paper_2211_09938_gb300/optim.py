"""Differentiable reconstruction and phase-only hologram optimisation.

The hologram-to-reconstruction map is linear (the Fresnel back-propagation of the
plan), so its backward pass is the forward point-source propagation of the layer
fields: both run in libcgh's tensor-core kernels, wrapped here in a
torch.autograd.Function.  PyTorch supplies the tensors, the Adam optimiser and
checkpoint files; it computes no part of the hologram path.
"""
import torch

from .cgh import phase_grad, phase_to_field


class PhaseReconstruction(torch.autograd.Function):
    """phase [holo, holo] float32  ->  composite amplitude [obj, obj] float32:
    H = exp(j phase), R_z = Fresnel back-propagation of H to layer z,
    amplitude(i, j) = |R_{layer(i,j)}(i, j)|.

    With checkpoint=True the per-layer fields are not kept between forward and
    backward; the backward recomputes them (activation checkpointing)."""

    @staticmethod
    def forward(ctx, phase, plan, layer, checkpoint=True):
        phase = phase.contiguous()
        H = phase_to_field(phase)
        F, amp = plan.reconstruct(H, layer)
        ctx.plan = plan
        ctx.layer = layer
        ctx.checkpoint = bool(checkpoint)
        if ctx.checkpoint:
            ctx.save_for_backward(phase)
        else:
            ctx.save_for_backward(phase, H, F)
        return amp

    @staticmethod
    def backward(ctx, g_amp):
        plan = ctx.plan
        if ctx.checkpoint:
            (phase,) = ctx.saved_tensors
            H = phase_to_field(phase)
            F, _ = plan.reconstruct(H, ctx.layer, amplitude=False)
        else:
            phase, H, F = ctx.saved_tensors
        gF = plan.amplitude_backward(F, ctx.layer, g_amp.contiguous().float())
        gH = plan.propagate(gF)
        return phase_grad(H, gH), None, None, None


def reconstruct_amplitude(phase, plan, layer, checkpoint=True):
    return PhaseReconstruction.apply(phase, plan, layer, checkpoint)


class PhaseReconstructionBatch(torch.autograd.Function):
    """phase [B, holo, holo] float32  ->  composite amplitudes [B, obj, obj] float32, as
    PhaseReconstruction per hologram, with each GEMM stage run once over the batch
    (cgh_reconstruct_batch; backward by cgh_amplitude_backward_batch and
    cgh_propagate_batch).  The same numbers as B single reconstructions."""

    @staticmethod
    def forward(ctx, phase, plan, layer, checkpoint=True):
        phase = phase.contiguous()
        H = phase_to_field(phase)
        F, amp = plan.reconstruct_batch(H, layer)
        ctx.plan = plan
        ctx.layer = layer
        ctx.checkpoint = bool(checkpoint)
        if ctx.checkpoint:
            ctx.save_for_backward(phase)
        else:
            ctx.save_for_backward(phase, H, F)
        return amp

    @staticmethod
    def backward(ctx, g_amp):
        plan = ctx.plan
        if ctx.checkpoint:
            (phase,) = ctx.saved_tensors
            H = phase_to_field(phase)
            F, _ = plan.reconstruct_batch(H, ctx.layer, amplitude=False)
        else:
            phase, H, F = ctx.saved_tensors
        gF = plan.amplitude_backward_batch(F, ctx.layer, g_amp.contiguous().float())
        gH = plan.propagate_batch(gF)
        return phase_grad(H, gH), None, None, None


def reconstruct_amplitudes(phase, plan, layer, checkpoint=True):
    """Composite amplitudes of a batch of phase-only holograms [B, holo, holo]."""
    return PhaseReconstructionBatch.apply(phase, plan, layer, checkpoint)


class ProgressiveOperator(torch.autograd.Function):
    """object [obj, obj] float32  ->  progressive hologram [holo, holo] complex64:
    H = sum_z E_z P_z(object [layer = z]) E_z^T (Eq. 3, Section 2 steps 2-5, for a real
    object), forward by cgh_progressive_apply.  The map is linear in the object, so the
    backward is its adjoint, cgh_adjoint: for a cotangent G of H (real-pair convention,
    dL/dRe H + j dL/dIm H, as torch passes it) the object gradient is
    Re(A^H G) = [layer = z] P_z Re(R_z), R_z the back-propagation of G to layer z."""

    @staticmethod
    def forward(ctx, obj, plan, lists, counts, layer):
        ctx.plan, ctx.lists, ctx.counts, ctx.layer = plan, lists, counts, layer
        return plan.progressive_apply(obj.contiguous().float(), lists, counts, layer)

    @staticmethod
    def backward(ctx, g_holo):
        g = ctx.plan.adjoint(g_holo.contiguous().to(torch.complex64), ctx.lists, ctx.counts, ctx.layer)
        return g, None, None, None, None


def progressive_hologram(obj, plan, lists, counts, layer):
    """Differentiable progressive hologram of a real object (see ProgressiveOperator)."""
    return ProgressiveOperator.apply(obj, plan, lists, counts, layer)


def weighted_loss(amp, target, weight, kappa):
    """sum w (amp / kappa - target)^2, accumulated in float64."""
    d = amp.double() / kappa - target.double()
    return (weight.double() * d * d).sum()


def fit_kappa(amp, target):
    """Least-squares scale of the amplitude onto the target: sum(a T) / sum(T^2)."""
    t = target.double()
    return float((amp.double() * t).sum() / (t * t).sum())


class PhaseOptimiser:
    """Adam over a batch of phase-only holograms [B, holo, holo] so that each one's
    reconstructed composite amplitude matches its target (weights per pixel, e.g. 4
    inside the saliency mask and 1 outside).  state_dict()/load_state_dict() (with
    torch.save/torch.load) checkpoint and resume the run; with a plan created with
    Plan.DETERMINISTIC a resumed run reproduces an uninterrupted one bit for bit.

    graph=True captures one whole step (the B reconstructions, the loss, the backward through
    libcgh's kernels and the fused Adam update) in a CUDA graph on the first step and replays it
    from then on: the ~130 launches of a step then cost one host call, where the eager loop is
    bound by the host's launch rate."""

    def __init__(self, plan, layer, targets, weights, phase0, lr=0.05, checkpoint=True, concurrent=False,
                 graph=False):
        self.plan = plan
        self.layer = layer
        self.targets = targets
        self.weights = weights
        self.checkpoint = checkpoint
        self.phase = phase0.detach().clone().float().contiguous().requires_grad_(True)
        self.use_graph = bool(graph) and not concurrent
        self.opt = torch.optim.Adam([self.phase], lr=lr, fused=True, capturable=self.use_graph)
        self.graph = None
        self.step_count = 0
        nb = self.phase.shape[0]
        # the loss's constants in float64, cast once
        self._t64 = torch.stack([targets[b] for b in range(nb)]).double()
        self._w64 = weights.double()
        # By default the batch goes through each GEMM stage at once (PhaseReconstructionBatch).
        # concurrent: the holograms run one by one on their own streams instead, each with its
        # own plan (plan scratch is per plan), so that their GEMMs and small kernels overlap on
        # the GPU; autograd runs every hologram's backward on the stream of its forward.
        # Measured at batch 4, 1024^2, 8 layers: 2.96 ms per Adam step against 2.66 ms one by
        # one in order (the four plans' operands compete for L2), so it is off by default.
        self.plans = [plan] + ([plan.clone() for _ in range(nb - 1)] if concurrent else [plan] * (nb - 1))
        self.streams = [torch.cuda.Stream() for _ in range(nb)] if concurrent else None
        with torch.no_grad():
            self.kappa = [fit_kappa(reconstruct_amplitude(self.phase[b], plan, layer, False), targets[b])
                          for b in range(nb)]
        self._set_kappa()

    def _set_kappa(self):
        # the scales as a device tensor [B, 1, 1], made outside any capture
        self._k64 = torch.tensor(self.kappa, dtype=torch.float64, device=self.phase.device).view(-1, 1, 1)

    def loss(self):
        nb = self.phase.shape[0]
        if self.streams is None:
            # the whole batch through each GEMM stage at once
            amps = reconstruct_amplitudes(self.phase, self.plan, self.layer, self.checkpoint)
            d = amps.double() / self._k64 - self._t64
            return (self._w64 * d * d).sum()
        cur = torch.cuda.current_stream()
        parts = []
        for b in range(nb):
            s = self.streams[b]
            s.wait_stream(cur)
            with torch.cuda.stream(s):
                amp = reconstruct_amplitude(self.phase[b], self.plans[b], self.layer, self.checkpoint)
                parts.append(weighted_loss(amp, self._t64[b], self._w64, self.kappa[b]))
        for s in self.streams:
            cur.wait_stream(s)
        return torch.stack(parts).sum()

    def _capture(self):
        """Warm up on a side stream (output buffers, the plan's lazily built operands, Adam's
        state), capture one step, then put the phase and Adam's state back as they were, so
        that the first replay is the next step."""
        phase0 = self.phase.detach().clone()
        state0 = [{k: v.clone() for k, v in st.items() if torch.is_tensor(v)} for st in self.opt.state.values()]
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            for _ in range(2):
                self.opt.zero_grad(set_to_none=True)
                self.loss().backward()
                self.opt.step()
        torch.cuda.current_stream().wait_stream(side)
        self.opt.zero_grad(set_to_none=True)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self._static_loss = self.loss()
            self._static_loss.backward()
            self.opt.step()
        with torch.no_grad():
            self.phase.copy_(phase0)
            for st, old in zip(self.opt.state.values(), state0 if state0 else [None] * len(self.opt.state)):
                for k, v in st.items():
                    if torch.is_tensor(v):
                        v.copy_(old[k]) if old else v.zero_()
        self.graph = g

    def step(self, sync=True):
        """One Adam step; returns the loss as a float, or with sync=False as a device tensor
        (no host synchronisation, so that the host queues the next steps while the GPU runs)."""
        if self.use_graph:
            if self.graph is None:
                self._capture()
            self.graph.replay()
            L = self._static_loss.detach()
            L = L if sync else L.clone()
        else:
            self.opt.zero_grad(set_to_none=True)
            L = self.loss()
            L.backward()
            self.opt.step()
            L = L.detach()
        self.step_count += 1
        return float(L) if sync else L

    def state_dict(self):
        return {"phase": self.phase.detach().clone(), "adam": self.opt.state_dict(),
                "step": self.step_count, "kappa": list(self.kappa)}

    def load_state_dict(self, st):
        with torch.no_grad():
            self.phase.copy_(st["phase"])
        self.opt.load_state_dict(st["adam"])
        self.step_count = int(st["step"])
        self.kappa = list(st["kappa"])
        self._set_kappa()
        self.graph = None  # the captured step holds the old state tensors: capture again
