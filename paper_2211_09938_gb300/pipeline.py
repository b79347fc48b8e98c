"""Streaming many scenes of one geometry from host memory to host holograms.

Each submitted scene is copied in (intensity, layer and saliency maps, pinned host
memory), taken through the whole progressive path (fringe tables, Haar DWT, block
selection, superposition; Section 2 steps 1-5) and copied back out.  The device buffers
come in `depth` slots used round robin: while one slot's hologram is copied out on the
copy stream, the next slot's inputs are copied in and its step runs.  Each slot's step is
one captured CUDA graph; for the tensor forms the selection and superposition inside it
are one cgh_progressive_step.

With `concurrent=True` every slot also has its own plan (plan scratch is per plan) and its
own compute streams, so the steps of consecutive scenes may overlap on the GPU: the small
latency-bound kernels of one scene (DWT, selection, compaction) then run beside the other
scene's GEMMs, which leave registers and threads free on every SM.  Every kernel is the
library's; this module only orders copies and graph replays with events.
"""
import torch

from .cgh import Plan


class _Slot:
    def __init__(self, plan, device, concurrent):
        obj = (plan.obj_h, plan.obj_w)
        self.plan = plan
        self.I = torch.empty(obj, dtype=torch.uint8, device=device)
        self.L = torch.empty(obj, dtype=torch.uint8, device=device)
        self.S = torch.empty(obj, dtype=torch.uint8, device=device)
        self.coeffs = torch.empty((plan.n_layers,) + obj, dtype=torch.int32, device=device)
        self.counts = torch.zeros((4, 2), dtype=torch.int32, device=device)
        self.lists = [torch.empty(plan.max_blocks(3 if k == 0 else k), dtype=torch.int32, device=device)
                      for k in range(4)]
        self.holo = torch.empty((plan.holo_h, plan.holo_w), dtype=torch.complex64, device=device)
        self.graph = None
        self.in_done = torch.cuda.Event()
        self.step_done = torch.cuda.Event()
        self.out_done = torch.cuda.Event()
        self.compute = torch.cuda.Stream(device) if concurrent else None
        self.side = (torch.cuda.Stream(device), torch.cuda.Stream(device)) if concurrent else None


class ProgressivePipeline:
    """plan: a Plan; thresholds: level -> uint8 threshold; form: superposition form.
    submit(hI, hL, hS, hH) copies the pinned host maps in, runs the step and copies the
    hologram into the pinned complex64 host tensor hH, all asynchronously; hH is complete
    once synchronize() returns (or the event returned by submit has completed).
    concurrent: one plan and one set of compute streams per slot, so that the steps of
    consecutive scenes overlap (the extra plans are clones of `plan`)."""

    def __init__(self, plan, thresholds, form="tc_fp16x3", depth=2, graphs=True, concurrent=False):
        self.plan = plan
        self.thresholds = dict(thresholds)
        self.form = form
        dev = plan.device
        self.compute = torch.cuda.Stream(dev)
        self.copy_in = torch.cuda.Stream(dev)
        self.copy_out = torch.cuda.Stream(dev)
        self.side = (torch.cuda.Stream(dev), torch.cuda.Stream(dev))
        plans = [plan] + [plan.clone() if concurrent else plan for _ in range(depth - 1)]
        self.slots = [_Slot(p, dev, concurrent) for p in plans]
        for sl in self.slots:
            if sl.compute is None:
                sl.compute, sl.side = self.compute, self.side
        self.k = 0
        # one eager pass per slot (plan scratch, operand planes), then the captured step
        for sl in self.slots:
            self._step(sl)
        for sl in self.slots:
            sl.compute.synchronize()
        if graphs:
            for sl in self.slots:
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g, stream=sl.compute):
                    self._step(sl)
                sl.graph = g
            for sl in self.slots:
                sl.compute.synchronize()

    def _step(self, sl):
        """The whole path on one slot: tables and DWT on side streams forked from the
        compute stream, the selection on it, then the superposition.  The tensor forms run
        selection and superposition as one cgh_progressive_step, which waits for the DWT only
        before it reads the coefficients; the direct form joins both side streams first."""
        st = sl.compute
        s_tab, s_dwt = sl.side
        plan = sl.plan
        fork = torch.cuda.Event()
        fork.record(st)
        s_tab.wait_event(fork)
        s_dwt.wait_event(fork)
        plan.build_tables(stream=s_tab)
        plan.haar_decompose(sl.I, sl.L, sl.coeffs, stream=s_dwt)
        j1, j2 = torch.cuda.Event(), torch.cuda.Event()
        j2.record(s_dwt)
        if self.form != "direct_lut":
            plan.progressive_step(sl.S, sl.L, sl.coeffs, self.thresholds, counts=sl.counts, lists=sl.lists,
                                       holo=sl.holo, form=self.form, coeffs_ready=j2, stream=st)
            j1.record(s_tab)
            st.wait_event(j1)
            return
        plan.progressive_lists(sl.S, sl.L, self.thresholds, counts=sl.counts, lists=sl.lists, stream=st)
        j1.record(s_tab)
        st.wait_event(j1)
        st.wait_event(j2)
        plan.progressive_hologram(sl.coeffs, sl.lists, sl.counts, holo=sl.holo, form=self.form, stream=st)

    def submit(self, hI, hL, hS, hH):
        sl = self.slots[self.k % len(self.slots)]
        self.k += 1
        # inputs: the slot's previous step must have read them
        self.copy_in.wait_event(sl.step_done)
        with torch.cuda.stream(self.copy_in):
            sl.I.copy_(hI, non_blocking=True)
            sl.L.copy_(hL, non_blocking=True)
            sl.S.copy_(hS, non_blocking=True)
        sl.in_done.record(self.copy_in)
        # step: inputs in, and the slot's previous hologram copied out
        sl.compute.wait_event(sl.in_done)
        sl.compute.wait_event(sl.out_done)
        if sl.graph is not None:
            with torch.cuda.stream(sl.compute):
                sl.graph.replay()
        else:
            self._step(sl)
        sl.step_done.record(sl.compute)
        self.copy_out.wait_event(sl.step_done)
        with torch.cuda.stream(self.copy_out):
            hH.copy_(sl.holo, non_blocking=True)
        sl.out_done.record(self.copy_out)
        return sl.out_done

    def synchronize(self):
        for s in [self.copy_in, self.compute, self.copy_out] + [sl.compute for sl in self.slots]:
            s.synchronize()

    def status(self):
        """First nonzero device status word of the slots' plans (cgh_status; read and cleared),
        else 0.  Synchronises."""
        self.synchronize()
        codes = [sl.plan.status() for sl in self.slots]
        return next((c for c in codes if c), 0)


__all__ = ["ProgressivePipeline", "Plan"]
