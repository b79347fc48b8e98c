"""Benchmark: saliency-progressive hologram generation on one GB300 (or N replicas).

A step is one pass of the whole hot path over one synthetic paper-scale scene
(object 512x512 uint8, 16 depth layers in [0.08, 0.20] m, union-of-3-ellipses
saliency, hologram 1024x1024 complex64, pitch 8 um, lambda 532 nm):
  fringe tables -> 3-level integer Haar DWT -> 4 saliency work lists ->
  progressive superposition (the chosen form).
Metric: equivalent point-wise work per second, obj_h*obj_w*holo_h*holo_w / t,
in Gpoint*px/s.

Prints ONE JSON line (rank 0).  --impl reference times the FP64 CPU oracle on the
same workload instead (the reference arm of this repository).
"""
import argparse
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

OBJ, HOLO, NLAYERS = 512, 1024, 16
WORKLOAD = "paper-scale progressive CGH: object 512x512 u8, 16 layers z in [0.08,0.20] m, " \
           "3-ellipse saliency (20-35%), 3 Haar levels, hologram 1024x1024 c64, p=8um, lambda=532nm"
UNITS_PER_STEP = OBJ * OBJ * HOLO * HOLO  # point*px equivalent work of one scene
METRIC = "Gpoint·px/s, saliency-progressive CGH at 1024² vs plain direct; % roofline"
UNIT = "Gpoint·px/s"
L2_FLUSH_BYTES = 512 << 20
E2E_DEPTH = 4  # device slots of the end-to-end pipeline (each with its own plan)


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


def reduce_max(x, device=None):
    """Max of a float over all ranks (identity without torch.distributed)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(units_per_step_per_rank, steps, world_size, max_ms):
    """Aggregate throughput of all ranks: every rank processes its own scene (weak
    scaling), the slowest rank's time bounds the job."""
    return units_per_step_per_rank * steps * world_size / (max_ms / 1e3) / 1e9


def kernel_source_hash(src_files, marker=None):
    """First 16 hex digits of the SHA-256 of the kernel's sources: whole files, or with a
    marker (text on the kernel's definition line) only the definition in the first file, from
    that line to the first closing brace at column 0 after it (the other files whole)."""
    import hashlib
    h = hashlib.sha256()
    for n, f in enumerate(src_files):
        text = open(os.path.join(ROOT, f), "rb").read()
        if marker and n == 0:
            i = text.find(marker.encode())
            if i < 0:
                raise KeyError(f"{marker} not in {f}")
            i = text.rfind(b"\n", 0, i) + 1
            j = text.find(b"\n}\n", i)
            text = text[i:] if j < 0 else text[i:j + 3]
        h.update(text)
    return h.hexdigest()[:16]


def kernel_traffic(key):
    """DRAM bytes per launch of `key` from the committed ncu summary (profiles/traffic.json),
    or None when the kernel's sources changed since those counters were taken."""
    try:
        entry = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))[key]
        ok = kernel_source_hash(entry["src_files"], entry.get("src_marker")) == entry["src_hash"]
        return entry["bytes"] if ok else None
    except Exception:
        return None


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons while the GPU works."""
    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.rows = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        self.t0 = time.time()

    def stop(self):
        if self.proc is None:
            return
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        for line in out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 10:
                continue
            try:
                self.rows.append(dict(sm=float(f[2]), max=float(f[3]), power=float(f[4]),
                                      hw=f[6], hwt=f[7], swt=f[8], pcap=f[9]))
            except ValueError:
                pass

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi samples"], "samples": 0}
        sms = sorted(r["sm"] for r in self.rows)
        reasons = set()
        for r in self.rows:
            if r["hw"].lower() == "active":
                reasons.add("hw_slowdown")
            if r["hwt"].lower() == "active":
                reasons.add("hw_thermal_slowdown")
            if r["swt"].lower() == "active":
                reasons.add("sw_thermal_slowdown")
            if r["pcap"].lower() == "active":
                reasons.add("sw_power_cap")
        return {"sm_mhz": sms[len(sms) // 2], "sm_max_mhz": max(r["max"] for r in self.rows),
                "reasons": sorted(reasons), "samples": len(self.rows),
                "power_w_max": max(r["power"] for r in self.rows)}


def scene_for_rank(rank):
    from synth import scenes
    return scenes.paper_scene(seed=2000 + rank)


# ---------------------------------------------------------------------------------------
# reference arm: the FP64 CPU oracle on the same workload


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import numpy as np
    from oracle import cgh_oracle as O
    from synth import scenes
    sc = scene_for_rank(0)
    g = O.geometry_of(sc)
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()

    def step():
        lists = O.progressive_lists(sc["saliency"], sc["layer"], g.n_layers, scenes.THRESHOLDS_U8)
        return O.progressive_hologram(sc["intensity"], sc["layer"], lists, g)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    value = UNITS_PER_STEP * args.steps / dt / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "form": "oracle residual-map FP64"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{args.steps} full paper-scale scenes (selection + residual-map hologram)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def cpu_baseline(budget_s=12.0):
    """The oracle as it stands, on whole paper-scale scenes, for about budget_s seconds."""
    from oracle import cgh_oracle as O
    from synth import scenes
    sc = scene_for_rank(0)
    g = O.geometry_of(sc)
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    n = 0
    t0 = time.perf_counter()
    H = None
    while True:
        lists = O.progressive_lists(sc["saliency"], sc["layer"], g.n_layers, scenes.THRESHOLDS_U8)
        H = O.progressive_hologram(sc["intensity"], sc["layer"], lists, g)
        n += 1
        if time.perf_counter() - t0 > budget_s or n >= 8:
            break
    dt = time.perf_counter() - t0
    # the plain point-wise hologram of the same scene in the oracle's separable FP64 form
    t1 = time.perf_counter()
    O.plain_pointwise_hologram(sc["intensity"], sc["layer"], g)
    dt_sep = time.perf_counter() - t1
    # and in its direct FP64 sum (every object point at every pixel), on 64 seeded pixels
    import numpy as np
    rng = np.random.default_rng(2000)
    pix = (rng.integers(0, HOLO, 64), rng.integers(0, HOLO, 64))
    t2 = time.perf_counter()
    O.plain_pointwise_hologram(sc["intensity"], sc["layer"], g, pixels=pix)
    dt_dir = time.perf_counter() - t2
    return {"value": UNITS_PER_STEP * n / dt / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n} whole paper-scale scene(s), selection + residual-map hologram, {dt:.1f} s "
                      f"(numpy: matrix products on the BLAS pool of {cores} threads, fringe evaluation on one)",
            "other_forms": {"pointwise_separable_fp64_ms": dt_sep * 1e3,
                            "pointwise_separable_fp64_value": UNITS_PER_STEP / dt_sep / 1e9,
                            "pointwise_direct_fp64_value": OBJ * OBJ * 64 / dt_dir / 1e9,
                            "pointwise_direct_fp64_sample": f"64 seeded hologram pixels, {dt_dir:.1f} s"}}, H


# ---------------------------------------------------------------------------------------
# secondary workloads (reported as fields of the same JSON line)


def progress(msg):
    """One line on stderr per bench phase (the JSON line goes to stdout)."""
    print(f"[bench {time.strftime('%H:%M:%S')}] {msg}", file=sys.stderr, flush=True)


def run_batch_workload(stream, form, count, reps):
    """64 scenes of uneven size (object edge in {128,256,512,1024}, hologram 2x, 4..32
    layers, ellipse saliency covering 5-60%) as one graph-captured batch."""
    import torch
    from paper_2211_09938_gb300 import Plan, autotune
    from paper_2211_09938_gb300.cgh import Batch
    from synth import scenes
    scs = scenes.batch_scenes(seed=4000, count=count)
    with torch.cuda.stream(stream):
        plans = [Plan.for_scene(sc, stream=stream) for sc in scs]
        I = [torch.from_numpy(sc["intensity"]).cuda() for sc in scs]
        L = [torch.from_numpy(sc["layer"]).cuda() for sc in scs]
        S = [torch.from_numpy(sc["saliency"]).cuda() for sc in scs]
        Hs = [torch.empty(sc["holo"], dtype=torch.complex64, device="cuda") for sc in scs]
        batch = Batch(plans, I, L, S, scenes.THRESHOLDS_U8, Hs, form=form, stream=stream)
    cache = os.path.join(ROOT, "paper_2211_09938_gb300", "_build", "autotune.json")
    os.makedirs(os.path.dirname(cache), exist_ok=True)
    progress("batch: created, autotuning")
    tuned = autotune.tune_batch(batch, plans, form, stream, cache_path=cache)
    progress(f"batch: tuned {tuned.get('tiles')}/{tuned['ksteps']}")
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        batch.run(stream=stream)
    for _ in range(3):
        with torch.cuda.stream(stream):
            g.replay()
    stream.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    with torch.cuda.stream(stream):
        for a, b in evs:
            a.record(stream)
            g.replay()
            b.record(stream)
    torch.cuda.synchronize()
    ms = sorted(a.elapsed_time(b) for a, b in evs)[reps // 2]
    work = sum(sc["intensity"].size * sc["holo"][0] * sc["holo"][1] for sc in scs)
    progress("batch: timed; per-scene latency")
    # per-scene latency: each scene alone as its own captured graph
    lat = []
    for k, sc in enumerate(scs):
        with torch.cuda.stream(stream):
            coeffs = torch.empty((len(sc["z"]),) + sc["intensity"].shape, dtype=torch.int32, device="cuda")
            counts = torch.zeros((4, 2), dtype=torch.int32, device="cuda")
            lists = [torch.empty(plans[k].max_blocks(3 if q == 0 else q), dtype=torch.int32, device="cuda")
                     for q in range(4)]

            def one():
                plans[k].haar_decompose(I[k], L[k], coeffs, stream=stream)
                plans[k].progressive_lists(S[k], L[k], scenes.THRESHOLDS_U8, counts=counts, lists=lists,
                                           stream=stream)
                plans[k].progressive_hologram(coeffs, lists, counts, holo=Hs[k], form=form, stream=stream)
            one()
        stream.synchronize()
        gk = torch.cuda.CUDAGraph()
        with torch.cuda.graph(gk, stream=stream):
            one()
        t = []
        for _ in range(5):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                a.record(stream)
                gk.replay()
                b.record(stream)
            torch.cuda.synchronize()
            t.append(a.elapsed_time(b))
        lat.append(sorted(t)[2])
        del gk
    lat = sorted(lat)
    batch.close()
    for p_ in plans:
        p_.close()
    return {"scenes": count, "form": form, "ms_per_batch": ms, "scenes_per_s": count / (ms / 1e3),
            "gpoint_px_per_s": work / (ms / 1e3) / 1e9,
            "latency_ms_p50": lat[len(lat) // 2], "latency_ms_p99": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
            "latency_note": "each scene alone as a captured graph (DWT, selection, superposition)",
            "autotuned_ksteps_per_unit": tuned["ksteps"], "autotuned_stage2_tiles": tuned.get("tiles"),
            "autotune_tried_ms": tuned.get("tried"),
            "sizes": sorted(set(sc["intensity"].shape[0] for sc in scs))}


def run_phase_opt_workload(stream, steps):
    """Phase-only optimisation: batch 4, hologram 1024^2, 8 layers, 512^2 blob target, loss
    weight 4 inside the saliency mask; phase initialised to arg of the progressive hologram."""
    import numpy as np
    import torch
    from paper_2211_09938_gb300 import Plan, optim
    from synth import scenes
    sc = scenes.random_scene(5000, 512, 1024, 8, sal_fraction=0.3)
    with torch.cuda.stream(stream):
        plan = Plan.for_scene(sc, stream=stream)
        L = torch.from_numpy(sc["layer"]).cuda()
        W = torch.from_numpy(np.where(sc["saliency"] > 0, 4.0, 1.0).astype(np.float32)).cuda()
        targets, phases = [], []
        for b in range(4):
            t = scenes.random_scene(5000 + b, 512, 1024, 8)["intensity"].astype(np.float32) / 255.0
            targets.append(torch.from_numpy(t).cuda())
            I = torch.from_numpy((t * 255).astype(np.uint8)).cuda()
            S = torch.from_numpy(sc["saliency"]).cuda()
            coeffs = plan.haar_decompose(I, L, stream=stream)
            lists, counts = plan.progressive_lists(S, L, scenes.THRESHOLDS_U8, stream=stream)
            H = plan.progressive_hologram(coeffs, lists, counts, form="tc_bf16x3", stream=stream)
            phases.append(torch.angle(H))
        T = torch.stack(targets)
        opt = optim.PhaseOptimiser(plan, L, T, W, torch.stack(phases), lr=0.05, checkpoint=True, graph=True)
        l0 = opt.step()
    stream.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        a.record(stream)
        t0 = time.perf_counter()
        for _ in range(steps):
            l1 = opt.step(sync=False)
        host_ms = (time.perf_counter() - t0) * 1e3 / steps
        b.record(stream)
    torch.cuda.synchronize()
    l1 = float(l1)
    ms = a.elapsed_time(b) / steps
    plan.close()
    # tensor-core work of one Adam step: per hologram and layer, the reconstruction
    # (8 Nh^2 No + 8 Nh No^2 flop for the two complex products), its recomputation in the
    # backward (checkpointing) and the propagation of the field cotangents (the same sizes),
    # each as 3 bf16 hi+lo products
    nh, no, nz, nb = 1024, 512, 8, 4
    flop = 3 * nb * nz * 3 * 8.0 * (nh * nh * no + nh * no * no)
    pk = peaks() or {}
    peak_tf = pk.get("bf16_tflops_sustained", pk.get("bf16_tflops", 1700.0))
    roof = {"bound": "tensor", "flop_per_adam_step": flop, "achieved": flop / (ms / 1e3) / 1e12,
            "peak": peak_tf, "unit": "TFLOP/s", "frac": flop / (ms / 1e3) / 1e12 / peak_tf,
            "peak_note": "measured cuBLAS bf16 dense, sustained (a seconds-long loop)"}
    return {"batch": 4, "holo": 1024, "layers": 8, "adam_steps": steps + 1, "adam_steps_timed": steps,
            "ms_per_adam_step": ms, "host_ms_per_adam_step": host_ms, "roofline": roof,
            "adam_steps_per_s": 1e3 / ms, "loss_first": l0, "loss_last": l1,
            "note": "forward reconstruction + amplitude backward + propagation of the 4 holograms, each GEMM "
                    "stage once over the (hologram, layer) pairs; fields recomputed in backward (checkpointing); "
                    "the whole step (loss, backward, fused Adam) captured in a CUDA graph and replayed"}


# ---------------------------------------------------------------------------------------
# our arm


def run_level_sweep(plan, coeffs, lists, counts, I, L, stream, form, flush):
    """Section 3's level sweep on the bench scene: for each cumulative stage (LLL, LL, L,
    object) the operator count (Table 2), the SSIM of the reconstructed amplitude against
    the plain point-wise hologram's (Table 3), and the device time of the stage's
    superposition with L2 flushed; reconstruction and SSIM run in the library's kernels."""
    import torch
    from paper_2211_09938_gb300 import Plan
    from paper_2211_09938_gb300.cgh import ssim
    with torch.cuda.stream(stream):
        _, ref = plan.reconstruct(plan.plain_direct(I, L, stream=stream), L, fields=False, stream=stream)
        out = []
        for stage, name in enumerate(Plan.LEVEL_STAGES):
            c = Plan.level_counts(counts, stage)
            H = plan.progressive_hologram(coeffs, lists, c, form=form, stream=stream)
            flush.fill_(1.0)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            ev[0].record(stream)
            plan.progressive_hologram(coeffs, lists, c, holo=H, form=form, stream=stream)
            ev[1].record(stream)
            _, A = plan.reconstruct(H, L, fields=False, stream=stream)
            s = ssim(A, ref, stream=stream)
            stream.synchronize()
            out.append({"stage": name, "operators": Plan.operator_count(c),
                        "ssim_vs_pointwise": s.item(), "superposition_ms": ev[0].elapsed_time(ev[1])})
    return {"form": form, "pointwise_operators": int(I.numel()), "stages": out}


def run_asm_workload(plan, H, L, stream, flush, reps=10):
    """Inverse angular-spectrum reconstruction of the bench hologram (Section 2, last
    paragraph) for both paddings: device ms per call with L2 flushed, the split between
    the forward FFT and the per-layer transfer + inverse FFTs, and the HBM bytes the
    four-kernel pipeline must move (hologram in; row spectra, spectrum, layer columns out
    and back; fields and amplitude out; the spectrum read from HBM once, its re-reads by
    the other layers served from L2) against the measured copy bandwidth."""
    import torch
    Z, No, Nh, s = plan.n_layers, plan.obj_h, plan.holo_h, plan.holo_h // plan.obj_h
    F = torch.empty((Z, No, No), dtype=torch.complex64, device="cuda")
    A = torch.empty((No, No), dtype=torch.float32, device="cuda")
    out = {}
    pk = peaks() or {}
    for pad in (2, 1):
        P = pad * Nh
        Lf = P // s
        with torch.cuda.stream(stream):
            for _ in range(3):
                plan.reconstruct_asm(H, L, F, A, pad=pad, stream=stream)
            plan.profile(True)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
            split = {"asm_fft": 0.0, "asm_inv": 0.0}
            for k in range(reps):
                flush.fill_(float(k))
                ev[k][0].record(stream)
                plan.reconstruct_asm(H, L, F, A, pad=pad, stream=stream)
                ev[k][1].record(stream)
                st = plan.profile_read(stream=stream)
                for key in split:
                    split[key] += st[key] / reps
            plan.profile(False)
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in ev) / reps
        nbytes = 8 * (Nh * Nh + 2 * Nh * P + 2 * P * P + 2 * Z * No * Lf + Z * No * No) + 4 * No * No + Z * No * No
        gbs = nbytes / (ms / 1e3) / 1e9
        out[f"pad{pad}"] = {"ms": ms, "stages_ms": split, "hbm_bytes_algorithmic": nbytes,
                            "achieved_GBps": gbs,
                            "frac_of_measured_hbm": gbs / pk["hbm_gbs"] if "hbm_gbs" in pk else None}
    return out


def run_rgb_workload(stream, form, flush, reps=10):
    """Colour frame: the bench scene's three colour channels (R, G, B at 638, 532 and 450
    nm) as one three-scene batch; device ms per colour frame with L2 flushed."""
    import numpy as np
    import torch
    from synth import scenes
    from paper_2211_09938_gb300.rgb import RGBHologram, WAVELENGTHS_RGB
    sc = scenes.rgb_scene(2002, OBJ, HOLO, NLAYERS)
    Ic = [torch.from_numpy(np.ascontiguousarray(sc["intensity"][c])).cuda() for c in range(3)]
    L = torch.from_numpy(sc["layer"]).cuda()
    S = torch.from_numpy(sc["saliency"]).cuda()
    holos = [torch.empty((HOLO, HOLO), dtype=torch.complex64, device="cuda") for _ in range(3)]
    with torch.cuda.stream(stream):
        rgb = RGBHologram((OBJ, OBJ), (HOLO, HOLO), sc["pitch"], sc["z"], Ic, L, S, scenes.THRESHOLDS_U8, holos,
                          form=form, stream=stream)
        for _ in range(3):
            rgb.run(stream)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        for k in range(reps):
            flush.fill_(float(k))
            ev[k][0].record(stream)
            rgb.run(stream)
            ev[k][1].record(stream)
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in ev) / reps
    rgb.close()
    return {"form": form, "wavelengths_nm": [w * 1e9 for w in WAVELENGTHS_RGB], "ms_per_colour_frame": ms,
            "value": 3 * UNITS_PER_STEP / (ms / 1e3) / 1e9, "unit": UNIT}


def run_precision_workload(stream, flush, forms=("tc_fp16x3", "tc_bf16x3", "tc_fp16x2", "direct_lut"), reps=5):
    """The precision configuration: the paper-scale 512x512 scene at a 2048x2048 hologram
    with 32 layers.  Per superposition form: device time of the superposition call (L2
    flushed before each), Gpoint*px/s, the stage-2 GEMM's roofline fraction (tensor forms),
    and rel-L2 / max-abs against the FP64 oracle for the full hologram and for every layer
    (each layer's own work lists).  The oracle's per-layer holograms sum to the full one."""
    import numpy as np
    import torch
    from oracle import cgh_oracle as O
    from paper_2211_09938_gb300 import Plan
    from synth import scenes
    obj, holo, nl = 512, 2048, 32
    sc = scenes.paper_scene(n_layers=nl, holo=holo)
    g = O.geometry_of(sc)
    pk = peaks() or {}
    peak_tf = pk.get("bf16_tflops", 1900.0)
    with torch.cuda.stream(stream):
        plan = Plan.for_scene(sc, stream=stream)
        I = torch.from_numpy(sc["intensity"]).cuda()
        L = torch.from_numpy(sc["layer"]).cuda()
        S = torch.from_numpy(sc["saliency"]).cuda()
        coeffs = plan.haar_decompose(I, L, stream=stream)
        lists, counts = plan.progressive_lists(S, L, scenes.THRESHOLDS_U8, stream=stream)
        H = torch.empty((holo, holo), dtype=torch.complex64, device="cuda")
    stream.synchronize()
    c = counts.cpu().numpy()
    host = [lists[k][:int(c[k, 0])].cpu().numpy() for k in range(4)]
    per_layer_lists = []
    for z in range(nl):
        sel = [x[(x >> 24) == z] for x in host]
        dl = [torch.from_numpy(np.concatenate([x, np.zeros(1, np.int32)]).astype(np.int32)).cuda() for x in sel]
        cnt = torch.tensor([[len(x), len(x)] for x in sel], dtype=torch.int32, device="cuda")
        per_layer_lists.append((sel, dl, cnt))
    out = {"workload": f"paper-scale scene {obj}x{obj}, {nl} layers z in [0.08,0.20] m, hologram {holo}x{holo}",
           "forms": {}}
    got = {}
    for form in forms:
        times, st2 = [], []
        for k in range(reps + 1):
            plan.profile(True)
            with torch.cuda.stream(stream):
                flush.fill_(float(k))
                e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
                e[0].record(stream)
                plan.progressive_hologram(coeffs, lists, counts, holo=H, form=form, stream=stream)
                e[1].record(stream)
            prof = plan.profile_read(stream=stream)
            plan.profile(False)
            if k:
                times.append(e[0].elapsed_time(e[1]))
                st2.append(prof.get("tc_fused", 0.0) or prof.get("tc_stage2", 0.0))
                fused_run = prof.get("tc_fused", 0.0) > 0
        ms = sorted(times)[len(times) // 2]
        ent = {"superposition_ms": ms, "value": obj * obj * holo * holo / (ms / 1e3) / 1e9, "unit": UNIT}
        if form != "direct_lut":
            kr, kc = plan.tc_layer_dims(stream=stream)
            prods = 2 if form == "tc_fp16x2" else 3
            flop = prods * 8.0 * holo * holo * sum(kr)
            if fused_run:
                flop += prods * 4.0 * holo * sum(a_ * b_ for a_, b_ in zip(kr, kc))
            k_ms = sorted(st2)[len(st2) // 2]
            ent["gemm"] = {"kernel": "k_tc_fused (both GEMM stages)" if fused_run else "k_tc_gemm stage 2",
                           "ms": k_ms, "achieved_tflops": flop / (k_ms / 1e3) / 1e12,
                           "frac_of_measured_bf16_peak": flop / (k_ms / 1e3) / 1e12 / peak_tf,
                           "k_contracted": sum(kr)}
        got[form] = H.cpu().numpy()
        layer_h = []
        for z in range(nl):
            _, dl, cnt = per_layer_lists[z]
            with torch.cuda.stream(stream):
                Hz = plan.progressive_hologram(coeffs, dl, cnt, form=form, stream=stream)
            stream.synchronize()
            layer_h.append(Hz.cpu().numpy())
        ent["_layers"] = layer_h
        out["forms"][form] = ent
    plan.close()
    # the FP64 oracle, layer by layer (its per-layer holograms sum to the full hologram)
    Href = np.zeros((holo, holo), np.complex128)
    for z in range(nl):
        Hz_ref = O.progressive_hologram(sc["intensity"], sc["layer"], per_layer_lists[z][0], g)
        Href += Hz_ref
        for form in forms:
            ent = out["forms"][form]
            Hz = ent["_layers"][z]
            ent.setdefault("per_layer_rel_l2", []).append(O.rel_l2(Hz, Hz_ref))
            ent.setdefault("per_layer_max_abs", []).append(float(np.max(np.abs(Hz - Hz_ref))))
    for form in forms:
        ent = out["forms"][form]
        del ent["_layers"]
        ent["rel_l2_vs_fp64_oracle"] = O.rel_l2(got[form], Href)
        ent["max_abs_vs_fp64_oracle"] = float(np.max(np.abs(got[form] - Href)))
        ent["per_layer_rel_l2_max"] = max(ent["per_layer_rel_l2"])
    out["max_abs_reference"] = float(np.max(np.abs(Href)))
    out["bars"] = {"fp32": 1e-5, "bf16_split": 1e-3}
    return out


def run_hbm_paths(stream, flush, reps=5):
    """The DWT (A2) and the four-list selection (A3) at an 8192 x 8192 object with 4 layers,
    where they are long enough to measure against HBM: algorithmic bytes 2 No^2 read and
    4 Z No^2 written (DWT), 2 No^2 read plus 4 bytes per list entry written (selection)."""
    import numpy as np
    import torch
    from paper_2211_09938_gb300 import Plan
    from synth import scenes
    n, Z = 8192, 4
    rng = np.random.default_rng(7000)
    pk = peaks() or {}
    with torch.cuda.stream(stream):
        plan = Plan((n, n), (n, n), 8e-6, 532e-9, [0.10, 0.11, 0.12, 0.13], stream=stream)
        I = torch.from_numpy(rng.integers(0, 256, size=(n, n), dtype=np.uint8)).cuda()
        L = torch.from_numpy(np.repeat(np.arange(Z, dtype=np.uint8), n // Z)[:, None].repeat(n, 1)).cuda()
        S = torch.from_numpy(rng.integers(0, 256, size=(n, n), dtype=np.uint8)).cuda()
        coeffs = torch.empty((Z, n, n), dtype=torch.int32, device="cuda")
        counts = torch.zeros((4, 2), dtype=torch.int32, device="cuda")
        lists = [torch.empty(plan.max_blocks(3 if k == 0 else k), dtype=torch.int32, device="cuda")
                 for k in range(4)]
        out = {}
        for name, fn in (("haar", lambda: plan.haar_decompose(I, L, coeffs, stream=stream)),
                         ("select", lambda: plan.progressive_lists(S, L, scenes.THRESHOLDS_U8, counts=counts,
                                                                   lists=lists, stream=stream))):
            fn()
            ms = 0.0
            for k in range(reps):
                flush.fill_(float(k))
                ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
                ev[0].record(stream)
                fn()
                ev[1].record(stream)
                ev[1].synchronize()
                ms += ev[0].elapsed_time(ev[1]) / reps
            if name == "haar":
                nbytes = 2 * n * n + 4 * Z * n * n
            else:
                nbytes = 2 * n * n + 4 * int(counts[:, 0].sum().item())
            gbs = nbytes / (ms / 1e3) / 1e9
            out[name] = {"ms": ms, "bytes_algorithmic": nbytes, "achieved_GBps": gbs,
                         "frac_of_measured_hbm": gbs / pk["hbm_gbs"] if "hbm_gbs" in pk else None}
    plan.close()
    return {"object": f"{n}x{n}, {Z} layers", **out}


def run_ours(args):
    import numpy as np
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    devn = torch.cuda.current_device()
    from paper_2211_09938_gb300 import Plan
    from synth import scenes

    sc = scene_for_rank(rank)
    stream = torch.cuda.Stream()
    form = args.form
    with torch.cuda.stream(stream):
        plan = Plan.for_scene(sc, stream=stream)
        I = torch.from_numpy(sc["intensity"]).cuda()
        L = torch.from_numpy(sc["layer"]).cuda()
        S = torch.from_numpy(sc["saliency"]).cuda()
        coeffs = torch.empty((NLAYERS, OBJ, OBJ), dtype=torch.int32, device="cuda")
        counts = torch.zeros((4, 2), dtype=torch.int32, device="cuda")
        lists = [torch.empty(plan.max_blocks(3 if k == 0 else k), dtype=torch.int32, device="cuda")
                 for k in range(4)]
        holo = torch.empty((HOLO, HOLO), dtype=torch.complex64, device="cuda")
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    tensor_form = form != "direct_lut"
    # fringe tables (FP64 point fringes, block tables) and the DWT, then: tensor forms, one
    # cgh_progressive_step (the single-launch selection, which also marks the operand flags,
    # compaction, inverse DWT, the two GEMMs); direct form, the three selection passes and
    # the direct kernel
    launches_per_step = 2 + 1 + (1 + 4 if tensor_form else 3 + 1)  # one fewer when the GEMMs are fused

    # The fringe-table build, the DWT and the block selection are independent: the first two
    # run on side streams forked from (and joined back into) the step's stream, which the
    # CUDA graph capture records as parallel branches.  The tensor-form step waits for the DWT
    # only before its inverse-DWT kernel (coeffs_ready), so the selection overlaps the DWT.
    s_tab, s_dwt = torch.cuda.Stream(), torch.cuda.Stream()

    def step(f=form):
        fork = torch.cuda.Event()
        fork.record(stream)
        s_tab.wait_event(fork)
        s_dwt.wait_event(fork)
        plan.build_tables(stream=s_tab)
        plan.haar_decompose(I, L, coeffs, stream=s_dwt)
        j1, j2 = torch.cuda.Event(), torch.cuda.Event()
        j2.record(s_dwt)
        if f != "direct_lut":
            plan.progressive_step(S, L, coeffs, scenes.THRESHOLDS_U8, counts=counts, lists=lists, holo=holo,
                                  form=f, coeffs_ready=j2, stream=stream)
            j1.record(s_tab)
            stream.wait_event(j1)
            return
        plan.progressive_lists(S, L, scenes.THRESHOLDS_U8, counts=counts, lists=lists, stream=stream)
        j1.record(s_tab)
        stream.wait_event(j1)
        stream.wait_event(j2)
        plan.progressive_hologram(coeffs, lists, counts, holo=holo, form=form, stream=stream)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    stream.synchronize()
    # the whole step as one CUDA graph (every launch of the path, no host work between)
    graph = None
    if not args.no_graph:
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            step()
        for _ in range(args.warmup):
            with torch.cuda.stream(stream):
                graph.replay()
        stream.synchronize()

    def run_step():
        if graph is not None:
            graph.replay()
        else:
            step()

    # ---- timed region: K steps, L2 flushed before each, device time from CUDA events
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    sampler = ClockSampler(devn)
    sampler.start()
    time.sleep(0.3)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    with torch.cuda.stream(stream):
        for k in range(args.steps):
            flush.fill_(float(k))
            evs[k][0].record(stream)
            run_step()
            evs[k][1].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if ws > 1:
        torch.distributed.barrier()
    sampler.stop()
    dev_ms = reduce_max(sum(a.elapsed_time(b) for a, b in evs), device="cuda")
    value = whole_job_value(UNITS_PER_STEP, args.steps, ws, dev_ms)

    # ---- the same step with the fp16x2 tensor form (fringe rounded once to fp16, data hi+lo,
    # two products per real product), timed the same way; its accuracy is reported beside the
    # other forms'
    fast = None
    if form != "direct_lut" and graph is not None and not args.skip_forms:
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                step("tc_fp16x2")
        stream.synchronize()
        g2 = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g2, stream=stream):
            step("tc_fp16x2")
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                g2.replay()
        stream.synchronize()
        evs2 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                for _ in range(args.steps)]
        with torch.cuda.stream(stream):
            for k in range(args.steps):
                flush.fill_(float(k))
                evs2[k][0].record(stream)
                g2.replay()
                evs2[k][1].record(stream)
        torch.cuda.synchronize()
        ms2 = reduce_max(sum(a.elapsed_time(b) for a, b in evs2), device="cuda")
        fast = {"form": "tc_fp16x2", "ms_per_step": ms2 / args.steps,
                "value": whole_job_value(UNITS_PER_STEP, args.steps, ws, ms2), "unit": UNIT,
                "note": "the same captured step, L2 flushed before each, with the fringe operand as its fp16 hi "
                        "planes (one rounding, unit roundoff 2^-11) and the data operand fp16 hi+lo: two "
                        "products per real product; rel-L2 in other_forms_rel_l2_vs_fp64_oracle (bar 1e-3)"}
        del g2

    # ---- a long steady run of the same captured step (L2 flushed before each), with the SM
    # clock sampled throughout: thousands of steps instead of the K of the timed region above
    steady = None
    if graph is not None and rank == 0 and args.steady_steps > 0:
        n_st = args.steady_steps
        sam = ClockSampler(devn)
        sam.start()
        time.sleep(0.3)
        ev_st = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_st)]
        with torch.cuda.stream(stream):
            for k in range(n_st):
                flush.fill_(float(k))
                ev_st[k][0].record(stream)
                graph.replay()
                ev_st[k][1].record(stream)
        torch.cuda.synchronize()
        sam.stop()
        t_st = sorted(a.elapsed_time(b) for a, b in ev_st)
        steady = {"steps": n_st, "ms_per_step_median": t_st[n_st // 2], "ms_per_step_p10": t_st[n_st // 10],
                  "ms_per_step_p99": t_st[min(n_st - 1, int(0.99 * n_st))],
                  "value_median": UNITS_PER_STEP / (t_st[n_st // 2] / 1e3) / 1e9, "unit": UNIT,
                  "clocks": sam.summary(),
                  "note": "the captured step replayed back to back, a 512 MiB L2 flush before each, SM clock "
                          "sampled every 100 ms over the run"}

    # ---- per-stage device times (CUDA events recorded by the library on `stream`),
    # L2 flushed before every repetition; the dominant kernel's average launch duration
    R = max(5, min(50, args.steps))
    plan.profile(True)
    stage_sum = {}
    for k in range(R):
        with torch.cuda.stream(stream):
            flush.fill_(float(k))
            step()
        for key, v in plan.profile_read(stream=stream).items():
            stage_sum[key] = stage_sum.get(key, 0.0) + v
    plan.profile(False)
    stages = {key: v / R for key, v in stage_sum.items() if v > 0}
    fused = stages.get("tc_fused", 0.0) > 0
    k_ms = stages.get("direct_lut" if form == "direct_lut" else ("tc_fused" if fused else "tc_stage2"), 0.0)

    c = counts.cpu().numpy()
    n_lll, n1, n2, n3 = (int(c[k, 0]) for k in range(4))
    rank1_terms = n_lll + 2 * (n1 + n2 + n3)
    # the detail-basis terms (an LLL block, or one of X, Y, D of a selected block) and the
    # paper's operators (an LLL block, or one residual cell: 4 per selected block)
    t_terms = n_lll + 3 * (n1 + n2 + n3)
    operators = Plan.operator_count(counts)
    step_ms = sorted(a.elapsed_time(b) for a, b in evs)
    from paper_2211_09938_gb300.cgh import probe_peaks
    unit_peaks = probe_peaks(stream=stream)
    pk = peaks() or {}
    clocks = sampler.summary()
    if form != "direct_lut":
        kr, kc = plan.tc_layer_dims(stream=stream)
        ksum = sum(kr)
        # stage 2: complex GEMM M = N = hologram edge, K = sum of the layers' compacted rows,
        # 8 flop per complex MAC, x3 for the hi+lo products (the algorithmic count of the form);
        # stage 1: per layer a complex x real GEMM, M = hologram edge, N = the layer's compacted
        # rows, K = its compacted columns, 4 flop per MAC, x3.  The fused launch runs both.
        stage2_flop = 3 * 8.0 * HOLO * HOLO * ksum
        stage1_flop = 3 * 4.0 * HOLO * sum(a_ * b_ for a_, b_ in zip(kr, kc))
        algo_flop = stage2_flop + (stage1_flop if fused else 0.0)
        peak_tf = pk.get("bf16_tflops", 1900.0)
        pairs = not fused and plan.stage2_tiles_used() == Plan.TILES_PAIR
        roof = {"bound": "tensor",
                "kernel": "k_tc_fused (both GEMM stages, one cooperative launch)" if fused
                else ("k_tc_gemm_pair<KIND_CC> (stage 2, a CTA pair per 256x128 tile)" if pairs
                      else "k_tc_gemm<KIND_CC,EPI_H> (stage 2, one CTA per 128x128 tile)"),
                "achieved": algo_flop / (k_ms / 1e3) / 1e12, "peak": peak_tf, "unit": "TFLOP/s",
                "frac": algo_flop / (k_ms / 1e3) / 1e12 / peak_tf,
                "traffic": kernel_traffic(("k_tc_fused" if fused else "k_tc_gemm_pair stage 2" if pairs
                                           else "k_tc_gemm stage 2") + f" ({form})"),
                "traffic_note": "ncu dram__bytes_read.sum + dram__bytes_write.sum per launch, from "
                                "profiles/traffic.json (the ncu summary it names); null if the kernel changed "
                                "since the counters were taken",
                "peak_note": "measured cuBLAS bf16 dense burst (MEASURED_PEAKS.json); fp16 has the same "
                             "nominal dense rate" if "bf16_tflops" in pk else "fallback 1.9 PFLOP/s",
                "kernel_ms": k_ms, "flop": algo_flop, "stage1_flop": stage1_flop, "stage2_flop": stage2_flop,
                "k_contracted": ksum, "k_other_axis": sum(kc),
                "k_note": "k_contracted: the sum over the layers of the compacted object rows or columns "
                          "that stage 2 contracts over (the smaller, chosen on the device); k_other_axis: "
                          "the other one"}
    if form == "direct_lut":
        # FP32 FFMA bound: 8 flop (4 FFMA) per rank-1 term and hologram pixel
        algo_flop = 8.0 * rank1_terms * HOLO * HOLO
        sms = torch.cuda.get_device_properties(devn).multi_processor_count
        peak_tf = unit_peaks["ffma_flops_per_s"] / 1e12
        roof = {"bound": "alu", "kernel": "k_direct_lut", "achieved": algo_flop / (k_ms / 1e3) / 1e12,
                "peak": peak_tf, "unit": "TFLOP/s",
                "frac": algo_flop / (k_ms / 1e3) / 1e12 / peak_tf, "traffic": kernel_traffic("k_direct_lut"),
                "peak_note": "FP32 FMA rate measured by the library's own microbenchmark (cgh_probe_ffma); "
                             f"derived {sms} SMs x 128 lanes x 2 flop x "
                             f"{pk.get('sm_max_mhz', 2070.0):.0f} MHz = "
                             f"{sms * 256 * pk.get('sm_max_mhz', 2070.0) * 1e6 / 1e12:.1f} TFLOP/s",
                "kernel_ms": k_ms}

    progress("step timed; end to end")
    # ---- end to end from pinned host inputs to the host hologram, every step: the library's
    # streaming pipeline (copies in and out on their own streams, overlapping the neighbouring
    # scenes' compute; two device slots, each step a captured graph)
    from paper_2211_09938_gb300.pipeline import ProgressivePipeline
    hI = torch.from_numpy(sc["intensity"]).pin_memory()
    hL = torch.from_numpy(sc["layer"]).pin_memory()
    hS = torch.from_numpy(sc["saliency"]).pin_memory()
    hH = [torch.empty((HOLO, HOLO), dtype=torch.complex64).pin_memory() for _ in range(2)]
    pipe = ProgressivePipeline(plan, scenes.THRESHOLDS_U8, form=form, depth=E2E_DEPTH, graphs=not args.no_graph,
                               concurrent=True)
    for k in range(3):
        pipe.submit(hI, hL, hS, hH[k % 2])
    pipe.synchronize()
    E = max(3, min(args.steps, 50))
    torch.cuda.synchronize()
    e0 = time.perf_counter()
    for k in range(E):
        pipe.submit(hI, hL, hS, hH[k % 2])
    pipe.synchronize()
    e2e_s = (time.perf_counter() - e0) / E
    if pipe.status() != 0:
        raise RuntimeError("end-to-end pipeline: a bounded device wait gave up (cgh_status)")
    e2e = {"value": UNITS_PER_STEP * ws / e2e_s / 1e9, "unit": UNIT,
           "h2d_bytes_per_step": 3 * OBJ * OBJ, "d2h_bytes_per_step": 8 * HOLO * HOLO,
           "note": f"ProgressivePipeline, {E2E_DEPTH} concurrent slots (one plan and compute stream each): "
                   "inputs copied in and the hologram copied out every step on copy streams, consecutive "
                   "scenes' steps overlapping on the GPU; no L2 flush between steps, the per-step working "
                   "set (fringe planes 128 MB per plan, coefficients 16 MB, stage-1 output 30 MB) exceeds "
                   "the 129 MB L2"}

    # ---- plain point-wise direct kernel on the same scene (the baseline the metric names)
    plain = None
    if not args.skip_plain:
        with torch.cuda.stream(stream):
            Hp = plan.plain_direct(I, L, stream=stream)
            pe = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            pe[0].record(stream)
            plan.plain_direct(I, L, holo=Hp, stream=stream)
            pe[1].record(stream)
        torch.cuda.synchronize()
        p_ms = pe[0].elapsed_time(pe[1])
        plain = {"ms": p_ms, "value": UNITS_PER_STEP / (p_ms / 1e3) / 1e9, "unit": UNIT,
                 "speedup_of_progressive_step": p_ms / (dev_ms / args.steps)}

    # ---- per-point depth (no depth layers) on the same object, continuous depth map
    pointcloud = None
    if rank == 0 and not args.skip_plain:
        D = torch.from_numpy(scenes.depth_map(2001, OBJ)).cuda()
        with torch.cuda.stream(stream):
            Hc = plan.pointcloud_direct(I, D, stream=stream)
            pe = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            pe[0].record(stream)
            plan.pointcloud_direct(I, D, holo=Hc, stream=stream)
            pe[1].record(stream)
        torch.cuda.synchronize()
        c_ms = pe[0].elapsed_time(pe[1])
        sms = torch.cuda.get_device_properties(devn).multi_processor_count
        # one SFU sine-cosine pair per point and pixel, against the pair rate the library's own
        # microbenchmark measures (cgh_probe_sfu)
        xu_peak = unit_peaks["sfu_pairs_per_s"] / 1e9
        c_val = UNITS_PER_STEP / (c_ms / 1e3) / 1e9
        pointcloud = {"ms": c_ms, "value": c_val, "unit": UNIT,
                      "roofline": {"bound": "xu", "achieved": c_val, "peak": xu_peak, "unit": UNIT,
                                   "frac": c_val / xu_peak,
                                   "peak_note": "sine-cosine pairs per second measured by cgh_probe_sfu; derived "
                                                f"{sms} SMs x 16 SFU lanes x max SM clock / 2 = "
                                                f"{sms * 16 * pk.get('sm_max_mhz', 2070.0) * 1e6 / 2 / 1e9:.0f} "
                                                "Gpair/s"}}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dev_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"direct_lut": "f32", "tc_bf16x3": "bf16", "tc_fp16x3": "fp16"}[form],
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "form": form, "l2": "flushed (512 MiB write) before every timed step",
                   "cuda_graph": graph is not None,
                   "luts": "one-axis fringe tables rebuilt every step (side stream); the tensor form's fringe "
                           "planes are derived from them once per plan (the paper's precomputed LUT blocks)",
                   "arithmetic": {"direct_lut": "FP32 FFMA", "tc_bf16x3": "bf16 hi+lo operands, 3 products, FP32 accumulation",
                                  "tc_fp16x3": "fp16 hi+lo operands, 3 products, FP32 accumulation"}[form],
                   "parallelism": f"replicas{ws}" if ws > 1 else "single GPU",
                   "work_lists": [n_lll, n1, n2, n3], "rank1_terms": rank1_terms},
        "roofline": roof, "clocks": clocks, "e2e": e2e,
        "gpu_launches": (launches_per_step - (1 if fused else 0)) * args.steps, "wall_s_timed_region": wall,
        "ms_per_step_p50": step_ms[len(step_ms) // 2], "ms_per_step_p99": step_ms[min(len(step_ms) - 1,
                                                                                     int(0.99 * len(step_ms)))],
        "algorithmic": {"terms": t_terms, "terms_px_per_s": t_terms * HOLO * HOLO / (dev_ms / args.steps / 1e3),
                        "operators": operators, "pointwise_operators": OBJ * OBJ,
                        "note": "terms: LLL blocks and the X, Y, D coefficients of selected blocks; operators: "
                                "LLL blocks and residual cells (4 per selected block), as counted in Section 3"},
        "unit_peaks_measured": unit_peaks,
    }
    line["stages_ms"] = stages
    if steady is not None:
        line["steady_state"] = steady
    if form != "direct_lut" and not args.skip_forms:
        # the same superposition with both stages in one cooperative launch (plan option)
        plan.set_fusion(True)
        s1, s2 = [], []
        for k in range(R):
            plan.profile(True)
            with torch.cuda.stream(stream):
                flush.fill_(float(k))
                plan.progressive_hologram(coeffs, lists, counts, holo=holo, form=form, stream=stream)
            pr = plan.profile_read(stream=stream)
            plan.profile(False)
            s1.append(pr.get("tc_fused", 0.0))
        plan.set_fusion(False)
        m1 = sorted(s1)[len(s1) // 2]
        fl = stage1_flop + stage2_flop
        line["fused_gemms"] = {
            "kernel": "k_tc_fused (both GEMM stages, one cooperative launch)", "ms": m1,
            "two_launches_ms": stages.get("tc_stage1", 0.0) + stages.get("tc_stage2", 0.0),
            "achieved_tflops": fl / (m1 / 1e3) / 1e12, "frac_of_measured_bf16_peak": fl / (m1 / 1e3) / 1e12 / peak_tf,
            "note": "plan option (cgh_plan_set_fusion); the step runs the two launches, because the cooperative "
                    "launch needs every SM and so gains nothing in the captured step and slows concurrent "
                    "pipelines; L2 flushed before each"}
    progress("e2e done; batch")
    if rank == 0 and ws == 1 and not args.skip_batch:
        line["batch"] = run_batch_workload(stream, form if form != "direct_lut" else "tc_bf16x3",
                                           args.batch_scenes, 10)
    progress("phase optimisation")
    if rank == 0 and ws == 1 and not args.skip_phase_opt:
        line["phase_opt"] = run_phase_opt_workload(stream, args.phase_opt_steps)
    if plain is not None:
        line["plain_direct"] = plain
    if pointcloud is not None:
        line["pointcloud_direct"] = pointcloud
    progress("HBM paths")
    if rank == 0 and not args.skip_hbm_paths:
        line["hbm_paths_8192"] = run_hbm_paths(stream, flush)
    progress("precision")
    if rank == 0 and ws == 1 and not args.skip_precision:
        line["precision"] = run_precision_workload(stream, flush)
    progress("rgb")
    if rank == 0 and not args.skip_rgb:
        line["rgb"] = run_rgb_workload(stream, form if form != "direct_lut" else "tc_bf16x3", flush)
    progress("angular spectrum")
    if rank == 0 and not args.skip_asm:
        line["asm_reconstruct"] = run_asm_workload(plan, holo, L, stream, flush)
    progress("level sweep")
    if rank == 0 and not args.skip_level_sweep:
        line["level_sweep"] = run_level_sweep(plan, coeffs, lists, counts, I, L, stream, form, flush)
    # the other superposition forms on the same scene (device ms of the superposition call)
    others, others_h = {}, {}
    for f in ("direct_lut", "tc_bf16x3", "tc_fp16x3", "tc_fp16x2"):
        if f == form or args.skip_forms:
            continue
        fe = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        with torch.cuda.stream(stream):
            plan.progressive_hologram(coeffs, lists, counts, holo=holo, form=f, stream=stream)
            flush.fill_(0.0)
            fe[0].record(stream)
            plan.progressive_hologram(coeffs, lists, counts, holo=holo, form=f, stream=stream)
            fe[1].record(stream)
        torch.cuda.synchronize()
        others[f] = fe[0].elapsed_time(fe[1])
        others_h[f] = holo.cpu().numpy()
    if others:
        line["other_forms_superposition_ms"] = others
    if fast is not None:
        line["fp16x2_step"] = fast
    progress("cpu baseline")
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cb, Href = cpu_baseline()
        line["cpu_baseline"] = cb
        from oracle import cgh_oracle as O
        # the hologram buffer holds the accumulated kernel-timing runs: recompute one step
        with torch.cuda.stream(stream):
            step()
        stream.synchronize()
        Hg = holo.cpu().numpy()
        line["accuracy"] = {"rel_l2_vs_fp64_oracle": O.rel_l2(Hg, Href),
                            "max_abs_vs_fp64_oracle": float(np.max(np.abs(Hg - Href))),
                            "max_abs_reference": float(np.max(np.abs(Href))),
                            "per_layer": per_layer_accuracy(plan, sc, coeffs, lists, counts, form, stream)}
        if others_h:
            line["other_forms_rel_l2_vs_fp64_oracle"] = {f: O.rel_l2(h, Href) for f, h in others_h.items()}
    if rank == 0:
        print(json.dumps(line), flush=True)
    plan.close()
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def per_layer_accuracy(plan, sc, coeffs, lists, counts, form, stream):
    """Each layer's hologram alone (the step's lists restricted to one layer) against the
    oracle's: rel-L2 and max-abs per layer."""
    import numpy as np
    import torch
    from oracle import cgh_oracle as O
    g = O.geometry_of(sc)
    c = counts.cpu().numpy()
    host = [lists[k][:int(c[k, 0])].cpu().numpy() for k in range(4)]
    rel, mabs = [], []
    for z in range(g.n_layers):
        sel = [x[(x >> 24) == z] for x in host]
        dev_lists = [torch.from_numpy(np.ascontiguousarray(x) if len(x) else np.zeros(1, np.int32)).cuda()
                     for x in sel]
        cnt = torch.tensor([[len(x), len(x)] for x in sel], dtype=torch.int32, device="cuda")
        with torch.cuda.stream(stream):
            Hz = plan.progressive_hologram(coeffs, dev_lists, cnt, form=form, stream=stream)
        stream.synchronize()
        Hz = Hz.cpu().numpy()
        Hr = O.progressive_hologram(sc["intensity"], sc["layer"], sel, g)
        rel.append(O.rel_l2(Hz, Hr))
        mabs.append(float(np.max(np.abs(Hz - Hr))))
    return {"rel_l2_max": max(rel), "rel_l2": rel, "max_abs": mabs,
            "note": "each layer's hologram alone (lists restricted to the layer) against the FP64 oracle's"}


def main():
    import faulthandler
    # should a phase ever stall, say where (stderr, every 4 minutes); the JSON line is unaffected
    faulthandler.dump_traceback_later(240, repeat=True, file=sys.stderr)
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--form", default="tc_fp16x3", choices=["direct_lut", "tc_bf16x3", "tc_fp16x3"])
    ap.add_argument("--skip-forms", action="store_true")
    ap.add_argument("--no-graph", action="store_true", help="launch the step eagerly instead of as a CUDA graph")
    ap.add_argument("--skip-batch", action="store_true", help="skip the 64-scene batch measurement")
    ap.add_argument("--batch-scenes", type=int, default=64)
    ap.add_argument("--skip-phase-opt", action="store_true", help="skip the phase-optimisation measurement")
    ap.add_argument("--phase-opt-steps", type=int, default=199,
                    help="timed Adam steps after the first (199: the 200-step loop of the optimisation workload)")
    ap.add_argument("--skip-plain", action="store_true")
    ap.add_argument("--skip-level-sweep", action="store_true")
    ap.add_argument("--skip-asm", action="store_true", help="skip the angular-spectrum reconstruction timing")
    ap.add_argument("--skip-rgb", action="store_true", help="skip the three-channel colour frame timing")
    ap.add_argument("--skip-hbm-paths", action="store_true", help="skip the DWT and selection at an 8192^2 object")
    ap.add_argument("--steady-steps", type=int, default=5000,
                    help="captured steps of the steady-state run (0: skip)")
    ap.add_argument("--skip-precision", action="store_true",
                    help="skip the 2048^2-hologram, 32-layer precision workload")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
