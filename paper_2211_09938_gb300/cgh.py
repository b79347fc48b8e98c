"""Thin ctypes binding of libcgh (include/cgh.h).

Argument marshalling only: every step of the hologram path runs in the CUDA
kernels of libcgh.so.  There is no CPU fallback; if the library is missing or no
GPU is usable, calls raise CghError.

Two layers:
* the raw C functions under their C names (``lib().cgh_plan_create`` ...), for
  callers that hold raw device pointers;
* ``Plan``, which owns a cgh_plan and takes torch CUDA tensors (PyTorch is used
  for device memory and streams only).
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcgh.so")

CGH_OK = 0
CGH_ERR_ARG = 1
CGH_ERR_CUDA = 2
CGH_ERR_UNSUPPORTED = 3
CGH_ERR_TIMEOUT = 4
CGH_ERR_NOMEM = 5

FORM_DIRECT_LUT = 0
FORM_TC_BF16X3 = 1
FORM_TC_FP16X3 = 2
FORM_TC_FP16X2 = 3
FORMS = {"direct_lut": FORM_DIRECT_LUT, "tc_bf16x3": FORM_TC_BF16X3, "tc_fp16x3": FORM_TC_FP16X3,
         "tc_fp16x2": FORM_TC_FP16X2}

# Every symbol include/cgh.h declares, with (restype, argtypes).
_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
SIGNATURES = {
    "cgh_last_error": (ctypes.c_char_p, []),
    "cgh_version": (_I, []),
    "cgh_plan_create": (_I, [ctypes.POINTER(_P), _I, _I, _I, _I, _D, _D, _I,
                             ctypes.POINTER(_D), _I, _I, _P]),
    "cgh_plan_destroy": (_I, [_P]),
    "cgh_plan_set_tuning": (_I, [_P, _I]),
    "cgh_plan_set_stage2_tiles": (_I, [_P, _I]),
    "cgh_plan_stage2_tiles_used": (_I, [_P, _P]),
    "cgh_plan_set_fusion": (_I, [_P, _I]),
    "cgh_plan_set_contraction": (_I, [_P, _I]),
    "cgh_build_tables": (_I, [_P, _P]),
    "cgh_haar_decompose": (_I, [_P, _P, _P, _P, _P]),
    "cgh_select_blocks": (_I, [_P, _P, _P, _I, _I, _P, _P, _I, _P]),
    "cgh_select_blocks_noalloc": (_I, [_P, _P, _I, _I, _I, _I, _I, _P, _P, _I, _P]),
    "cgh_select_progressive": (_I, [_P, _P, _P, ctypes.POINTER(_I), ctypes.POINTER(_P),
                                    ctypes.POINTER(_I), _P, _P]),
    "cgh_progressive_hologram": (_I, [_P, _P, ctypes.POINTER(_P), _P, _P, _I, _I, _P]),
    "cgh_progressive_step": (_I, [_P, _P, _P, _P, _P, ctypes.POINTER(_I), ctypes.POINTER(_P),
                                  ctypes.POINTER(_I), _P, _P, _I, _I, _P]),
    "cgh_plain_direct": (_I, [_P, _P, _P, _P, _P]),
    "cgh_pointcloud_direct": (_I, [_P, _P, _P, _P, _I, _P]),
    "cgh_reconstruct": (_I, [_P, _P, _P, _P, _P, _P]),
    "cgh_reconstruct_asm": (_I, [_P, _P, _P, _P, _P, _I, _I, _P]),
    "cgh_propagate": (_I, [_P, _P, _P, _I, _P]),
    "cgh_adjoint": (_I, [_P, _P, ctypes.POINTER(_P), _P, _P, _P, _P]),
    "cgh_progressive_apply": (_I, [_P, _P, ctypes.POINTER(_P), _P, _P, _P, _I, _P]),
    "cgh_amplitude_backward": (_I, [_P, _P, _P, _P, _P, _P]),
    "cgh_reconstruct_batch": (_I, [_P, _P, _I, _P, _P, _P, _P]),
    "cgh_propagate_batch": (_I, [_P, _P, _I, _P, _I, _P]),
    "cgh_amplitude_backward_batch": (_I, [_P, _P, _I, _P, _P, _P, _P]),
    "cgh_phase_to_field": (_I, [_P, _P, ctypes.c_longlong, _P]),
    "cgh_phase_grad": (_I, [_P, _P, _P, ctypes.c_longlong, _P]),
    "cgh_ssim": (_I, [_P, _P, _I, _I, _I, _P, _P, _P]),
    "cgh_status": (_I, [_P, ctypes.POINTER(_I), _P]),
    "cgh_selftest_timeout": (_I, [_P, _I, _P]),
    "cgh_selftest_grid_barrier": (_I, [_P, _I, _I, _I, _P, _P]),
    "cgh_probe_sfu": (_I, [_P, _I, ctypes.c_longlong, _P]),
    "cgh_probe_ffma": (_I, [_P, _I, ctypes.c_longlong, _P]),
    "cgh_tc_selftest_gemm": (_I, [_P, _P, _P, _I, _I, _I, _I, _P]),
    "cgh_batch_create": (_I, [ctypes.POINTER(_P), ctypes.POINTER(_P), _I, ctypes.POINTER(_P),
                              ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_I),
                              ctypes.POINTER(_P), _I, _P]),
    "cgh_batch_run": (_I, [_P, _P]),
    "cgh_batch_set_stage2_tiles": (_I, [_P, _I]),
    "cgh_batch_set_tuning": (_I, [_P, _I]),
    "cgh_batch_lists": (_I, [_P, _I, ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_P)]),
    "cgh_batch_destroy": (_I, [_P]),
    "cgh_profile": (_I, [_P, _I]),
    "cgh_profile_read": (_I, [_P, ctypes.POINTER(ctypes.c_float), _P]),
    "cgh_tc_layer_dims": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(_I), _P]),
}

_lib = None


class CghError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libcgh error {code}: {msg}")
        self.code = code


def lib():
    """Load libcgh.so (built in-tree by __graft_entry__.build()); raise if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise CghError(CGH_ERR_CUDA, f"{LIB_PATH} is not built; run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def check(rc):
    if rc != CGH_OK:
        raise CghError(rc, lib().cgh_last_error().decode(errors="replace"))


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Plan:
    """A cgh_plan for one scene geometry.  Tensors passed in must be contiguous CUDA
    tensors of the dtypes include/cgh.h states; outputs are allocated by the caller or
    by the convenience helpers below (torch.empty on the plan's device)."""

    DETERMINISTIC = 1
    LAYER_FACTOR = 2  # keep exp(jkz)/z of Eq. 1 per layer (cgh.h: CGH_PLAN_LAYER_FACTOR)

    def __init__(self, obj_shape, holo_shape, pitch, wavelength, z, levels=3, stream=None, flags=0):
        import torch
        self.obj_h, self.obj_w = int(obj_shape[0]), int(obj_shape[1])
        self.holo_h, self.holo_w = int(holo_shape[0]), int(holo_shape[1])
        self.pitch, self.wavelength, self.levels, self.flags = float(pitch), float(wavelength), int(levels), int(flags)
        self.z = [float(v) for v in z]
        self.n_layers = len(self.z)
        self.device = torch.device("cuda", torch.cuda.current_device())
        zs = (ctypes.c_double * self.n_layers)(*self.z)
        h = ctypes.c_void_p()
        check(lib().cgh_plan_create(ctypes.byref(h), self.obj_h, self.obj_w, self.holo_h, self.holo_w,
                                    float(pitch), float(wavelength), self.n_layers, zs, levels, int(flags),
                                    _stream(stream)))
        self.handle = h

    @classmethod
    def for_scene(cls, scene, stream=None, flags=0):
        if scene.get("layer_factor", False):
            flags |= cls.LAYER_FACTOR
        return cls(scene["intensity"].shape[-2:], scene["holo"], scene["pitch"], scene["wavelength"],
                   scene["z"], stream=stream, flags=flags)

    def clone(self, stream=None):
        """A new plan of the same geometry and flags, with its own scratch (so that two scenes
        can be in flight at once, one per plan)."""
        return Plan((self.obj_h, self.obj_w), (self.holo_h, self.holo_w), self.pitch, self.wavelength, self.z,
                    levels=self.levels, stream=stream, flags=self.flags)

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            lib().cgh_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- C calls -------------------------------------------------------------------
    CONTRACT_AUTO, CONTRACT_ROWS, CONTRACT_COLS = 0, 1, 2

    def set_contraction(self, order):
        """Contraction order of the tensor form (cgh_plan_set_contraction): CONTRACT_AUTO,
        CONTRACT_ROWS or CONTRACT_COLS."""
        check(lib().cgh_plan_set_contraction(self.handle, int(order)))

    TILES_AUTO, TILES_CTA, TILES_PAIR = 0, 1, 2

    def set_stage2_tiles(self, tiles):
        """cgh_plan_set_stage2_tiles: TILES_AUTO, TILES_CTA (128x128 per CTA) or TILES_PAIR
        (256x128 per CTA pair, tcgen05 cta_group::2)."""
        check(lib().cgh_plan_set_stage2_tiles(self.handle, int(tiles)))

    def stage2_tiles_used(self):
        """cgh_plan_stage2_tiles_used: TILES_CTA or TILES_PAIR, the tile shape of the last
        two-launch separable call's stage 2 (TILES_AUTO before any)."""
        v = ctypes.c_int(0)
        check(lib().cgh_plan_stage2_tiles_used(self.handle, ctypes.byref(v)))
        return v.value

    def set_fusion(self, fused):
        """cgh_plan_set_fusion: both GEMM stages in one cooperative launch (True) or two
        launches (False, default)."""
        check(lib().cgh_plan_set_fusion(self.handle, 1 if fused else 0))

    def set_tuning(self, max_ksteps_per_chain):
        check(lib().cgh_plan_set_tuning(self.handle, int(max_ksteps_per_chain)))

    def build_tables(self, stream=None):
        check(lib().cgh_build_tables(self.handle, _stream(stream)))

    def haar_decompose(self, intensity, layer, coeffs=None, stream=None):
        import torch
        if coeffs is None:
            coeffs = torch.empty((self.n_layers, self.obj_h, self.obj_w), dtype=torch.int32,
                                 device=self.device)
        check(lib().cgh_haar_decompose(self.handle, _ptr(intensity), _ptr(layer), _ptr(coeffs),
                                       _stream(stream)))
        return coeffs

    def max_blocks(self, level):
        return self.n_layers * (self.obj_h >> level) * (self.obj_w >> level)

    def select_blocks(self, saliency, layer, threshold, level, out=None, count=None,
                      capacity=None, stream=None):
        import torch
        if capacity is None:
            capacity = self.max_blocks(level) if out is None else out.numel()
        if out is None:
            out = torch.empty(max(capacity, 1), dtype=torch.int32, device=self.device)
        if count is None:
            count = torch.empty(2, dtype=torch.int32, device=self.device)
        check(lib().cgh_select_blocks(self.handle, _ptr(saliency), _ptr(layer), int(threshold),
                                      int(level), _ptr(out), _ptr(count), int(capacity),
                                      _stream(stream)))
        return out, count

    def progressive_lists(self, saliency, layer, thresholds, counts=None, lists=None, stream=None):
        """The four work lists [LLL, level 1, level 2, level 3] and their int32[4][2]
        counts (cgh_select_progressive); thresholds maps level -> uint8 threshold."""
        import torch
        if counts is None:
            counts = torch.zeros((4, 2), dtype=torch.int32, device=self.device)
        if lists is None:
            lists = [torch.empty(self.max_blocks(3 if k == 0 else k), dtype=torch.int32,
                                 device=self.device) for k in range(4)]
        thr = (ctypes.c_int * 3)(*[int(thresholds[l]) for l in (1, 2, 3)])
        ptrs = (ctypes.c_void_p * 4)(*[l.data_ptr() for l in lists])
        caps = (ctypes.c_int * 4)(*[l.numel() for l in lists])
        check(lib().cgh_select_progressive(self.handle, _ptr(saliency), _ptr(layer), thr, ptrs, caps,
                                           _ptr(counts), _stream(stream)))
        return lists, counts

    LEVEL_STAGES = ("LLL", "LL", "L", "object")
    _STAGE_LISTS = ((0,), (0, 3), (0, 3, 2), (0, 3, 2, 1))

    @classmethod
    def level_counts(cls, counts, stage):
        """Counts for the cumulative hologram at one stage of the progression of Section 2
        (steps 2-5): 0 = LLL blocks only, 1 = + level-3 residuals (LL), 2 = + level 2 (L),
        3 = + level 1 (object level, the full progressive hologram).  Lists left out get
        zero counts; the lists themselves are not touched."""
        c = counts.clone()
        for k in range(4):
            if k not in cls._STAGE_LISTS[stage]:
                c[k].zero_()
        return c

    @staticmethod
    def operator_count(counts):
        """Section 3's operator count of the lists whose device counts are given: one LUT
        block multiplied, shifted and added per LLL block, and one per residual-map cell,
        i.e. four per selected detail block (the one-level inverse DWT of a selected block
        is a 2x2 grid of cells).  Reads the counts back to the host."""
        n = [int(v) for v in counts[:, 0].cpu().tolist()]
        return n[0] + 4 * sum(n[1:])

    def progressive_hologram(self, coeffs, lists, counts, holo=None, accumulate=False,
                             form="direct_lut", stream=None):
        import torch
        if holo is None:
            holo = torch.empty((self.holo_h, self.holo_w), dtype=torch.complex64, device=self.device)
        arr = (ctypes.c_void_p * 4)(*[l.data_ptr() for l in lists])
        f = FORMS[form] if isinstance(form, str) else int(form)
        check(lib().cgh_progressive_hologram(self.handle, _ptr(coeffs), arr, _ptr(counts), _ptr(holo),
                                             1 if accumulate else 0, f, _stream(stream)))
        return holo

    def progressive_step(self, saliency, layer, coeffs, thresholds, counts=None, lists=None, holo=None,
                         accumulate=False, form="tc_fp16x3", coeffs_ready=None, stream=None):
        """Selection and superposition in one call (cgh_progressive_step): the outputs of
        progressive_lists followed by progressive_hologram.  coeffs_ready: a torch.cuda.Event
        the call waits for after the selection, before it reads coeffs (a DWT on another
        stream then overlaps the selection).  Returns (holo, lists, counts)."""
        import torch
        if counts is None:
            counts = torch.zeros((4, 2), dtype=torch.int32, device=self.device)
        if lists is None:
            lists = [torch.empty(self.max_blocks(3 if k == 0 else k), dtype=torch.int32,
                                 device=self.device) for k in range(4)]
        if holo is None:
            holo = torch.empty((self.holo_h, self.holo_w), dtype=torch.complex64, device=self.device)
        thr = (ctypes.c_int * 3)(*[int(thresholds[l]) for l in (1, 2, 3)])
        ptrs = (ctypes.c_void_p * 4)(*[l.data_ptr() for l in lists])
        caps = (ctypes.c_int * 4)(*[l.numel() for l in lists])
        f = FORMS[form] if isinstance(form, str) else int(form)
        ev = None if coeffs_ready is None else ctypes.c_void_p(coeffs_ready.cuda_event)
        check(lib().cgh_progressive_step(self.handle, _ptr(saliency), _ptr(layer), _ptr(coeffs), ev, thr, ptrs,
                                         caps, _ptr(counts), _ptr(holo), 1 if accumulate else 0, f,
                                         _stream(stream)))
        return holo, lists, counts

    def plain_direct(self, intensity, layer, holo=None, stream=None):
        import torch
        if holo is None:
            holo = torch.empty((self.holo_h, self.holo_w), dtype=torch.complex64, device=self.device)
        check(lib().cgh_plain_direct(self.handle, _ptr(intensity), _ptr(layer), _ptr(holo),
                                     _stream(stream)))
        return holo

    def pointcloud_direct(self, intensity, depth, holo=None, accumulate=False, stream=None):
        """Point-wise hologram with a depth (float32 metres) per object pixel
        (cgh_pointcloud_direct); pixels with depth <= 0 or non-finite are no point."""
        import torch
        if holo is None:
            holo = torch.empty((self.holo_h, self.holo_w), dtype=torch.complex64, device=self.device)
        check(lib().cgh_pointcloud_direct(self.handle, _ptr(intensity), _ptr(depth), _ptr(holo),
                                          1 if accumulate else 0, _stream(stream)))
        return holo

    def reconstruct(self, holo, layer=None, fields=True, amplitude=True, stream=None):
        """(fields [Z, obj, obj] complex64 or None, amplitude [obj, obj] float32 or None).
        `fields` / `amplitude` may also be preallocated tensors."""
        import torch
        if fields is True:
            fields = torch.empty((self.n_layers, self.obj_h, self.obj_w), dtype=torch.complex64,
                                 device=self.device)
        if amplitude is True:
            amplitude = torch.empty((self.obj_h, self.obj_w), dtype=torch.float32, device=self.device)
        f = fields if fields is not False else None
        a = amplitude if amplitude is not False else None
        check(lib().cgh_reconstruct(self.handle, _ptr(holo), _ptr(f), _ptr(layer), _ptr(a),
                                    _stream(stream)))
        return f, a

    def reconstruct_asm(self, holo, layer=None, fields=True, amplitude=True, pad=2, band_limit=False,
                        stream=None):
        """Inverse angular-spectrum reconstruction (cgh_reconstruct_asm): (fields [Z, obj, obj]
        complex64 or None, amplitude [obj, obj] float32 or None)."""
        import torch
        if fields is True:
            fields = torch.empty((self.n_layers, self.obj_h, self.obj_w), dtype=torch.complex64,
                                 device=self.device)
        if amplitude is True:
            amplitude = torch.empty((self.obj_h, self.obj_w), dtype=torch.float32, device=self.device)
        f = fields if fields is not False else None
        a = amplitude if amplitude is not False else None
        check(lib().cgh_reconstruct_asm(self.handle, _ptr(holo), _ptr(f), _ptr(layer), _ptr(a), int(pad),
                                        1 if band_limit else 0, _stream(stream)))
        return f, a

    def reconstruct_batch(self, holos, layer=None, fields=True, amplitude=True, stream=None):
        """cgh_reconstruct_batch: holos [n, holo, holo] complex64 -> (fields [n, Z, obj, obj]
        complex64 or None, amplitude [n, obj, obj] float32 or None)."""
        import torch
        n = holos.shape[0]
        if fields is True:
            fields = torch.empty((n, self.n_layers, self.obj_h, self.obj_w), dtype=torch.complex64,
                                 device=self.device)
        if amplitude is True:
            amplitude = torch.empty((n, self.obj_h, self.obj_w), dtype=torch.float32, device=self.device)
        f = fields if fields is not False else None
        a = amplitude if amplitude is not False else None
        check(lib().cgh_reconstruct_batch(self.handle, _ptr(holos), int(n), _ptr(f), _ptr(layer), _ptr(a),
                                          _stream(stream)))
        return f, a

    def propagate_batch(self, fields, holos=None, accumulate=False, stream=None):
        """cgh_propagate_batch: fields [n, Z, obj, obj] complex64 -> holos [n, holo, holo]."""
        import torch
        n = fields.shape[0]
        if holos is None:
            holos = torch.empty((n, self.holo_h, self.holo_w), dtype=torch.complex64, device=self.device)
        check(lib().cgh_propagate_batch(self.handle, _ptr(fields), int(n), _ptr(holos), 1 if accumulate else 0,
                                        _stream(stream)))
        return holos

    def amplitude_backward_batch(self, fields, layer, grad_amp, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty_like(fields)
        check(lib().cgh_amplitude_backward_batch(self.handle, _ptr(fields), int(fields.shape[0]), _ptr(layer),
                                                 _ptr(grad_amp), _ptr(out), _stream(stream)))
        return out

    def propagate(self, fields, holo=None, accumulate=False, stream=None):
        import torch
        if holo is None:
            holo = torch.empty((self.holo_h, self.holo_w), dtype=torch.complex64, device=self.device)
        check(lib().cgh_propagate(self.handle, _ptr(fields), _ptr(holo), 1 if accumulate else 0,
                                  _stream(stream)))
        return holo

    def adjoint(self, grad_holo, lists, counts, layer, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty((self.obj_h, self.obj_w), dtype=torch.float32, device=self.device)
        arr = (ctypes.c_void_p * 4)(*[l.data_ptr() for l in lists])
        check(lib().cgh_adjoint(self.handle, _ptr(grad_holo), arr, _ptr(counts), _ptr(layer), _ptr(out),
                                _stream(stream)))
        return out

    def progressive_apply(self, obj, lists, counts, layer, holo=None, accumulate=False, stream=None):
        """cgh_progressive_apply: the progressive operator on a real (float32) object; the
        linear map whose adjoint is `adjoint`."""
        import torch
        if holo is None:
            holo = torch.empty((self.holo_h, self.holo_w), dtype=torch.complex64, device=self.device)
        arr = (ctypes.c_void_p * 4)(*[l.data_ptr() for l in lists])
        check(lib().cgh_progressive_apply(self.handle, _ptr(obj), arr, _ptr(counts), _ptr(layer), _ptr(holo),
                                          1 if accumulate else 0, _stream(stream)))
        return holo

    def amplitude_backward(self, fields, layer, grad_amp, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty_like(fields)
        check(lib().cgh_amplitude_backward(self.handle, _ptr(fields), _ptr(layer), _ptr(grad_amp),
                                           _ptr(out), _stream(stream)))
        return out

    PROF_SLOTS = ["tables", "haar", "select", "direct_lut", "tc_prep", "tc_stage1", "tc_stage2",
                  "plain", "recon", "propagate", "asm_fft", "asm_inv", "pointcloud", "tc_fused"]

    def profile(self, enable=True):
        check(lib().cgh_profile(self.handle, 1 if enable else 0))

    def profile_read(self, stream=None):
        """Per-stage device ms of the most recent run of each stage (synchronises)."""
        ms = (ctypes.c_float * len(self.PROF_SLOTS))()
        check(lib().cgh_profile_read(self.handle, ms, _stream(stream)))
        return dict(zip(self.PROF_SLOTS, list(ms)))

    def tc_layer_dims(self, stream=None):
        kr = (ctypes.c_int * self.n_layers)()
        kc = (ctypes.c_int * self.n_layers)()
        check(lib().cgh_tc_layer_dims(self.handle, kr, kc, _stream(stream)))
        return list(kr), list(kc)

    def selftest_timeout(self, limit_us, stream=None):
        check(lib().cgh_selftest_timeout(self.handle, int(limit_us), _stream(stream)))

    def selftest_grid_barrier(self, ctas, absent_cta, limit_us, crossed, stream=None):
        """The selection's bounded grid barrier with `ctas` cooperative CTAs, one of them
        (absent_cta >= 0) never arriving; crossed: device int32 counter of CTAs that crossed."""
        check(lib().cgh_selftest_grid_barrier(self.handle, int(ctas), int(absent_cta), int(limit_us),
                                              _ptr(crossed), _stream(stream)))

    def status(self, stream=None):
        v = ctypes.c_int(0)
        check(lib().cgh_status(self.handle, ctypes.byref(v), _stream(stream)))
        return v.value


def tc_selftest_gemm(A, B, fp16=False, stream=None):
    """C = A @ B.T on the tcgen05 path (diagnostic); A [M,K], B [N,K] bf16/fp16 CUDA tensors."""
    import torch
    M, K = A.shape
    N = B.shape[0]
    C = torch.empty((M, N), dtype=torch.float32, device=A.device)
    check(lib().cgh_tc_selftest_gemm(_ptr(A), _ptr(B), _ptr(C), M, N, K, 1 if fp16 else 0,
                                     _stream(stream)))
    return C


def probe_peaks(iters=4096, stream=None):
    """Measured peaks of the SFU and FP32 FMA units (cgh_probe_sfu / cgh_probe_ffma), timed
    with CUDA events: {"sfu_pairs_per_s", "ffma_flops_per_s"}.  Synchronises."""
    import torch
    dev = torch.cuda.current_device()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    grid = sms * 8
    sink = torch.empty(grid * 256, dtype=torch.float32, device="cuda")
    st = stream or torch.cuda.current_stream()
    out = {}
    for name, fn, per in (("sfu_pairs_per_s", lib().cgh_probe_sfu, 8), ("ffma_flops_per_s", lib().cgh_probe_ffma, 64)):
        check(fn(_ptr(sink), grid, 64, _stream(st)))  # warm-up
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        with torch.cuda.stream(st):
            ev[0].record(st)
            check(fn(_ptr(sink), grid, int(iters), _stream(st)))
            ev[1].record(st)
        ev[1].synchronize()
        out[name] = grid * 256.0 * iters * per / (ev[0].elapsed_time(ev[1]) / 1e3)
    return out


def phase_to_field(phase, out=None, stream=None):
    """exp(j*phase) on the GPU (cgh_phase_to_field); phase float32 CUDA tensor."""
    import torch
    if out is None:
        out = torch.empty(phase.shape, dtype=torch.complex64, device=phase.device)
    check(lib().cgh_phase_to_field(_ptr(phase), _ptr(out), phase.numel(), _stream(stream)))
    return out


def phase_grad(field, grad_field, out=None, stream=None):
    """Im(grad_field * conj(field)) (cgh_phase_grad)."""
    import torch
    if out is None:
        out = torch.empty(field.shape, dtype=torch.float32, device=field.device)
    check(lib().cgh_phase_grad(_ptr(field), _ptr(grad_field), _ptr(out), field.numel(), _stream(stream)))
    return out


def ssim(x, y, normalize=True, out=None, stream=None):
    """Mean SSIM of two float32 [h, w] CUDA images (cgh_ssim); returns a device float64
    scalar tensor (read it with .item())."""
    import torch
    h, w = x.shape
    if out is None:
        out = torch.empty((), dtype=torch.float64, device=x.device)
    scratch = torch.empty(2, dtype=torch.int32, device=x.device) if normalize else None
    check(lib().cgh_ssim(_ptr(x), _ptr(y), h, w, 1 if normalize else 0, _ptr(out),
                         _ptr(scratch) if scratch is not None else None, _stream(stream)))
    return out


class Batch:
    """cgh_batch: many scenes (each with its Plan) run as one batch.  Inputs and outputs
    are bound at creation; run() enqueues every scene's hologram with one persistent
    launch per GEMM stage across all scenes."""

    def __init__(self, plans, intensity, layer, saliency, thresholds, holos, form="tc_fp16x3",
                 stream=None):
        n = len(plans)
        self.plans = list(plans)
        self._keep = (list(intensity), list(layer), list(saliency), list(holos))
        P = ctypes.c_void_p
        arr = lambda xs: (P * n)(*[x.data_ptr() for x in xs])
        thr = (ctypes.c_int * 3)(*[int(thresholds[l]) for l in (1, 2, 3)])
        h = P()
        check(lib().cgh_batch_create(ctypes.byref(h), (P * n)(*[p.handle.value for p in plans]), n,
                                     arr(intensity), arr(layer), arr(saliency), thr, arr(holos),
                                     FORMS[form] if isinstance(form, str) else int(form), _stream(stream)))
        self.handle = h
        self.holos = list(holos)

    def run(self, stream=None):
        check(lib().cgh_batch_run(self.handle, _stream(stream)))

    def set_tuning(self, ksteps_per_unit):
        check(lib().cgh_batch_set_tuning(self.handle, int(ksteps_per_unit)))

    def set_stage2_tiles(self, tiles):
        """Plan.TILES_CTA (128x128 per CTA) or Plan.TILES_PAIR (256x128 per CTA pair)."""
        check(lib().cgh_batch_set_stage2_tiles(self.handle, int(tiles)))

    def lists(self, k):
        """(lists [4] as raw device pointers, counts pointer, coeffs pointer) of scene k."""
        P = ctypes.c_void_p
        lp = (P * 4)()
        cp, kp = P(), P()
        check(lib().cgh_batch_lists(self.handle, int(k), lp, ctypes.byref(cp), ctypes.byref(kp)))
        return [lp[i] for i in range(4)], cp.value, kp.value

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            lib().cgh_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
