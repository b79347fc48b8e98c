"""Colour holograms: the three colour channels of one scene, each a saliency-progressive
hologram at its own wavelength (the paper computes a single colour channel, Section 3; the
method applies per channel unchanged, with the channel's wavelength in the fringe rate
a_z = p^2 / (2 lambda z) of Eq. 1).

The channels share the object geometry, the depth layers and the saliency map; each has
its own plan (fringe tables and operand planes depend on lambda).  The three channels run
as one cgh_batch, so each GEMM stage is one persistent launch across the channels."""
from .cgh import Batch, Plan

# Red, green and blue laser lines (metres); any three wavelengths may be given instead.
WAVELENGTHS_RGB = (638e-9, 532e-9, 450e-9)


class RGBHologram:
    """Three-channel progressive hologram bound to device buffers.

    intensity_rgb: three uint8 [obj_h, obj_w] CUDA tensors (R, G, B); layer, saliency:
    uint8 [obj_h, obj_w] CUDA tensors shared by the channels; holos: three complex64
    [holo_h, holo_w] CUDA tensors (outputs).  run() enqueues all three holograms."""

    def __init__(self, obj_shape, holo_shape, pitch, z, intensity_rgb, layer, saliency, thresholds, holos,
                 wavelengths=WAVELENGTHS_RGB, form="tc_fp16x3", stream=None, flags=0):
        if len(intensity_rgb) != 3 or len(holos) != 3 or len(wavelengths) != 3:
            raise ValueError("three channels expected")
        self.wavelengths = tuple(float(w) for w in wavelengths)
        self.plans = [Plan(obj_shape, holo_shape, pitch, lam, z, stream=stream, flags=flags)
                      for lam in self.wavelengths]
        self.holos = list(holos)
        self.batch = Batch(self.plans, list(intensity_rgb), [layer] * 3, [saliency] * 3, thresholds,
                           self.holos, form=form, stream=stream)

    def run(self, stream=None):
        self.batch.run(stream)
        return self.holos

    def reconstruct(self, layer, stream=None):
        """Per-channel composite amplitude [3 x (obj_h, obj_w)] of the current holograms
        (Fresnel back-propagation at each channel's wavelength)."""
        return [p.reconstruct(h, layer, fields=False, stream=stream)[1] for p, h in zip(self.plans, self.holos)]

    def close(self):
        self.batch.close()
        for p in self.plans:
            p.close()
