"""Seeded synthetic scenes for saliency-progressive CGH.

These generators stand in for the paper's ECSSD sample objects (Section 3) and
its PoolNet saliency maps (Section 1, Fig. 3), neither of which exists here.
They draw random numbers only: no hologram, wavelet or selection arithmetic
lives in this module, so the CPU oracle and the CUDA path can both be fed from
it without sharing any of the method's code.

A scene is a dict with
  intensity  uint8 [obj_h, obj_w]   object intensity (the point amplitudes)
  layer      uint8 [obj_h, obj_w]   depth-layer index of every object point
  saliency   uint8 [obj_h, obj_w]   0..255 saliency map (255 = most salient)
  z          float64 [n_layers]     distance of each depth layer (metres)
  holo       (holo_h, holo_w)       hologram size in pixels
  pitch, wavelength                 metres
Seeds follow the rule seed = 1000 * config_index + scene_index.
"""
import numpy as np

PITCH = 8e-6
WAVELENGTH = 532e-9


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _blobs(rng, n, count, sigma_lo, sigma_hi, peak_lo, peak_hi):
    yy, xx = np.mgrid[0:n, 0:n].astype(np.float64)
    img = np.zeros((n, n))
    for _ in range(count):
        cy, cx = rng.uniform(0.15, 0.85, size=2) * n
        sig = rng.uniform(sigma_lo, sigma_hi) * n
        peak = rng.uniform(peak_lo, peak_hi)
        img += peak * np.exp(-((yy - cy) ** 2 + (xx - cx) ** 2) / (2.0 * sig * sig))
    return img


def _depth_layers(rng, n, n_layers):
    """Smooth depth field from 3 broad blobs, normalised to [0,1], quantised."""
    field = _blobs(rng, n, 3, 0.20, 0.40, 0.5, 1.0)
    lo, hi = field.min(), field.max()
    d = (field - lo) / (hi - lo) if hi > lo else np.zeros_like(field)
    return np.clip(np.floor(d * n_layers), 0, n_layers - 1).astype(np.uint8)


def _ellipse(n, cy, cx, ay, ax, theta=0.0):
    yy, xx = np.mgrid[0:n, 0:n].astype(np.float64)
    yy = yy + 0.5 - cy
    xx = xx + 0.5 - cx
    c, s = np.cos(theta), np.sin(theta)
    u = c * xx + s * yy
    v = -s * xx + c * yy
    return (u / ax) ** 2 + (v / ay) ** 2 <= 1.0


def centred_ellipse_saliency(n, area_fraction):
    """255 inside a centred ellipse of the given area fraction, 0 outside."""
    a = 0.32 * n
    b = area_fraction * n * n / (np.pi * a)
    if b > 0.5 * n:  # keep the ellipse inside the frame for large fractions
        b = 0.5 * n
        a = area_fraction * n * n / (np.pi * b)
    m = _ellipse(n, n / 2.0, n / 2.0, b, a)
    return (m * 255).astype(np.uint8)


def union_ellipses_saliency(rng, n, k=3, lo=0.20, hi=0.35, max_tries=1000):
    """Union of k seeded ellipses, rejection-sampled until its area is in [lo, hi]."""
    for _ in range(max_tries):
        m = np.zeros((n, n), bool)
        for _ in range(k):
            cy, cx = rng.uniform(0.2, 0.8, size=2) * n
            ay, ax = rng.uniform(0.08, 0.30, size=2) * n
            m |= _ellipse(n, cy, cx, ay, ax, rng.uniform(0, np.pi))
        frac = m.mean()
        if lo <= frac <= hi:
            return (m * 255).astype(np.uint8)
    raise RuntimeError("saliency rejection sampling did not converge")


def graded_saliency(rng, n):
    """Smooth 0..255 saliency (for threshold tests; not a benchmark config)."""
    f = _blobs(rng, n, 4, 0.08, 0.25, 0.3, 1.0)
    f = f / f.max()
    return np.clip(np.round(f * 255), 0, 255).astype(np.uint8)


def tiny_scene(seed=1000, n=64, holo=256, n_layers=4):
    """64x64 object, 4 layers at 0.10..0.13 m, 25% ellipse saliency, 256^2 hologram."""
    rng = _rng(seed)
    img = rng.uniform(0.0, 40.0, size=(n, n)) + _blobs(rng, n, 6, 0.04, 0.12, 120, 215)
    intensity = np.clip(np.round(img), 0, 255).astype(np.uint8)
    layer = _depth_layers(rng, n, n_layers)
    sal = centred_ellipse_saliency(n, 0.25)
    z = np.array([0.10, 0.11, 0.12, 0.13][:n_layers] if n_layers <= 4 else
                 np.linspace(0.10, 0.13, n_layers), dtype=np.float64)
    return dict(intensity=intensity, layer=layer, saliency=sal, z=z,
                holo=(holo, holo), pitch=PITCH, wavelength=WAVELENGTH)


def paper_scene(seed=2000, n=512, holo=1024, n_layers=16):
    """Paper-scale scene: blobs plus 8 hard-edged rectangles, 16 layers in [0.08, 0.20] m,
    saliency = union of 3 ellipses covering 20-35% of the object."""
    rng = _rng(seed)
    img = rng.uniform(0.0, 40.0, size=(n, n)) + _blobs(rng, n, 6, 0.04, 0.12, 120, 215)
    for _ in range(8):
        h, w = rng.integers(n // 16, n // 4, size=2)
        y0 = rng.integers(0, n - h)
        x0 = rng.integers(0, n - w)
        img[y0:y0 + h, x0:x0 + w] = rng.uniform(60, 255)
    intensity = np.clip(np.round(img), 0, 255).astype(np.uint8)
    layer = _depth_layers(rng, n, n_layers)
    sal = union_ellipses_saliency(rng, n)
    z = np.linspace(0.08, 0.20, n_layers)
    return dict(intensity=intensity, layer=layer, saliency=sal, z=z,
                holo=(holo, holo), pitch=PITCH, wavelength=WAVELENGTH)


def random_scene(seed, n, holo, n_layers, sal_fraction=None, graded=False):
    """Generic seeded scene of any size (tests and the batched workload)."""
    rng = _rng(seed)
    img = rng.uniform(0.0, 40.0, size=(n, n)) + _blobs(rng, n, 6, 0.04, 0.12, 120, 215)
    intensity = np.clip(np.round(img), 0, 255).astype(np.uint8)
    layer = _depth_layers(rng, n, n_layers)
    if graded:
        sal = graded_saliency(rng, n)
    else:
        frac = 0.25 if sal_fraction is None else sal_fraction
        sal = centred_ellipse_saliency(n, frac)
    z = np.linspace(0.08, 0.20, n_layers) if n_layers > 1 else np.array([0.10])
    return dict(intensity=intensity, layer=layer, saliency=sal, z=z,
                holo=(holo, holo), pitch=PITCH, wavelength=WAVELENGTH)


def depth_map(seed, n, z_lo=0.08, z_hi=0.20, holes=0.0):
    """Continuous per-pixel depth (float32 metres) for the per-point-depth path: a smooth
    field from 3 broad blobs scaled to [z_lo, z_hi] plus a small seeded jitter; a fraction
    `holes` of pixels gets no depth (NaN, 0 or negative) at random."""
    rng = _rng(seed)
    f = _blobs(rng, n, 3, 0.20, 0.40, 0.5, 1.0)
    lo, hi = f.min(), f.max()
    d = (f - lo) / (hi - lo) if hi > lo else np.zeros_like(f)
    z = z_lo + (z_hi - z_lo) * np.clip(d + rng.normal(0.0, 0.01, size=d.shape), 0.0, 1.0)
    z = z.astype(np.float32)
    if holes > 0:
        pick = rng.uniform(size=z.shape) < holes
        kind = rng.integers(0, 3, size=z.shape)
        z[pick & (kind == 0)] = np.nan
        z[pick & (kind == 1)] = 0.0
        z[pick & (kind == 2)] = -0.05
    return z


def rgb_scene(seed, n, holo, n_layers):
    """Colour scene: a random_scene whose intensity becomes three correlated channels
    (uint8 [3, n, n], R G B): the grey image scaled by seeded per-channel gains plus
    per-channel blobs and noise; layers and saliency are shared by the channels."""
    sc = random_scene(seed, n, holo, n_layers)
    rng = _rng(seed + 1)
    base = sc["intensity"].astype(np.float64)
    chans = []
    for _ in range(3):
        g = rng.uniform(0.5, 1.0)
        img = g * base + _blobs(rng, n, 3, 0.05, 0.15, 20, 80) + rng.normal(0.0, 4.0, size=base.shape)
        chans.append(np.clip(np.round(img), 0, 255).astype(np.uint8))
    sc["intensity"] = np.stack(chans)
    return sc


def batch_scenes(seed=4000, count=64):
    """Batched workload: uneven object edges from {128,256,512,1024}, hologram 2x,
    4..32 layers each, ellipse saliency with area fraction U[0.05, 0.6]."""
    rng = _rng(seed)
    out = []
    for k in range(count):
        n = int(rng.choice([128, 256, 512, 1024]))
        zl = int(rng.integers(4, 33))
        frac = float(rng.uniform(0.05, 0.6))
        out.append(random_scene(seed + 1 + k, n, 2 * n, zl, sal_fraction=frac))
    return out


THRESHOLDS_U8 = {3: 127, 2: 178, 1: 229}
"""Per-level saliency thresholds on the uint8 scale: floor(255 * t) for
t = 0.5 (level-3 details), 0.7 (level 2), 0.9 (level 1); the coarse LLL band
takes every occupied block (Section 3 threshold values, Section 2 steps 2-5)."""
