"""Plain FP64 CPU oracle for saliency-progressive point-source CGH.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline leg may import or run this module.  The CUDA library never calls
it and shares no code, table or constant generator with it.

What it computes (arXiv 2211.09938, "Progressive hologram generation based on
object saliency"):

* Point-source hologram, Eq. 1 (Section 2) in its paraxial (Fresnel) form: an
  object point of amplitude A at hologram-pixel coordinates (s*i, s*j) on the
  plane at distance z adds A * exp(j*pi*p^2*((m-s*i)^2 + (n-s*j)^2)/(lambda*z))
  to hologram pixel (m, n).  The 1/r amplitude and the constant exp(j*k*z)
  are dropped (a per-layer constant); the phase sign is +.  With
  a_z = p^2 / (2*lambda*z) (cycles per squared pixel offset) the fringe of one
  offset is f_z(d) = exp(j*2*pi*frac(a_z*d^2)) and the 2-D point fringe
  factorises as f_z(dm) * f_z(dn).
* Object -> three-level Haar wavelet decomposition, Eq. 2 and Section 2 step 1,
  unnormalised integer form: on every 2x2 cell [a b; c d] (rows i, columns j)
  S = a+b+c+d, X = a-b+c-d (difference along columns), Y = a+b-c-d
  (difference along rows), D = a-b-c+d; recurse on S.  Mallat layout.
* Saliency quantisation, Section 2 step 1: block maximum over 2^l x 2^l.
* Progressive superposition, Eq. 3 and Section 2 steps 2-5, in the paper's
  residual-map form: H = sum over LLL points of (LLL/64) * (8x8 block
  fringe), then for level l = 3, 2, 1 the residual map (one-level inverse
  DWT with zero low band of the details of the salient blocks) is superposed
  with 2^(l-1) x 2^(l-1) block fringes.  Block fringes are sums of point
  fringes evaluated here in FP64.
* Eq. 1's amplitude 1/r and carrier exp(jkr) are a per-layer constant for a layer;
  they are dropped by default and kept, as exp(j 2 pi frac(z/lambda)) / z per layer,
  when the geometry asks for them (layer_factor).
* Depth: every object pixel belongs to one depth layer; the per-layer object
  plane is A_z = I * [layer == z] and each plane has its own DWT and fringes
  (the per-depth extension sketched at the end of Section 2).
* Reconstruction (Section 2, last paragraph) by Fresnel back-propagation,
  i.e. the adjoint of the per-layer forward operator, or by the inverse angular
  spectrum method the paper names, and SSIM (Section 3) after Wang et al. 2004.

Readings where the paper is silent or garbled (distance term of Eq. 1, sign,
amplitude, thresholds, saliency scale, residual definition, depth handling,
sampling) are listed in the design notes of the repository; the code below
follows them.

Every function here is pinned by tests/test_oracle_pins.py against closed
forms, invariants, brute force or values the paper prints.
"""
import numpy as np

# ----------------------------------------------------------------------------
# geometry


class Geometry:
    """Object/hologram sampling (reading: object pixel (i, j) sits at hologram
    pixel (s*i, s*j) with s = holo/obj an integer; Table 1 of the paper is an
    image that is not available)."""

    def __init__(self, obj_shape, holo_shape, pitch, wavelength, z, layer_factor=False):
        self.obj_h, self.obj_w = int(obj_shape[0]), int(obj_shape[1])
        self.holo_h, self.holo_w = int(holo_shape[0]), int(holo_shape[1])
        if self.holo_h % self.obj_h or self.holo_w % self.obj_w:
            raise ValueError("hologram size must be an integer multiple of the object size")
        self.s = self.holo_h // self.obj_h
        if self.holo_w // self.obj_w != self.s:
            raise ValueError("the sampling stride must be the same along both axes")
        self.pitch = float(pitch)
        self.wavelength = float(wavelength)
        self.z = np.asarray(z, dtype=np.float64).reshape(-1)
        self.layer_factor = bool(layer_factor)

    @property
    def n_layers(self):
        return self.z.size

    def a(self, k):
        """Fresnel rate a_z = p^2 / (2 lambda z) in cycles per squared pixel offset."""
        return fresnel_rate(self.pitch, self.wavelength, self.z[k])

    def factor(self, k):
        """Per-layer factor of Eq. 1 that the default reading drops: exp(j k z) / z for the
        layer's distance (only with layer_factor), else 1."""
        return layer_factor(self.wavelength, self.z[k]) if self.layer_factor else 1.0


def geometry_of(scene):
    n_h, n_w = scene["intensity"].shape[-2:]
    return Geometry((n_h, n_w), scene["holo"], scene["pitch"], scene["wavelength"], scene["z"],
                    scene.get("layer_factor", False))


def layer_factor(wavelength, z):
    """exp(j 2 pi z / lambda) / z: Eq. 1's amplitude 1/r and carrier exp(j k r) at r = z,
    with the carrier's phase reduced to frac(z / lambda) cycles in FP64."""
    x = np.asarray(z, dtype=np.float64) / wavelength
    return np.exp(2j * np.pi * (x - np.floor(x))) / np.asarray(z, dtype=np.float64)


def fresnel_rate(pitch, wavelength, z):
    """a_z such that the paraxial phase pi*(d*p)^2/(lambda*z) equals 2*pi*a_z*d^2 (Eq. 1)."""
    return pitch * pitch / (2.0 * wavelength * z)


def _phase_cycles(a, d2):
    """frac(a * d2) in [-1/2, 1/2] cycles, d2 an exact integer squared offset."""
    x = a * np.asarray(d2, dtype=np.int64).astype(np.float64)
    return x - np.round(x)


def point_fringe_1d(delta, a):
    """f(d) = exp(j 2 pi frac(a d^2)) for integer offsets d (Eq. 1, paraxial, one axis)."""
    d = np.asarray(delta, dtype=np.int64)
    return np.exp(2j * np.pi * _phase_cycles(a, d * d))


def point_fringe_2d(dm, dn, a):
    """Fringe of one object point at integer pixel offsets (dm, dn), evaluated from the
    full squared distance dm^2 + dn^2 (no factorisation)."""
    dm = np.asarray(dm, dtype=np.int64)
    dn = np.asarray(dn, dtype=np.int64)
    return np.exp(2j * np.pi * _phase_cycles(a, dm * dm + dn * dn))


# ----------------------------------------------------------------------------
# Haar DWT (Eq. 2, Section 2 step 1)


def haar_forward(A, levels=3):
    """Unnormalised integer Haar DWT in Mallat layout.

    Level 1 acts on the whole plane; level l+1 acts on the low (S) quadrant of
    level l.  Quadrants at each level (h x w the current S size):
    S -> [:h/2, :w/2], X -> [:h/2, w/2:], Y -> [h/2:, :w/2], D -> [h/2:, w/2:].
    """
    C = np.array(A, dtype=np.int64, copy=True)
    h, w = C.shape
    for _ in range(levels):
        if h % 2 or w % 2:
            raise ValueError("object size must be divisible by 2^levels")
        S = C[:h, :w].copy()
        a = S[0::2, 0::2]
        b = S[0::2, 1::2]
        c = S[1::2, 0::2]
        d = S[1::2, 1::2]
        h2, w2 = h // 2, w // 2
        C[:h2, :w2] = a + b + c + d
        C[:h2, w2:w] = a - b + c - d
        C[h2:h, :w2] = a + b - c - d
        C[h2:h, w2:w] = a - b - c + d
        h, w = h2, w2
    return C


def haar_inverse(C, levels=3):
    """Exact integer inverse of haar_forward (each 2x2 synthesis divides by 4 exactly)."""
    C = np.array(C, dtype=np.int64, copy=True)
    H, W = C.shape
    for l in range(levels, 0, -1):
        h, w = H >> l, W >> l
        S = C[:h, :w]
        X = C[:h, w:2 * w]
        Y = C[h:2 * h, :w]
        D = C[h:2 * h, w:2 * w]
        out = np.empty((2 * h, 2 * w), dtype=np.int64)
        for (r, c, sx, sy) in ((0, 0, 1, 1), (0, 1, -1, 1), (1, 0, 1, -1), (1, 1, -1, -1)):
            num = S + sx * X + sy * Y + sx * sy * D
            if np.any(num % 4):
                raise ValueError("coefficients are not those of an integer image")
            out[r::2, c::2] = num // 4
        C[:2 * h, :2 * w] = out
    return C


def haar_synthesis_scaled(C, keep, levels=3):
    """4^levels times the inverse DWT of C with the detail coefficients of the blocks
    not kept set to zero.  keep[l] is a boolean [H>>l, W>>l] map of the level-l blocks
    whose (X, Y, D) are used.  Integer result (the scaled inverse never divides)."""
    C = np.asarray(C, dtype=np.int64)
    H, W = C.shape
    L = levels
    V = C[:H >> L, :W >> L].copy()  # 4^L * block mean at level L equals the level-L sum
    for l in range(L, 0, -1):
        h, w = H >> l, W >> l
        k = keep[l].astype(np.int64)
        X = C[:h, w:2 * w] * k
        Y = C[h:2 * h, :w] * k
        D = C[h:2 * h, w:2 * w] * k
        f = 4 ** (L - l)
        out = np.empty((2 * h, 2 * w), dtype=np.int64)
        for (r, c, sx, sy) in ((0, 0, 1, 1), (0, 1, -1, 1), (1, 0, 1, -1), (1, 1, -1, -1)):
            out[r::2, c::2] = V + f * (sx * X + sy * Y + sx * sy * D)
        V = out
    return V


def haar_forward_real(x, levels=3):
    """haar_forward on a real (float64) plane; same butterflies, no rounding issue."""
    C = np.array(x, dtype=np.float64, copy=True)
    h, w = C.shape
    for _ in range(levels):
        S = C[:h, :w].copy()
        a, b, c, d = S[0::2, 0::2], S[0::2, 1::2], S[1::2, 0::2], S[1::2, 1::2]
        h2, w2 = h // 2, w // 2
        C[:h2, :w2] = a + b + c + d
        C[:h2, w2:w] = a - b + c - d
        C[h2:h, :w2] = a + b - c - d
        C[h2:h, w2:w] = a - b - c + d
        h, w = h2, w2
    return C


def haar_synthesis_real(C, keep, levels=3):
    """Real inverse DWT with unkept details zeroed (haar_synthesis_scaled / 4^levels)."""
    C = np.asarray(C, dtype=np.float64)
    H, W = C.shape
    V = C[:H >> levels, :W >> levels].copy()
    for l in range(levels, 0, -1):
        h, w = H >> l, W >> l
        k = keep[l].astype(np.float64)
        X = C[:h, w:2 * w] * k
        Y = C[h:2 * h, :w] * k
        D = C[h:2 * h, w:2 * w] * k
        out = np.empty((2 * h, 2 * w))
        for (r, c, sx, sy) in ((0, 0, 1, 1), (0, 1, -1, 1), (1, 0, 1, -1), (1, 1, -1, -1)):
            out[r::2, c::2] = (V + sx * X + sy * Y + sx * sy * D) / 4.0
        V = out
    return V


# ----------------------------------------------------------------------------
# saliency quantisation and block selection (Section 2 steps 1-5)


def block_max(sal, level):
    """Saliency quantised to the level-l grid by the maximum over 2^l x 2^l blocks."""
    k = 1 << level
    h, w = sal.shape
    return np.asarray(sal).reshape(h // k, k, w // k, k).max(axis=(1, 3))


def block_occupied(layer, z, level):
    """True where depth layer z owns at least one pixel of the 2^l x 2^l block."""
    k = 1 << level
    h, w = layer.shape
    return (np.asarray(layer) == z).reshape(h // k, k, w // k, k).any(axis=(1, 3))


def selected_mask(saliency, layer, z, threshold, level):
    """Blocks of layer z taken at this level: occupied and (threshold < 0 or the block
    maximum of the saliency strictly above the threshold)."""
    occ = block_occupied(layer, z, level)
    if threshold < 0:
        return occ
    return occ & (block_max(saliency, level) > threshold)


def pack_entry(z, by, bx):
    return (int(z) << 24) | (int(by) << 12) | int(bx)


def unpack_entry(e):
    e = int(e)
    return (e >> 24) & 0x7F, (e >> 12) & 0xFFF, e & 0xFFF


def select_blocks(saliency, layer, n_layers, threshold, level):
    """Ordered work list of selected blocks: layer-major, then block row, then block
    column, each packed as (z << 24) | (by << 12) | bx."""
    out = []
    for z in range(n_layers):
        m = selected_mask(saliency, layer, z, threshold, level)
        for by in range(m.shape[0]):
            for bx in range(m.shape[1]):
                if m[by, bx]:
                    out.append(pack_entry(z, by, bx))
    return np.array(out, dtype=np.int32)


def masks_from_lists(lists, n_layers, obj_shape, levels=3):
    """Per-layer boolean keep maps from packed lists; lists[0] is the LLL list, lists[l]
    the level-l detail list."""
    H, W = obj_shape
    out = {}
    for key in range(levels + 1):
        lvl = levels if key == 0 else key
        m = np.zeros((n_layers, H >> lvl, W >> lvl), dtype=bool)
        for e in np.asarray(lists[key]).reshape(-1):
            z, by, bx = unpack_entry(e)
            m[z, by, bx] = True
        out[key] = m
    return out


def progressive_lists(saliency, layer, n_layers, thresholds, levels=3):
    """The four work lists of the method: [LLL (every occupied block), level-3, level-2,
    level-1 details], thresholds given per level on the uint8 saliency scale."""
    lists = [select_blocks(saliency, layer, n_layers, -1, levels)]
    for l in range(1, levels + 1):
        lists.append(select_blocks(saliency, layer, n_layers, thresholds[l], l))
    return lists


def object_planes(intensity, layer, n_layers):
    """A_z = I * [layer == z] (int64 planes)."""
    I = np.asarray(intensity, dtype=np.int64)
    L = np.asarray(layer)
    return np.stack([I * (L == z) for z in range(n_layers)])


def progressive_object(intensity, layer, lists, n_layers, levels=3):
    """Per-layer progressively reconstructed object A^_z: the inverse DWT of the layer
    plane with only the selected detail blocks kept.  Returns 4^levels * A^_z (int64)."""
    planes = object_planes(intensity, layer, n_layers)
    masks = masks_from_lists(lists, n_layers, planes.shape[1:], levels)
    out = np.empty_like(planes)
    H, W = planes.shape[1:]
    for z in range(n_layers):
        C = haar_forward(planes[z], levels)
        C[:H >> levels, :W >> levels] *= masks[0][z]  # LLL blocks not listed are dropped
        keep = {l: masks[l][z] for l in range(1, levels + 1)}
        out[z] = haar_synthesis_scaled(C, keep, levels)
    return out


# ----------------------------------------------------------------------------
# holograms


def block_fringe_rows(geom, k, a, n_cells, length):
    """Row factor of a k x k uniform block: b[r, m] = sum_{t<k} f(m - s*(k*r + t)).
    The LUT hologram block of Section 2 (Fig. 1) is the outer product of a row and
    a column factor of this kind."""
    m = np.arange(length, dtype=np.int64)[None, :]
    out = np.zeros((n_cells, length), dtype=np.complex128)
    r = np.arange(n_cells, dtype=np.int64)[:, None]
    for t in range(k):
        out += point_fringe_1d(m - geom.s * (k * r + t), a)
    return out


def superpose_cells(geom, a, k, values):
    """Hologram of a grid of uniform k x k cells with per-pixel values values[r, c]:
    sum_{r,c} values[r, c] * Blk_k(m - s*k*r, n - s*k*c)."""
    Bx = block_fringe_rows(geom, k, a, values.shape[0], geom.holo_h)
    By = block_fringe_rows(geom, k, a, values.shape[1], geom.holo_w)
    return Bx.T @ (values.astype(np.complex128) @ By)


def progressive_hologram(intensity, layer, lists, geom, levels=3):
    """Progressive hologram in the residual-map form of Section 2 steps 2-5.

    Step 2: every LLL point (every occupied block of the layer) is superposed with the
    8x8 block fringe times its per-pixel value LLL/64.  Steps 3-5, for l = 3, 2, 1:
    the residual map at level l-1 is the one-level inverse DWT of the selected detail
    blocks with the low band set to zero; every residual cell is superposed with the
    2^(l-1) x 2^(l-1) block fringe times its per-pixel value."""
    planes = object_planes(intensity, layer, geom.n_layers)
    masks = masks_from_lists(lists, geom.n_layers, planes.shape[1:], levels)
    H = np.zeros((geom.holo_h, geom.holo_w), dtype=np.complex128)
    Ho, Wo = planes.shape[1:]
    for z in range(geom.n_layers):
        a = geom.a(z)
        Hz = np.zeros_like(H)
        C = haar_forward(planes[z], levels)
        hL, wL = Ho >> levels, Wo >> levels
        lll = C[:hL, :wL] * masks[0][z]
        kL = 1 << levels
        Hz += superpose_cells(geom, a, kL, lll / float(kL * kL))
        for l in range(levels, 0, -1):
            h, w = Ho >> l, Wo >> l
            keep = masks[l][z]
            if not keep.any():
                continue
            X = C[:h, w:2 * w] * keep
            Y = C[h:2 * h, :w] * keep
            D = C[h:2 * h, w:2 * w] * keep
            res4 = np.empty((2 * h, 2 * w), dtype=np.int64)  # 4 x residual in level-(l-1) sums
            for (r, c, sx, sy) in ((0, 0, 1, 1), (0, 1, -1, 1), (1, 0, 1, -1), (1, 1, -1, -1)):
                res4[r::2, c::2] = sx * X + sy * Y + sx * sy * D
            k = 1 << (l - 1)
            # residual sum of a level-(l-1) cell is res4/4, spread over k*k pixels
            Hz += superpose_cells(geom, a, k, res4 / float(4 * k * k))
        H += geom.factor(z) * Hz
    return H


def pointwise_hologram_separable(planes, geom):
    """Full point-source hologram of real object planes: sum_z E_z A_z E_z^T with
    E_z[m, i] = f_z(m - s*i)."""
    planes = np.asarray(planes, dtype=np.float64)
    H = np.zeros((geom.holo_h, geom.holo_w), dtype=np.complex128)
    mi = np.arange(geom.holo_h)[:, None] - geom.s * np.arange(planes.shape[1])[None, :]
    nj = np.arange(geom.holo_w)[:, None] - geom.s * np.arange(planes.shape[2])[None, :]
    for z in range(planes.shape[0]):
        if not np.any(planes[z]):
            continue
        Ex = point_fringe_1d(mi, geom.a(z))
        Ey = point_fringe_1d(nj, geom.a(z))
        H += geom.factor(z) * (Ex @ planes[z] @ Ey.T)
    return H


def pointwise_hologram_direct(planes, geom, pixels=None):
    """Brute-force point-source sum over every object point, with the 2-D fringe
    evaluated from the full squared distance (Eq. 1, paraxial).  pixels: optional
    (m, n) index arrays; default every hologram pixel."""
    planes = np.asarray(planes, dtype=np.float64)
    if pixels is None:
        mm, nn = np.meshgrid(np.arange(geom.holo_h), np.arange(geom.holo_w), indexing="ij")
        mm, nn = mm.reshape(-1), nn.reshape(-1)
        shape = (geom.holo_h, geom.holo_w)
    else:
        mm = np.asarray(pixels[0], dtype=np.int64).reshape(-1)
        nn = np.asarray(pixels[1], dtype=np.int64).reshape(-1)
        shape = mm.shape
    out = np.zeros(mm.shape, dtype=np.complex128)
    for z in range(planes.shape[0]):
        ii, jj = np.nonzero(planes[z])
        if ii.size == 0:
            continue
        amp = planes[z][ii, jj]
        a = geom.a(z)
        c = geom.factor(z)
        for p in range(mm.size):
            out[p] += c * np.sum(amp * point_fringe_2d(mm[p] - geom.s * ii, nn[p] - geom.s * jj, a))
    return out.reshape(shape)


def plain_pointwise_hologram(intensity, layer, geom, pixels=None):
    """Plain point-wise hologram of the whole object (no wavelet, no saliency): the
    1x1-LUT column of Section 3.  Direct sum at the given pixels, else separable."""
    planes = object_planes(intensity, layer, geom.n_layers)
    if pixels is not None:
        return pointwise_hologram_direct(planes, geom, pixels)
    return pointwise_hologram_separable(planes, geom)


def pointcloud_hologram(intensity, depth, geom, pixels=None):
    """Point-source hologram of an object whose every pixel has its own depth: Eq. 1 in
    its paraxial form, for the 3-D extension sketched at the end of Section 2 without
    quantising depth into layers.  Pixel (i, j) with a finite depth z_ij > 0 (metres) is a
    point of amplitude intensity(i, j) at hologram pixel (s i, s j) on the plane at z_ij,
    with its own rate a_ij = p^2 / (2 lambda z_ij); other pixels are no point.  Direct sum
    at the given pixels ((m, n) index arrays; default every hologram pixel), each fringe
    from the exact integer squared distance."""
    I = np.asarray(intensity, dtype=np.float64)
    zz = np.asarray(depth, dtype=np.float64)
    valid = np.isfinite(zz) & (zz > 0)
    ii, jj = np.nonzero(valid)
    amp = I[ii, jj] * (layer_factor(geom.wavelength, zz[ii, jj]) if geom.layer_factor else 1.0)
    a = fresnel_rate(geom.pitch, geom.wavelength, zz[ii, jj])
    if pixels is None:
        mm, nn = np.meshgrid(np.arange(geom.holo_h), np.arange(geom.holo_w), indexing="ij")
        mm, nn = mm.reshape(-1), nn.reshape(-1)
        shape = (geom.holo_h, geom.holo_w)
    else:
        mm = np.asarray(pixels[0], dtype=np.int64).reshape(-1)
        nn = np.asarray(pixels[1], dtype=np.int64).reshape(-1)
        shape = mm.shape
    out = np.zeros(mm.shape, dtype=np.complex128)
    for p in range(mm.size):
        dm = mm[p] - geom.s * ii
        dn = nn[p] - geom.s * jj
        out[p] = np.sum(amp * np.exp(2j * np.pi * _phase_cycles(a, dm * dm + dn * dn)))
    return out.reshape(shape)


# ----------------------------------------------------------------------------
# reconstruction, adjoint, quality


def reconstruct_fields(H, geom, n_obj=None):
    """Fresnel back-propagation of the hologram to every layer, sampled on the object
    grid: R_z = conj(c_z) E_z^H H conj(E_z), the adjoint of A -> c_z E_z A E_z^T (c_z the
    layer factor, 1 unless the geometry keeps it)."""
    oh, ow = n_obj if n_obj is not None else (geom.holo_h // geom.s, geom.holo_w // geom.s)
    mi = np.arange(geom.holo_h)[:, None] - geom.s * np.arange(oh)[None, :]
    nj = np.arange(geom.holo_w)[:, None] - geom.s * np.arange(ow)[None, :]
    R = np.empty((geom.n_layers, oh, ow), dtype=np.complex128)
    for z in range(geom.n_layers):
        Ex = point_fringe_1d(mi, geom.a(z))
        Ey = point_fringe_1d(nj, geom.a(z))
        R[z] = np.conj(geom.factor(z)) * (Ex.conj().T @ H @ Ey.conj())
    return R


def asm_transfer(geom, k, P, band_limit=False):
    """Angular-spectrum transfer function that back-propagates the hologram plane by z_k
    (to layer k's plane) on a P x P DFT grid of pitch p (Section 2, last paragraph:
    inverse angular spectrum at the scene's own parameters).  A plane wave of spatial frequency (fx, fy) advances by
    2 pi z sqrt(1/lambda^2 - fx^2 - fy^2) over a distance z; back-propagation takes that
    phase off.  The common carrier exp(j 2 pi z / lambda) is removed (the holograms here
    omit it), so T = exp(-j 2 pi z (sqrt(1/lambda^2 - f^2) - 1/lambda)); evanescent
    frequencies (f >= 1/lambda) get 0.  band_limit additionally zeroes |fx| or |fy| above
    1 / (lambda sqrt((2 df z)^2 + 1)), df = 1/(P p) (Matsushima and Shimobaba 2009)."""
    f = np.fft.fftfreq(P, d=geom.pitch)
    fx, fy = f[None, :], f[:, None]
    lam, z = geom.wavelength, geom.z[k]
    arg = 1.0 / lam ** 2 - fx ** 2 - fy ** 2
    prop = arg > 0
    T = np.where(prop, np.exp(-2j * np.pi * z * (np.sqrt(np.where(prop, arg, 0.0)) - 1.0 / lam)), 0.0)
    if band_limit:
        df = 1.0 / (P * geom.pitch)
        flim = 1.0 / (lam * np.sqrt((2.0 * df * z) ** 2 + 1.0))
        T = T * ((np.abs(fx) <= flim) & (np.abs(fy) <= flim))
    return T


def asm_reconstruct_fields(H, geom, pad=2, band_limit=False):
    """Reconstruction by the inverse angular spectrum method (Section 2, last paragraph),
    sampled on the object grid: the hologram is zero-padded to P = pad * holo (pad 2 makes
    the DFT's circular convolution a linear one), transformed, multiplied by each layer's
    back-propagation transfer function, inverse transformed and read at the object
    pixels (s i, s j).  Scaled by p^2 / (lambda z) so that an unbounded Fresnel point
    fringe of amplitude A comes back as A at its point (the Fresnel kernel's
    1 / (j lambda z) per unit area, which the holograms omit)."""
    H = np.asarray(H, dtype=np.complex128)
    P = pad * geom.holo_h
    if geom.holo_h != geom.holo_w:
        raise ValueError("square holograms only")
    Hp = np.zeros((P, P), dtype=np.complex128)
    Hp[:geom.holo_h, :geom.holo_w] = H
    X = np.fft.fft2(Hp)
    oh, ow = geom.holo_h // geom.s, geom.holo_w // geom.s
    R = np.empty((geom.n_layers, oh, ow), dtype=np.complex128)
    for k in range(geom.n_layers):
        U = np.fft.ifft2(X * asm_transfer(geom, k, P, band_limit))
        scale = geom.pitch ** 2 / (geom.wavelength * geom.z[k])
        R[k] = scale * U[:geom.s * oh:geom.s, :geom.s * ow:geom.s]
    return R


def propagate_fields(fields, geom):
    """Point-source hologram of complex layer fields (Eq. 1 per layer, paraxial):
    H = sum_z c_z E_z F_z E_z^T; the adjoint of reconstruct_fields."""
    fields = np.asarray(fields, dtype=np.complex128)
    H = np.zeros((geom.holo_h, geom.holo_w), dtype=np.complex128)
    mi = np.arange(geom.holo_h)[:, None] - geom.s * np.arange(fields.shape[1])[None, :]
    nj = np.arange(geom.holo_w)[:, None] - geom.s * np.arange(fields.shape[2])[None, :]
    for z in range(fields.shape[0]):
        Ex = point_fringe_1d(mi, geom.a(z))
        Ey = point_fringe_1d(nj, geom.a(z))
        H += geom.factor(z) * (Ex @ fields[z] @ Ey.T)
    return H


def phase_opt_loss(phase, target, weight, layer, geom, kappa):
    """Phase-only hologram loss: H = exp(j phase), a = composite amplitude of the Fresnel
    reconstruction, L = sum w (a / kappa - T)^2."""
    H = np.exp(1j * np.asarray(phase, dtype=np.float64))
    a = composite_amplitude(reconstruct_fields(H, geom, np.shape(layer)), layer)
    return float(np.sum(weight * (a / kappa - target) ** 2))


def phase_opt_grad(phase, target, weight, layer, geom, kappa):
    """Analytic dL/dphase of phase_opt_loss by the chain rule: dL/da = 2 w (a/kappa - T)/kappa;
    dL/dR_z = dL/da * R/|R| on the pixels of layer z; dL/dH = propagate_fields(dL/dR)
    (adjoint of the reconstruction); dL/dphase = Im(dL/dH * conj(H))."""
    H = np.exp(1j * np.asarray(phase, dtype=np.float64))
    L = np.asarray(layer).astype(np.int64)
    R = reconstruct_fields(H, geom, L.shape)
    ii, jj = np.indices(L.shape)
    Rl = R[L, ii, jj]
    a = np.abs(Rl)
    ga = 2.0 * weight * (a / kappa - target) / kappa
    gR = np.zeros_like(R)
    unit = np.where(a > 0, Rl / np.where(a > 0, a, 1.0), 0.0)
    gR[L, ii, jj] = ga * unit
    gH = propagate_fields(gR, geom)
    return np.imag(gH * np.conj(H))


def composite_amplitude(R, layer):
    """|R_{layer(i,j)}(i, j)|: each object pixel read on its own layer."""
    L = np.asarray(layer).astype(np.int64)
    ii, jj = np.indices(L.shape)
    return np.abs(R[L, ii, jj])


def progressive_adjoint(G, layer, lists, geom, levels=3):
    """Adjoint of the real-input progressive operator I -> H: for a hologram-space
    cotangent G returns dL/dI = sum_z [layer == z] * P_z(Re R_z), R_z the
    back-propagated field and P_z = IDWT o mask o DWT the per-layer progressive
    approximation (an orthogonal projection for the Haar basis, hence self-adjoint)."""
    L = np.asarray(layer)
    R = reconstruct_fields(G, geom, L.shape)
    masks = masks_from_lists(lists, geom.n_layers, L.shape, levels)
    out = np.zeros(L.shape, dtype=np.float64)
    for z in range(geom.n_layers):
        keep = {l: masks[l][z] for l in range(1, levels + 1)}
        C = haar_forward_real(np.real(R[z]), levels)
        C[:L.shape[0] >> levels, :L.shape[1] >> levels] *= masks[0][z]
        Pz = haar_synthesis_real(C, keep, levels)
        out += Pz * (L == z)
    return out


def progressive_hologram_real(x, layer, lists, geom, levels=3):
    """The progressive operator on a real-valued object x (Eq. 3 is linear in the object):
    H = sum_z E_z P_z(x [layer == z]) E_z^T with P_z = IDWT o mask o DWT, the layer's
    progressive approximation.  For an integer object it is progressive_hologram; its
    adjoint is progressive_adjoint."""
    x = np.asarray(x, dtype=np.float64)
    L = np.asarray(layer)
    masks = masks_from_lists(lists, geom.n_layers, L.shape, levels)
    planes = np.zeros((geom.n_layers,) + L.shape, dtype=np.float64)
    for z in range(geom.n_layers):
        keep = {l: masks[l][z] for l in range(1, levels + 1)}
        C = haar_forward_real(x * (L == z), levels)
        C[:L.shape[0] >> levels, :L.shape[1] >> levels] *= masks[0][z]
        planes[z] = haar_synthesis_real(C, keep, levels)
    return pointwise_hologram_separable(planes, geom)


def _gauss_window(size=11, sigma=1.5):
    t = np.arange(size) - (size - 1) / 2.0
    g = np.exp(-t * t / (2 * sigma * sigma))
    return g / g.sum()


def _filter_valid(x, g):
    """Separable 'valid' correlation of x with the window g along both axes."""
    k = g.size
    tmp = sum(g[t] * x[t:x.shape[0] - k + 1 + t, :] for t in range(k))
    return sum(g[t] * tmp[:, t:x.shape[1] - k + 1 + t] for t in range(k))


def ssim(x, y, data_range=1.0, k1=0.01, k2=0.03, win=11, sigma=1.5):
    """Mean SSIM (Wang et al. 2004) with an 11x11 Gaussian window of sigma 1.5."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    g = _gauss_window(win, sigma)
    c1 = (k1 * data_range) ** 2
    c2 = (k2 * data_range) ** 2
    mx, my = _filter_valid(x, g), _filter_valid(y, g)
    sxx = _filter_valid(x * x, g) - mx * mx
    syy = _filter_valid(y * y, g) - my * my
    sxy = _filter_valid(x * y, g) - mx * my
    s = ((2 * mx * my + c1) * (2 * sxy + c2)) / ((mx * mx + my * my + c1) * (sxx + syy + c2))
    return float(s.mean())


def operator_count(lists):
    """Operator count of Section 3: one operator = one LUT block multiplied, shifted and
    added.  LLL blocks count once; a residual map at level l has 4 cells per selected
    detail block, each superposed once."""
    return int(len(lists[0]) + 4 * sum(len(x) for x in lists[1:]))


def detail_term_count(lists):
    """Number of coefficient terms of the detail-basis form: one per LLL block and three
    (X, Y, D) per selected detail block."""
    return int(len(lists[0]) + 3 * sum(len(x) for x in lists[1:]))


def rel_l2(x, ref):
    x = np.asarray(x, dtype=np.complex128)
    ref = np.asarray(ref, dtype=np.complex128)
    den = np.linalg.norm(ref.reshape(-1))
    return float(np.linalg.norm((x - ref).reshape(-1)) / (den if den > 0 else 1.0))
