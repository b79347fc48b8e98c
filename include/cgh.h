/*
 * cgh.h - C ABI of libcgh, saliency-progressive point-source hologram generation
 * (Rafiei & Shirani, "Progressive hologram generation based on object saliency",
 * arXiv 2211.09938) on NVIDIA GB300 (sm_103a).
 *
 * Conventions shared by every call
 * --------------------------------
 * - Every data pointer is a DEVICE pointer owned by the caller unless a call says
 *   otherwise; the library never frees caller memory.  Arrays are dense, row-major,
 *   C order, with no padding between rows.
 * - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *   Calls only enqueue work on that stream and return; they never synchronise
 *   except where a call says so.  Counts produced on the device stay there.
 * - Return value: CGH_OK (0) or an error code below; cgh_last_error() gives a
 *   thread-local message for the last failing call of the calling thread.
 *   Argument errors are detected on the host before anything is enqueued.
 *   CGH_ERR_CUDA reports a CUDA launch or API error (no CPU fallback exists: with
 *   no usable GPU every call fails with CGH_ERR_CUDA).
 * - Geometry: object obj_h x obj_w pixels (multiples of 8), hologram holo_h x holo_w
 *   pixels, with holo_h = s*obj_h and holo_w = s*obj_w for one integer stride s >= 1.
 *   Object pixel (i, j) sits at hologram pixel (s*i, s*j).  Pixel pitch p, wavelength
 *   lambda, depth layers z_0..z_{Z-1} (metres), 1 <= Z <= 64.
 * - Point fringe (Eq. 1 of the paper, paraxial form, 1/r and exp(jkz) dropped): the
 *   hologram of a unit point at (i, j) on layer z is
 *       f_z(m - s*i) * f_z(n - s*j),   f_z(d) = exp(j*2*pi*frac(a_z*d^2)),
 *       a_z = p^2 / (2*lambda*z).
 * - Holograms are complex64 (float2: re, im) [holo_h][holo_w].
 */
#ifndef CGH_H
#define CGH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------------- */
#define CGH_OK 0
#define CGH_ERR_ARG 1          /* invalid argument (NULL, size, range)               */
#define CGH_ERR_CUDA 2         /* CUDA API / launch error, or no usable GPU          */
#define CGH_ERR_UNSUPPORTED 3  /* valid but not supported by this build / device      */
#define CGH_ERR_TIMEOUT 4      /* a bounded device-side wait gave up (see cgh_status) */
#define CGH_ERR_NOMEM 5        /* device allocation failed                            */

/* ---- superposition forms (cgh_progressive_hologram `form`) ------------------------ */
/* Detail-basis direct form on CUDA cores, FP32: every LLL block and every selected
 * detail block is added as row-factor x column-factor products read from the fringe
 * tables (Eq. 3, Section 2 steps 2-5).                                               */
#define CGH_FORM_DIRECT_LUT 0
/* Separable dense form on tcgen05 tensor cores: per layer H += E_z * A^_z * E_z^T,
 * A^_z the progressively reconstructed object plane (inverse DWT of the LLL band and
 * the selected detail blocks), operands split into hi+lo halves (3 products) with
 * FP32 accumulation in tensor memory.                                                */
#define CGH_FORM_TC_BF16X3 1   /* bf16 hi+lo                                            */
#define CGH_FORM_TC_FP16X3 2   /* fp16 hi+lo                                            */
/* The same separable form with the fringe operand rounded once to fp16 (its hi planes
 * only) and the data operand fp16 hi+lo: two products per real product instead of three,
 * a third fewer MMAs and operand bytes.  The fringe's own fp16 rounding (2^-12) then bounds
 * the error (a few 1e-4 rel-L2, against 1e-3 for the split paths).  Single scenes only
 * (cgh_batch_* take the two forms above).                                              */
#define CGH_FORM_TC_FP16X2 3

/* ---- plan --------------------------------------------------------------------------- */
/* Plan flag: every output element is written by one CTA in a fixed order (no split-K
 * atomics), so results are bit-reproducible run to run; the split forms are faster.  The
 * unsplit FP32 accumulation chains are longer: fp16 hi+lo then reaches ~2e-5 rel-L2 on a
 * 512x512 object with 16 layers (the split default stays below 1e-5). */
#define CGH_PLAN_DETERMINISTIC 1
/* Plan flag: keep Eq. 1's amplitude 1/r and carrier exp(jkr) at r = z as a per-layer factor
 * c_z = exp(j*2*pi*frac(z/lambda)) / z (the default reading drops this constant of each
 * layer).  Every hologram and reconstruction of the plan includes it (the reconstructions
 * as conj(c_z), the adjoint); the point-wise per-point-depth call takes each point's own
 * exp(j*2*pi*frac(z/lambda)) / z.  cgh_reconstruct_asm treats the hologram as given. */
#define CGH_PLAN_LAYER_FACTOR 2

typedef struct cgh_plan cgh_plan;

/* Thread-local message describing the last error of the calling thread ("" if none). */
const char* cgh_last_error(void);

/* Library version (major*10000 + minor*100 + patch). */
int cgh_version(void);

/*
 * cgh_plan_create - geometry, fringe tables and scratch for one scene shape.
 * Paper: Section 2 ("hologram blocks ... precomputed in LUT using eq. 1", 8x8, 4x4,
 * 2x2 and 1x1 blocks) and Table 1 (scene specification).
 *   out          receives the plan (host pointer to a library-owned object)
 *   obj_h, obj_w object size, multiples of 8 (3 Haar levels), 8..8192
 *   holo_h, holo_w hologram size, s*obj_h and s*obj_w for an integer s, <= 16384
 *   pitch_m, wavelength_m  pixel pitch and wavelength (metres, > 0)
 *   n_layers     Z, 1..64;   z_m  HOST array of Z layer distances (metres, > 0)
 *   levels       number of Haar levels; must be 3 (the paper's choice)
 *   flags        0, or CGH_PLAN_DETERMINISTIC and / or CGH_PLAN_LAYER_FACTOR
 *   stream       stream on which the fringe tables are built
 * The plan allocates device memory (tables, scratch, status word) with cudaMalloc on
 * the current device and builds the fringe tables with cgh_build_tables on `stream`.
 * Errors: CGH_ERR_ARG, CGH_ERR_NOMEM, CGH_ERR_CUDA.  On error *out is NULL.
 */
int cgh_plan_create(cgh_plan** out, int obj_h, int obj_w, int holo_h, int holo_w,
                    double pitch_m, double wavelength_m, int n_layers, const double* z_m,
                    int levels, int flags, void* stream);

/*
 * cgh_plan_set_tuning - cap on the 32-wide K steps accumulated in one tensor-memory chain of
 * the stage-2 GEMM (0 = automatic: 32 for fp16 hi+lo, 128 for bf16 hi+lo).  Longer chains are faster;
 * the tensor pipe's FP32 accumulation error grows with the chain length (about 2e-5 rel-L2
 * for ~14k-term chains at a 2048x2048 hologram with 32 layers), shorter chains add their
 * partial sums in L2 with round-to-nearest atomics.  Applies to later calls of the plan.
 */
int cgh_plan_set_tuning(cgh_plan* plan, int max_ksteps_per_chain);

/*
 * cgh_plan_set_contraction - order of the separable tensor form's two GEMMs.
 * H = sum_z E_z A^_z E_z^T can be contracted over the layers' compacted object rows
 * (stage 2 K = sum of the row counts) or, for a square object, over their columns (the
 * transposed problem, H written transposed); the cost of stage 2 follows that K.
 *   CGH_CONTRACT_AUTO  (default) on the device, per call: columns when their sum is smaller
 *   CGH_CONTRACT_ROWS  always rows;  CGH_CONTRACT_COLS  columns whenever the object is square
 * Results agree to rounding.  Applies to later calls of the plan.  The paper has no
 * counterpart (it superposes block fringes directly).
 */
/*
 * cgh_plan_set_stage2_tiles - tile shape of the separable form's stage-2 GEMM.
 *   CGH_TILES_AUTO  (default) CTA pairs when the call splits K stream-K style (not with
 *                   CGH_PLAN_DETERMINISTIC), the device holds CTA pairs and the hologram
 *                   has at least 64 tiles of 128 x 128 (1024 x 1024 and larger)
 *   CGH_TILES_CTA   one CTA per 128 x 128 output tile
 *   CGH_TILES_PAIR  two CTAs of a cluster per 256 x 128 output tile (tcgen05 cta_group::2:
 *                   each CTA stages its 128 rows of the fringe operand and half of the data
 *                   operand, so the data operand is staged once per pair); falls back to
 *                   one CTA per tile where pairs do not apply
 * Results agree to rounding.  Applies to later calls of the plan.  The paper has no
 * counterpart (a tuning knob of the GPU contraction).
 */
#define CGH_TILES_AUTO 0
#define CGH_TILES_CTA 1
#define CGH_TILES_PAIR 2
int cgh_plan_set_stage2_tiles(cgh_plan* plan, int tiles);

/*
 * cgh_plan_stage2_tiles_used - *tiles = the tile shape the plan's last separable-form call
 * with two GEMM launches ran stage 2 with: CGH_TILES_CTA or CGH_TILES_PAIR (CGH_TILES_AUTO
 * before the first such call, and unchanged by fused or batched calls).  Host-side state,
 * recorded when the launch is enqueued; nothing is synchronised.  CGH_ERR_ARG for a NULL
 * argument.  The paper has no counterpart (it reports which GPU kernel a call used).
 */
int cgh_plan_stage2_tiles_used(const cgh_plan* plan, int* tiles);

/*
 * cgh_plan_set_fusion - 1: the separable form's two GEMM stages run as one cooperative
 * persistent launch in which each CTA does its share of stage 1 and then its stream-K share
 * of stage 2, each stage-2 chain first waiting (bounded) until every stage-1 tile of the
 * layers it reads is stored; used when the call splits K stream-K style (not with
 * CGH_PLAN_DETERMINISTIC), the stage-2 tiles are not forced to CTA pairs, and the grid fits
 * on the device at once.  0 (default): two launches (stage 2 on CTA pairs by default).  The
 * fused launch saves ~4 us of a 512 -> 1024, 16-layer superposition on its own, but needs
 * every SM, so it neither starts early behind the preceding kernel nor overlaps another
 * stream's work (a captured step gains nothing; concurrent pipelines lose).  Results agree
 * to rounding.  Applies to later calls of the plan.  The paper has no counterpart (a
 * scheduling choice of the GPU path).
 */
int cgh_plan_set_fusion(cgh_plan* plan, int fused);

#define CGH_CONTRACT_AUTO 0
#define CGH_CONTRACT_ROWS 1
#define CGH_CONTRACT_COLS 2
int cgh_plan_set_contraction(cgh_plan* plan, int order);

/* Frees the plan and its device memory (synchronises the device first).  NULL is a no-op. */
int cgh_plan_destroy(cgh_plan* plan);

/*
 * cgh_build_tables - (re)build the plan's fringe tables on `stream`.
 * Paper: Section 2 (LUT hologram blocks of 2^l x 2^l points from Eq. 1).
 * For every layer z, level l in 0..3 and offset d in [-s*obj, holo) the plan stores the
 * one-axis block fringes
 *     b_l(d) = sum_{t < 2^l} f_z(d - s*t)
 *     w_l(d) = sum_{t < 2^(l-1)} f_z(d - s*t) - sum_{2^(l-1) <= t < 2^l} f_z(d - s*t)
 * (b_0 = f_z), whose outer products are the hologram blocks of a uniform block and of
 * the Haar detail functions.  The phase frac(a_z*d^2) is formed in FP64 from the exact
 * integer d^2 and range-reduced before the FP32 cast.  plan_create already calls it.
 */
int cgh_build_tables(cgh_plan* plan, void* stream);

/*
 * cgh_haar_decompose - per-layer 3-level integer Haar DWT.
 * Paper: Eq. 2 and Section 2 step 1.  For every layer z the plane
 * A_z(i,j) = intensity(i,j) * [layer_idx(i,j) == z] is decomposed with the unnormalised
 * sum/difference Haar on 2x2 cells [a b; c d] (rows i, columns j):
 *     S = a+b+c+d, X = a-b+c-d, Y = a+b-c-d, D = a-b-c+d, recursing on S.
 *   intensity  uint8 [obj_h][obj_w];  layer_idx uint8 [obj_h][obj_w] (values >= Z own no layer)
 *   coeffs     int32 [Z][obj_h][obj_w] output, Mallat layout per layer: at level l
 *              (h = obj_h>>l, w = obj_w>>l) X in [0,h)x[w,2w), Y in [h,2h)x[0,w),
 *              D in [h,2h)x[w,2w); LLL (S of level 3) in [0,obj_h>>3)x[0,obj_w>>3).
 * Bit-exact.  Errors: CGH_ERR_ARG (NULL), CGH_ERR_CUDA.
 */
int cgh_haar_decompose(const cgh_plan* plan, const uint8_t* intensity, const uint8_t* layer_idx,
                       int32_t* coeffs, void* stream);

/*
 * cgh_select_blocks - saliency quantisation, block selection and ordered compaction.
 * Paper: Section 2 step 1 (saliency map quantised to the level grids by the block
 * maximum) and steps 2-5 (blocks above a threshold get that level's hologram).
 * A level-l block (2^l x 2^l pixels) of layer z is selected iff layer z owns at least
 * one of its pixels and (threshold < 0 or max(saliency over the block) > threshold).
 *   saliency   uint8 [obj_h][obj_w] (may be NULL when threshold < 0), 8-byte aligned
 *   layer_idx  uint8 [obj_h][obj_w], 8-byte aligned (blocks are read a row at a time)
 *   threshold  -1 (occupancy only: the LLL list) or 0..255 (strict comparison)
 *   level      1..3
 *   list       int32 [capacity] output, entries (z << 24) | (by << 12) | bx in
 *              ascending order of z, then block row by, then block column bx
 *   d_count    int32 [2] output: d_count[0] = entries written = min(total, capacity),
 *              d_count[1] = total number of selected blocks
 *   capacity   >= 0
 * Uses plan scratch for per-chunk counts (calls that share a plan must be ordered on
 * one stream).  Bit-exact.  Errors: CGH_ERR_ARG, CGH_ERR_CUDA.
 */
int cgh_select_blocks(const cgh_plan* plan, const uint8_t* saliency, const uint8_t* layer_idx,
                      int threshold, int level, int32_t* list, int32_t* d_count, int capacity,
                      void* stream);

/*
 * cgh_select_blocks_noalloc - cgh_select_blocks without a plan and without allocating.
 * The paper has no counterpart: this entry point exists for callers that cannot call
 * cudaMalloc (for example an embedder whose device memory budget is fixed and reserved
 * at start-up and must not grow afterwards) and so cannot create a plan.  Like every
 * entry point here it calls the CUDA runtime, so it must not be called from inside a
 * stream host function (cudaLaunchHostFunc), where CUDA calls are not allowed.
 * Same selection, order, output format, d_count[2] semantics and bit-exact results as
 * cgh_select_blocks for the same inputs.
 *   obj_h, obj_w  object size (multiples of 8, 8..8192);  n_layers  Z, 1..64
 *   other arguments as for cgh_select_blocks (device pointers, caller-owned)
 * Scratch: a static device array built into the library (2 MiB per GPU that loads the
 * library, held until the process exits).  Limit: n_layers * ceil(blocks at `level` /
 * 256) <= 262144, e.g. 64 layers of a 2048x2048 object at level 1; larger requests
 * return CGH_ERR_ARG with a message and enqueue nothing.
 * Allocates nothing: no cudaMalloc, no cudaFree, no allocating library routine.  The
 * array is placed when the library's module is first loaded on a device, which under
 * lazy module loading (the CUDA default) can be this entry point's first call there.
 * That first call on each device also looks up the array's device address with
 * cudaGetSymbolAddress (with that device current).  So make one call per device at
 * start-up, before any stream capture and before the memory budget is fixed.  The
 * looked-up address is cached for the life of the process and does not survive
 * cudaDeviceReset: do not call this entry point after resetting its device.  All calls on a device share the one array: calls that may overlap on
 * the GPU (different streams, or different host threads) race and must be serialised
 * by the caller.
 * Errors: CGH_ERR_ARG, CGH_ERR_UNSUPPORTED (device ordinal >= 64), CGH_ERR_CUDA.
 */
int cgh_select_blocks_noalloc(const uint8_t* saliency, const uint8_t* layer_idx, int obj_h, int obj_w,
                              int n_layers, int threshold, int level, int32_t* list, int32_t* d_count,
                              int capacity, void* stream);

/*
 * cgh_select_progressive - the four work lists of one progressive hologram in one go.
 * Paper: Section 2 steps 1-5 (the LLL band takes every block; the detail levels take the
 * blocks above their saliency thresholds).  Same results as four cgh_select_blocks calls:
 *   lists[0]  LLL list    = cgh_select_blocks(threshold -1, level 3)
 *   lists[l]  level l     = cgh_select_blocks(thresholds[l-1], level l), l = 1, 2, 3
 *   saliency, layer_idx  uint8 [obj_h][obj_w], 8-byte aligned
 *   thresholds  HOST int[3] (levels 1, 2, 3), each -1..255
 *   lists       HOST array of 4 device pointers;  capacities  HOST int[4]
 *   d_counts    device int32 [4][2] output, ([written, total] per list, as d_count of
 *               cgh_select_blocks); directly usable by cgh_progressive_hologram
 * Runs the compaction once for all four lists: one cooperative launch with a single grid
 * barrier when the count tables are small (see cgh_progressive_step), else three passes.
 * Uses plan scratch.  Bit-exact.  Errors: CGH_ERR_ARG, CGH_ERR_CUDA.
 */
int cgh_select_progressive(const cgh_plan* plan, const uint8_t* saliency, const uint8_t* layer_idx,
                           const int* thresholds, int32_t* const* lists, const int* capacities,
                           int32_t* d_counts, void* stream);

/*
 * cgh_progressive_hologram - progressive superposition of the selected blocks.
 * Paper: Eq. 3 (hologram = sum of the holograms of the Haar basis functions times their
 * coefficients) and Section 2 steps 2-5.
 *   H(m,n) = sum_z [ sum_{LLL list} LLL/64 * b_3(m-u) b_3(n-v)
 *            + sum_{l=1..3} sum_{level-l list} 4^-l (X b_l(m-u) w_l(n-v)
 *                                               + Y w_l(m-u) b_l(n-v) + D w_l(m-u) w_l(n-v)) ]
 *   with u = s*2^l*by, v = s*2^l*bx for a block (z, by, bx) of level l.
 *   coeffs    int32 [Z][obj_h][obj_w] from cgh_haar_decompose
 *   lists     HOST array of 4 device pointers: lists[0] = LLL list (level-3 blocks),
 *             lists[l] = level-l detail list, l = 1..3 (format of cgh_select_blocks)
 *   d_counts  int32 [4][2] device array, d_counts[2k] = entries in lists[k] (the
 *             d_count[0] written by cgh_select_blocks); [2k+1] is ignored.  Each list
 *             must hold d_counts[2k] entries.  A count outside [0, Z * blocks at the
 *             list's level] cannot come from the selection: the kernels clamp it to that
 *             range (never reading past the plan's largest possible list) and record
 *             CGH_ERR_ARG in the plan's status word (read with cgh_status).
 *   holo      complex64 [holo_h][holo_w] output
 *   accumulate 0: holo = H;  1: holo += H
 *   form      CGH_FORM_* (the tensor-core forms use plan scratch)
 * Errors: CGH_ERR_ARG, CGH_ERR_UNSUPPORTED (form), CGH_ERR_CUDA; device-side count errors
 * through cgh_status as above.
 */
int cgh_progressive_hologram(const cgh_plan* plan, const int32_t* coeffs,
                             const int32_t* const* lists, const int32_t* d_counts,
                             float* holo, int accumulate, int form, void* stream);

/*
 * cgh_progressive_step - block selection and progressive superposition in one call.
 * Paper: Section 2 steps 1-5 (selection of the LLL band and of the detail blocks above
 * their saliency thresholds) followed by Eq. 3 (superposition of the selected blocks).
 * Same outputs as cgh_select_progressive(saliency, layer_idx, thresholds, lists,
 * capacities, d_counts) followed by cgh_progressive_hologram(coeffs, lists, d_counts,
 * holo, accumulate, form):
 *   lists, d_counts  the four work lists and their [written, total] counts, bit-exact
 *   holo             the hologram of the written list entries
 * Arguments as for those two calls (saliency, layer_idx 8-byte aligned; thresholds,
 * lists, capacities HOST arrays; all four lists non-NULL), plus
 *   coeffs_ready  a cudaEvent_t or NULL: when given, `stream` waits for it after the
 *                 selection and before coeffs is first read, so that a DWT running on
 *                 another stream overlaps the selection
 * For the tensor-core forms, when the selection's count tables are small (at most 8192
 * per-layer chunk counts per list and a grid the device holds at once, e.g. a 512x512
 * object with 16 layers), the selection runs as one cooperative launch with a single grid
 * barrier and marks the operands' selection flags itself, so the lists are not read back.  Its wait is bounded:
 * on timeout it records CGH_ERR_TIMEOUT in the status word (cgh_status); the plan's
 * barrier state is then undefined and the plan must be destroyed.  Uses plan scratch.
 * Errors: CGH_ERR_ARG, CGH_ERR_UNSUPPORTED (form), CGH_ERR_CUDA.
 */
int cgh_progressive_step(const cgh_plan* plan, const uint8_t* saliency, const uint8_t* layer_idx,
                         const int32_t* coeffs, const void* coeffs_ready, const int* thresholds,
                         int32_t* const* lists, const int* capacities, int32_t* d_counts, float* holo,
                         int accumulate, int form, void* stream);

/*
 * cgh_plain_direct - plain point-wise hologram, no wavelet and no saliency.
 * Paper: Eq. 1 (the fully point-wise "1x1 LUT" hologram of Section 3, M x N operators).
 *   H(m,n) = sum_{(i,j)} intensity(i,j) * exp(j*2*pi*frac(a_{z(i,j)} * ((m-s*i)^2 + (n-s*j)^2)))
 * with z(i,j) = layer_idx(i,j) (pixels with layer >= Z are skipped).  The phase is
 * reduced exactly in 64-bit fixed point (a_z mod 1 scaled by 2^64) and evaluated with
 * the hardware sine/cosine (SFU).
 *   holo complex64 [holo_h][holo_w] output (overwritten).
 * Errors: CGH_ERR_ARG, CGH_ERR_CUDA.
 */
int cgh_plain_direct(const cgh_plan* plan, const uint8_t* intensity, const uint8_t* layer_idx,
                     float* holo, void* stream);

/*
 * cgh_pointcloud_direct - point-wise hologram with a depth per object point.
 * Paper: Eq. 1 (paraxial) for the 3-D scenes the end of Section 2 extends the method to,
 * here without quantising depth into the plan's layers.  Object pixel (i, j) with a finite
 * depth z_ij > 0 is a point of amplitude intensity(i, j) at hologram pixel (s*i, s*j):
 *   holo(m,n) (+)= sum_{i,j} intensity(i,j) * exp(j*2*pi*frac(a_ij*((m-s*i)^2 + (n-s*j)^2))),
 *   a_ij = p^2 / (2*lambda*z_ij)   (formed in FP64, then reduced exactly in 64-bit fixed point)
 * Pixels with depth <= 0, NaN or infinite are no point.  The plan's layer distances are not
 * used; a depth map holding them reproduces cgh_plain_direct bit for bit.  FP32 SFU
 * sine/cosine per (point, pixel), as cgh_plain_direct.
 *   intensity  uint8 [obj_h][obj_w];  depth_m float [obj_h][obj_w] (metres)
 *   holo       complex64 [holo_h][holo_w], overwritten (accumulate = 0) or added to (1)
 * Errors: CGH_ERR_ARG, CGH_ERR_CUDA.
 */
int cgh_pointcloud_direct(const cgh_plan* plan, const uint8_t* intensity, const float* depth_m, float* holo,
                          int accumulate, void* stream);

/*
 * cgh_reconstruct - Fresnel back-propagation of a hologram to every layer.
 * Paper: Section 2 last paragraph (numerical reconstruction; the paper uses the inverse
 * angular spectrum, this library uses the Fresnel adjoint of Eq. 1 on the object grid).
 *   R_z(i,j) = sum_{m,n} holo(m,n) * conj(f_z(m-s*i) * f_z(n-s*j))
 * computed as (E_z^H holo) conj(E_z) on the tensor cores (bf16 hi+lo operands, 3 products,
 * FP32 accumulation).  Square object and hologram, object edge a multiple of 32.
 *   holo       complex64 [holo_h][holo_w]
 *   fields     complex64 [Z][obj_h][obj_w] output, or NULL (then plan scratch is used)
 *   layer_idx  uint8 [obj_h][obj_w] (needed when amplitude != NULL)
 *   amplitude  float [obj_h][obj_w] output |R_{layer(i,j)}(i,j)| (0 where layer >= Z), or NULL
 * The first call builds the plan's geometry operands (conj(E_z), E_z: 3 x 8*Z*obj*holo bytes).
 * Errors: CGH_ERR_ARG, CGH_ERR_UNSUPPORTED (geometry), CGH_ERR_NOMEM, CGH_ERR_CUDA.
 */
int cgh_reconstruct(const cgh_plan* plan, const float* holo, float* fields,
                    const uint8_t* layer_idx, float* amplitude, void* stream);

/*
 * cgh_reconstruct_batch - cgh_reconstruct of n_holo holograms in one pass: both GEMM stages
 * run once over the (hologram, layer) pairs, which fills the GPU better than n_holo calls.
 * No counterpart in the paper (the batch of phase-only holograms of the optimisation).
 *   holos      complex64 [n_holo][holo_h][holo_w]
 *   fields     complex64 [n_holo][Z][obj_h][obj_w] output, or NULL (plan scratch)
 *   layer_idx  uint8 [obj_h][obj_w], shared by the holograms (needed when amplitude != NULL)
 *   amplitude  float [n_holo][obj_h][obj_w] output, or NULL
 * 1 <= n_holo <= 64.  The plan keeps scratch for the largest batch seen: a call with a larger
 * batch than before reallocates it and synchronises `stream` (make it outside stream capture).
 * The results equal n_holo calls of cgh_reconstruct bit for bit.  Errors: as cgh_reconstruct.
 */
int cgh_reconstruct_batch(const cgh_plan* plan, const float* holos, int n_holo, float* fields,
                          const uint8_t* layer_idx, float* amplitude, void* stream);

/*
 * cgh_reconstruct_asm - reconstruction by the inverse angular spectrum method, the one the
 * paper renders its results with (Section 2, last paragraph: "inverse angular spectrum ...
 * using the same parameters of the scene").
 *   P = pad * holo edge; the hologram is zero-padded to P x P (pad 2: linear convolution),
 *   X = DFT_PxP(holo); per layer z
 *     T_z(fx, fy) = exp(-j*2*pi*z*(sqrt(1/lambda^2 - fx^2 - fy^2) - 1/lambda)),
 *     fx, fy = signed DFT index / (P*p); 0 for evanescent waves and, with band_limit = 1,
 *     for |fx| or |fy| above 1/(lambda*sqrt((2*z/(P*p))^2 + 1)) (Matsushima-Shimobaba
 *     band limit);
 *     R_z(i, j) = p^2/(lambda*z) * IDFT_PxP(X * T_z)(s*i, s*j)   (IDFT normalised by 1/P^2).
 * The carrier exp(j*2*pi*z/lambda) is left out of T_z (the holograms omit it) and the
 * p^2/(lambda*z) factor makes an unbounded point fringe reconstruct to its amplitude.
 * All arithmetic FP32: hand-written shared-memory FFTs (radix 16), the phase of T_z
 * reduced exactly in 64-bit fixed point.  Square power-of-two hologram, s in {1, 2, 4, 8},
 * P and P/s in [64, 4096].
 *   holo       complex64 [holo_h][holo_w]
 *   fields     complex64 [Z][obj_h][obj_w] output, or NULL
 *   layer_idx  uint8 [obj_h][obj_w] (needed when amplitude != NULL)
 *   amplitude  float [obj_h][obj_w] output |R_{layer(i,j)}(i,j)| (0 where layer >= Z), or NULL
 *   pad        1 or 2;  band_limit 0 or 1
 * The first call for a padding allocates the plan's buffers (8*(holo*P + P*P + Z*obj*P/s)
 * bytes) and synchronises `stream` once; later calls only enqueue.
 * Errors: CGH_ERR_ARG, CGH_ERR_UNSUPPORTED (geometry), CGH_ERR_NOMEM, CGH_ERR_CUDA.
 */
int cgh_reconstruct_asm(const cgh_plan* plan, const float* holo, float* fields, const uint8_t* layer_idx,
                        float* amplitude, int pad, int band_limit, void* stream);

/*
 * cgh_propagate - point-source hologram of complex layer fields: the adjoint of
 * cgh_reconstruct.  Paper: Eq. 1 (the superposition of point fringes, layer by layer).
 *   holo(m,n) (+)= sum_z sum_{i,j} fields[z](i,j) * f_z(m-s*i) * f_z(n-s*j)
 * = sum_z E_z F_z E_z^T on the tensor cores (bf16 hi+lo, 3 products, FP32 accumulation).
 *   fields      complex64 [Z][obj_h][obj_w];  holo complex64 [holo_h][holo_w] output
 *   accumulate  0: holo = result;  1: holo += result
 * Same geometry limits and operands as cgh_reconstruct.  Errors: as cgh_reconstruct.
 */
int cgh_propagate(const cgh_plan* plan, const float* fields, float* holo, int accumulate, void* stream);

/*
 * cgh_propagate_batch - cgh_propagate of n_holo field stacks: the first GEMM stage runs once
 * over the (hologram, layer) pairs, the second once per hologram.  No counterpart in the paper.
 *   fields  complex64 [n_holo][Z][obj_h][obj_w];  holos complex64 [n_holo][holo_h][holo_w]
 *   accumulate  0: holos = result;  1: holos += result
 * 1 <= n_holo <= 64; scratch as cgh_reconstruct_batch.  With a plan created with
 * CGH_PLAN_DETERMINISTIC the results equal n_holo calls of cgh_propagate bit for bit.
 * Errors: as cgh_reconstruct.
 */
int cgh_propagate_batch(const cgh_plan* plan, const float* fields, int n_holo, float* holos, int accumulate,
                        void* stream);

/*
 * cgh_adjoint - adjoint of the (real-input) progressive operator intensity -> hologram.
 * Paper: Eq. 3 (the hologram is linear in the object), Section 2 steps 2-5.
 * For a hologram-space cotangent G:
 *   grad_object(i,j) = [P_z Re(R_z)](i,j),  z = layer(i,j),
 * with R_z = cgh_reconstruct(G) and P_z the layer's progressive approximation: 3-level Haar
 * of Re R_z, LLL blocks outside lists[0] and detail blocks outside lists[1..3] set to zero,
 * inverse Haar (an orthogonal projection in the Haar basis, hence self-adjoint).
 *   grad_holo  complex64 [holo_h][holo_w];  lists, d_counts as for cgh_progressive_hologram
 *   layer_idx  uint8 [obj_h][obj_w];  grad_object float [obj_h][obj_w] output (0 off-layer)
 * Errors: as cgh_reconstruct.
 */
int cgh_adjoint(const cgh_plan* plan, const float* grad_holo, const int32_t* const* lists,
                const int32_t* d_counts, const uint8_t* layer_idx, float* grad_object, void* stream);

/*
 * cgh_progressive_apply - the progressive operator applied to a real-valued object: the
 * linear map whose adjoint is cgh_adjoint.  Paper: Eq. 3 (the hologram is the sum of the
 * holograms of the Haar basis functions times their coefficients), Section 2 steps 2-5.
 *   H = sum_z E_z P_z(object * [layer_idx = z]) E_z^T,   E_z[m][i] = f_z(m - s*i)
 * with P_z the layer's progressive approximation (3-level Haar, LLL blocks outside lists[0]
 * and detail blocks outside lists[1..3] set to zero, inverse Haar).  For an integer object
 * this is the hologram cgh_progressive_hologram computes; here the object may be any real
 * image, which makes the operator differentiable with respect to it.
 *   object     float [obj_h][obj_w];  layer_idx uint8 [obj_h][obj_w]
 *   lists, d_counts  as for cgh_progressive_hologram
 *   holo       complex64 [holo_h][holo_w] output;  accumulate 0: holo = H, 1: holo += H
 * Runs on the tensor cores (bf16 hi+lo, 3 products, FP32 accumulation), through the same
 * operands as cgh_propagate; uses plan scratch.  Geometry limits as cgh_reconstruct.
 * Errors: CGH_ERR_ARG, CGH_ERR_UNSUPPORTED (geometry), CGH_ERR_CUDA.
 */
int cgh_progressive_apply(const cgh_plan* plan, const float* object, const int32_t* const* lists,
                          const int32_t* d_counts, const uint8_t* layer_idx, float* holo, int accumulate,
                          void* stream);

/*
 * cgh_amplitude_backward - cotangent of the composite amplitude |R_{layer(i,j)}(i,j)| with
 * respect to the layer fields: grad_fields[z](i,j) = grad_amp(i,j) * R_z(i,j) / |R_z(i,j)|
 * where z = layer(i,j) and R_z(i,j) != 0, else 0 (real-pair convention: d/dRe + j d/dIm).
 *   fields complex64 [Z][obj_h][obj_w]; layer_idx uint8 [obj_h][obj_w]; grad_amp float
 *   [obj_h][obj_w]; grad_fields complex64 [Z][obj_h][obj_w] output.
 * The paper has no counterpart (differentiation of the reconstruction for optimisation).
 */
int cgh_amplitude_backward(const cgh_plan* plan, const float* fields, const uint8_t* layer_idx,
                           const float* grad_amp, float* grad_fields, void* stream);

/*
 * cgh_amplitude_backward_batch - cgh_amplitude_backward of n_holo field stacks (fields and
 * grad_fields [n_holo][Z][obj_h][obj_w], grad_amp [n_holo][obj_h][obj_w], one layer map).
 * No counterpart in the paper.  Errors: CGH_ERR_ARG, CGH_ERR_CUDA.
 */
int cgh_amplitude_backward_batch(const cgh_plan* plan, const float* fields, int n_holo, const uint8_t* layer_idx,
                                 const float* grad_amp, float* grad_fields, void* stream);

/*
 * cgh_phase_to_field / cgh_phase_grad - phase-only holograms: field = exp(j*phase) and, for
 * a real-pair cotangent g of the field, d/dphase = Im(g * conj(field)).  Elementwise over n
 * values (phase float[n], field / grad_field complex64 [n], grad_phase float[n]).
 * The paper has no counterpart (phase-only hologram optimisation).
 */
int cgh_phase_to_field(const float* phase, float* field, long long n, void* stream);
int cgh_phase_grad(const float* field, const float* grad_field, float* grad_phase, long long n, void* stream);

/*
 * cgh_ssim - mean SSIM of two reconstructed amplitude images, the quality measure of
 * Section 3 (Table 3: each progressive level against the fully point-wise reconstruction).
 * Wang et al. 2004 with an 11x11 Gaussian window (sigma 1.5) over the valid positions,
 * K1 = 0.01, K2 = 0.03, data range 1.
 *   x, y       device float [h][w] row-major, non-negative (amplitudes)
 *   normalize  1: each image is divided by its own maximum first (amplitudes of different
 *              holograms differ in scale); 0: used as given
 *   out_mean   device double[1], overwritten with the mean SSIM
 *   scratch    device 8 bytes (two uint32 maxima) when normalize = 1, else may be NULL
 * Stream-ordered; the caller owns every buffer.
 * Errors: CGH_ERR_ARG (NULL pointer, h or w outside [11, 65536]), CGH_ERR_CUDA.
 */
int cgh_ssim(const float* x, const float* y, int h, int w, int normalize, double* out_mean, void* scratch,
             void* stream);

/*
 * cgh_tc_selftest_gemm - diagnostic: C = A * B^T through the tensor-core machinery of the
 * separable form (TMA loads with 64-byte swizzle, shared-memory descriptors, tcgen05.mma
 * with FP32 accumulation in tensor memory), one real product, no hi+lo split.
 * The paper has no counterpart; it exists to test that machinery in isolation.
 *   A       16-bit [M][K] row-major (bf16 or fp16 bit patterns), 16-byte aligned
 *   B       16-bit [N][K] row-major, 16-byte aligned
 *   C       float [M][N] output (overwritten)
 *   K       a positive multiple of 32;  is_fp16  0 = bf16, 1 = fp16
 * Errors: CGH_ERR_ARG, CGH_ERR_CUDA.
 */
int cgh_tc_selftest_gemm(const uint16_t* A, const uint16_t* B, float* C, int M, int N, int K, int is_fp16,
                         void* stream);

/* ---- batches ----------------------------------------------------------------------- */
typedef struct cgh_batch cgh_batch;

/*
 * cgh_batch_create - many scenes, each with its own plan, run as one batch.
 * Paper: Section 2 steps 1-5 for every scene; the batch is this library's scheduling.
 * For scene k: plans[k], device inputs intensity[k], layer_idx[k], saliency[k] (uint8
 * [obj_h][obj_w] of that plan), output holos[k] (complex64 [holo_h][holo_w]), shared
 * thresholds (HOST int[3], levels 1, 2, 3).  The buffers are bound at creation and reused by
 * every cgh_batch_run (fill the inputs, run, read the outputs), so a run can be captured in
 * a CUDA graph.  form: CGH_FORM_TC_BF16X3 or CGH_FORM_TC_FP16X3.  The batch allocates the
 * per-scene coefficients and work lists and its launch tables (which take each plan's
 * contraction order as set at creation); it does not own the plans.  1 <= n <= 1024, at most
 * 65535 scene layers in all.  Holograms 16-byte aligned with an even pixel count.
 * Errors: CGH_ERR_ARG, CGH_ERR_UNSUPPORTED (form), CGH_ERR_NOMEM, CGH_ERR_CUDA.
 */
int cgh_batch_create(cgh_batch** out, cgh_plan* const* plans, int n, const uint8_t* const* intensity,
                     const uint8_t* const* layer_idx, const uint8_t* const* saliency, const int* thresholds,
                     float* const* holos, int form, void* stream);

/*
 * cgh_batch_run - enqueue one progressive hologram per scene, with a fixed number of
 * launches whatever the number of scenes: one clear of the selection flags and holograms,
 * one DWT, the three selection passes (counts, scan, ordered scatter, which also marks the
 * tensor-core flags), one compaction and one inverse-DWT operand build, each walking all
 * scenes; then ONE persistent stage-1 launch and ONE persistent stage-2 launch whose work
 * units span every scene (uneven sizes and work lists included).
 */
int cgh_batch_run(cgh_batch* batch, void* stream);

/*
 * cgh_batch_set_tuning - target number of 32-wide K steps per stage-2 work unit (splits of
 * each scene's K); synchronises the device and re-uploads the work descriptors.  Chosen by
 * the autotuner of the Python package; default 32.
 */
int cgh_batch_set_tuning(cgh_batch* batch, int ksteps_per_unit);

/*
 * cgh_batch_set_stage2_tiles - tile shape of the batch's stage-2 launch: CGH_TILES_CTA (or
 * CGH_TILES_AUTO, the default) one CTA per 128 x 128 tile, CGH_TILES_PAIR two CTAs of a
 * cluster per 256 x 128 tile (tcgen05 cta_group::2; one CTA per tile where the device holds
 * no pair).  Chosen by the autotuner of the Python package with the K steps per unit.
 * Applies to later runs (no synchronisation needed).  The paper has no counterpart.
 */
int cgh_batch_set_stage2_tiles(cgh_batch* batch, int tiles);

/* cgh_batch_lists - device pointers of scene k's work lists [4], counts int32[4][2] and
 * coefficients (owned by the batch; valid after a run has completed). */
int cgh_batch_lists(const cgh_batch* batch, int scene, int32_t** lists, int32_t** d_counts, int32_t** coeffs);

/* Frees the batch (synchronises the device first).  NULL is a no-op. */
int cgh_batch_destroy(cgh_batch* batch);

/* ---- profiling -------------------------------------------------------------------- */
/* Stage slots of cgh_profile_read. */
#define CGH_PROF_TABLES 0      /* fringe-table build                    */
#define CGH_PROF_HAAR 1        /* Haar DWT                              */
#define CGH_PROF_SELECT 2      /* block selection (all passes)          */
#define CGH_PROF_DIRECT_LUT 3  /* direct-form superposition             */
#define CGH_PROF_TC_PREP 4     /* tensor form: flags, compaction, operands */
#define CGH_PROF_TC_STAGE1 5   /* tensor form: stage-1 GEMM             */
#define CGH_PROF_TC_STAGE2 6   /* tensor form: stage-2 GEMM             */
#define CGH_PROF_PLAIN 7       /* plain point-wise kernel               */
#define CGH_PROF_RECON 8       /* reconstruction                        */
#define CGH_PROF_PROPAGATE 9   /* propagation of layer fields            */
#define CGH_PROF_ASM_FFT 10    /* angular spectrum: forward 2-D FFT      */
#define CGH_PROF_ASM_INV 11    /* angular spectrum: transfer + inverse FFTs */
#define CGH_PROF_POINTCLOUD 12 /* per-point depth direct kernel          */
#define CGH_PROF_TC_FUSED 13   /* tensor form: both GEMM stages in one launch */
#define CGH_PROF_SLOTS 14

/*
 * cgh_profile - enable (1) or disable (0) CUDA-event timing around the plan's internal
 * launches.  While enabled, every call records a start and a stop event around each stage
 * it runs, on the call's stream.  The paper has no counterpart (instrumentation).
 */
int cgh_profile(cgh_plan* plan, int enable);

/*
 * cgh_profile_read - synchronise `stream`, then write into ms[CGH_PROF_SLOTS] (host) the
 * device time in milliseconds of each stage's most recent run since profiling was enabled
 * (0 for stages that did not run), and clear the record.
 */
int cgh_profile_read(cgh_plan* plan, float* ms, void* stream);

/*
 * cgh_tc_layer_dims - synchronise `stream` and copy to host the per-layer padded compacted
 * counts used by the last tensor-form call (kr[Z], kc[Z], host arrays); zeros before the
 * first such call.  kr is along the stage-2 contraction axis (object rows, or object columns
 * when that call contracted over columns, see cgh_plan_set_contraction), kc along the other.
 * Their sums size the tensor-core GEMMs.
 */
int cgh_tc_layer_dims(const cgh_plan* plan, int* kr, int* kc, void* stream);

/*
 * cgh_probe_sfu / cgh_probe_ffma - microbenchmarks for the roofline peaks of the direct
 * kernels (the paper has no counterpart).  `grid` CTAs of 256 threads; every thread runs
 * iters x 8 independent SFU sine-cosine pairs (__sincosf on [0, 1.1]), or iters x 32 FP32
 * fused multiply-adds (16 packed FP32x2 chains); sink (device float[grid*256]) receives one
 * value per thread.  Time the call with CUDA events on `stream`: pairs (or flops = 2 x FMAs)
 * per second give the measured peak that the point-wise (or detail-basis direct) kernel is
 * compared with.  Errors: CGH_ERR_ARG (NULL sink, grid outside 1..2^20, iters outside
 * 1..2^32), CGH_ERR_CUDA.
 */
int cgh_probe_sfu(float* sink, int grid, long long iters, void* stream);
int cgh_probe_ffma(float* sink, int grid, long long iters, void* stream);

/*
 * cgh_selftest_timeout - failure-detection self-test (the paper has no counterpart).
 * Enqueues a kernel whose bounded device wait, the same one the tensor-core pipeline uses,
 * waits on a barrier that nothing completes; after limit_us microseconds (1..1000000) it
 * gives up, records CGH_ERR_TIMEOUT in the plan's status word and returns, so no GPU hangs
 * and the context stays usable.  Read the result with cgh_status.
 */
int cgh_selftest_timeout(const cgh_plan* plan, int limit_us, void* stream);

/*
 * cgh_selftest_grid_barrier - failure-detection self-test of the single-launch selection's
 * grid barrier (the paper has no counterpart).  Launches `ctas` CTAs (2 .. the number the
 * device holds at once, as for the selection) cooperatively; every CTA except absent_cta
 * crosses the same bounded grid barrier the selection uses (a plan-owned barrier word of
 * its own, cleared first; absent_cta = -1: every CTA arrives).  A CTA that crosses adds 1
 * to *d_crossed (device int32, caller-owned, not cleared here).  With a CTA absent the
 * barrier never completes: each waiting CTA gives up after limit_us microseconds
 * (1..1000000), records CGH_ERR_TIMEOUT in the plan's status word and returns, so no GPU
 * hangs.  Read the status with cgh_status.  Errors: CGH_ERR_ARG, CGH_ERR_CUDA.
 */
int cgh_selftest_grid_barrier(const cgh_plan* plan, int ctas, int absent_cta, int limit_us,
                              int32_t* d_crossed, void* stream);

/*
 * cgh_status - read and clear the plan's device status word (synchronises `stream`).
 * Bounded device-side waits that give up record CGH_ERR_TIMEOUT there instead of
 * hanging.  *status_out receives CGH_OK or the recorded code.
 */
int cgh_status(const cgh_plan* plan, int* status_out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* CGH_H */
