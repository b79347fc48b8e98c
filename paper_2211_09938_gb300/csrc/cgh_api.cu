// C ABI of libcgh: argument checking, plan lifetime, error reporting and launches.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "cgh_internal.h"

static thread_local char g_err[512] = "";

int cgh_fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

int cgh_cuda_check(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return CGH_OK;
  if (e == cudaErrorMemoryAllocation)
    return cgh_fail(CGH_ERR_NOMEM, "%s: %s", what, cudaGetErrorString(e));
  return cgh_fail(CGH_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CHECK_CUDA(expr, what)                          \
  do {                                                  \
    int _rc = cgh_cuda_check((expr), (what));           \
    if (_rc != CGH_OK) return _rc;                      \
  } while (0)

extern "C" {

const char* cgh_last_error(void) { return g_err; }

int cgh_version(void) { return 10000; }

int cgh_plan_destroy(cgh_plan* p) {
  if (!p) return CGH_OK;
  cudaDeviceSynchronize();
  if (p->prof_ev[0][0])
    for (int k = 0; k < CGH_PROF_SLOTS; ++k) {
      cudaEventDestroy(p->prof_ev[k][0]);
      cudaEventDestroy(p->prof_ev[k][1]);
    }
  tc_destroy(p);
  field_destroy(p);
  eops_destroy(p);
  asm_destroy(p);
  cudaFree(p->d_tab);
  cudaFree(p->d_f64);
  cudaFree(p->d_a_frac);
  cudaFree(p->d_a_fixed);
  cudaFree(p->d_lf_half);
  cudaFree(p->d_lf_full);
  cudaFree(p->d_status);
  cudaFree(p->d_chunk_cnt);
  cudaFree(p->d_chunk_off);
  cudaFree(p->d_sel_bar);
  cudaFree(p->d_ml_rec);
  cudaFree(p->d_ml_wt);
  free(p);
  return CGH_OK;
}

int cgh_plan_set_tuning(cgh_plan* p, int max_ksteps) {
  if (!p || max_ksteps < 0) return cgh_fail(CGH_ERR_ARG, "cgh_plan_set_tuning: bad argument");
  p->max_ksteps = max_ksteps;
  return CGH_OK;
}

int cgh_plan_set_stage2_tiles(cgh_plan* p, int tiles) {
  if (!p || tiles < CGH_TILES_AUTO || tiles > CGH_TILES_PAIR)
    return cgh_fail(CGH_ERR_ARG, "cgh_plan_set_stage2_tiles: bad argument");
  p->stage2_tiles = tiles;
  return CGH_OK;
}

int cgh_plan_stage2_tiles_used(const cgh_plan* p, int* tiles) {
  if (!p || !tiles) return cgh_fail(CGH_ERR_ARG, "cgh_plan_stage2_tiles_used: bad argument");
  *tiles = p->stage2_used;
  return CGH_OK;
}

int cgh_plan_set_fusion(cgh_plan* p, int fused) {
  if (!p || fused < 0 || fused > 1) return cgh_fail(CGH_ERR_ARG, "cgh_plan_set_fusion: bad argument");
  p->fusion = fused;
  return CGH_OK;
}

int cgh_plan_set_contraction(cgh_plan* p, int order) {
  if (!p || order < CGH_CONTRACT_AUTO || order > CGH_CONTRACT_COLS)
    return cgh_fail(CGH_ERR_ARG, "cgh_plan_set_contraction: bad argument");
  p->contraction = order;
  return CGH_OK;
}

int cgh_build_tables(cgh_plan* p, void* stream) {
  if (!p) return cgh_fail(CGH_ERR_ARG, "cgh_build_tables: plan is NULL");
  prof_mark(p, CGH_PROF_TABLES, 0, (cudaStream_t)stream);
  CHECK_CUDA(launch_build_tables(p, (cudaStream_t)stream), "cgh_build_tables launch");
  prof_mark(p, CGH_PROF_TABLES, 1, (cudaStream_t)stream);
  return CGH_OK;
}

int cgh_plan_create(cgh_plan** out, int obj_h, int obj_w, int holo_h, int holo_w, double pitch_m,
                    double wavelength_m, int n_layers, const double* z_m, int levels, int flags,
                    void* stream) {
  if (!out) return cgh_fail(CGH_ERR_ARG, "cgh_plan_create: out is NULL");
  *out = NULL;
  if (levels != CGH_LEVELS)
    return cgh_fail(CGH_ERR_UNSUPPORTED, "cgh_plan_create: levels must be 3 (got %d)", levels);
  if (obj_h < 8 || obj_w < 8 || obj_h % 8 || obj_w % 8 || obj_h > 8192 || obj_w > 8192)
    return cgh_fail(CGH_ERR_ARG, "cgh_plan_create: object %dx%d must be multiples of 8 in [8, 8192]",
                    obj_h, obj_w);
  if (holo_h <= 0 || holo_w <= 0 || holo_h % obj_h || holo_w % obj_w ||
      holo_h / obj_h != holo_w / obj_w || holo_h > 16384 || holo_w > 16384)
    return cgh_fail(CGH_ERR_ARG,
                    "cgh_plan_create: hologram %dx%d must be s*object (%dx%d) for one integer s, <= 16384",
                    holo_h, holo_w, obj_h, obj_w);
  if (!(pitch_m > 0) || !(wavelength_m > 0))
    return cgh_fail(CGH_ERR_ARG, "cgh_plan_create: pitch and wavelength must be > 0");
  if (n_layers < 1 || n_layers > CGH_MAX_LAYERS)
    return cgh_fail(CGH_ERR_ARG, "cgh_plan_create: n_layers %d outside [1, %d]", n_layers, CGH_MAX_LAYERS);
  if (!z_m) return cgh_fail(CGH_ERR_ARG, "cgh_plan_create: z_m is NULL");
  for (int k = 0; k < n_layers; ++k)
    if (!(z_m[k] > 0)) return cgh_fail(CGH_ERR_ARG, "cgh_plan_create: z[%d] must be > 0", k);
  if (flags & ~(CGH_PLAN_DETERMINISTIC | CGH_PLAN_LAYER_FACTOR))
    return cgh_fail(CGH_ERR_ARG, "cgh_plan_create: unknown flags 0x%x", flags);

  cgh_plan* p = (cgh_plan*)calloc(1, sizeof(cgh_plan));
  if (!p) return cgh_fail(CGH_ERR_NOMEM, "cgh_plan_create: host allocation failed");
  p->obj_h = obj_h;
  p->obj_w = obj_w;
  p->holo_h = holo_h;
  p->holo_w = holo_w;
  p->s = holo_h / obj_h;
  p->n_layers = n_layers;
  p->levels = levels;
  p->deterministic = (flags & CGH_PLAN_DETERMINISTIC) ? 1 : 0;
  p->layer_factor = (flags & CGH_PLAN_LAYER_FACTOR) ? 1 : 0;
  p->pitch = pitch_m;
  p->wavelength = wavelength_m;
  for (int k = 0; k < n_layers; ++k) {
    const double a = pitch_m * pitch_m / (2.0 * wavelength_m * z_m[k]);
    const double fr = a - floor(a);
    p->z[k] = z_m[k];
    p->a_frac[k] = fr;
    const double x = floor(ldexp(fr, 64) + 0.5);
    p->a_fixed[k] = x >= 18446744073709551616.0 ? 0ull : (uint64_t)x;
  }
  const int nmax = holo_h > holo_w ? holo_h : holo_w;
  const int omax = obj_h > obj_w ? obj_h : obj_w;
  p->tab_off = p->s * omax;
  p->tab_len = nmax + p->tab_off;
  cudaGetDevice(&p->device);

  int rc = CGH_OK;
#define PLAN_TRY(expr, what)                     \
  do {                                           \
    rc = cgh_cuda_check((expr), (what));         \
    if (rc != CGH_OK) {                          \
      cgh_plan_destroy(p);                       \
      return rc;                                 \
    }                                            \
  } while (0)
  PLAN_TRY(cudaMalloc(&p->d_tab, (size_t)n_layers * CGH_TAB_PER_LAYER * p->tab_len * sizeof(float2)),
           "cgh_plan_create: tables");
  p->f_len = p->tab_len + 7 * p->s;
  PLAN_TRY(cudaMalloc(&p->d_f64, (size_t)n_layers * p->f_len * sizeof(double2)), "cgh_plan_create: fringe");
  PLAN_TRY(basic_init_attributes(), "cgh_plan_create: kernel attributes");
  if (tc_init_attributes() != CGH_OK || field_init_attributes() != CGH_OK || asm_init_attributes() != CGH_OK) {
    cgh_plan_destroy(p);
    return CGH_ERR_CUDA;
  }
  PLAN_TRY(cudaMalloc(&p->d_a_frac, CGH_MAX_LAYERS * sizeof(double)), "cgh_plan_create: a_frac");
  PLAN_TRY(cudaMalloc(&p->d_a_fixed, CGH_MAX_LAYERS * sizeof(unsigned long long)), "cgh_plan_create: a_fixed");
  PLAN_TRY(cudaMalloc(&p->d_status, sizeof(int)), "cgh_plan_create: status");
  // room for the four selections of one progressive call (LLL, levels 1, 2, 3)
  p->max_chunks = select_num_chunks(obj_h, obj_w, 1) + select_num_chunks(obj_h, obj_w, 2) +
                  2 * select_num_chunks(obj_h, obj_w, 3);
  PLAN_TRY(cudaMalloc(&p->d_chunk_cnt, (size_t)n_layers * p->max_chunks * sizeof(int)),
           "cgh_plan_create: chunk counts");
  PLAN_TRY(cudaMalloc(&p->d_chunk_off, (size_t)n_layers * p->max_chunks * sizeof(int)),
           "cgh_plan_create: chunk offsets");
  PLAN_TRY(cudaMemcpy(p->d_a_frac, p->a_frac, CGH_MAX_LAYERS * sizeof(double), cudaMemcpyHostToDevice),
           "cgh_plan_create: copy a_frac");
  PLAN_TRY(cudaMemcpy(p->d_a_fixed, p->a_fixed, CGH_MAX_LAYERS * sizeof(unsigned long long),
                      cudaMemcpyHostToDevice),
           "cgh_plan_create: copy a_fixed");
  PLAN_TRY(cudaMemset(p->d_status, 0, sizeof(int)), "cgh_plan_create: status clear");
  PLAN_TRY(cudaMalloc(&p->d_sel_bar, 2 * sizeof(unsigned)), "cgh_plan_create: selection barrier");
  PLAN_TRY(cudaMemset(p->d_sel_bar, 0, 2 * sizeof(unsigned)), "cgh_plan_create: selection barrier clear");
  if (obj_h % 8 == 0 && (obj_w / 8) % 256 == 0) {  // the multi-level selection's scratch
    PLAN_TRY(cudaMalloc(&p->d_ml_rec, (size_t)(obj_h / 8) * (obj_w / 8) * sizeof(uint2)),
             "cgh_plan_create: selection records");
    PLAN_TRY(cudaMalloc(&p->d_ml_wt, (size_t)(obj_h / 8) * (obj_w / 8) / 256 * 8 * n_layers * sizeof(uint4)),
             "cgh_plan_create: selection row totals");
  }
  {
    int sms = 0;
    PLAN_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device), "cgh_plan_create: SM count");
    p->sel_coop_ctas = select_fused_ctas_per_sm() * sms;
  }
  if (p->layer_factor) {
    // c_z = exp(j 2 pi frac(z/lambda)) / z; its square root goes into the point fringe of
    // both axes (so every separable product carries c_z once), c_z itself into the
    // point-wise kernel
    double2 half[CGH_MAX_LAYERS];
    float2 full[CGH_MAX_LAYERS];
    double mag_max = 0.0;
    for (int k = 0; k < n_layers; ++k) {
      const double x = z_m[k] / wavelength_m, fr = x - floor(x);
      half[k] = make_double2(cos(M_PI * fr) / sqrt(z_m[k]), sin(M_PI * fr) / sqrt(z_m[k]));
      full[k] = make_float2((float)(cos(2.0 * M_PI * fr) / z_m[k]), (float)(sin(2.0 * M_PI * fr) / z_m[k]));
      if (1.0 / sqrt(z_m[k]) > mag_max) mag_max = 1.0 / sqrt(z_m[k]);
    }
    p->lf_extra = mag_max > 1.0 ? (int)ceil(log2(mag_max)) : 0;
    PLAN_TRY(cudaMalloc(&p->d_lf_half, n_layers * sizeof(double2)), "cgh_plan_create: layer factor");
    PLAN_TRY(cudaMalloc(&p->d_lf_full, n_layers * sizeof(float2)), "cgh_plan_create: layer factor");
    PLAN_TRY(cudaMemcpy(p->d_lf_half, half, n_layers * sizeof(double2), cudaMemcpyHostToDevice),
             "cgh_plan_create: layer factor");
    PLAN_TRY(cudaMemcpy(p->d_lf_full, full, n_layers * sizeof(float2), cudaMemcpyHostToDevice),
             "cgh_plan_create: layer factor");
  }
  PLAN_TRY(launch_build_tables(p, (cudaStream_t)stream), "cgh_plan_create: table build");
#undef PLAN_TRY
  *out = p;
  return CGH_OK;
}

int cgh_haar_decompose(const cgh_plan* p, const uint8_t* intensity, const uint8_t* layer_idx,
                       int32_t* coeffs, void* stream) {
  if (!p || !intensity || !layer_idx || !coeffs)
    return cgh_fail(CGH_ERR_ARG, "cgh_haar_decompose: NULL argument");
  if (((uintptr_t)coeffs & 15) || ((uintptr_t)intensity & 7) || ((uintptr_t)layer_idx & 7))
    return cgh_fail(CGH_ERR_ARG, "cgh_haar_decompose: coeffs must be 16-byte and inputs 8-byte aligned");
  prof_mark(p, CGH_PROF_HAAR, 0, (cudaStream_t)stream);
  CHECK_CUDA(launch_haar(p, intensity, layer_idx, coeffs, (cudaStream_t)stream), "cgh_haar_decompose");
  prof_mark(p, CGH_PROF_HAAR, 1, (cudaStream_t)stream);
  return CGH_OK;
}

int cgh_select_blocks(const cgh_plan* p, const uint8_t* saliency, const uint8_t* layer_idx,
                      int threshold, int level, int32_t* list, int32_t* d_count, int capacity,
                      void* stream) {
  if (!p || !layer_idx || !d_count || (capacity > 0 && !list))
    return cgh_fail(CGH_ERR_ARG, "cgh_select_blocks: NULL argument");
  if (level < 1 || level > CGH_LEVELS) return cgh_fail(CGH_ERR_ARG, "cgh_select_blocks: level %d not in 1..3", level);
  if (threshold < -1 || threshold > 255)
    return cgh_fail(CGH_ERR_ARG, "cgh_select_blocks: threshold %d not in -1..255", threshold);
  if (threshold >= 0 && !saliency) return cgh_fail(CGH_ERR_ARG, "cgh_select_blocks: saliency is NULL");
  if (capacity < 0) return cgh_fail(CGH_ERR_ARG, "cgh_select_blocks: capacity < 0");
  if (((uintptr_t)layer_idx & 7) || (threshold >= 0 && ((uintptr_t)saliency & 7)))
    return cgh_fail(CGH_ERR_ARG, "cgh_select_blocks: saliency and layer_idx must be 8-byte aligned");
  prof_mark(p, CGH_PROF_SELECT, 0, (cudaStream_t)stream);
  const SelCoop coop = plan_sel_coop(p);
  CHECK_CUDA(launch_select(p->obj_h, p->obj_w, p->n_layers, threshold >= 0 ? saliency : NULL, layer_idx,
                           threshold, level, list, d_count, capacity, p->d_chunk_cnt, p->d_chunk_off,
                           (cudaStream_t)stream, &coop),
             "cgh_select_blocks");
  prof_mark(p, CGH_PROF_SELECT, 1, (cudaStream_t)stream);
  return CGH_OK;
}

// The four selections of one progressive call (LLL, levels 1, 2, 3) from the host arguments.
static int progressive_tasks(const int* thresholds, int32_t* const* lists, const int* capacities, int32_t* d_counts,
                             SelTasks* T, const char* name) {
  memset(T, 0, sizeof(*T));
  T->n = 4;
  for (int k = 0; k < 4; ++k) {
    if (capacities[k] < 0) return cgh_fail(CGH_ERR_ARG, "%s: capacities[%d] < 0", name, k);
    if (capacities[k] > 0 && !lists[k]) return cgh_fail(CGH_ERR_ARG, "%s: lists[%d] is NULL", name, k);
    const int thr = k == 0 ? -1 : thresholds[k - 1];
    if (thr < -1 || thr > 255) return cgh_fail(CGH_ERR_ARG, "%s: threshold %d not in -1..255", name, thr);
    T->t[k].level = k == 0 ? CGH_LEVELS : k;
    T->t[k].threshold = thr;
    T->t[k].capacity = capacities[k];
    T->t[k].list = lists[k];
    T->t[k].count = d_counts + 2 * k;
  }
  return CGH_OK;
}

int cgh_select_progressive(const cgh_plan* p, const uint8_t* saliency, const uint8_t* layer_idx,
                           const int* thresholds, int32_t* const* lists, const int* capacities,
                           int32_t* d_counts, void* stream) {
  if (!p || !saliency || !layer_idx || !thresholds || !lists || !capacities || !d_counts)
    return cgh_fail(CGH_ERR_ARG, "cgh_select_progressive: NULL argument");
  if (((uintptr_t)layer_idx & 7) || ((uintptr_t)saliency & 7))
    return cgh_fail(CGH_ERR_ARG, "cgh_select_progressive: saliency and layer_idx must be 8-byte aligned");
  SelTasks T;
  int rc = progressive_tasks(thresholds, lists, capacities, d_counts, &T, "cgh_select_progressive");
  if (rc != CGH_OK) return rc;
  prof_mark(p, CGH_PROF_SELECT, 0, (cudaStream_t)stream);
  const SelCoop coop = plan_sel_coop(p);
  CHECK_CUDA(launch_select_tasks(p->obj_h, p->obj_w, p->n_layers, saliency, layer_idx, T, p->d_chunk_cnt,
                                 p->d_chunk_off, (cudaStream_t)stream, &coop),
             "cgh_select_progressive");
  prof_mark(p, CGH_PROF_SELECT, 1, (cudaStream_t)stream);
  return CGH_OK;
}

int cgh_progressive_step(const cgh_plan* p, const uint8_t* saliency, const uint8_t* layer_idx,
                         const int32_t* coeffs, const void* coeffs_ready, const int* thresholds,
                         int32_t* const* lists, const int* capacities, int32_t* d_counts, float* holo,
                         int accumulate, int form, void* stream) {
  if (!p || !saliency || !layer_idx || !coeffs || !thresholds || !lists || !capacities || !d_counts || !holo)
    return cgh_fail(CGH_ERR_ARG, "cgh_progressive_step: NULL argument");
  for (int k = 0; k < 4; ++k)
    if (!lists[k]) return cgh_fail(CGH_ERR_ARG, "cgh_progressive_step: lists[%d] is NULL", k);
  if (((uintptr_t)layer_idx & 7) || ((uintptr_t)saliency & 7))
    return cgh_fail(CGH_ERR_ARG, "cgh_progressive_step: saliency and layer_idx must be 8-byte aligned");
  if (((uintptr_t)holo & 7)) return cgh_fail(CGH_ERR_ARG, "cgh_progressive_step: holo must be 8-byte aligned");
  SelTasks T;
  int rc = progressive_tasks(thresholds, lists, capacities, d_counts, &T, "cgh_progressive_step");
  if (rc != CGH_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  if (form == CGH_FORM_TC_BF16X3 || form == CGH_FORM_TC_FP16X3 || form == CGH_FORM_TC_FP16X2)
    return tc_progressive_step(p, saliency, layer_idx, coeffs, (cudaEvent_t)coeffs_ready, T, lists, d_counts,
                               (float2*)holo, accumulate, form, st);
  if (form != CGH_FORM_DIRECT_LUT) return cgh_fail(CGH_ERR_UNSUPPORTED, "cgh_progressive_step: unknown form %d", form);
  rc = cgh_select_progressive(p, saliency, layer_idx, thresholds, lists, capacities, d_counts, stream);
  if (rc != CGH_OK) return rc;
  if (coeffs_ready)
    CHECK_CUDA(cudaStreamWaitEvent(st, (cudaEvent_t)coeffs_ready, 0), "cgh_progressive_step: wait for coeffs");
  return cgh_progressive_hologram(p, coeffs, lists, d_counts, holo, accumulate, form, stream);
}

int cgh_progressive_hologram(const cgh_plan* p, const int32_t* coeffs, const int32_t* const* lists,
                             const int32_t* d_counts, float* holo, int accumulate, int form,
                             void* stream) {
  if (!p || !coeffs || !lists || !d_counts || !holo)
    return cgh_fail(CGH_ERR_ARG, "cgh_progressive_hologram: NULL argument");
  for (int k = 0; k < 4; ++k)
    if (!lists[k]) return cgh_fail(CGH_ERR_ARG, "cgh_progressive_hologram: lists[%d] is NULL", k);
  if (((uintptr_t)holo & 7)) return cgh_fail(CGH_ERR_ARG, "cgh_progressive_hologram: holo must be 8-byte aligned");
  cudaStream_t st = (cudaStream_t)stream;
  if (form == CGH_FORM_DIRECT_LUT) {
    if (!accumulate)
      CHECK_CUDA(cudaMemsetAsync(holo, 0, (size_t)p->holo_h * p->holo_w * sizeof(float2), st),
                 "cgh_progressive_hologram: clear");
    prof_mark(p, CGH_PROF_DIRECT_LUT, 0, st);
    CHECK_CUDA(launch_direct_lut(p, coeffs, lists, d_counts, (float2*)holo, st), "cgh_progressive_hologram");
    prof_mark(p, CGH_PROF_DIRECT_LUT, 1, st);
    return CGH_OK;
  }
  if (form == CGH_FORM_TC_BF16X3 || form == CGH_FORM_TC_FP16X3 || form == CGH_FORM_TC_FP16X2)
    return tc_progressive(p, coeffs, lists, d_counts, (float2*)holo, accumulate, form, st);
  return cgh_fail(CGH_ERR_UNSUPPORTED, "cgh_progressive_hologram: unknown form %d", form);
}

int cgh_plain_direct(const cgh_plan* p, const uint8_t* intensity, const uint8_t* layer_idx, float* holo,
                     void* stream) {
  if (!p || !intensity || !layer_idx || !holo) return cgh_fail(CGH_ERR_ARG, "cgh_plain_direct: NULL argument");
  prof_mark(p, CGH_PROF_PLAIN, 0, (cudaStream_t)stream);
  CHECK_CUDA(launch_plain_direct(p, intensity, layer_idx, (float2*)holo, (cudaStream_t)stream),
             "cgh_plain_direct");
  prof_mark(p, CGH_PROF_PLAIN, 1, (cudaStream_t)stream);
  return CGH_OK;
}

int cgh_pointcloud_direct(const cgh_plan* p, const uint8_t* intensity, const float* depth_m, float* holo,
                          int accumulate, void* stream) {
  if (!p || !intensity || !depth_m || !holo) return cgh_fail(CGH_ERR_ARG, "cgh_pointcloud_direct: NULL argument");
  if (accumulate != 0 && accumulate != 1)
    return cgh_fail(CGH_ERR_ARG, "cgh_pointcloud_direct: accumulate %d not 0 or 1", accumulate);
  if ((uintptr_t)holo & 7) return cgh_fail(CGH_ERR_ARG, "cgh_pointcloud_direct: holo must be 8-byte aligned");
  prof_mark(p, CGH_PROF_POINTCLOUD, 0, (cudaStream_t)stream);
  CHECK_CUDA(launch_pointcloud_direct(p, intensity, depth_m, (float2*)holo, accumulate, (cudaStream_t)stream),
             "cgh_pointcloud_direct");
  prof_mark(p, CGH_PROF_POINTCLOUD, 1, (cudaStream_t)stream);
  return CGH_OK;
}

int cgh_reconstruct_batch(const cgh_plan* p, const float* holos, int n_holo, float* fields,
                          const uint8_t* layer_idx, float* amplitude, void* stream) {
  if (!p || !holos) return cgh_fail(CGH_ERR_ARG, "cgh_reconstruct: NULL argument");
  if (n_holo < 1) return cgh_fail(CGH_ERR_ARG, "cgh_reconstruct: %d holograms", n_holo);
  if (amplitude && !layer_idx) return cgh_fail(CGH_ERR_ARG, "cgh_reconstruct: amplitude needs layer_idx");
  if (!fields && !amplitude) return cgh_fail(CGH_ERR_ARG, "cgh_reconstruct: nothing to compute");
  if (((uintptr_t)holos & 7) || ((uintptr_t)fields & 7))
    return cgh_fail(CGH_ERR_ARG, "cgh_reconstruct: complex arrays must be 8-byte aligned");
  return tc_reconstruct(p, (const float2*)holos, n_holo, (float2*)fields, layer_idx, amplitude,
                        (cudaStream_t)stream);
}

int cgh_reconstruct(const cgh_plan* p, const float* holo, float* fields, const uint8_t* layer_idx,
                    float* amplitude, void* stream) {
  return cgh_reconstruct_batch(p, holo, 1, fields, layer_idx, amplitude, stream);
}

int cgh_propagate_batch(const cgh_plan* p, const float* fields, int n_holo, float* holos, int accumulate,
                        void* stream) {
  if (!p || !fields || !holos) return cgh_fail(CGH_ERR_ARG, "cgh_propagate: NULL argument");
  if (n_holo < 1) return cgh_fail(CGH_ERR_ARG, "cgh_propagate: %d holograms", n_holo);
  if (((uintptr_t)holos & 7) || ((uintptr_t)fields & 7))
    return cgh_fail(CGH_ERR_ARG, "cgh_propagate: complex arrays must be 8-byte aligned");
  return field_propagate(p, (const float2*)fields, n_holo, (float2*)holos, accumulate, (cudaStream_t)stream);
}

int cgh_propagate(const cgh_plan* p, const float* fields, float* holo, int accumulate, void* stream) {
  return cgh_propagate_batch(p, fields, 1, holo, accumulate, stream);
}

int cgh_adjoint(const cgh_plan* p, const float* grad_holo, const int32_t* const* lists, const int32_t* d_counts,
                const uint8_t* layer_idx, float* grad_object, void* stream) {
  if (!p || !grad_holo || !lists || !d_counts || !layer_idx || !grad_object)
    return cgh_fail(CGH_ERR_ARG, "cgh_adjoint: NULL argument");
  for (int k = 0; k < 4; ++k)
    if (!lists[k]) return cgh_fail(CGH_ERR_ARG, "cgh_adjoint: lists[%d] is NULL", k);
  return field_adjoint(p, (const float2*)grad_holo, lists, d_counts, layer_idx, grad_object, (cudaStream_t)stream);
}

int cgh_progressive_apply(const cgh_plan* p, const float* object, const int32_t* const* lists,
                          const int32_t* d_counts, const uint8_t* layer_idx, float* holo, int accumulate,
                          void* stream) {
  if (!p || !object || !lists || !d_counts || !layer_idx || !holo)
    return cgh_fail(CGH_ERR_ARG, "cgh_progressive_apply: NULL argument");
  for (int k = 0; k < 4; ++k)
    if (!lists[k]) return cgh_fail(CGH_ERR_ARG, "cgh_progressive_apply: lists[%d] is NULL", k);
  if ((uintptr_t)holo & 7) return cgh_fail(CGH_ERR_ARG, "cgh_progressive_apply: holo must be 8-byte aligned");
  return field_forward(p, object, lists, d_counts, layer_idx, (float2*)holo, accumulate, (cudaStream_t)stream);
}

int cgh_amplitude_backward_batch(const cgh_plan* p, const float* fields, int n_holo, const uint8_t* layer_idx,
                                 const float* grad_amp, float* grad_fields, void* stream) {
  if (!p || !fields || !layer_idx || !grad_amp || !grad_fields)
    return cgh_fail(CGH_ERR_ARG, "cgh_amplitude_backward: NULL argument");
  if (n_holo < 1) return cgh_fail(CGH_ERR_ARG, "cgh_amplitude_backward: %d holograms", n_holo);
  return field_amplitude_backward(p, (const float2*)fields, n_holo, layer_idx, grad_amp, (float2*)grad_fields,
                                  (cudaStream_t)stream);
}

int cgh_amplitude_backward(const cgh_plan* p, const float* fields, const uint8_t* layer_idx, const float* grad_amp,
                           float* grad_fields, void* stream) {
  return cgh_amplitude_backward_batch(p, fields, 1, layer_idx, grad_amp, grad_fields, stream);
}

int cgh_profile(cgh_plan* p, int enable) {
  if (!p) return cgh_fail(CGH_ERR_ARG, "cgh_profile: plan is NULL");
  if (enable && !p->prof_ev[0][0])
    for (int k = 0; k < CGH_PROF_SLOTS; ++k) {
      CHECK_CUDA(cudaEventCreate(&p->prof_ev[k][0]), "cgh_profile: event");
      CHECK_CUDA(cudaEventCreate(&p->prof_ev[k][1]), "cgh_profile: event");
    }
  p->prof_on = enable ? 1 : 0;
  for (int k = 0; k < CGH_PROF_SLOTS; ++k) p->prof_used[k] = 0;
  return CGH_OK;
}

int cgh_profile_read(cgh_plan* p, float* ms, void* stream) {
  if (!p || !ms) return cgh_fail(CGH_ERR_ARG, "cgh_profile_read: NULL argument");
  CHECK_CUDA(cudaStreamSynchronize((cudaStream_t)stream), "cgh_profile_read: sync");
  for (int k = 0; k < CGH_PROF_SLOTS; ++k) {
    ms[k] = 0.f;
    if (p->prof_used[k]) CHECK_CUDA(cudaEventElapsedTime(&ms[k], p->prof_ev[k][0], p->prof_ev[k][1]),
                                    "cgh_profile_read: elapsed");
    p->prof_used[k] = 0;
  }
  return CGH_OK;
}

int cgh_tc_layer_dims(const cgh_plan* p, int* kr, int* kc, void* stream) {
  if (!p || !kr || !kc) return cgh_fail(CGH_ERR_ARG, "cgh_tc_layer_dims: NULL argument");
  return tc_layer_dims(p, kr, kc, (cudaStream_t)stream);
}

int cgh_status(const cgh_plan* p, int* status_out, void* stream) {
  if (!p || !status_out) return cgh_fail(CGH_ERR_ARG, "cgh_status: NULL argument");
  int v = 0;
  CHECK_CUDA(cudaMemcpyAsync(&v, p->d_status, sizeof(int), cudaMemcpyDeviceToHost, (cudaStream_t)stream),
             "cgh_status: read");
  CHECK_CUDA(cudaMemsetAsync(p->d_status, 0, sizeof(int), (cudaStream_t)stream), "cgh_status: clear");
  CHECK_CUDA(cudaStreamSynchronize((cudaStream_t)stream), "cgh_status: sync");
  *status_out = v;
  return CGH_OK;
}

}  // extern "C"

extern "C" int cgh_selftest_grid_barrier(const cgh_plan* p, int ctas, int absent_cta, int limit_us,
                                         int32_t* d_crossed, void* stream) {
  if (!p || !d_crossed || limit_us < 1 || limit_us > 1000000 || ctas < 2 || absent_cta < -1 ||
      absent_cta >= ctas)
    return cgh_fail(CGH_ERR_ARG, "cgh_selftest_grid_barrier: plan or d_crossed NULL, ctas < 2, absent_cta "
                                 "outside -1..ctas-1 or limit outside 1..1000000 us");
  if (ctas > p->sel_coop_ctas)
    return cgh_fail(CGH_ERR_ARG, "cgh_selftest_grid_barrier: %d CTAs exceed the %d the device holds at once",
                    ctas, p->sel_coop_ctas);
  return cgh_cuda_check(launch_grid_barrier_selftest(p->d_sel_bar + 1, p->d_status, d_crossed, ctas,
                                                     1000ull * (unsigned long long)limit_us, absent_cta,
                                                     (cudaStream_t)stream),
                        "cgh_selftest_grid_barrier");
}
