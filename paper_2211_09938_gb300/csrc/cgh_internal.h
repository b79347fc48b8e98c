// Internal declarations shared by the translation units of libcgh.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

#include "../../include/cgh.h"

#define CGH_MAX_LAYERS 64
#define CGH_LEVELS 3

// Offsets of the four tables kept per layer: level l (0..3) x kind (0 = b, 1 = w).
#define CGH_TAB_PER_LAYER 8

struct cgh_plan {
  int obj_h, obj_w, holo_h, holo_w, s, n_layers, levels;
  int deterministic;  // CGH_PLAN_DETERMINISTIC: no split-K atomics
  int layer_factor;   // CGH_PLAN_LAYER_FACTOR: keep exp(jkz)/z per layer
  int max_ksteps;     // cgh_plan_set_tuning: cap on K steps per stage-2 chain (0 = automatic)
  int contraction;    // cgh_plan_set_contraction: CGH_CONTRACT_AUTO / _ROWS / _COLS
  int stage2_tiles;   // cgh_plan_set_stage2_tiles: CGH_TILES_AUTO / _CTA / _PAIR
  int stage2_used;    // the tile shape the last two-launch separable call ran stage 2 with
  int fusion;         // cgh_plan_set_fusion(plan, 1): both GEMM stages in one cooperative launch
  double pitch, wavelength;
  double z[CGH_MAX_LAYERS];
  double a_frac[CGH_MAX_LAYERS];     // frac(a_z) in [0,1)
  uint64_t a_fixed[CGH_MAX_LAYERS];  // round(frac(a_z) * 2^64)
  int device;

  // Fringe tables: float2 tab[Z][4 levels][2 kinds][tab_len], offset d -> index d + tab_off.
  int tab_len, tab_off;
  float2* d_tab;
  double2* d_f64;  // FP64 point fringe f_z(d), d in [-(tab_off + 7s), tab_len - tab_off)
  int f_len;
  double* d_a_frac;
  unsigned long long* d_a_fixed;
  double2* d_lf_half;  // layer factor: sqrt(c_z) folded into the point fringe (null without the flag)
  float2* d_lf_full;   // layer factor c_z for the point-wise kernel (null without the flag)
  int lf_extra;        // fp16 headroom: extra power of two taken off stage 1 (>= 0)

  // Status word for bounded device waits.
  int* d_status;

  // Scratch for block compaction: per (layer, chunk) counts and offsets; the fused
  // selection's grid-barrier word and the largest grid it may launch.
  int* d_chunk_cnt;
  int* d_chunk_off;
  int max_chunks;
  unsigned* d_sel_bar;  // [0]: the fused selection's grid barrier; [1]: its self-test's
  uint2* d_ml_rec;      // multi-level selection: one record per 8x8 block (null below 2048-pixel rows)
  uint4* d_ml_wt;       // multi-level selection: row totals per (CTA, warp, layer)
  int sel_coop_ctas;

  // Separable tensor-core path (allocated lazily by the first call that needs it).
  struct cgh_tc_state* tc;
  // Reconstruction / propagation operands and scratch (allocated lazily).
  struct cgh_field_state* fs;
  // Fringe operand planes E_z by rows / columns, per dtype (allocated lazily).
  struct cgh_eops* eops;
  // Angular-spectrum reconstruction buffers (allocated lazily).
  struct cgh_asm_state* asmst;

  // CUDA-event profiling of the internal stages (cgh_profile).
  int prof_on;
  int prof_used[CGH_PROF_SLOTS];
  cudaEvent_t prof_ev[CGH_PROF_SLOTS][2];
};

// Records the start / stop event of a profiled stage when profiling is on.
static inline void prof_mark(const cgh_plan* pc, int slot, int stop, cudaStream_t st) {
  cgh_plan* p = const_cast<cgh_plan*>(pc);
  if (!p->prof_on) return;
  cudaEventRecord(p->prof_ev[slot][stop], st);
  if (stop) p->prof_used[slot] = 1;
}

// Programmatic dependent launch: a kernel launched with launch_pdl may start while its
// predecessor in the stream finishes; pdl_wait() blocks until that predecessor has
// completed and its memory is visible, pdl_trigger() lets the successor start.  Kernels
// call pdl_wait() before reading anything a predecessor wrote, and pdl_trigger() only
// after their own wait, so data written two or more kernels back is always complete when a
// kernel starts.  Both are no-ops for ordinary launches.
#ifdef __CUDACC__
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... Exp, typename... Act>
static inline cudaError_t launch_pdl(void (*k)(Exp...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                                     Act&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, std::forward<Act>(args)...);
}
#endif

#ifdef __CUDACC__
// A work list's device count, clamped to [0, cmax] (cmax: the plan's largest possible list
// at that level, layers x blocks).  A count outside that range cannot come from the
// selection; it is recorded as CGH_ERR_ARG in the plan's status word (first error wins)
// instead of being walked past the list.
__device__ __forceinline__ int clamp_list_count(int c, int cmax, int* status) {
  if (c >= 0 && c <= cmax) return c;
  if (status) atomicCAS(status, 0, CGH_ERR_ARG);
  return c < 0 ? 0 : cmax;
}
#endif

// Thread-local error message helpers (cgh_api.cu).
int cgh_fail(int code, const char* fmt, ...);
int cgh_cuda_check(cudaError_t e, const char* what);

// Chunk size (blocks) of the ordered compaction.
#define CGH_SEL_CHUNK 256

// One block selection (a level, a threshold, an output list) inside a launch.
#define SEL_FLAGS_NONE 0
#define SEL_FLAGS_LLL 1     // mark occ3 / rowband / colband (the LLL list)
#define SEL_FLAGS_DETAIL 2  // mark sel[level] (a detail list)
struct SelTask {
  int level, threshold, capacity;
  int nchunks, chunk0, cnt_off;  // filled by launch_select_tasks
  int flag_kind;                 // SEL_FLAGS_*: tensor-core flags the fused selection marks
  int32_t* list;
  int32_t* count;
};
struct SelTasks {
  SelTask t[4];
  int n;
};
// Selection scratch of a plan: the fused single-launch selection's grid-barrier word, its
// status word and the largest grid the device holds at once (0: use the three-pass
// selection); the multi-level selection's block records (two words per 8x8 block of the
// object) and its per-warp row totals (eight warps x layers x four words per CTA of 256
// blocks); null: the multi-level passes are not used.
struct SelCoop {
  unsigned* bar;
  int* status;
  int max_ctas;
  uint2* ml_rec;
  uint4* ml_wt;
};

// Kernel launchers (kernels_basic.cu).  All asynchronous on `st`.
cudaError_t launch_build_tables(const cgh_plan* p, cudaStream_t st);
cudaError_t launch_haar(const cgh_plan* p, const uint8_t* I, const uint8_t* L, int32_t* coef,
                        cudaStream_t st);
cudaError_t launch_select(int obj_h, int obj_w, int n_layers, const uint8_t* sal, const uint8_t* L,
                          int threshold, int level, int32_t* list, int32_t* d_count, int capacity,
                          int* chunk_cnt, int* chunk_off, cudaStream_t st, const SelCoop* coop = nullptr);
cudaError_t launch_direct_lut(const cgh_plan* p, const int32_t* coef, const int32_t* const* lists,
                              const int32_t* d_counts, float2* holo, cudaStream_t st);
cudaError_t launch_plain_direct(const cgh_plan* p, const uint8_t* I, const uint8_t* L, float2* holo,
                                cudaStream_t st);
cudaError_t launch_pointcloud_direct(const cgh_plan* p, const uint8_t* I, const float* depth, float2* holo,
                                     int accumulate, cudaStream_t st);
int select_num_chunks(int obj_h, int obj_w, int level);
struct TcFlags;
cudaError_t launch_select_tasks(int obj_h, int obj_w, int n_layers, const uint8_t* sal, const uint8_t* L,
                                SelTasks T, int* chunk_cnt, int* chunk_off, cudaStream_t st,
                                const SelCoop* coop = nullptr, const TcFlags* fl = nullptr,
                                bool* flags_done = nullptr);
int select_fused_ctas_per_sm();
cudaError_t launch_grid_barrier_selftest(unsigned* bar, int* status, int* crossed, int ctas,
                                         unsigned long long limit_ns, int absent, cudaStream_t st);
static inline SelCoop plan_sel_coop(const cgh_plan* p) {
  return SelCoop{p->d_sel_bar, p->d_status, p->sel_coop_ctas, p->d_ml_rec, p->d_ml_wt};
}
cudaError_t basic_init_attributes();
int tc_init_attributes();

// Selection flags of one progressive call: occ3 [Z][H/8][W/8] (LLL list), rowband
// [Z][H/8], colband [Z][W/8], sel[l] [Z][H>>l][W>>l] for l = 1..3 (detail lists).
struct TcFlags {
  uint8_t *occ3, *rowband, *colband, *sel[4];
};

// Batches (one launch per preparation kernel across scenes).
struct HaarItem {  // one (scene, layer) plane of the batched DWT
  const uint8_t* I;
  const uint8_t* L;
  int32_t* coef;
  int H, W, z;
};
struct SelTaskB {  // one selection of one scene of the batched selection
  SelTask t;       // chunk0 and cnt_off over the whole batch
  const uint8_t* sal;
  const uint8_t* L;
  int H, W, Z;
  TcFlags fl;
};
cudaError_t launch_haar_batch(const HaarItem* d_items, int n_items, int max_h, int max_w, cudaStream_t st);
cudaError_t launch_select_batch(const SelTaskB* d_tasks, int n_tasks, int total_chunks, int max_scan_blocks,
                                int* chunk_cnt, int* chunk_off, cudaStream_t st);
int select_scan_blocks(int n_layers, int nchunks);

// Separable tensor-core path (kernels_tc.cu).
int tc_progressive(const cgh_plan* p, const int32_t* coef, const int32_t* const* lists,
                   const int32_t* d_counts, float2* holo, int accumulate, int form, cudaStream_t st);
int tc_reconstruct(const cgh_plan* p, const float2* holo, int n, float2* fields, const uint8_t* L,
                   float* amp, cudaStream_t st);
void tc_destroy(cgh_plan* p);
int tc_layer_dims(const cgh_plan* p, int* kr, int* kc, cudaStream_t st);
int tc_progressive_step(const cgh_plan* p, const uint8_t* sal, const uint8_t* L, const int32_t* coef,
                        cudaEvent_t coef_ready, SelTasks T,
                        const int32_t* const* lists, const int32_t* d_counts, float2* holo, int accumulate,
                        int form, cudaStream_t st);
int tc_build_flags(const cgh_plan* p, const int32_t* const* lists, const int32_t* d_counts, TcFlags* out,
                   cudaStream_t st);

// Fields: reconstruction, propagation, adjoints (kernels_field.cu).
int field_init_attributes();
int field_propagate(const cgh_plan* p, const float2* fields, int n, float2* holo, int accumulate, cudaStream_t st);
int field_forward(const cgh_plan* p, const float* obj, const int32_t* const* lists, const int32_t* d_counts,
                  const uint8_t* L, float2* holo, int accumulate, cudaStream_t st);
int field_adjoint(const cgh_plan* p, const float2* grad_holo, const int32_t* const* lists,
                  const int32_t* d_counts, const uint8_t* L, float* grad_obj, cudaStream_t st);
int field_amplitude_backward(const cgh_plan* p, const float2* fields, int n, const uint8_t* L,
                             const float* grad_amp, float2* grad_fields, cudaStream_t st);
void field_destroy(cgh_plan* p);
struct CUtensorMap_st;
int eops_get(const cgh_plan* p, int f16, const struct CUtensorMap_st** mEZ, const struct CUtensorMap_st** mEZt,
             cudaStream_t st);
// The fringe planes' hi parts only (re_hi, im_hi), as maps over the same memory.
int eops_get_hi(const cgh_plan* p, int f16, const struct CUtensorMap_st** mEZh,
                const struct CUtensorMap_st** mEZth, cudaStream_t st);
void eops_destroy(cgh_plan* p);

// Angular-spectrum reconstruction (kernels_asm.cu).
int asm_init_attributes();
void asm_destroy(cgh_plan* p);
