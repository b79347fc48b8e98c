// Allocation-free variant of the block selection (cgh_select_blocks_noalloc).
//
// Some callers cannot call cudaMalloc: an embedder whose device memory budget is fixed
// and reserved at start-up, and which must not see device memory grow afterwards, or a
// caller that shares the device with an allocator it does not own.  They cannot create
// a plan, because a plan allocates its tables and scratch.  This entry point needs no
// plan.  Its only scratch, the per-(layer, chunk) counts and offsets of the ordered
// compaction, lives in the file-scope device array below.  The array is placed in
// device memory when this module is first loaded on a device; with lazy module loading
// (the CUDA default) that can be this entry point's first call on the device, so a
// caller with a fixed budget makes one call per device at start-up.  Every GPU that has
// loaded the module keeps the array until the process exits.
#include <mutex>

#include "cgh_internal.h"

// Capacity of the shared scratch in ints: counts in the first half, offsets in the
// second.  n_layers * ceil(blocks_at_level / 256) may not exceed the half.
#define CGH_NOALLOC_HALF 262144

static __device__ __align__(256) int g_noalloc_scratch[2 * CGH_NOALLOC_HALF];

// Host-side device addresses of g_noalloc_scratch, one per device ordinal, filled by
// the first call on that device.  The array's name in host code is only a stand-in for
// the symbol and must never be handed to a kernel.  The cached address belongs to the
// device's primary context: after cudaDeviceReset the module is loaded again and the
// address may change, so the entry point must not be used after a reset in the same
// process.
#define CGH_NOALLOC_MAX_DEVICES 64
static int* g_scratch_ptr[CGH_NOALLOC_MAX_DEVICES];
static std::mutex g_scratch_mu;

static int noalloc_scratch(int** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cgh_cuda_check(e, "cgh_select_blocks_noalloc: cudaGetDevice");
  if (dev < 0 || dev >= CGH_NOALLOC_MAX_DEVICES)
    return cgh_fail(CGH_ERR_UNSUPPORTED, "cgh_select_blocks_noalloc: device ordinal %d too large", dev);
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);  // the current device is `dev`
    if (e != cudaSuccess || !p)
      return cgh_cuda_check(e != cudaSuccess ? e : cudaErrorInvalidSymbol,
                            "cgh_select_blocks_noalloc: cudaGetSymbolAddress");
    g_scratch_ptr[dev] = (int*)p;
  }
  *out = g_scratch_ptr[dev];
  return CGH_OK;
}

extern "C" int cgh_select_blocks_noalloc(const uint8_t* saliency, const uint8_t* layer_idx, int obj_h,
                                         int obj_w, int n_layers, int threshold, int level,
                                         int32_t* list, int32_t* d_count, int capacity, void* stream) {
  if (!layer_idx || !d_count || (capacity > 0 && !list))
    return cgh_fail(CGH_ERR_ARG, "cgh_select_blocks_noalloc: NULL argument");
  if (obj_h < 8 || obj_w < 8 || obj_h % 8 || obj_w % 8 || obj_h > 8192 || obj_w > 8192)
    return cgh_fail(CGH_ERR_ARG, "cgh_select_blocks_noalloc: object %dx%d must be multiples of 8 in [8, 8192]",
                    obj_h, obj_w);
  if (n_layers < 1 || n_layers > CGH_MAX_LAYERS)
    return cgh_fail(CGH_ERR_ARG, "cgh_select_blocks_noalloc: n_layers %d outside [1, %d]", n_layers,
                    CGH_MAX_LAYERS);
  if (level < 1 || level > CGH_LEVELS)
    return cgh_fail(CGH_ERR_ARG, "cgh_select_blocks_noalloc: level %d not in 1..3", level);
  if (threshold < -1 || threshold > 255)
    return cgh_fail(CGH_ERR_ARG, "cgh_select_blocks_noalloc: threshold %d not in -1..255", threshold);
  if (threshold >= 0 && !saliency)
    return cgh_fail(CGH_ERR_ARG, "cgh_select_blocks_noalloc: saliency is NULL");
  if (capacity < 0) return cgh_fail(CGH_ERR_ARG, "cgh_select_blocks_noalloc: capacity < 0");
  if (((uintptr_t)layer_idx & 7) || (threshold >= 0 && ((uintptr_t)saliency & 7)))
    return cgh_fail(CGH_ERR_ARG, "cgh_select_blocks_noalloc: saliency and layer_idx must be 8-byte aligned");
  const long long need = (long long)n_layers * select_num_chunks(obj_h, obj_w, level);
  if (need > CGH_NOALLOC_HALF)
    return cgh_fail(CGH_ERR_ARG,
                    "cgh_select_blocks_noalloc: n_layers * ceil(blocks/256) = %lld exceeds the static "
                    "scratch limit of %d (64 layers of a 2048x2048 object at level 1 just fit); use "
                    "cgh_select_blocks",
                    need, CGH_NOALLOC_HALF);
  int* scratch = nullptr;
  int rc = noalloc_scratch(&scratch);
  if (rc != CGH_OK) return rc;
  // Every count and offset the kernels read is written earlier in the same call, so
  // the contents left by a previous call need no clearing.
  return cgh_cuda_check(launch_select(obj_h, obj_w, n_layers, threshold >= 0 ? saliency : NULL, layer_idx,
                                      threshold, level, list, d_count, capacity, scratch,
                                      scratch + CGH_NOALLOC_HALF, (cudaStream_t)stream),
                        "cgh_select_blocks_noalloc");
}
