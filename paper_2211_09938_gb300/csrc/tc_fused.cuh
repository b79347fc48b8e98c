// Both GEMM stages of the separable form in one cooperative, persistent launch.
//
// Every CTA first runs its share of stage 1 (per layer: Y_z^T = E_z[:, cols] A^_z[rows,
// cols]^T, stored by TMA), publishing each finished tile in a per-layer counter, then its
// stream-K slice of stage 2 (H += sum over the concatenated layer rows of E Y^T).  Stage 2
// reads stage 1's output one layer at a time: before the first load of a K step of layer z
// the producer waits (bounded) until every stage-1 tile of layer z has been published.
// So stage 2 starts on a CTA as soon as that CTA's stage-1 tiles are done and the layers
// it needs are complete, instead of after the last stage-1 tile of the grid, and the
// second launch, its prologue and pipeline fill disappear (an option of the plan: the
// cooperative launch occupies every SM, so it cannot overlap other streams' kernels).  The launch is cooperative, so
// all CTAs are resident and the waits always end (every stage-1 tile is owned by a running
// CTA that waits for nothing in stage 1).  The hologram is cleared by every CTA at the
// start; stage 2 adds into it only after every CTA has cleared its share (a second counter).
// The counters are zeroed by the compaction kernel two launches earlier.
#pragma once
#include "tc_gemm.cuh"

__device__ __forceinline__ int ld_acquire_gpu_s32(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void fence_proxy_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

// Bounded wait until *p >= target; gives up on the CTA's abort flag or after TC_WAIT_NS
// (CGH_ERR_TIMEOUT in *status).
__device__ __forceinline__ bool wait_counter(const int* p, int target, volatile int* abort_flag, int* status) {
  if (ld_acquire_gpu_s32(p) >= target) return true;
  const uint64_t t0 = global_timer();
  while (ld_acquire_gpu_s32(p) < target) {
    __nanosleep(200);
    if (*abort_flag) return false;
    if (global_timer() - t0 > TC_WAIT_NS) {
      *abort_flag = 1;
      if (status) atomicExch(status, CGH_ERR_TIMEOUT);
      return false;
    }
  }
  return true;
}

// Stage 1 of the fused launch: the one-problem source whose finished tiles are published.
struct FusedStage1Src : TcSingleSrc {
  int* layer_done;
  __device__ bool publishes() const { return true; }
  // called by one thread once the tile's stores are complete; orders them (written through
  // the async proxy) before the counter that stage-2 loads (async proxy again) depend on
  __device__ void tile_stored(const TileInfo& ti) const {
    fence_proxy_async_global();
    __threadfence();
    atomicAdd(layer_done + ti.layer, 1);
  }
};

// Stage 2 of the fused launch: waits, per layer, for stage 1's tiles, and before its first
// output for every CTA's clearing of the hologram.
struct FusedStage2Src : TcSingleSrc {
  const int* layer_done;
  const int* zero_done;
  const int* s_need;  // stage-1 tiles per layer
  int n_ctas;
  mutable unsigned long long ready;  // layers this thread has seen complete (bits >= Z set)
  mutable bool zeroed;
  // At the first K step of a chain: wait for every layer the chain reads, then one proxy
  // fence (it orders the TMA loads that follow after the counters; a fence per layer would
  // drain the load pipeline once per layer).
  __device__ bool before_load(const TileInfo& ti, int kt, volatile int* abort_flag) const {
    if (kt != 0 || ready == ~0ull) return true;
    const int r0 = ti.k_lo, r1 = ti.k_lo + ti.nk * TC_BK;  // rows of the concatenated layers' K
    bool fresh = false;
    for (int z = 0; z < a->n_layers; ++z) {
      if (s_off[z + 1] <= r0 || s_off[z] >= r1 || ((ready >> z) & 1ull)) continue;
      if (!wait_counter(layer_done + z, s_need[z], abort_flag, a->status)) return false;
      ready |= 1ull << z;
      fresh = true;
    }
    if (fresh) fence_proxy_async_global();
    return true;
  }
  __device__ bool before_epilogue(volatile int* abort_flag) const {
    if (zeroed) return true;
    if (!wait_counter(zero_done, n_ctas, abort_flag, a->status)) return false;
    zeroed = true;
    return true;
  }
};

template <int K1, int K2>
constexpr size_t fused_smem_bytes() {
  return tc_smem_bytes<K1, EPI_Y>() > tc_smem_bytes<K2, EPI_H>() ? tc_smem_bytes<K1, EPI_Y>()
                                                                 : tc_smem_bytes<K2, EPI_H>();
}

// K1 / K2: the kinds of stage 1 (CR or CR2) and stage 2 (CC or CC2).  args1: stage-1
// arguments (mode 1, with the regions to clear); args2: stage-2 arguments (mode 2,
// stream-K).  mapA1 / mapB1: stage-1 operands; mapY: the stage-1 output (stored by stage 1,
// B operand of stage 2); mapA2: stage-2 A operand.  sync[0..Z): per-layer published
// stage-1 tiles, sync[CGH_MAX_LAYERS]: CTAs that have cleared their share.
template <int K1, int K2, bool F16>
__global__ void __launch_bounds__(192, 1) k_tc_fused(const __grid_constant__ CUtensorMap mapA1,
                                                      const __grid_constant__ CUtensorMap mapB1,
                                                      const __grid_constant__ CUtensorMap mapY,
                                                      const __grid_constant__ CUtensorMap mapA2,
                                                      const TcGemmArgs args1, const TcGemmArgs args2, int* sync) {
  constexpr int NST1 = tc_nst<K1, EPI_Y>(), NST2 = tc_nst<K2, EPI_H>();
  extern __shared__ uint8_t tc_smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)tc_smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t bar1[2 * NST1 + 5], bar2[2 * NST2 + 5];
  __shared__ uint32_t s_tmem;
  __shared__ volatile int s_abort;
  __shared__ int s_off[CGH_MAX_LAYERS + 1];
  __shared__ int s_toff[CGH_MAX_LAYERS + 1];
  __shared__ int s_kr[CGH_MAX_LAYERS];
  __shared__ int s_need[CGH_MAX_LAYERS];
  pdl_wait();
  const int Z = args1.n_layers;
  if (threadIdx.x < Z) s_kr[threadIdx.x] = args1.kr_pad[threadIdx.x];
  __syncthreads();
  if (threadIdx.x == 0) {
    int o = 0, u = 0;
    s_off[0] = 0;
    s_toff[0] = 0;
    for (int q = 0; q < Z; ++q) {
      const int kr = s_kr[q];
      s_off[q + 1] = (o += kr);
      s_toff[q + 1] = (u += args1.tm * ((kr + TC_BN - 1) / TC_BN));
      s_need[q] = s_toff[q + 1] - s_toff[q];
    }
  }
  if (threadIdx.x >= 64) {  // clear this CTA's share of the hologram and of the flags
    const long long t0 = (long long)blockIdx.x * 128 + (threadIdx.x - 64), nt = (long long)gridDim.x * 128;
#pragma unroll 1
    for (int r = 0; r < 2; ++r)
      for (long long i = t0; i < args1.zero_n[r]; i += nt) args1.zero_ptr[r][i] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(sync + CGH_MAX_LAYERS, 1);
  }
  {
    FusedStage1Src src1{{&mapA1, &mapB1, &mapY, &args1, s_off, 0, s_toff}, sync};
    tc_gemm_body<K1, EPI_Y, F16, FusedStage1Src, true, false>(src1, smem, bar1, bar1 + NST1, bar1 + 2 * NST1,
                                                               bar1 + 2 * NST1 + 2, bar1 + 2 * NST1 + 4, &s_tmem,
                                                               &s_abort);
  }
  {
    FusedStage2Src src2{{&mapA2, &mapY, &mapY, &args2, s_off, s_off[Z], s_toff}, sync, sync + CGH_MAX_LAYERS,
                        s_need, (int)gridDim.x, Z >= 64 ? 0ull : (~0ull << Z), false};
    tc_gemm_body<K2, EPI_H, F16, FusedStage2Src, false, true>(src2, smem, bar2, bar2 + NST2, bar2 + 2 * NST2,
                                                               bar2 + 2 * NST2 + 2, bar2 + 2 * NST2 + 4, &s_tmem,
                                                               &s_abort);
  }
}

template <int K1, int K2, bool F16>
static cudaError_t set_fused_attr() {
  return cudaFuncSetAttribute(k_tc_fused<K1, K2, F16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)fused_smem_bytes<K1, K2>());
}

// CTAs of the fused kernel the device holds at once (one per SM), cached per kernel.
template <int K1, int K2, bool F16>
static int fused_max_ctas() {
  static int n = -1;
  if (n < 0) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tc_fused<K1, K2, F16>, 192,
                                                      fused_smem_bytes<K1, K2>()) != cudaSuccess) {
      cudaGetLastError();
      per_sm = 0;
    }
    n = per_sm * tc_num_sms();
  }
  return n;
}

// One cooperative launch over min(SMs, what the device holds) CTAs; a2.streamk must be > 0.
// Returns cudaErrorNotSupported when the grid cannot be resident at once.
template <int K1, int K2, bool F16>
static cudaError_t launch_fused(const CUtensorMap& a1, const CUtensorMap& b1, const CUtensorMap& y,
                                const CUtensorMap& a2, TcGemmArgs g1, dim3 tiles1, TcGemmArgs g2, dim3 tiles2,
                                int* sync, cudaStream_t st) {
  g1.tm = (int)tiles1.x;
  g1.tn = (int)tiles1.y;
  g1.tz = (int)tiles1.z;
  g2.tm = (int)tiles2.x;
  g2.tn = (int)tiles2.y;
  g2.tz = (int)tiles2.z;
  const int grid = tc_num_sms();
  if (g2.streamk <= 0 || fused_max_ctas<K1, K2, F16>() < grid) return cudaErrorNotSupported;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(192);
  cfg.dynamicSmemBytes = fused_smem_bytes<K1, K2>();
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  return cudaLaunchKernelEx(&cfg, k_tc_fused<K1, K2, F16>, a1, b1, y, a2, g1, g2, sync);
}
