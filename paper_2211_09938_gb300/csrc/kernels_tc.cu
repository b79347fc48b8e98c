// Separable tensor-core form of the progressive superposition (tcgen05 + TMA + TMEM).
//
// Per layer z the progressive hologram is the point-source hologram of the progressively
// reconstructed object plane A^_z (inverse Haar DWT of the LLL band and of the selected
// detail blocks), so by Eq. 1's separability
//     H = sum_z E_z A^_z E_z^T,    E_z[m][i] = f_z(m - s*i),
// which equals the detail-basis sum of Eq. 3 exactly (linearity).  Two GEMM stages:
//   stage 1 (per layer):  Y_z^T[n][k] = sum_j E_z[n][j_c] A^_z[i_k][j_c]
//                         (rows i_k / columns j_c: the 8-pixel bands of the layer's LLL blocks)
//   stage 2 (all layers): H[m][n]    += sum_kappa E_{z(kappa)}[m][i_kappa] Y^T[n][kappa]
// Operands are real planes in bf16 or fp16, each value split x = hi + lo; a real product is
// hi*hi + hi*lo + lo*hi (three MMAs) with FP32 accumulation in tensor memory; a complex
// product is four real ones (the imaginary-times-imaginary term negated through the
// instruction descriptor).  A^_z is 64x an integer <= 16320, exact in hi + lo.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "cgh_internal.h"

#define TC_BM 128
#define TC_BN 128
#define TC_BK 32                            // K elements per pipeline stage (64-byte rows)
#define TC_PLANE_BYTES (128 * TC_BK * 2)    // one 128-row plane tile: 8 KiB
#define TC_WAIT_NS 2000000000ull            // bounded waits: 2 s, then CGH_ERR_TIMEOUT

enum { KIND_TEST = 0, KIND_CR = 1, KIND_CC = 2 };
enum { EPI_H = 0, EPI_Y = 1, EPI_C = 2 };

// ------------------------------------------------------------------------------------
// PTX helpers

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t global_timer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for the phase `parity` of `bar` to complete.  Gives up after TC_WAIT_NS or when
// another role has raised the CTA's abort flag; a timeout records CGH_ERR_TIMEOUT.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                                  int* status) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_timer();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*abort_flag) return false;
    if (global_timer() - t0 > TC_WAIT_NS) {
      *abort_flag = 1;
      if (status) atomicExch(status, CGH_ERR_TIMEOUT);
      return false;
    }
  }
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1,
                                            int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor of a K-major tile with 64-byte swizzling: 128 rows of
// 64 bytes, 8-row groups 512 bytes apart (stride byte offset), version bits 46-47 = 1,
// layout type 4 (SWIZZLE_64B) in bits 61-63.  The leading byte offset is unused for
// swizzled K-major layouts (encoded 1).
__device__ __forceinline__ uint64_t sdesc_sw64(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(512 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)4 << 61);
}

// Instruction descriptor, kind::f16: D = F32 (bits 4-5 = 1), A/B type (bits 7-9, 10-12:
// 0 = F16, 1 = BF16), negate A (bit 13), both K-major (bits 15, 16 = 0), N >> 3 in bits
// 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t idesc_f16(int is_bf16, int neg_a, int M, int N) {
  return (1u << 4) | ((uint32_t)is_bf16 << 7) | ((uint32_t)is_bf16 << 10) | ((uint32_t)neg_a << 13) |
         ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
      "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
        "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
        "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
        "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
}

__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// ------------------------------------------------------------------------------------
// the GEMM kernel

struct TcGemmArgs {
  int mode;          // 1: stage 1 (grid z = layer), 2: stage 2 (grid z = K split), 0: test
  int a_rows_per_z;  // stage 1: rows of A per layer (hologram width)
  const int* kr_pad; // [Z] padded compacted row counts
  const int* kc_pad; // [Z] padded compacted column counts
  int n_layers;
  int M, N, K;       // test: sizes; stages: M and N of the output (K from the device)
  int tm, tn, tz;    // work units: M tiles x N tiles x (layers | K splits | 1)
  float scale;
  float2* H;         // EPI_H: complex output [M][N]
  int ldh;
  int h_vec4;        // H rows 16-byte aligned: add pairs of pixels with float4 atomics
  uint16_t* Y;       // EPI_Y: 4 planes [plane][M][ldy]
  long long y_plane;
  int ldy;
  float* C;          // EPI_C: real output [M][N]
  int ldc;
  int* status;
};

template <int KIND>
struct TcCfg;
template <>
struct TcCfg<KIND_TEST> {
  static constexpr int NA = 1, NB = 1, NST = 8;  // > 114 KiB: one CTA (and one TMEM owner) per SM
};
template <>
struct TcCfg<KIND_CR> {
  static constexpr int NA = 4, NB = 2, NST = 4;
};
template <>
struct TcCfg<KIND_CC> {
  static constexpr int NA = 4, NB = 4, NST = 3;
};

template <int KIND>
constexpr size_t tc_smem_bytes() {
  return (size_t)TcCfg<KIND>::NST * (TcCfg<KIND>::NA + TcCfg<KIND>::NB) * TC_PLANE_BYTES + 1024;
}

// Products of one 16-wide K slice.  Plane order of complex operands: re_hi, re_lo, im_hi,
// im_lo; of real operands: hi, lo.  Accumulator 0 holds the real part (columns 0..127 of
// the TMEM allocation), accumulator 1 the imaginary part (columns 128..255).
template <int KIND>
__device__ __forceinline__ void issue_products(uint32_t tmem, uint32_t a_base, uint32_t b_base, int kk,
                                               uint32_t id_pos, uint32_t id_neg, bool first) {
  auto A = [&](int p) { return sdesc_sw64(a_base + p * TC_PLANE_BYTES + kk * 32); };
  auto B = [&](int p) { return sdesc_sw64(b_base + p * TC_PLANE_BYTES + kk * 32); };
  const uint32_t d0 = tmem, d1 = tmem + 128;
  const uint32_t f = first ? 0u : 1u;
  if (KIND == KIND_TEST) {
    mma_f16(d0, A(0), B(0), id_pos, f);
  } else if (KIND == KIND_CR) {
    mma_f16(d0, A(0), B(0), id_pos, f);
    mma_f16(d0, A(0), B(1), id_pos, 1);
    mma_f16(d0, A(1), B(0), id_pos, 1);
    mma_f16(d1, A(2), B(0), id_pos, f);
    mma_f16(d1, A(2), B(1), id_pos, 1);
    mma_f16(d1, A(3), B(0), id_pos, 1);
  } else {
    mma_f16(d0, A(0), B(0), id_pos, f);
    mma_f16(d0, A(0), B(1), id_pos, 1);
    mma_f16(d0, A(1), B(0), id_pos, 1);
    mma_f16(d0, A(2), B(2), id_neg, 1);
    mma_f16(d0, A(2), B(3), id_neg, 1);
    mma_f16(d0, A(3), B(2), id_neg, 1);
    mma_f16(d1, A(0), B(2), id_pos, f);
    mma_f16(d1, A(0), B(3), id_pos, 1);
    mma_f16(d1, A(1), B(2), id_pos, 1);
    mma_f16(d1, A(2), B(0), id_pos, 1);
    mma_f16(d1, A(2), B(1), id_pos, 1);
    mma_f16(d1, A(3), B(0), id_pos, 1);
  }
}

template <bool F16>
__device__ __forceinline__ void split_hi_lo(float x, uint16_t& hi, uint16_t& lo) {
  if (F16) {
    const __half h = __float2half_rn(x);
    const __half l = __float2half_rn(x - __half2float(h));
    hi = __half_as_ushort(h);
    lo = __half_as_ushort(l);
  } else {
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    const __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
    hi = __bfloat16_as_ushort(h);
    lo = __bfloat16_as_ushort(l);
  }
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

struct TileInfo {
  int a_row, b_row, k_lo, nk, out_row0, out_col0, n_valid;
};

// Work unit t of the persistent grid: (mt fastest, then nt, then the layer / K split).
// Returns false for units with nothing to do; every role decodes identically.
__device__ __forceinline__ bool decode_tile(const TcGemmArgs& a, int t, const int* s_off, int ktot, TileInfo& ti) {
  const int mt = t % a.tm, r = t / a.tm, nt = r % a.tn, zz = r / a.tn;
  ti.out_row0 = mt * TC_BM;
  ti.n_valid = TC_BN;
  if (a.mode == 1) {
    const int krz = s_off[zz + 1] - s_off[zz];
    ti.n_valid = min(TC_BN, krz - nt * TC_BN);
    if (ti.n_valid <= 0) return false;
    ti.a_row = zz * a.a_rows_per_z + mt * TC_BM;
    ti.b_row = s_off[zz] + nt * TC_BN;
    ti.k_lo = 0;
    ti.nk = a.kc_pad[zz] / TC_BK;
    ti.out_col0 = s_off[zz] + nt * TC_BN;
  } else if (a.mode == 2) {
    const int nkt = ktot / TC_BK, S = a.tz;
    const int k0 = (int)((long long)nkt * zz / S), k1 = (int)((long long)nkt * (zz + 1) / S);
    ti.a_row = mt * TC_BM;
    ti.b_row = nt * TC_BN;
    ti.k_lo = k0 * TC_BK;
    ti.nk = k1 - k0;
    ti.out_col0 = nt * TC_BN;
  } else {
    ti.a_row = mt * TC_BM;
    ti.b_row = nt * TC_BN;
    ti.k_lo = 0;
    ti.nk = a.K / TC_BK;
    ti.out_col0 = nt * TC_BN;
  }
  return ti.nk > 0;
}

// Persistent warp-specialised GEMM.  Warp 0 (one lane) streams operand tiles with TMA
// through an NST-deep shared-memory ring; warp 1 owns the tensor memory (512 columns:
// two accumulator buffers of Re | Im) and one lane issues the MMAs; warps 2-5 drain a
// finished buffer (TMEM -> registers -> global) while the next tile accumulates in the
// other buffer.
template <int KIND, int EPI, bool F16>
__global__ void __launch_bounds__(192, 1) k_tc_gemm(const __grid_constant__ CUtensorMap mapA,
                                                     const __grid_constant__ CUtensorMap mapB,
                                                     const TcGemmArgs args) {
  using Cfg = TcCfg<KIND>;
  constexpr int NA = Cfg::NA, NB = Cfg::NB, NST = Cfg::NST;
  constexpr uint32_t STAGE = (NA + NB) * TC_PLANE_BYTES;
  extern __shared__ uint8_t tc_smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)tc_smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full_bar[NST], empty_bar[NST], tfull_bar[2], tempty_bar[2], done_bar;
  __shared__ uint32_t s_tmem;
  __shared__ volatile int s_abort;
  __shared__ int s_off[CGH_MAX_LAYERS + 1];

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int total = args.tm * args.tn * args.tz;

  if (threadIdx.x == 0) {
    for (int s = 0; s < NST; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull_bar[b], 1);
      mbar_init(&tempty_bar[b], 4);
    }
    mbar_init(&done_bar, 1);
    s_abort = 0;
    int o = 0;
    s_off[0] = 0;
    if (args.mode != 0)
      for (int q = 0; q < args.n_layers; ++q) s_off[q + 1] = (o += args.kr_pad[q]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(&s_tmem))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  const uint32_t smem_base = smem_u32(smem);
  const int ktot = args.mode == 2 ? s_off[args.n_layers] : 0;

  if (warp == 0) {
    if (lane == 0) {
      // ---- TMA producer
      int it = 0;
      bool issued[NST];
      uint32_t issued_ph[NST];
      for (int s = 0; s < NST; ++s) issued[s] = false, issued_ph[s] = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < total && ok; t += gridDim.x) {
        TileInfo ti;
        if (!decode_tile(args, t, s_off, ktot, ti)) continue;
        for (int kt = 0; kt < ti.nk; ++kt, ++it) {
          const int s = it % NST;
          const uint32_t ph = (uint32_t)(it / NST) & 1u;
          if (!mbar_wait_bounded(&empty_bar[s], ph ^ 1u, &s_abort, args.status)) {
            ok = false;
            break;
          }
          uint8_t* st = smem + s * STAGE;
          mbar_arrive_expect_tx(&full_bar[s], STAGE);
          tma_load_3d(st, &mapA, &full_bar[s], ti.k_lo + kt * TC_BK, ti.a_row, 0);
          tma_load_3d(st + NA * TC_PLANE_BYTES, &mapB, &full_bar[s], ti.k_lo + kt * TC_BK, ti.b_row, 0);
          issued[s] = true;
          issued_ph[s] = ph;
        }
      }
      if (s_abort) {  // let copies in flight land before shared memory goes away
        for (int s = 0; s < NST; ++s)
          if (issued[s]) {
            const uint64_t t0 = global_timer();
            while (!mbar_try_wait(&full_bar[s], issued_ph[s]) && global_timer() - t0 < TC_WAIT_NS) {
            }
          }
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      // ---- MMA issuer
      const uint32_t id_pos = idesc_f16(F16 ? 0 : 1, 0, TC_BM, TC_BN);
      const uint32_t id_neg = idesc_f16(F16 ? 0 : 1, 1, TC_BM, TC_BN);
      int it = 0, local = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < total && ok; t += gridDim.x) {
        TileInfo ti;
        if (!decode_tile(args, t, s_off, ktot, ti)) continue;
        const int buf = local & 1;
        const uint32_t use_ph = (uint32_t)(local >> 1) & 1u;
        if (!mbar_wait_bounded(&tempty_bar[buf], use_ph ^ 1u, &s_abort, args.status)) break;
        tc_fence_after();
        const uint32_t acc = tmem + buf * 256;
        for (int kt = 0; kt < ti.nk; ++kt, ++it) {
          const int s = it % NST;
          const uint32_t ph = (uint32_t)(it / NST) & 1u;
          if (!mbar_wait_bounded(&full_bar[s], ph, &s_abort, args.status)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a_base = smem_base + s * STAGE;
          const uint32_t b_base = a_base + NA * TC_PLANE_BYTES;
#pragma unroll
          for (int kk = 0; kk < TC_BK / 16; ++kk)
            issue_products<KIND>(acc, a_base, b_base, kk, id_pos, id_neg, kt == 0 && kk == 0);
          mma_commit(&empty_bar[s]);
        }
        mma_commit(&tfull_bar[buf]);
        ++local;
      }
      // every MMA issued above completes before the accumulators are released
      mma_commit(&done_bar);
      const uint64_t t0 = global_timer();
      while (!mbar_try_wait(&done_bar, 0) && global_timer() - t0 < TC_WAIT_NS) {
      }
    }
    __syncwarp();
  } else {
    // ---- epilogue warps 2..5: TMEM lane quarter (warp % 4) -> 32 output rows
    const int quarter = warp & 3;
    int local = 0;
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
      TileInfo ti;
      if (!decode_tile(args, t, s_off, ktot, ti)) continue;
      const int buf = local & 1;
      const uint32_t ph = (uint32_t)(local >> 1) & 1u;
      bool have = mbar_wait_bounded(&tfull_bar[buf], ph, &s_abort, args.status);
      have = __all_sync(0xffffffffu, have && !s_abort);  // tcgen05.ld below is warp-collective
      if (!have) break;
      tc_fence_after();
      const int row = ti.out_row0 + quarter * 32 + lane;
      const uint32_t t_lane = tmem + buf * 256 + ((uint32_t)(quarter * 32) << 16);
#pragma unroll 1
      for (int c0 = 0; c0 < TC_BN; c0 += 32) {
        uint32_t re[32], im[32];
        tmem_ld32(t_lane + c0, re);
        if (KIND != KIND_TEST) tmem_ld32(t_lane + 128 + c0, im);
        tmem_ld_wait();
        if (EPI == EPI_H) {
          if (row < args.M) {
            float2* dst = args.H + (size_t)row * args.ldh + ti.out_col0 + c0;
            const int nv = min(32, args.N - (ti.out_col0 + c0));
            if (nv == 32 && args.h_vec4) {
#pragma unroll
              for (int j = 0; j < 32; j += 2) {
                float4 v = make_float4(__uint_as_float(re[j]) * args.scale, __uint_as_float(im[j]) * args.scale,
                                       __uint_as_float(re[j + 1]) * args.scale,
                                       __uint_as_float(im[j + 1]) * args.scale);
                atomicAdd(reinterpret_cast<float4*>(dst + j), v);
              }
            } else {
#pragma unroll
              for (int j = 0; j < 32; ++j)
                if (j < nv)
                  atomicAdd(dst + j, make_float2(__uint_as_float(re[j]) * args.scale,
                                                 __uint_as_float(im[j]) * args.scale));
            }
          }
        } else if (EPI == EPI_Y) {
          if (row < args.M) {
            const int nv = min(32, ti.n_valid - c0);
            uint16_t* base = args.Y + (size_t)row * args.ldy + ti.out_col0 + c0;
            if (nv == 32) {  // 64 contiguous bytes per plane: four 16-byte stores each
              uint32_t prh[16], prl[16], pih[16], pil[16];
#pragma unroll
              for (int j = 0; j < 32; j += 2) {
                uint16_t a0, a1, b0, b1, c0h, c1h, d0, d1;
                split_hi_lo<F16>(__uint_as_float(re[j]) * args.scale, a0, b0);
                split_hi_lo<F16>(__uint_as_float(re[j + 1]) * args.scale, a1, b1);
                split_hi_lo<F16>(__uint_as_float(im[j]) * args.scale, c0h, d0);
                split_hi_lo<F16>(__uint_as_float(im[j + 1]) * args.scale, c1h, d1);
                prh[j / 2] = (uint32_t)a0 | ((uint32_t)a1 << 16);
                prl[j / 2] = (uint32_t)b0 | ((uint32_t)b1 << 16);
                pih[j / 2] = (uint32_t)c0h | ((uint32_t)c1h << 16);
                pil[j / 2] = (uint32_t)d0 | ((uint32_t)d1 << 16);
              }
              uint4* q0 = reinterpret_cast<uint4*>(base);
              uint4* q1 = reinterpret_cast<uint4*>(base + args.y_plane);
              uint4* q2 = reinterpret_cast<uint4*>(base + 2 * args.y_plane);
              uint4* q3 = reinterpret_cast<uint4*>(base + 3 * args.y_plane);
#pragma unroll
              for (int v = 0; v < 4; ++v) {
                q0[v] = make_uint4(prh[4 * v], prh[4 * v + 1], prh[4 * v + 2], prh[4 * v + 3]);
                q1[v] = make_uint4(prl[4 * v], prl[4 * v + 1], prl[4 * v + 2], prl[4 * v + 3]);
                q2[v] = make_uint4(pih[4 * v], pih[4 * v + 1], pih[4 * v + 2], pih[4 * v + 3]);
                q3[v] = make_uint4(pil[4 * v], pil[4 * v + 1], pil[4 * v + 2], pil[4 * v + 3]);
              }
            } else {
#pragma unroll
              for (int j = 0; j < 32; ++j)
                if (j < nv) {
                  uint16_t rh, rl, ih, il;
                  split_hi_lo<F16>(__uint_as_float(re[j]) * args.scale, rh, rl);
                  split_hi_lo<F16>(__uint_as_float(im[j]) * args.scale, ih, il);
                  base[j] = rh;
                  base[args.y_plane + j] = rl;
                  base[2 * args.y_plane + j] = ih;
                  base[3 * args.y_plane + j] = il;
                }
            }
          }
        } else {
          if (row < args.M) {
#pragma unroll
            for (int j = 0; j < 32; ++j)
              if (ti.out_col0 + c0 + j < args.N)
                args.C[(size_t)row * args.ldc + ti.out_col0 + c0 + j] = __uint_as_float(re[j]) * args.scale;
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty_bar[buf]);
      ++local;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
  }
}

// ------------------------------------------------------------------------------------
// operand preparation kernels

// Scratch flags: occ3 [Z][H/8][W/8] (LLL list), rowband [Z][H/8], colband [Z][W/8],
// sel_l [Z][H>>l][W>>l] for l = 1..3 (detail lists).
struct TcFlags {
  uint8_t *occ3, *rowband, *colband, *sel[4];
};

__global__ void k_tc_scatter(const int32_t* __restrict__ l0, const int32_t* __restrict__ l1,
                             const int32_t* __restrict__ l2, const int32_t* __restrict__ l3,
                             const int32_t* __restrict__ d_counts, TcFlags fl, int H, int W, int Z) {
  const int li = blockIdx.y;
  const int32_t* lst = li == 0 ? l0 : li == 1 ? l1 : li == 2 ? l2 : l3;
  const int level = li == 0 ? 3 : li;
  const int cnt = d_counts[2 * li];
  const int hl = H >> level, wl = W >> level;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < cnt; e += gridDim.x * blockDim.x) {
    const int ent = lst[e];
    const int z = (ent >> 24) & 0x7F, by = (ent >> 12) & 0xFFF, bx = ent & 0xFFF;
    if (z >= Z || by >= hl || bx >= wl) continue;  // corrupt entries add nothing
    if (li == 0) {
      fl.occ3[((size_t)z * hl + by) * wl + bx] = 1;
      fl.rowband[(size_t)z * hl + by] = 1;
      fl.colband[(size_t)z * wl + bx] = 1;
    } else {
      fl.sel[level][((size_t)z * hl + by) * wl + bx] = 1;
    }
  }
}

// Exclusive scan of 0/1 flags over up to 1024 bands (one CTA of 1024 threads).
__device__ int block_scan_flags(int f, int* s_warp, int* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned bal = __ballot_sync(0xffffffffu, f);
  const int wpre = __popc(bal & ((1u << lane) - 1u));
  if (lane == 0) s_warp[warp] = __popc(bal);
  __syncthreads();
  if (warp == 0) {
    const int v = s_warp[lane];
    int inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += t;
    }
    s_warp[lane] = inc - v;
    if (lane == 31) s_warp[32] = inc;
  }
  __syncthreads();
  const int r = s_warp[warp] + wpre;
  *total = s_warp[32];
  __syncthreads();
  return r;
}

// Per layer: compacted object rows / columns (8-pixel bands of the layer's LLL blocks),
// padded with -1 to a multiple of 32.
__global__ void __launch_bounds__(1024) k_tc_compact(TcFlags fl, int H, int W, int* __restrict__ rows,
                                                     int* __restrict__ cols, int* __restrict__ kr_pad,
                                                     int* __restrict__ kc_pad, int ld_rows, int ld_cols) {
  __shared__ int s_warp[33];
  const int z = blockIdx.x, t = threadIdx.x;
  for (int axis = 0; axis < 2; ++axis) {
    const int nb = axis == 0 ? (H >> 3) : (W >> 3);
    const uint8_t* band = axis == 0 ? fl.rowband + (size_t)z * (H >> 3) : fl.colband + (size_t)z * (W >> 3);
    int* out = axis == 0 ? rows + (size_t)z * ld_rows : cols + (size_t)z * ld_cols;
    const int f = t < nb ? band[t] : 0;
    int total;
    const int r = block_scan_flags(f, s_warp, &total);
    if (f)
      for (int q = 0; q < 8; ++q) out[8 * r + q] = 8 * t + q;
    const int cnt = 8 * total, pad = (cnt + 31) & ~31;
    if (t < pad - cnt) out[cnt + t] = -1;
    if (t == 0) (axis == 0 ? kr_pad : kc_pad)[z] = pad;
    __syncthreads();
  }
}

// 64 x A^_z at (rows[k], cols[c]) from the Haar coefficients and the selection flags:
// V = LLL + sum_{l=3,2,1} 4^(3-l) [selected] (sx X + sy Y + sx sy D), with sx = -1 for the
// right child column and sy = -1 for the lower child row of the level-l cell.  One thread
// builds 8 consecutive compacted columns: they are one 8-pixel band of the object (or all
// padding), so they share one LLL block, one level-3 block, two level-2 and four level-1
// blocks.
template <bool F16>
__global__ void k_tc_idwt(const int32_t* __restrict__ coef, TcFlags fl, const int* __restrict__ rows,
                          const int* __restrict__ cols, const int* __restrict__ kr_pad,
                          const int* __restrict__ kc_pad, int H, int W, int ld_rows, int ld_cols,
                          uint16_t* __restrict__ B1, long long b1_plane, int ldb1) {
  const int z = blockIdx.z;
  const int c = 8 * (blockIdx.x * blockDim.x + threadIdx.x);
  const int k = blockIdx.y * blockDim.y + threadIdx.y;
  if (k >= kr_pad[z] || c >= kc_pad[z]) return;
  int off = 0;
  for (int q = 0; q < z; ++q) off += kr_pad[q];
  const int i = rows[(size_t)z * ld_rows + k], j0 = cols[(size_t)z * ld_cols + c];
  int V[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) V[q] = 0;
  if (i >= 0 && j0 >= 0) {
    const int32_t* P = coef + (size_t)z * H * W;
    const int h3 = H >> 3, w3 = W >> 3, by3 = i >> 3, bx3 = j0 >> 3;
    const size_t f3 = ((size_t)z * h3 + by3) * w3 + bx3;
    if (fl.occ3[f3]) {
      const int LL = P[(size_t)by3 * W + bx3];
#pragma unroll
      for (int q = 0; q < 8; ++q) V[q] = LL;
    }
    if (fl.sel[3][f3]) {
      const int X = P[(size_t)by3 * W + w3 + bx3], Y = P[(size_t)(h3 + by3) * W + bx3],
                D = P[(size_t)(h3 + by3) * W + w3 + bx3];
      const int sy = ((i >> 2) & 1) ? -1 : 1;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int sx = (q >> 2) ? -1 : 1;
        V[q] += sx * X + sy * Y + sx * sy * D;
      }
    }
    const int h2 = H >> 2, w2 = W >> 2, by2 = i >> 2, sy2 = ((i >> 1) & 1) ? -1 : 1;
#pragma unroll
    for (int g = 0; g < 2; ++g) {
      const int bx2 = (j0 >> 2) + g;
      if (fl.sel[2][((size_t)z * h2 + by2) * w2 + bx2]) {
        const int X = P[(size_t)by2 * W + w2 + bx2], Y = P[(size_t)(h2 + by2) * W + bx2],
                  D = P[(size_t)(h2 + by2) * W + w2 + bx2];
#pragma unroll
        for (int q = 4 * g; q < 4 * g + 4; ++q) {
          const int sx = ((q >> 1) & 1) ? -1 : 1;
          V[q] += 4 * (sx * X + sy2 * Y + sx * sy2 * D);
        }
      }
    }
    const int h1 = H >> 1, w1 = W >> 1, by1 = i >> 1, sy1 = (i & 1) ? -1 : 1;
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      const int bx1 = (j0 >> 1) + g;
      if (fl.sel[1][((size_t)z * h1 + by1) * w1 + bx1]) {
        const int X = P[(size_t)by1 * W + w1 + bx1], Y = P[(size_t)(h1 + by1) * W + bx1],
                  D = P[(size_t)(h1 + by1) * W + w1 + bx1];
#pragma unroll
        for (int q = 2 * g; q < 2 * g + 2; ++q) {
          const int sx = (q & 1) ? -1 : 1;
          V[q] += 16 * (sx * X + sy1 * Y + sx * sy1 * D);
        }
      }
    }
  }
  uint32_t hi[4], lo[4];
#pragma unroll
  for (int q = 0; q < 8; q += 2) {
    uint16_t h0, l0, h1v, l1v;
    split_hi_lo<F16>((float)V[q], h0, l0);
    split_hi_lo<F16>((float)V[q + 1], h1v, l1v);
    hi[q / 2] = (uint32_t)h0 | ((uint32_t)h1v << 16);
    lo[q / 2] = (uint32_t)l0 | ((uint32_t)l1v << 16);
  }
  uint16_t* dst = B1 + (size_t)(off + k) * ldb1 + c;
  *reinterpret_cast<uint4*>(dst) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
  *reinterpret_cast<uint4*>(dst + b1_plane) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
}

// E operand planes: out[p][z*rows_per_z + r][c] = split(f_z(r - s*idx[z][c])) for c below the
// layer's padded count (idx < 0: zero).  stage 1: idx = columns, rows = hologram width;
// stage 2 (z_off_from_counts): column index off_z + c, rows = hologram height, z block 0.
template <bool F16>
__global__ void k_tc_gather_e(const float2* __restrict__ tab, int tab_len, int tab_off, int s,
                              const int* __restrict__ idx, int ld_idx, const int* __restrict__ cnt_pad,
                              int rows_out, int stage2, uint16_t* __restrict__ E, long long e_plane, int lde) {
  // one thread: 8 consecutive columns (padded counts are multiples of 32), 16-byte stores
  const int z = blockIdx.z;
  const int c = 8 * (blockIdx.x * blockDim.x + threadIdx.x);
  const int r = blockIdx.y * blockDim.y + threadIdx.y;
  if (r >= rows_out || c >= cnt_pad[z]) return;
  int col = c;
  size_t row = (size_t)z * rows_out + r;
  if (stage2) {
    int off = 0;
    for (int q = 0; q < z; ++q) off += cnt_pad[q];
    col = off + c;
    row = r;
  }
  const float2* T = tab + (size_t)(z * 4 + 0) * 2 * tab_len + tab_off + r;
  uint32_t w[4][4];
#pragma unroll
  for (int q = 0; q < 8; q += 2) {
    uint16_t h[2][4];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int i = idx[(size_t)z * ld_idx + c + q + u];
      const float2 v = i >= 0 ? T[-s * i] : make_float2(0.f, 0.f);
      split_hi_lo<F16>(v.x, h[u][0], h[u][1]);
      split_hi_lo<F16>(v.y, h[u][2], h[u][3]);
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) w[p][q / 2] = (uint32_t)h[0][p] | ((uint32_t)h[1][p] << 16);
  }
  uint16_t* dst = E + row * lde + col;
#pragma unroll
  for (int p = 0; p < 4; ++p)
    *reinterpret_cast<uint4*>(dst + p * e_plane) = make_uint4(w[p][0], w[p][1], w[p][2], w[p][3]);
}

// ------------------------------------------------------------------------------------
// host side

static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
static std::mutex g_encode_mu;

static int get_encoder() {
  std::lock_guard<std::mutex> lock(g_encode_mu);
  if (g_encode) return CGH_OK;
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
  if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
    return cgh_fail(CGH_ERR_CUDA, "cuTensorMapEncodeTiled unavailable (%s)", cudaGetErrorString(e));
  g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  return CGH_OK;
}

// 3-D map over `planes` planes of a [rows][k_alloc] 16-bit matrix; box 32 x 128 x planes,
// 64-byte swizzle (matches sdesc_sw64).
static int make_plane_map(CUtensorMap* map, const void* base, int planes, long long rows, long long k_alloc) {
  if (get_encoder() != CGH_OK) return CGH_ERR_CUDA;
  if (((uintptr_t)base & 15) || (k_alloc * 2) % 16)
    return cgh_fail(CGH_ERR_ARG, "tensor map: base must be 16-byte aligned and rows a multiple of 16 bytes");
  cuuint64_t dims[3] = {(cuuint64_t)k_alloc, (cuuint64_t)rows, (cuuint64_t)planes};
  cuuint64_t strides[2] = {(cuuint64_t)(k_alloc * 2), (cuuint64_t)(rows * k_alloc * 2)};
  cuuint32_t box[3] = {TC_BK, 128, (cuuint32_t)planes};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_UINT16, 3, const_cast<void*>(base), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return cgh_fail(CGH_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return CGH_OK;
}

template <int KIND, int EPI, bool F16>
static cudaError_t set_gemm_attr() {
  return cudaFuncSetAttribute(k_tc_gemm<KIND, EPI, F16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)tc_smem_bytes<KIND>());
}

// Shared-memory opt-in of every GEMM instantiation on the current device; called outside
// any stream capture (plan creation), so that launches inside a captured graph need no
// attribute calls.
int tc_init_attributes() {
  cudaError_t e;
  if ((e = set_gemm_attr<KIND_TEST, EPI_C, false>()) != cudaSuccess ||
      (e = set_gemm_attr<KIND_TEST, EPI_C, true>()) != cudaSuccess ||
      (e = set_gemm_attr<KIND_CR, EPI_Y, false>()) != cudaSuccess ||
      (e = set_gemm_attr<KIND_CR, EPI_Y, true>()) != cudaSuccess ||
      (e = set_gemm_attr<KIND_CC, EPI_H, false>()) != cudaSuccess ||
      (e = set_gemm_attr<KIND_CC, EPI_H, true>()) != cudaSuccess)
    return cgh_cuda_check(e, "tensor-core kernel attributes");
  return CGH_OK;
}

static int tc_num_sms();

template <int KIND, int EPI, bool F16>
static cudaError_t launch_gemm(const CUtensorMap& ma, const CUtensorMap& mb, TcGemmArgs a, dim3 tiles,
                               cudaStream_t st) {
  a.tm = (int)tiles.x;
  a.tn = (int)tiles.y;
  a.tz = (int)tiles.z;
  const long long units = (long long)a.tm * a.tn * a.tz;
  const int grid = (int)(units < tc_num_sms() ? units : tc_num_sms());
  if (grid <= 0) return cudaSuccess;
  k_tc_gemm<KIND, EPI, F16><<<grid, 192, tc_smem_bytes<KIND>(), st>>>(ma, mb, a);
  return cudaGetLastError();
}

struct cgh_tc_state {
  int kc_alloc, kr_alloc, ktot_alloc;
  uint8_t* flags;  // one block: occ3 | rowband | colband | sel1 | sel2 | sel3
  size_t flags_bytes;
  TcFlags fl;
  int *rows, *cols, *kr_pad, *kc_pad;
  uint16_t *A1, *A2, *B1, *Y;
  long long a1_plane, a2_plane, b1_plane, y_plane;
  CUtensorMap mA1, mA2, mB1, mY;
};

static int tc_ensure(const cgh_plan* pc) {
  cgh_plan* p = const_cast<cgh_plan*>(pc);
  if (p->tc) return CGH_OK;
  cgh_tc_state* t = (cgh_tc_state*)calloc(1, sizeof(cgh_tc_state));
  if (!t) return cgh_fail(CGH_ERR_NOMEM, "tensor-core state: host allocation");
  const int H = p->obj_h, W = p->obj_w, Z = p->n_layers;
  t->kc_alloc = (W + 31) & ~31;
  t->kr_alloc = (H + 31) & ~31;
  t->ktot_alloc = Z * t->kr_alloc;
  const size_t n3 = (size_t)Z * (H >> 3) * (W >> 3);
  const size_t sz_sel[4] = {0, (size_t)Z * (H >> 1) * (W >> 1), (size_t)Z * (H >> 2) * (W >> 2), n3};
  t->flags_bytes = n3 + (size_t)Z * (H >> 3) + (size_t)Z * (W >> 3) + sz_sel[1] + sz_sel[2] + sz_sel[3];
  int rc = CGH_OK;
#define TC_TRY(expr, what)                  \
  do {                                      \
    rc = cgh_cuda_check((expr), (what));    \
    if (rc != CGH_OK) goto fail;            \
  } while (0)
  TC_TRY(cudaMalloc(&t->flags, t->flags_bytes), "tensor-core scratch: flags");
  t->fl.occ3 = t->flags;
  t->fl.rowband = t->fl.occ3 + n3;
  t->fl.colband = t->fl.rowband + (size_t)Z * (H >> 3);
  t->fl.sel[0] = nullptr;
  t->fl.sel[1] = t->fl.colband + (size_t)Z * (W >> 3);
  t->fl.sel[2] = t->fl.sel[1] + sz_sel[1];
  t->fl.sel[3] = t->fl.sel[2] + sz_sel[2];
  TC_TRY(cudaMalloc(&t->rows, (size_t)Z * t->kr_alloc * sizeof(int)), "tensor-core scratch: rows");
  TC_TRY(cudaMalloc(&t->cols, (size_t)Z * t->kc_alloc * sizeof(int)), "tensor-core scratch: cols");
  TC_TRY(cudaMalloc(&t->kr_pad, CGH_MAX_LAYERS * sizeof(int)), "tensor-core scratch: kr");
  TC_TRY(cudaMalloc(&t->kc_pad, CGH_MAX_LAYERS * sizeof(int)), "tensor-core scratch: kc");
  t->a1_plane = (long long)Z * p->holo_w * t->kc_alloc;
  t->a2_plane = (long long)p->holo_h * t->ktot_alloc;
  t->b1_plane = (long long)t->ktot_alloc * t->kc_alloc;
  t->y_plane = (long long)p->holo_w * t->ktot_alloc;
  TC_TRY(cudaMalloc(&t->A1, 4 * t->a1_plane * sizeof(uint16_t)), "tensor-core scratch: A1");
  TC_TRY(cudaMalloc(&t->A2, 4 * t->a2_plane * sizeof(uint16_t)), "tensor-core scratch: A2");
  TC_TRY(cudaMalloc(&t->B1, 2 * t->b1_plane * sizeof(uint16_t)), "tensor-core scratch: B1");
  TC_TRY(cudaMalloc(&t->Y, 4 * t->y_plane * sizeof(uint16_t)), "tensor-core scratch: Y");
  if ((rc = make_plane_map(&t->mA1, t->A1, 4, (long long)Z * p->holo_w, t->kc_alloc)) != CGH_OK) goto fail;
  if ((rc = make_plane_map(&t->mB1, t->B1, 2, t->ktot_alloc, t->kc_alloc)) != CGH_OK) goto fail;
  if ((rc = make_plane_map(&t->mA2, t->A2, 4, p->holo_h, t->ktot_alloc)) != CGH_OK) goto fail;
  if ((rc = make_plane_map(&t->mY, t->Y, 4, p->holo_w, t->ktot_alloc)) != CGH_OK) goto fail;
#undef TC_TRY
  p->tc = t;
  return CGH_OK;
fail:
  p->tc = t;
  tc_destroy(p);
  return rc;
}

void tc_destroy(cgh_plan* p) {
  cgh_tc_state* t = p->tc;
  if (!t) return;
  cudaFree(t->flags);
  cudaFree(t->rows);
  cudaFree(t->cols);
  cudaFree(t->kr_pad);
  cudaFree(t->kc_pad);
  cudaFree(t->A1);
  cudaFree(t->A2);
  cudaFree(t->B1);
  cudaFree(t->Y);
  free(t);
  p->tc = nullptr;
}

static int g_tc_sms = 0;

static int tc_num_sms() {
  if (!g_tc_sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_tc_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_tc_sms <= 0) g_tc_sms = 148;
  }
  return g_tc_sms;
}

// K splits of stage 2: fill at least two waves of one CTA per SM with a small tail,
// keeping at least 8 K steps per CTA at the largest possible K.
static int stage2_splits(int tiles, int kmax_steps) {
  // units are taken round-robin by one persistent CTA per SM: pick the fewest splits that
  // give every SM at least one unit and leave under 10% of the last round idle
  const int sms = tc_num_sms();
  int best = 1;
  double best_eff = 0;
  for (int S = 1; S <= 32 && S * 4 <= kmax_steps; ++S) {
    const double rounds = (double)S * tiles / sms;
    const double eff = rounds / ceil(rounds);
    if (S * tiles >= sms && eff >= 0.9) return S;
    if (eff > best_eff + 1e-9) best_eff = eff, best = S;
  }
  return best;
}

template <bool F16>
static int tc_run(const cgh_plan* p, const int32_t* coef, const int32_t* const* lists, const int32_t* d_counts,
                  float2* holo, int accumulate, cudaStream_t st) {
  cgh_tc_state* t = p->tc;
  const int H = p->obj_h, W = p->obj_w, Z = p->n_layers;
  cudaError_t e;
#define TC_CK(expr, what)                                   \
  do {                                                      \
    int _rc = cgh_cuda_check((expr), (what));               \
    if (_rc != CGH_OK) return _rc;                          \
  } while (0)
  prof_mark(p, CGH_PROF_TC_PREP, 0, st);
  TC_CK(cudaMemsetAsync(t->flags, 0, t->flags_bytes, st), "tc: clear flags");
  k_tc_scatter<<<dim3(64, 4), 256, 0, st>>>(lists[0], lists[1], lists[2], lists[3], d_counts, t->fl, H, W, Z);
  TC_CK(cudaGetLastError(), "tc: scatter");
  k_tc_compact<<<Z, 1024, 0, st>>>(t->fl, H, W, t->rows, t->cols, t->kr_pad, t->kc_pad, t->kr_alloc, t->kc_alloc);
  TC_CK(cudaGetLastError(), "tc: compact");
  {
    dim3 blk(8, 32), grid((t->kc_alloc / 8 + 7) / 8, (t->kr_alloc + 31) / 32, Z);
    k_tc_idwt<F16><<<grid, blk, 0, st>>>(coef, t->fl, t->rows, t->cols, t->kr_pad, t->kc_pad, H, W, t->kr_alloc,
                                         t->kc_alloc, t->B1, t->b1_plane, t->kc_alloc);
    TC_CK(cudaGetLastError(), "tc: idwt");
  }
  {
    dim3 blk(8, 32), grid((t->kc_alloc / 8 + 7) / 8, (p->holo_w + 31) / 32, Z);
    k_tc_gather_e<F16><<<grid, blk, 0, st>>>(p->d_tab, p->tab_len, p->tab_off, p->s, t->cols, t->kc_alloc,
                                             t->kc_pad, p->holo_w, 0, t->A1, t->a1_plane, t->kc_alloc);
    TC_CK(cudaGetLastError(), "tc: gather E1");
    dim3 grid2((t->kr_alloc / 8 + 7) / 8, (p->holo_h + 31) / 32, Z);
    k_tc_gather_e<F16><<<grid2, blk, 0, st>>>(p->d_tab, p->tab_len, p->tab_off, p->s, t->rows, t->kr_alloc,
                                              t->kr_pad, p->holo_h, 1, t->A2, t->a2_plane, t->ktot_alloc);
    TC_CK(cudaGetLastError(), "tc: gather E2");
  }
  prof_mark(p, CGH_PROF_TC_PREP, 1, st);
  // stage 1: Y^T = E_z[:, cols] * A^_z[rows, cols]^T / 64, scaled by 2^-4 for fp16 headroom
  const float s1 = F16 ? 1.0f / 1024.0f : 1.0f / 64.0f;
  const float s2 = F16 ? 16.0f : 1.0f;
  {
    TcGemmArgs a;
    memset(&a, 0, sizeof(a));
    a.mode = 1;
    a.a_rows_per_z = p->holo_w;
    a.kr_pad = t->kr_pad;
    a.kc_pad = t->kc_pad;
    a.n_layers = Z;
    a.M = p->holo_w;
    a.N = t->ktot_alloc;
    a.scale = s1;
    a.Y = t->Y;
    a.y_plane = t->y_plane;
    a.ldy = t->ktot_alloc;
    a.status = p->d_status;
    dim3 grid((p->holo_w + TC_BM - 1) / TC_BM, (t->kr_alloc + TC_BN - 1) / TC_BN, Z);
    prof_mark(p, CGH_PROF_TC_STAGE1, 0, st);
    e = launch_gemm<KIND_CR, EPI_Y, F16>(t->mA1, t->mB1, a, grid, st);
    prof_mark(p, CGH_PROF_TC_STAGE1, 1, st);
    TC_CK(e, "tc: stage-1 GEMM");
  }
  if (!accumulate) TC_CK(cudaMemsetAsync(holo, 0, (size_t)p->holo_h * p->holo_w * sizeof(float2), st), "tc: clear");
  {
    TcGemmArgs a;
    memset(&a, 0, sizeof(a));
    a.mode = 2;
    a.kr_pad = t->kr_pad;
    a.n_layers = Z;
    a.M = p->holo_h;
    a.N = p->holo_w;
    a.scale = s2;
    a.H = holo;
    a.ldh = p->holo_w;
    a.h_vec4 = ((p->holo_w & 1) == 0) && (((uintptr_t)holo & 15) == 0);
    a.status = p->d_status;
    const int tm = (p->holo_h + TC_BM - 1) / TC_BM, tn = (p->holo_w + TC_BN - 1) / TC_BN;
    const int S = stage2_splits(tm * tn, t->ktot_alloc / TC_BK);
    prof_mark(p, CGH_PROF_TC_STAGE2, 0, st);
    e = launch_gemm<KIND_CC, EPI_H, F16>(t->mA2, t->mY, a, dim3(tm, tn, S), st);
    prof_mark(p, CGH_PROF_TC_STAGE2, 1, st);
    TC_CK(e, "tc: stage-2 GEMM");
  }
#undef TC_CK
  return CGH_OK;
}

int tc_progressive(const cgh_plan* p, const int32_t* coef, const int32_t* const* lists, const int32_t* d_counts,
                   float2* holo, int accumulate, int form, cudaStream_t st) {
  if (p->obj_h > 8192 || p->obj_w > 8192)
    return cgh_fail(CGH_ERR_UNSUPPORTED, "tensor-core form: object too large");
  int rc = tc_ensure(p);
  if (rc != CGH_OK) return rc;
  if (form == CGH_FORM_TC_FP16X3) return tc_run<true>(p, coef, lists, d_counts, holo, accumulate, st);
  return tc_run<false>(p, coef, lists, d_counts, holo, accumulate, st);
}

int tc_layer_dims(const cgh_plan* p, int* kr, int* kc, cudaStream_t st) {
  const int Z = p->n_layers;
  if (!p->tc) {
    for (int z = 0; z < Z; ++z) kr[z] = kc[z] = 0;
    return CGH_OK;
  }
  int rc = cgh_cuda_check(cudaMemcpyAsync(kr, p->tc->kr_pad, Z * sizeof(int), cudaMemcpyDeviceToHost, st),
                          "cgh_tc_layer_dims: copy");
  if (rc != CGH_OK) return rc;
  rc = cgh_cuda_check(cudaMemcpyAsync(kc, p->tc->kc_pad, Z * sizeof(int), cudaMemcpyDeviceToHost, st),
                      "cgh_tc_layer_dims: copy");
  if (rc != CGH_OK) return rc;
  return cgh_cuda_check(cudaStreamSynchronize(st), "cgh_tc_layer_dims: sync");
}

int tc_reconstruct(const cgh_plan*, const float2*, float2*, const uint8_t*, float*, cudaStream_t) {
  return cgh_fail(CGH_ERR_UNSUPPORTED, "reconstruction not built");
}

extern "C" int cgh_tc_selftest_gemm(const uint16_t* A, const uint16_t* B, float* C, int M, int N, int K,
                                    int is_fp16, void* stream) {
  if (!A || !B || !C) return cgh_fail(CGH_ERR_ARG, "cgh_tc_selftest_gemm: NULL argument");
  if (M <= 0 || N <= 0 || K <= 0 || K % TC_BK)
    return cgh_fail(CGH_ERR_ARG, "cgh_tc_selftest_gemm: M, N > 0 and K a positive multiple of 32 required");
  CUtensorMap ma, mb;
  int rc = make_plane_map(&ma, A, 1, M, K);
  if (rc != CGH_OK) return rc;
  rc = make_plane_map(&mb, B, 1, N, K);
  if (rc != CGH_OK) return rc;
  rc = tc_init_attributes();
  if (rc != CGH_OK) return rc;
  TcGemmArgs a;
  memset(&a, 0, sizeof(a));
  a.mode = 0;
  a.M = M;
  a.N = N;
  a.K = K;
  a.scale = 1.0f;
  a.C = C;
  a.ldc = N;
  a.status = nullptr;
  dim3 grid((M + TC_BM - 1) / TC_BM, (N + TC_BN - 1) / TC_BN, 1);
  cudaError_t e = is_fp16 ? launch_gemm<KIND_TEST, EPI_C, true>(ma, mb, a, grid, (cudaStream_t)stream)
                          : launch_gemm<KIND_TEST, EPI_C, false>(ma, mb, a, grid, (cudaStream_t)stream);
  return cgh_cuda_check(e, "cgh_tc_selftest_gemm");
}
