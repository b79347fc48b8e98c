// tcgen05 GEMM engine shared by the tensor-core translation units of libcgh: PTX helpers,
// the persistent warp-specialised kernel and its host-side launch / tensor-map helpers.
// Every translation unit that includes it gets its own instantiations (and must opt them
// in to large shared memory with set_gemm_attr before launching).
#pragma once
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

// Operand kinds.  CR: complex fringe x real data (stage 1), CC: complex x complex (stage 2),
// both with every operand split hi + lo (three products per real product).  CR2 / CC2: the
// same with the fringe operand as its hi planes only (re_hi, im_hi) and the data operand
// hi + lo, two products per real product (fringe_hi x data_hi + fringe_hi x data_lo); the
// fringe's own rounding then bounds the error.
enum { KIND_TEST = 0, KIND_CR = 1, KIND_CC = 2, KIND_CR2 = 3, KIND_CC2 = 4 };
enum { EPI_H = 0, EPI_Y = 1, EPI_C = 2, EPI_F = 3 };

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
                                                  int* status, uint64_t limit_ns = TC_WAIT_NS) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_timer();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*abort_flag) return false;
    if (global_timer() - t0 > limit_ns) {
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
  int mode;          // 1: stage 1 (layers, compacted), 2: split K, 3: per-layer batch, 0: test
  int a_rows_per_z;  // modes 1, 3: row offset of A per layer
  int b_rows_per_z;  // mode 3: row offset of B per layer
  int out_rows_per_z, out_cols_per_z;  // mode 3: output offsets per layer
  int a_zmod, b_zdiv, b_zmod;  // mode 3, stacked problems: A's layer is zz % a_zmod and B's
                               // (zz / b_zdiv) % b_zmod (0: zz itself), zz the unit's layer
  const int* kr_pad; // [Z] padded compacted row counts
  const int* kc_pad; // [Z] padded compacted column counts
  int n_layers;
  int M, N, K;       // test: sizes; stages: M and N of the output (K from the device)
  int tm, tn, tz;    // work units: M tiles x N tiles x (layers | K splits | 1)
  int streamk;       // mode 2: equal slices of the (tile, K step) space per CTA instead of units,
                     // cut into chains of at most `streamk` K steps (tensor-memory accumulation
                     // error grows with the chain length)
  const int* a_kmap; // optional: A's K coordinate of every 32-wide K step (mode 1: per layer,
  int a_kmap_ld;     // a_kmap_ld entries apart; mode 2: one map over the concatenated K)
  float scale;
  float2* H;         // EPI_H: complex output [M][N]
  int ldh;
  int h_vec4;        // H rows 16-byte aligned: add pairs of pixels with float4 atomics
  const int* h_transposed;  // EPI_H, optional device flag: add C[m][n] into H[n][m] (square H)
  uint16_t* Y;       // EPI_Y: 4 planes [plane][M][ldy]
  long long y_plane;
  int ldy;
  int y_rows;        // EPI_Y: rows of the output tensor (the store map's row extent)
  float* C;          // EPI_C: real output [M][N]
  int ldc;
  float2* F;         // EPI_F: complex output rows (plain stores)
  int ldf;
  int* status;
  float4* zero_ptr[2];    // single-problem launches: regions the epilogue warps clear before their
  long long zero_n[2];    // first tile (float4 counts; for the next kernels or the next call)
  int a_early;            // single-problem launches: no grid of the last two wrote A or the K
                          // sizes and maps, so the first A loads may start before the wait
                          // for the previous grid
};

template <int KIND>
struct TcCfg;
template <>
struct TcCfg<KIND_TEST> {
  static constexpr int NA = 1, NB = 1;
};
template <>
struct TcCfg<KIND_CR> {
  static constexpr int NA = 4, NB = 2;
};
template <>
struct TcCfg<KIND_CC> {
  static constexpr int NA = 4, NB = 4;
};
template <>
struct TcCfg<KIND_CR2> {
  static constexpr int NA = 2, NB = 2;
};
template <>
struct TcCfg<KIND_CC2> {
  static constexpr int NA = 2, NB = 4;
};

// Epilogue staging for EPI_Y: 32-column chunks of the four output planes (128 rows x
// 64 bytes x 4 planes each), written by the epilogue warps and stored by TMA.  KIND_CR keeps
// one chunk buffer so that its operand ring gets a fourth stage (its loads, not its
// epilogue, bound it); the other kinds double-buffer the chunks.
#define TC_STAGE_Y_BYTES (4 * TC_PLANE_BYTES)
template <int KIND>
constexpr int tc_stage_y_bufs() {
  return KIND == KIND_CR || KIND == KIND_CR2 ? 1 : 2;
}

// Pipeline depth per kind and epilogue, sized so that one CTA per SM fits in shared memory
// (and owns the tensor memory): > 114 KiB, <= 227 KiB.
template <int KIND, int EPI>
constexpr int tc_nst() {
  return KIND == KIND_TEST ? 8
                           : (EPI == EPI_Y ? (KIND == KIND_CR ? 4 : KIND == KIND_CR2 ? 6 : 2)
                                           : (KIND == KIND_CR || KIND == KIND_CC2 ? 4 : 3));
}

template <int KIND, int EPI>
constexpr size_t tc_smem_bytes() {
  return (size_t)tc_nst<KIND, EPI>() * (TcCfg<KIND>::NA + TcCfg<KIND>::NB) * TC_PLANE_BYTES +
         (EPI == EPI_Y ? tc_stage_y_bufs<KIND>() * TC_STAGE_Y_BYTES : 0) + 1024;
}

__device__ __forceinline__ void tma_store_3d(const CUtensorMap* map, const void* src, int c0, int c1, int c2) {
  asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%2, %3, %4}], [%1];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(smem_u32(src)), "r"(c0), "r"(c1), "r"(c2)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read1() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// AND of `pred` over the four epilogue warps (named barrier 2), uniform result
__device__ __forceinline__ bool epi_all(bool pred) {
  uint32_t out;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "barrier.red.and.pred q, 2, 128, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(out)
      : "r"((uint32_t)pred)
      : "memory");
  return out != 0;
}
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// named barrier of the four epilogue warps (ids 0 is __syncthreads)
__device__ __forceinline__ void epi_barrier() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

// Products of one 16-wide K slice.  Plane order of complex operands: re_hi, re_lo, im_hi,
// im_lo; of real operands: hi, lo.  Accumulator 0 holds the real part (columns 0..127 of
// the TMEM allocation), accumulator 1 the imaginary part (columns 128..255).
// The descriptors of a stage's operand tiles differ from the stage's base descriptors only
// in the start-address field (address >> 4, 14 bits; shared-memory offsets stay below
// 256 KiB, so adding the tile offset >> 4 never carries out of it): one 64-bit add each,
// which keeps the single issuing thread ahead of the tensor pipe.
template <int KIND>
__device__ __forceinline__ void issue_products(uint32_t tmem, uint64_t a_desc, uint64_t b_desc, int kk,
                                               uint32_t id_pos, uint32_t id_neg, bool first) {
  auto A = [&](int p) { return a_desc + (uint64_t)((p * TC_PLANE_BYTES + kk * 32) >> 4); };
  auto B = [&](int p) { return b_desc + (uint64_t)((p * TC_PLANE_BYTES + kk * 32) >> 4); };
  const uint32_t d0 = tmem, d1 = tmem + 128;
  const uint32_t f = first ? 0u : 1u;
  if (KIND == KIND_TEST) {
    mma_f16(d0, A(0), B(0), id_pos, f);
  } else if (KIND == KIND_CR2) {
    // A: re_hi, im_hi; B: hi, lo
    mma_f16(d0, A(0), B(0), id_pos, f);
    mma_f16(d0, A(0), B(1), id_pos, 1);
    mma_f16(d1, A(1), B(0), id_pos, f);
    mma_f16(d1, A(1), B(1), id_pos, 1);
  } else if (KIND == KIND_CC2) {
    // A: re_hi, im_hi; B: re_hi, re_lo, im_hi, im_lo
    mma_f16(d0, A(0), B(0), id_pos, f);
    mma_f16(d0, A(0), B(1), id_pos, 1);
    mma_f16(d0, A(1), B(2), id_neg, 1);
    mma_f16(d0, A(1), B(3), id_neg, 1);
    mma_f16(d1, A(0), B(2), id_pos, f);
    mma_f16(d1, A(0), B(3), id_pos, 1);
    mma_f16(d1, A(1), B(0), id_pos, 1);
    mma_f16(d1, A(1), B(1), id_pos, 1);
  } else if (KIND == KIND_CR) {
    // the two accumulators' products interleaved (each accumulator's own order unchanged),
    // so that consecutive MMAs never depend on each other's result
    mma_f16(d0, A(0), B(0), id_pos, f);
    mma_f16(d1, A(2), B(0), id_pos, f);
    mma_f16(d0, A(0), B(1), id_pos, 1);
    mma_f16(d1, A(2), B(1), id_pos, 1);
    mma_f16(d0, A(1), B(0), id_pos, 1);
    mma_f16(d1, A(3), B(0), id_pos, 1);
  } else {
    mma_f16(d0, A(0), B(0), id_pos, f);
    mma_f16(d1, A(0), B(2), id_pos, f);
    mma_f16(d0, A(0), B(1), id_pos, 1);
    mma_f16(d1, A(0), B(3), id_pos, 1);
    mma_f16(d0, A(1), B(0), id_pos, 1);
    mma_f16(d1, A(1), B(2), id_pos, 1);
    mma_f16(d0, A(2), B(2), id_neg, 1);
    mma_f16(d1, A(2), B(0), id_pos, 1);
    mma_f16(d0, A(2), B(3), id_neg, 1);
    mma_f16(d1, A(2), B(1), id_pos, 1);
    mma_f16(d0, A(3), B(2), id_neg, 1);
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
  int a_row, b_row, k_lo, nk, out_row0, out_col0, n_valid, row_lim, col_lim, item;
  int layer;       // mode 1: the tile's layer
  const int* akm;  // A's K coordinate per K step of this tile, or null (= k_lo + 32 kt)
};

// Work unit t of the persistent grid: (mt fastest, then nt, then the layer / K split).
// Returns false for units with nothing to do; every role decodes identically.
// Mode 1 (per layer, compacted): tile (mt, nt) of layer zz.
__device__ __forceinline__ bool decode_stage1(const TcGemmArgs& a, int mt, int nt, int zz, const int* s_off,
                                              TileInfo& ti) {
  const int krz = s_off[zz + 1] - s_off[zz];
  ti.n_valid = min(TC_BN, krz - nt * TC_BN);
  if (ti.n_valid <= 0) return false;
  ti.layer = zz;
  ti.a_row = zz * a.a_rows_per_z + mt * TC_BM;
  ti.b_row = s_off[zz] + nt * TC_BN;
  ti.k_lo = 0;
  ti.nk = __ldcg(a.kc_pad + zz) / TC_BK;
  ti.out_col0 = s_off[zz] + nt * TC_BN;
  ti.col_lim = ti.out_col0 + ti.n_valid;
  if (a.a_kmap) ti.akm = a.a_kmap + (size_t)zz * a.a_kmap_ld;
  return ti.nk > 0;
}

__device__ __forceinline__ bool decode_tile(const TcGemmArgs& a, int t, const int* s_off, int ktot, TileInfo& ti) {
  const int mt = t % a.tm, r = t / a.tm, nt = r % a.tn, zz = r / a.tn;
  ti.out_row0 = mt * TC_BM;
  ti.n_valid = TC_BN;
  ti.row_lim = a.M;
  ti.col_lim = a.N;
  ti.akm = nullptr;
  if (a.mode == 3) {
    const int za = a.a_zmod ? zz % a.a_zmod : zz;
    int zb = a.b_zdiv ? zz / a.b_zdiv : zz;
    if (a.b_zmod) zb %= a.b_zmod;
    ti.a_row = za * a.a_rows_per_z + mt * TC_BM;
    ti.b_row = zb * a.b_rows_per_z + nt * TC_BN;
    ti.k_lo = 0;
    ti.nk = a.K / TC_BK;
    ti.out_row0 = zz * a.out_rows_per_z + mt * TC_BM;
    ti.out_col0 = zz * a.out_cols_per_z + nt * TC_BN;
    ti.row_lim = zz * a.out_rows_per_z + a.M;
    ti.col_lim = zz * a.out_cols_per_z + a.N;
    ti.n_valid = min(TC_BN, ti.col_lim - ti.out_col0);
    return ti.nk > 0 && ti.n_valid > 0;
  }
  if (a.mode == 1) {
    return decode_stage1(a, mt, nt, zz, s_off, ti);
  } else if (a.mode == 2) {
    const int nkt = ktot / TC_BK, S = a.tz;
    const int k0 = (int)((long long)nkt * zz / S), k1 = (int)((long long)nkt * (zz + 1) / S);
    ti.a_row = mt * TC_BM;
    ti.b_row = nt * TC_BN;
    ti.k_lo = k0 * TC_BK;
    ti.nk = k1 - k0;
    ti.out_col0 = nt * TC_BN;
    if (a.a_kmap) ti.akm = a.a_kmap + k0;
  } else {
    ti.a_row = mt * TC_BM;
    ti.b_row = nt * TC_BN;
    ti.k_lo = 0;
    ti.nk = a.K / TC_BK;
    ti.out_col0 = nt * TC_BN;
  }
  return ti.nk > 0;
}

// Barriers of an NST-deep ring, the two accumulator buffers and the drain, and (ALLOC) the
// 512 tensor-memory columns, then a CTA barrier.  Touches nothing another grid writes.
template <int NST, bool ALLOC>
__device__ __forceinline__ void tc_gemm_setup(uint64_t* full_bar, uint64_t* empty_bar, uint64_t* tfull_bar,
                                              uint64_t* tempty_bar, uint64_t* done_bar, uint32_t* s_tmem_p,
                                              volatile int* s_abort_p) {
  if (threadIdx.x == 0) {
    for (int s = 0; s < NST; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull_bar[b], 1);
      mbar_init(&tempty_bar[b], 4);
    }
    mbar_init(done_bar, 1);
    *s_abort_p = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (ALLOC && (threadIdx.x >> 5) == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(s_tmem_p))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
}

// Persistent warp-specialised GEMM.  Warp 0 (one lane) streams operand tiles with TMA
// through an NST-deep shared-memory ring; warp 1 owns the tensor memory (512 columns:
// two accumulator buffers of Re | Im) and one lane issues the MMAs; warps 2-5 drain a
// finished buffer (TMEM -> registers -> global) while the next tile accumulates in the
// other buffer.
// TMEM: ALLOC allocates the 512 columns at the start (else *s_tmem_p holds an allocation
// made earlier in the kernel), DEALLOC frees them at the end (else they stay allocated for
// a later body in the same kernel).  SETUP: the body initialises its barriers, allocates and
// then waits for the previous grid; else the kernel has done the first two (tc_gemm_setup)
// and, with EARLY, every role waits for the previous grid itself: the producer first issues
// the A loads of its first ring stages when src.a_early() (A and the K maps come from grids
// two or more back), and the epilogue warps clear src's regions (src.zero_idle) after the wait.  Hooks of the source: before_load(ti, kt) runs in the
// producer before the loads of K step kt (it may wait, bounded, for inputs that other CTAs
// produce; false aborts), before_epilogue() before a tile's output is written (false
// aborts), tile_stored(ti) after a tile's EPI_Y stores are complete and visible.
template <int KIND, int EPI, bool F16, class Src, bool ALLOC = true, bool DEALLOC = true, bool SETUP = true,
          bool EARLY = false>
__device__ __forceinline__ void tc_gemm_body(const Src& src, uint8_t* smem, uint64_t* full_bar, uint64_t* empty_bar,
                                             uint64_t* tfull_bar, uint64_t* tempty_bar, uint64_t* done_bar,
                                             uint32_t* s_tmem_p, volatile int* s_abort_p) {
  using Cfg = TcCfg<KIND>;
  constexpr int NA = Cfg::NA, NB = Cfg::NB, NST = tc_nst<KIND, EPI>();
  constexpr uint32_t STAGE = (NA + NB) * TC_PLANE_BYTES;
  volatile int& s_abort = *s_abort_p;
  uint8_t* const stage_y = smem + NST * STAGE;  // EPI_Y staging (tc_stage_y_bufs x TC_STAGE_Y_BYTES)
  constexpr int YBUFS = tc_stage_y_bufs<KIND>();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int* const status = src.status();

  if constexpr (SETUP) {
    tc_gemm_setup<NST, ALLOC>(full_bar, empty_bar, tfull_bar, tempty_bar, done_bar, s_tmem_p, s_abort_p);
    pdl_wait();  // barriers and tensor memory are set up; operands may now be read
  }
  const uint32_t tmem = *s_tmem_p;
  const uint32_t smem_base = smem_u32(smem);

  if (EARLY && warp != 0) {
    pdl_wait();
    pdl_trigger();
  }
  if (warp == 0) {
    if (EARLY && lane != 0) {
      pdl_wait();
      pdl_trigger();
    }
    if (lane == 0) {
      // ---- TMA producer
      int it = 0;
      bool issued[NST];
      uint32_t issued_ph[NST];
      for (int s = 0; s < NST; ++s) issued[s] = false, issued_ph[s] = 0;
      bool ok = true;
      TileInfo ti;
      // EARLY: the A halves of the first tile's first ring stages (fresh barriers: no wait
      // for a free slot) go out before the wait for the previous grid
      int npre = 0;
      if constexpr (EARLY) {
        if (src.a_early()) {
          int c0 = src.begin();
          if (src.next(c0, ti)) {
            const CUtensorMap* mA = src.mapA(ti);
            npre = min(NST, ti.nk);
            for (int kt = 0; kt < npre; ++kt) {
              mbar_arrive_expect_tx(&full_bar[kt], STAGE);
              tma_load_3d(smem + kt * STAGE, mA, &full_bar[kt], ti.akm ? __ldcg(ti.akm + kt) : ti.k_lo + kt * TC_BK,
                          ti.a_row, 0);
              issued[kt] = true;
            }
          }
        }
        pdl_wait();
        pdl_trigger();
      }
      for (int cur = src.begin(); ok && src.next(cur, ti);) {
        const CUtensorMap* mA = src.mapA(ti);
        const CUtensorMap* mB = src.mapB(ti);
        src.acquire_maps(mA, mB);
        for (int kt = 0; kt < ti.nk; ++kt, ++it) {
          const int s = it % NST;
          const uint32_t ph = (uint32_t)(it / NST) & 1u;
          const bool pre = it < npre;  // A already in flight, barrier armed
          if ((!pre && !mbar_wait_bounded(&empty_bar[s], ph ^ 1u, &s_abort, status)) ||
              !src.before_load(ti, kt, &s_abort)) {
            ok = false;
            break;
          }
          uint8_t* st = smem + s * STAGE;
          if (!pre) {
            mbar_arrive_expect_tx(&full_bar[s], STAGE);
            tma_load_3d(st, mA, &full_bar[s], ti.akm ? ti.akm[kt] : ti.k_lo + kt * TC_BK, ti.a_row, 0);
          }
          tma_load_3d(st + NA * TC_PLANE_BYTES, mB, &full_bar[s], ti.k_lo + kt * TC_BK, ti.b_row, 0);
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
      TileInfo ti;
      for (int cur = src.begin(); ok && src.next(cur, ti);) {
        const int buf = local & 1;
        const uint32_t use_ph = (uint32_t)(local >> 1) & 1u;
        if (!mbar_wait_bounded(&tempty_bar[buf], use_ph ^ 1u, &s_abort, status)) break;
        tc_fence_after();
        const uint32_t acc = tmem + buf * 256;
        for (int kt = 0; kt < ti.nk; ++kt, ++it) {
          const int s = it % NST;
          const uint32_t ph = (uint32_t)(it / NST) & 1u;
          if (!mbar_wait_bounded(&full_bar[s], ph, &s_abort, status)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a_base = smem_base + s * STAGE;
          const uint64_t a_desc = sdesc_sw64(a_base), b_desc = sdesc_sw64(a_base + NA * TC_PLANE_BYTES);
#pragma unroll
          for (int kk = 0; kk < TC_BK / 16; ++kk)
            issue_products<KIND>(acc, a_desc, b_desc, kk, id_pos, id_neg, kt == 0 && kk == 0);
          mma_commit(&empty_bar[s]);
        }
        mma_commit(&tfull_bar[buf]);
        ++local;
      }
      // every MMA issued above completes before the accumulators are released
      mma_commit(done_bar);
      const uint64_t t0 = global_timer();
      while (!mbar_try_wait(done_bar, 0) && global_timer() - t0 < TC_WAIT_NS) {
      }
    }
    __syncwarp();
  } else {
    // ---- epilogue warps 2..5: TMEM lane quarter (warp % 4) -> 32 output rows
    if constexpr (EARLY) src.zero_idle(threadIdx.x - 64);
    const int quarter = warp & 3;
    int local = 0, chunk = 0;
    bool prev_committed = false;  // (issuing thread) the previous chunk committed a store
    TileInfo ti;
    for (int cur = src.begin(); src.next(cur, ti);) {
      const TcGemmArgs& args = src.args(ti);
      const int buf = local & 1;
      const uint32_t ph = (uint32_t)(local >> 1) & 1u;
      bool have = mbar_wait_bounded(&tfull_bar[buf], ph, &s_abort, status) && src.before_epilogue(&s_abort);
      // one decision for all four epilogue warps: tcgen05.ld is warp-collective and the
      // staged stores meet at named barriers
      have = epi_all(have && !s_abort);
      if (!have) break;
      tc_fence_after();
      const int row = ti.out_row0 + quarter * 32 + lane;
      const uint32_t t_lane = tmem + buf * 256 + ((uint32_t)(quarter * 32) << 16);
      // TMA stores write whole 128-row boxes: only where no row of the box belongs to
      // another layer (rows past the tensor's end are clipped by the store itself)
      const bool use_tma_y = EPI == EPI_Y && (ti.out_row0 + TC_BM <= ti.row_lim || ti.row_lim >= args.y_rows);
#pragma unroll 1
      for (int c0 = 0; c0 < TC_BN; c0 += 32, ++chunk) {
        uint32_t re[32], im[32];
        tmem_ld32(t_lane + c0, re);
        if (KIND != KIND_TEST) tmem_ld32(t_lane + 128 + c0, im);
        tmem_ld_wait();
        if (EPI == EPI_H && args.h_transposed && *args.h_transposed) {
          // transposed problem: C[m][n] belongs at H[n][m]; the 32 lanes hold 32 consecutive
          // m, so each atomic instruction covers 256 contiguous bytes of one H row
          if (row < ti.row_lim) {
            const int nv = min(32, ti.col_lim - (ti.out_col0 + c0));
            float2* dst = args.H + (size_t)(ti.out_col0 + c0) * args.ldh + row;
#pragma unroll
            for (int j = 0; j < 32; ++j)
              if (j < nv)
                atomicAdd(dst + (size_t)j * args.ldh,
                          make_float2(__uint_as_float(re[j]) * args.scale, __uint_as_float(im[j]) * args.scale));
          }
        } else if (EPI == EPI_H || EPI == EPI_F) {
          if (row < ti.row_lim) {
            float2* dst = (EPI == EPI_H ? args.H + (size_t)row * args.ldh : args.F + (size_t)row * args.ldf) +
                          ti.out_col0 + c0;
            const int nv = min(32, ti.col_lim - (ti.out_col0 + c0));
            if (nv == 32 && args.h_vec4) {
#pragma unroll
              for (int j = 0; j < 32; j += 2) {
                float4 v = make_float4(__uint_as_float(re[j]) * args.scale, __uint_as_float(im[j]) * args.scale,
                                       __uint_as_float(re[j + 1]) * args.scale,
                                       __uint_as_float(im[j + 1]) * args.scale);
                if (EPI == EPI_H)
                  atomicAdd(reinterpret_cast<float4*>(dst + j), v);
                else
                  *reinterpret_cast<float4*>(dst + j) = v;
              }
            } else {
#pragma unroll
              for (int j = 0; j < 32; ++j)
                if (j < nv) {
                  const float2 v = make_float2(__uint_as_float(re[j]) * args.scale, __uint_as_float(im[j]) * args.scale);
                  if (EPI == EPI_H)
                    atomicAdd(dst + j, v);
                  else
                    dst[j] = v;
                }
            }
          }
        } else if (EPI == EPI_Y) {
          const int nv = min(32, ti.n_valid - c0);
          if (use_tma_y) {
            // stage the chunk (64-byte swizzled, as the tensor map stores it), then one TMA store
            uint8_t* buf = stage_y + (chunk % YBUFS) * TC_STAGE_Y_BYTES;
            if (lane == 0 && quarter == 0) {  // the buffer's previous store has read its data
              if (YBUFS == 2 && prev_committed)
                bulk_wait_read1();
              else
                bulk_wait_read0();
            }
            epi_barrier();
            const int r = quarter * 32 + lane;
            uint32_t w[4][16];
#pragma unroll
            for (int j = 0; j < 32; j += 2) {
              uint16_t a0, a1, b0, b1, c0h, c1h, d0, d1;
              split_hi_lo<F16>(__uint_as_float(re[j]) * args.scale, a0, b0);
              split_hi_lo<F16>(__uint_as_float(re[j + 1]) * args.scale, a1, b1);
              split_hi_lo<F16>(__uint_as_float(im[j]) * args.scale, c0h, d0);
              split_hi_lo<F16>(__uint_as_float(im[j + 1]) * args.scale, c1h, d1);
              w[0][j / 2] = (uint32_t)a0 | ((uint32_t)a1 << 16);
              w[1][j / 2] = (uint32_t)b0 | ((uint32_t)b1 << 16);
              w[2][j / 2] = (uint32_t)c0h | ((uint32_t)c1h << 16);
              w[3][j / 2] = (uint32_t)d0 | ((uint32_t)d1 << 16);
            }
#pragma unroll
            for (int pl = 0; pl < 4; ++pl)
#pragma unroll
              for (int q = 0; q < 4; ++q) {
                const int sw = q ^ ((r >> 1) & 3);
                *reinterpret_cast<uint4*>(buf + pl * TC_PLANE_BYTES + r * 64 + sw * 16) =
                    make_uint4(w[pl][4 * q], w[pl][4 * q + 1], w[pl][4 * q + 2], w[pl][4 * q + 3]);
              }
            fence_async_smem();
            epi_barrier();
            if (lane == 0 && quarter == 0) {
              prev_committed = nv > 0;
              if (nv > 0) {
                tma_store_3d(src.mapC(ti), buf, ti.out_col0 + c0, ti.out_row0, 0);
                bulk_commit();
              }
            }
          } else if (row < ti.row_lim) {
            uint16_t* base = args.Y + (size_t)row * args.ldy + ti.out_col0 + c0;
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
      if (EPI == EPI_Y && src.publishes()) {
        // the tile's stores (staged TMA stores and direct stores) complete and visible, then
        // published once
        if (lane == 0 && quarter == 0) bulk_wait_all();
        __threadfence();
        epi_barrier();
        if (lane == 0 && quarter == 0) src.tile_stored(ti);
      }
    }
    if (EPI == EPI_Y && lane == 0 && quarter == 0) bulk_wait_all();  // staged stores complete
  }
  tc_fence_before();
  __syncthreads();
  if (DEALLOC && warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
  }
}

// Work units of one problem: tensor maps and arguments in kernel parameters, per-layer K
// offsets in shared memory.
struct TcSingleSrc {
  const CUtensorMap* ma;
  const CUtensorMap* mb;
  const CUtensorMap* mc;
  const TcGemmArgs* a;
  const int* s_off;
  int ktot;
  const int* s_toff;  // mode 1: first unit of every layer over the non-empty tiles only
  __device__ int total() const { return a->mode == 1 ? s_toff[a->n_layers] : a->tm * a->tn * a->tz; }
  __device__ bool decode(int t, TileInfo& ti) const {
    ti.item = 0;
    if (a->mode == 1) {
      // round robin over the layers' non-empty tiles only, so that no CTA draws more
      // than its share of real work
      int zz = 0;
      while (zz + 1 < a->n_layers && t >= s_toff[zz + 1]) ++zz;
      const int local = t - s_toff[zz];
      ti.out_row0 = (local % a->tm) * TC_BM;
      ti.row_lim = a->M;
      ti.akm = nullptr;
      return decode_stage1(*a, local % a->tm, local / a->tm, zz, s_off, ti);
    }
    return decode_tile(*a, t, s_off, ktot, ti);
  }
  // Units of this CTA.  Round robin over the work units, or (stream-K, split-K mode) one
  // contiguous slice of the (tile, K step) space cut at tile boundaries.
  __device__ int begin() const {
    if (a->mode == 2 && a->streamk) {
      const long long W = (long long)a->tm * a->tn * (ktot / TC_BK);
      return (int)(W * blockIdx.x / gridDim.x);
    }
    return blockIdx.x;
  }
  __device__ bool next(int& cur, TileInfo& ti) const {
    if (a->mode == 2 && a->streamk) {
      const int nkt = ktot / TC_BK;
      const long long W = (long long)a->tm * a->tn * nkt;
      const int w1 = (int)(W * (blockIdx.x + 1) / gridDim.x);
      if (nkt <= 0 || cur >= w1) return false;
      const int tile = cur / nkt, kk = cur - tile * nkt;
      const int seg = min(min(w1, (tile + 1) * nkt) - cur, a->streamk);
      const int mt = tile % a->tm, nt = tile / a->tm;
      ti.item = 0;
      ti.akm = a->a_kmap ? a->a_kmap + kk : nullptr;
      ti.a_row = mt * TC_BM;
      ti.b_row = nt * TC_BN;
      ti.k_lo = kk * TC_BK;
      ti.nk = seg;
      ti.out_row0 = mt * TC_BM;
      ti.out_col0 = nt * TC_BN;
      ti.n_valid = TC_BN;
      ti.row_lim = a->M;
      ti.col_lim = a->N;
      cur += seg;
      return true;
    }
    for (; cur < total(); cur += gridDim.x)
      if (decode(cur, ti)) {
        cur += gridDim.x;
        return true;
      }
    return false;
  }
  __device__ const CUtensorMap* mapA(const TileInfo&) const { return ma; }
  __device__ const CUtensorMap* mapB(const TileInfo&) const { return mb; }
  __device__ const CUtensorMap* mapC(const TileInfo&) const { return mc; }
  __device__ void acquire_maps(const CUtensorMap*, const CUtensorMap*) const {}
  __device__ const TcGemmArgs& args(const TileInfo&) const { return *a; }
  __device__ int* status() const { return a->status; }
  __device__ bool before_load(const TileInfo&, int, volatile int*) const { return true; }
  __device__ bool before_epilogue(volatile int*) const { return true; }
  __device__ bool publishes() const { return false; }
  __device__ void tile_stored(const TileInfo&) const {}
  __device__ bool a_early() const { return a->a_early != 0; }
  // the epilogue warps, idle until the first tile has accumulated, clear the regions asked for
  __device__ void zero_idle(int e) const {
    const long long t0 = (long long)blockIdx.x * 128 + e, nt = (long long)gridDim.x * 128;
#pragma unroll 1
    for (int r = 0; r < 2; ++r)
      for (long long i = t0; i < a->zero_n[r]; i += nt) a->zero_ptr[r][i] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
};

template <int KIND, int EPI, bool F16>
__global__ void __launch_bounds__(192, 1) k_tc_gemm(const __grid_constant__ CUtensorMap mapA,
                                                     const __grid_constant__ CUtensorMap mapB,
                                                     const __grid_constant__ CUtensorMap mapC,
                                                     const TcGemmArgs args) {
  constexpr int NST = tc_nst<KIND, EPI>();
  extern __shared__ uint8_t tc_smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)tc_smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full_bar[NST], empty_bar[NST], tfull_bar[2], tempty_bar[2], done_bar;
  __shared__ uint32_t s_tmem;
  __shared__ volatile int s_abort;
  __shared__ int s_off[CGH_MAX_LAYERS + 1];
  __shared__ int s_toff[CGH_MAX_LAYERS + 1];
  __shared__ int s_kr[CGH_MAX_LAYERS];
  // barriers, tensor memory and the per-layer sizes (written by the compaction, two or more
  // grids back) before the wait for the previous grid: a CTA that starts while the previous
  // grid's last CTAs run does all of this, and issues its first A loads, in the meantime.  The
  // sizes are loaded in parallel (a serial loop of global loads in thread 0 would cost a
  // memory latency per layer before any role starts).
  tc_gemm_setup<NST, true>(full_bar, empty_bar, tfull_bar, tempty_bar, &done_bar, &s_tmem, &s_abort);
  if (args.kr_pad && threadIdx.x < args.n_layers) s_kr[threadIdx.x] = __ldcg(args.kr_pad + threadIdx.x);
  __syncthreads();
  if (threadIdx.x == 0) {
    int o = 0, u = 0;
    s_off[0] = 0;
    s_toff[0] = 0;
    if (args.kr_pad)
      for (int q = 0; q < args.n_layers; ++q) {
        const int kr = s_kr[q];
        s_off[q + 1] = (o += kr);
        s_toff[q + 1] = (u += args.tm * ((kr + TC_BN - 1) / TC_BN));
      }
  }
  __syncthreads();
  TcSingleSrc src{&mapA, &mapB, &mapC, &args, s_off,
                  args.mode == 2 ? (args.kr_pad ? s_off[args.n_layers] : args.K) : 0, s_toff};
  tc_gemm_body<KIND, EPI, F16, TcSingleSrc, true, true, false, true>(src, smem, full_bar, empty_bar, tfull_bar,
                                                                     tempty_bar, &done_bar, &s_tmem, &s_abort);
}

// One problem of a batch, in global memory: its tensor maps, arguments, first work unit
// and per-layer K offsets (filled on the device once the compaction has run).
struct alignas(128) TcBatchItem {
  CUtensorMap ma;
  CUtensorMap mb;
  CUtensorMap mc;
  CUtensorMap mb64;  // stage 2 on CTA pairs: B with 64-row boxes
  TcGemmArgs a;
  int unit0;
  int unit0p;        // stage 2 on CTA pairs: first pair unit
  int koff[CGH_MAX_LAYERS + 1];
};

// Work units of many problems: unit t belongs to the last item whose first unit is <= t
// (binary search over the items' first units, read from global memory).
struct TcBatchSrc {
  const TcBatchItem* items;
  int n, tot;
  int* st;
  __device__ int total() const { return tot; }
  __device__ int begin() const { return blockIdx.x; }
  __device__ bool next(int& cur, TileInfo& ti) const {
    for (; cur < tot; cur += gridDim.x)
      if (decode(cur, ti)) {
        cur += gridDim.x;
        return true;
      }
    return false;
  }
  __device__ bool decode(int t, TileInfo& ti) const {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (items[mid].unit0 <= t)
        lo = mid;
      else
        hi = mid - 1;
    }
    ti.item = lo;
    const TcBatchItem& it = items[lo];
    const int ktot = it.a.mode == 2 ? (it.a.kr_pad ? it.koff[it.a.n_layers] : it.a.K) : 0;
    return decode_tile(it.a, t - it.unit0, it.koff, ktot, ti);
  }
  __device__ const CUtensorMap* mapA(const TileInfo& ti) const { return &items[ti.item].ma; }
  __device__ const CUtensorMap* mapB(const TileInfo& ti) const { return &items[ti.item].mb; }
  __device__ const CUtensorMap* mapC(const TileInfo& ti) const { return &items[ti.item].mc; }
  __device__ void acquire_maps(const CUtensorMap* a, const CUtensorMap* b) const {
    // tensor maps written to global memory by a copy before the launch
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(reinterpret_cast<uint64_t>(a))
                 : "memory");
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(reinterpret_cast<uint64_t>(b))
                 : "memory");
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(
                     reinterpret_cast<uint64_t>(a + 2))
                 : "memory");  // the store map follows the two load maps in the item
  }
  __device__ const TcGemmArgs& args(const TileInfo& ti) const { return items[ti.item].a; }
  __device__ int* status() const { return st; }
  __device__ bool before_load(const TileInfo&, int, volatile int*) const { return true; }
  __device__ bool before_epilogue(volatile int*) const { return true; }
  __device__ bool publishes() const { return false; }
  __device__ void tile_stored(const TileInfo&) const {}
};

#define TC_BATCH_MAX 1024

template <int KIND, int EPI, bool F16>
__global__ void __launch_bounds__(192, 1) k_tc_gemm_batch(const TcBatchItem* __restrict__ items, int n,
                                                           int total, int* status) {
  constexpr int NST = tc_nst<KIND, EPI>();
  extern __shared__ uint8_t tc_smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)tc_smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full_bar[NST], empty_bar[NST], tfull_bar[2], tempty_bar[2], done_bar;
  __shared__ uint32_t s_tmem;
  __shared__ volatile int s_abort;
  pdl_wait();
  TcBatchSrc src{items, n, total, status};
  tc_gemm_body<KIND, EPI, F16>(src, smem, full_bar, empty_bar, tfull_bar, tempty_bar, &done_bar, &s_tmem,
                               &s_abort);
}

// ------------------------------------------------------------------------------------
// host helpers

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

// 3-D map over `planes` planes of a [rows][k_alloc] 16-bit matrix; box 32 x box_rows x
// planes, 64-byte swizzle (matches sdesc_sw64).
static int make_plane_map(CUtensorMap* map, const void* base, int planes, long long rows, long long k_alloc,
                          int box_rows = 128) {
  if (get_encoder() != CGH_OK) return CGH_ERR_CUDA;
  if (((uintptr_t)base & 15) || (k_alloc * 2) % 16)
    return cgh_fail(CGH_ERR_ARG, "tensor map: base must be 16-byte aligned and rows a multiple of 16 bytes");
  cuuint64_t dims[3] = {(cuuint64_t)k_alloc, (cuuint64_t)rows, (cuuint64_t)planes};
  cuuint64_t strides[2] = {(cuuint64_t)(k_alloc * 2), (cuuint64_t)(rows * k_alloc * 2)};
  cuuint32_t box[3] = {TC_BK, (cuuint32_t)box_rows, (cuuint32_t)planes};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_UINT16, 3, const_cast<void*>(base), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return cgh_fail(CGH_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return CGH_OK;
}

// The hi planes (0 and 2: re_hi, im_hi) of a 4-plane hi+lo operand as a 2-plane map over
// the same memory.
static int make_hi_plane_map(CUtensorMap* map, const void* base, long long rows, long long k_alloc) {
  if (get_encoder() != CGH_OK) return CGH_ERR_CUDA;
  if (((uintptr_t)base & 15) || (k_alloc * 2) % 16)
    return cgh_fail(CGH_ERR_ARG, "tensor map: base must be 16-byte aligned and rows a multiple of 16 bytes");
  cuuint64_t dims[3] = {(cuuint64_t)k_alloc, (cuuint64_t)rows, 2};
  cuuint64_t strides[2] = {(cuuint64_t)(k_alloc * 2), (cuuint64_t)(2 * rows * k_alloc * 2)};
  cuuint32_t box[3] = {TC_BK, 128, 2};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_UINT16, 3, const_cast<void*>(base), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return cgh_fail(CGH_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return CGH_OK;
}

template <int KIND, int EPI, bool F16>
static cudaError_t set_gemm_attr() {
  cudaError_t e = cudaFuncSetAttribute(k_tc_gemm<KIND, EPI, F16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)tc_smem_bytes<KIND, EPI>());
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_tc_gemm_batch<KIND, EPI, F16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)tc_smem_bytes<KIND, EPI>());
}

template <int KIND, int EPI, bool F16>
static cudaError_t launch_gemm(const CUtensorMap& ma, const CUtensorMap& mb, const CUtensorMap& mc, TcGemmArgs a,
                               dim3 tiles, cudaStream_t st) {
  a.tm = (int)tiles.x;
  a.tn = (int)tiles.y;
  a.tz = (int)tiles.z;
  const long long units = a.streamk ? (long long)tc_num_sms() : (long long)a.tm * a.tn * a.tz;
  const int grid = (int)(units < tc_num_sms() ? units : tc_num_sms());
  if (grid <= 0) return cudaSuccess;
  return launch_pdl(k_tc_gemm<KIND, EPI, F16>, dim3(grid), dim3(192), tc_smem_bytes<KIND, EPI>(), st, ma, mb, mc,
                    a);
}

