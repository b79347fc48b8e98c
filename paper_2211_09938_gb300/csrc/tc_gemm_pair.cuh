// Stage-2 GEMM on CTA pairs (tcgen05 cta_group::2): the two CTAs of a cluster share one
// 256 x 128 output tile.  Each CTA stages its own 128 rows of A and half (64 rows) of B;
// one thread of the even CTA issues MMAs of M = 256, N = 128, K = 16 that read both CTAs'
// shared memory and accumulate each CTA's 128 rows in its own tensor memory.  Per SM this
// is the same MMA work as a 128 x 128 tile on one CTA, but B is staged once per pair
// instead of once per CTA, so every MMA reads 6 KiB of shared memory per SM instead of
// 8 KiB and the TMA writes and L2 reads of B halve: the shared-memory traffic per MMA
// (operand reads plus TMA writes) drops by a quarter.
//
// Barriers.  full[s] lives in the even CTA: its producer arms it with both CTAs' bytes and
// both producers' TMA loads complete on it (.cta_group::2 lets a load signal the peer's
// barrier).  empty[s] and tfull[b] exist in both CTAs and are signalled by one multicast
// commit from the MMA thread.  tempty[b] lives in the even CTA and counts the four
// epilogue warps of each CTA (the odd CTA's arrive remotely).  Every wait is bounded.
#pragma once
#include "tc_gemm.cuh"

#define TC_PAIR_A_PLANE (128 * TC_BK * 2)  // 8 KiB: 128 rows of A per CTA
#define TC_PAIR_B_PLANE (64 * TC_BK * 2)   // 4 KiB: 64 rows of B per CTA

__device__ __forceinline__ uint32_t cluster_ctarank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

// All threads of both CTAs of the cluster (release / acquire).
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Shared::cluster address of the variable at shared::cta address `a` in CTA `rank`.
__device__ __forceinline__ uint32_t mapa_rank(uint32_t a, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}

__device__ __forceinline__ void mbar_arrive_remote(uint32_t cluster_addr) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}

// TMA load into this CTA's shared memory that completes on an mbarrier of either CTA of
// the pair (bar: shared::cluster address).
__device__ __forceinline__ void tma_load_3d_pair(void* dst, const CUtensorMap* map, uint32_t bar, int c0, int c1,
                                                 int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}

__device__ __forceinline__ void mma_f16_pair(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

// Arrive once on the mbarrier at this shared::cta offset in every CTA of `mask` when all
// MMAs issued so far by this thread have completed.
__device__ __forceinline__ void mma_commit_pair(uint64_t* bar, uint16_t mask) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
          smem_u32(bar)),
      "h"(mask)
      : "memory");
}

// Products of one 16-wide K slice (see issue_products): A planes 8 KiB apart, B planes
// 4 KiB apart (64 rows per CTA).
template <int KIND>
__device__ __forceinline__ void issue_products_pair(uint32_t tmem, uint64_t a_desc, uint64_t b_desc, int kk,
                                                    uint32_t id_pos, uint32_t id_neg, bool first) {
  auto A = [&](int p) { return a_desc + (uint64_t)((p * TC_PAIR_A_PLANE + kk * 32) >> 4); };
  auto B = [&](int p) { return b_desc + (uint64_t)((p * TC_PAIR_B_PLANE + kk * 32) >> 4); };
  const uint32_t d0 = tmem, d1 = tmem + 128;
  const uint32_t f = first ? 0u : 1u;
  if (KIND == KIND_CC2) {
    mma_f16_pair(d0, A(0), B(0), id_pos, f);
    mma_f16_pair(d0, A(0), B(1), id_pos, 1);
    mma_f16_pair(d0, A(1), B(2), id_neg, 1);
    mma_f16_pair(d0, A(1), B(3), id_neg, 1);
    mma_f16_pair(d1, A(0), B(2), id_pos, f);
    mma_f16_pair(d1, A(0), B(3), id_pos, 1);
    mma_f16_pair(d1, A(1), B(0), id_pos, 1);
    mma_f16_pair(d1, A(1), B(1), id_pos, 1);
  } else {
    // the two accumulators' products interleaved (each accumulator's own order unchanged)
    mma_f16_pair(d0, A(0), B(0), id_pos, f);
    mma_f16_pair(d1, A(0), B(2), id_pos, f);
    mma_f16_pair(d0, A(0), B(1), id_pos, 1);
    mma_f16_pair(d1, A(0), B(3), id_pos, 1);
    mma_f16_pair(d0, A(1), B(0), id_pos, 1);
    mma_f16_pair(d1, A(1), B(2), id_pos, 1);
    mma_f16_pair(d0, A(2), B(2), id_neg, 1);
    mma_f16_pair(d1, A(2), B(0), id_pos, 1);
    mma_f16_pair(d0, A(2), B(3), id_neg, 1);
    mma_f16_pair(d1, A(2), B(1), id_pos, 1);
    mma_f16_pair(d0, A(3), B(2), id_neg, 1);
    mma_f16_pair(d1, A(3), B(0), id_pos, 1);
  }
}

template <int KIND>
constexpr int pair_nst() {
  return KIND == KIND_CC ? 4 : 6;
}
template <int KIND>
constexpr uint32_t pair_stage_bytes() {
  return TcCfg<KIND>::NA * TC_PAIR_A_PLANE + TcCfg<KIND>::NB * TC_PAIR_B_PLANE;
}
template <int KIND>
constexpr size_t pair_smem_bytes() {
  return (size_t)pair_nst<KIND>() * pair_stage_bytes<KIND>() + 1024;
}

// Stream-K slice of one pair over the (pair tile, K step) space, cut into chains of at most
// a.streamk K steps at tile boundaries.  Both CTAs of the pair decode the same sequence;
// `rank` selects the CTA's 128 rows of A and 64 rows of B.
struct PairSlice {
  const TcGemmArgs* a;
  long long cur, end;
  int nkt, tmp;
  __device__ bool next(uint32_t rank, TileInfo& ti) {
    const TcGemmArgs& a = *this->a;
    if (nkt <= 0 || cur >= end) return false;
    const long long tile = cur / nkt;
    const int kk = (int)(cur - tile * nkt);
    const int seg = (int)min(min(end, (tile + 1) * nkt) - cur, (long long)a.streamk);
    const int mtp = (int)(tile % tmp), nt = (int)(tile / tmp);
    ti.item = 0;
    ti.akm = a.a_kmap ? a.a_kmap + kk : nullptr;
    ti.a_row = (2 * mtp + (int)rank) * TC_BM;
    ti.b_row = nt * TC_BN + 64 * (int)rank;
    ti.k_lo = kk * TC_BK;
    ti.nk = seg;
    ti.out_row0 = ti.a_row;
    ti.out_col0 = nt * TC_BN;
    ti.n_valid = TC_BN;
    ti.row_lim = a.M;
    ti.col_lim = a.N;
    cur += seg;
    return true;
  }
};

// The body of stage 2 on CTA pairs over a source of work units (PairSingleSrc: one problem,
// stream-K; PairBatchSrc: the units of a batch of problems).  Each role iterates its own
// copy of src.iter(); both CTAs of a pair decode the same sequence.  EARLY: the kernel has
// loaded the K sizes before the wait for the previous grid (they come from grids two or more
// back), the barriers and tensor memory are set up before that wait too, and each producer
// issues its A halves of the first ring stages (the fringe planes) before it; only the B
// halves, the stage-1 output, wait.
template <int KIND, bool F16, class PSrc, bool EARLY = false>
__device__ __forceinline__ void tc_gemm_pair_body(const PSrc& src) {
  using Cfg = TcCfg<KIND>;
  constexpr int NA = Cfg::NA, NST = pair_nst<KIND>();
  constexpr uint32_t STAGE = pair_stage_bytes<KIND>();
  extern __shared__ uint8_t tc_smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)tc_smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full_bar[NST], empty_bar[NST], tfull_bar[2], tempty_bar[2], done_bar;
  __shared__ uint32_t s_tmem;
  __shared__ volatile int s_abort_v;
  volatile int& s_abort = s_abort_v;
  const uint32_t rank = cluster_ctarank();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int* const status = src.status();

  if (threadIdx.x == 0) {
    for (int s = 0; s < NST; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull_bar[b], 1);
      mbar_init(&tempty_bar[b], 8);
    }
    mbar_init(&done_bar, 1);
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(&s_tmem))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync_all();  // both CTAs' barriers exist before any remote signal
  tc_fence_after();
  if constexpr (!EARLY) pdl_wait();  // the K sizes and the stage-1 output come from earlier kernels
  const uint32_t tmem = s_tmem;
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
      // ---- TMA producer (both CTAs): own rows of A and B, completing on the even CTA's full[s]
      const uint32_t full0 = mapa_rank(smem_u32(&full_bar[0]), 0);
      int it = 0;
      bool issued[NST];
      uint32_t issued_ph[NST];
      for (int s = 0; s < NST; ++s) issued[s] = false, issued_ph[s] = 0;
      bool ok = true;
      TileInfo ti;
      // EARLY: the A halves of the first unit's first ring stages (fresh barriers: no wait for
      // a free slot) go out before the wait for the previous grid
      int npre = 0;
      if constexpr (EARLY) {
        auto s0 = src.iter();
        if (src.a_early() && s0.next(rank, ti)) {
          const CUtensorMap* mA = src.mapA(ti);
          npre = min(NST, ti.nk);
          for (int kt = 0; kt < npre; ++kt) {
            if (rank == 0) mbar_arrive_expect_tx(&full_bar[kt], 2 * STAGE);
            tma_load_3d_pair(smem + kt * STAGE, mA, full0 + 8u * kt, ti.akm ? __ldcg(ti.akm + kt) : ti.k_lo + kt * TC_BK,
                             ti.a_row, 0);
            issued[kt] = true;
          }
        }
        pdl_wait();
        pdl_trigger();
      }
      auto sl = src.iter();
      while (ok && sl.next(rank, ti)) {
        const CUtensorMap* mA = src.mapA(ti);
        const CUtensorMap* mB = src.mapB(ti);
        src.acquire_maps(mA, mB);
        for (int kt = 0; kt < ti.nk; ++kt, ++it) {
          const int s = it % NST;
          const uint32_t ph = (uint32_t)(it / NST) & 1u;
          const bool pre = it < npre;  // A already in flight, barrier armed
          if (!pre && !mbar_wait_bounded(&empty_bar[s], ph ^ 1u, &s_abort, status)) {
            ok = false;
            break;
          }
          uint8_t* st = smem + s * STAGE;
          if (!pre) {
            if (rank == 0) mbar_arrive_expect_tx(&full_bar[s], 2 * STAGE);
            tma_load_3d_pair(st, mA, full0 + 8u * s, ti.akm ? ti.akm[kt] : ti.k_lo + kt * TC_BK, ti.a_row, 0);
          }
          tma_load_3d_pair(st + NA * TC_PAIR_A_PLANE, mB, full0 + 8u * s, ti.k_lo + kt * TC_BK, ti.b_row, 0);
          issued[s] = true;
          issued_ph[s] = ph;
        }
      }
      if (s_abort && rank == 0) {  // let copies in flight land before shared memory goes away
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
    if (lane == 0 && rank == 0) {
      // ---- MMA issuer (even CTA only): M = 256 over the pair, N = 128
      const uint32_t id_pos = idesc_f16(F16 ? 0 : 1, 0, 2 * TC_BM, TC_BN);
      const uint32_t id_neg = idesc_f16(F16 ? 0 : 1, 1, 2 * TC_BM, TC_BN);
      int it = 0, local = 0;
      bool ok = true;
      TileInfo ti;
      auto sl = src.iter();
      while (ok && sl.next(rank, ti)) {
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
          const uint64_t a_desc = sdesc_sw64(a_base), b_desc = sdesc_sw64(a_base + NA * TC_PAIR_A_PLANE);
#pragma unroll
          for (int kk = 0; kk < TC_BK / 16; ++kk)
            issue_products_pair<KIND>(acc, a_desc, b_desc, kk, id_pos, id_neg, kt == 0 && kk == 0);
          mma_commit_pair(&empty_bar[s], 0x3);
        }
        mma_commit_pair(&tfull_bar[buf], 0x3);
        ++local;
      }
      // every MMA issued above completes before the accumulators are released
      mma_commit_pair(&done_bar, 0x1);
      const uint64_t t0 = global_timer();
      while (!mbar_try_wait(&done_bar, 0) && global_timer() - t0 < TC_WAIT_NS) {
      }
    }
    __syncwarp();
  } else {
    // ---- epilogue warps 2..5 (both CTAs): TMEM lane quarter (warp % 4) -> 32 output rows
    const int quarter = warp & 3;
    const uint32_t tempty0 = mapa_rank(smem_u32(&tempty_bar[0]), 0);
    int local = 0;
    TileInfo ti;
    auto sl = src.iter();
    while (sl.next(rank, ti)) {
      const TcGemmArgs& args = src.args(ti);
      const int buf = local & 1;
      const uint32_t ph = (uint32_t)(local >> 1) & 1u;
      bool have = mbar_wait_bounded(&tfull_bar[buf], ph, &s_abort, status);
      have = epi_all(have && !s_abort);
      if (!have) break;
      tc_fence_after();
      const int row = ti.out_row0 + quarter * 32 + lane;
      const uint32_t t_lane = tmem + buf * 256 + ((uint32_t)(quarter * 32) << 16);
#pragma unroll 1
      for (int c0 = 0; c0 < TC_BN; c0 += 32) {
        uint32_t re[32], im[32];
        tmem_ld32(t_lane + c0, re);
        tmem_ld32(t_lane + 128 + c0, im);
        tmem_ld_wait();
        const int nv = min(32, ti.col_lim - (ti.out_col0 + c0));
        if (args.h_transposed && *args.h_transposed) {
          // transposed problem: C[m][n] belongs at H[n][m]; the 32 lanes hold 32 consecutive
          // m, so each atomic instruction covers 256 contiguous bytes of one H row
          if (row < ti.row_lim) {
            float2* dst = args.H + (size_t)(ti.out_col0 + c0) * args.ldh + row;
#pragma unroll
            for (int j = 0; j < 32; ++j)
              if (j < nv)
                atomicAdd(dst + (size_t)j * args.ldh,
                          make_float2(__uint_as_float(re[j]) * args.scale, __uint_as_float(im[j]) * args.scale));
          }
        } else if (row < ti.row_lim) {
          float2* dst = args.H + (size_t)row * args.ldh + ti.out_col0 + c0;
          if (nv == 32 && args.h_vec4) {
#pragma unroll
            for (int j = 0; j < 32; j += 2)
              atomicAdd(reinterpret_cast<float4*>(dst + j),
                        make_float4(__uint_as_float(re[j]) * args.scale, __uint_as_float(im[j]) * args.scale,
                                    __uint_as_float(re[j + 1]) * args.scale, __uint_as_float(im[j + 1]) * args.scale));
          } else {
#pragma unroll
            for (int j = 0; j < 32; ++j)
              if (j < nv)
                atomicAdd(dst + j,
                          make_float2(__uint_as_float(re[j]) * args.scale, __uint_as_float(im[j]) * args.scale));
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        if (rank == 0)
          mbar_arrive(&tempty_bar[buf]);
        else
          mbar_arrive_remote(tempty0 + 8u * buf);
      }
      ++local;
    }
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync_all();  // no remote signal or shared-memory read of the pair is left in flight
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
  }
}

// One problem: stream-K slices of the (pair tile, K step) space.
struct PairSingleSrc {
  const CUtensorMap* ma;
  const CUtensorMap* mb;
  const TcGemmArgs* a;
  PairSlice slice;
  __device__ PairSlice iter() const { return slice; }
  __device__ const CUtensorMap* mapA(const TileInfo&) const { return ma; }
  __device__ const CUtensorMap* mapB(const TileInfo&) const { return mb; }
  __device__ void acquire_maps(const CUtensorMap*, const CUtensorMap*) const {}
  __device__ const TcGemmArgs& args(const TileInfo&) const { return *a; }
  __device__ int* status() const { return a->status; }
  __device__ bool a_early() const { return a->a_early != 0; }
};

template <int KIND, bool F16>
__global__ void __launch_bounds__(192, 1) k_tc_gemm_pair(const __grid_constant__ CUtensorMap mapA,
                                                          const __grid_constant__ CUtensorMap mapB,
                                                          const TcGemmArgs args) {
  __shared__ int s_kr[CGH_MAX_LAYERS];
  __shared__ int s_ktot;
  // the K sizes come from the compaction, two or more grids back: read before the wait for
  // the previous grid, which the body's roles make themselves
  if (threadIdx.x < args.n_layers) s_kr[threadIdx.x] = __ldcg(args.kr_pad + threadIdx.x);
  __syncthreads();
  if (threadIdx.x == 0) {
    int o = 0;
    for (int q = 0; q < args.n_layers; ++q) o += s_kr[q];
    s_ktot = o;
  }
  __syncthreads();
  PairSingleSrc src{&mapA, &mapB, &args, {}};
  {
    const int npairs = gridDim.x >> 1, pair = blockIdx.x >> 1;
    src.slice.a = &args;
    src.slice.nkt = s_ktot / TC_BK;
    src.slice.tmp = (args.tm + 1) >> 1;
    const long long W = (long long)src.slice.tmp * args.tn * src.slice.nkt;
    src.slice.cur = W * pair / npairs;
    src.slice.end = W * (pair + 1) / npairs;
  }
  tc_gemm_pair_body<KIND, F16, PairSingleSrc, true>(src);
}

// The stage-2 units of a batch on CTA pairs: per item (pair tiles along M) x (tiles along
// N) x (K splits), found by binary search over the items' first pair units.
struct PairBatchSrc {
  const TcBatchItem* items;
  int n, tot;
  int* st;
  struct Iter {
    const PairBatchSrc* s;
    int cur;
    __device__ bool next(uint32_t rank, TileInfo& ti) {
      const int npairs = gridDim.x >> 1;
      for (; cur < s->tot; cur += npairs)
        if (s->decode(cur, rank, ti)) {
          cur += npairs;
          return true;
        }
      return false;
    }
  };
  __device__ Iter iter() const { return Iter{this, (int)(blockIdx.x >> 1)}; }
  __device__ bool decode(int t, uint32_t rank, TileInfo& ti) const {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (items[mid].unit0p <= t)
        lo = mid;
      else
        hi = mid - 1;
    }
    const TcBatchItem& it = items[lo];
    const TcGemmArgs& a = it.a;
    const int local = t - it.unit0p, tmp = (a.tm + 1) >> 1;
    const int mtp = local % tmp, r = local / tmp, nt = r % a.tn, split = r / a.tn;
    const int nkt = it.koff[a.n_layers] / TC_BK, S = a.tz;
    const int k0 = (int)((long long)nkt * split / S), k1 = (int)((long long)nkt * (split + 1) / S);
    ti.item = lo;
    ti.akm = a.a_kmap ? a.a_kmap + k0 : nullptr;
    ti.a_row = (2 * mtp + (int)rank) * TC_BM;
    ti.b_row = nt * TC_BN + 64 * (int)rank;
    ti.k_lo = k0 * TC_BK;
    ti.nk = k1 - k0;
    ti.out_row0 = ti.a_row;
    ti.out_col0 = nt * TC_BN;
    ti.n_valid = TC_BN;
    ti.row_lim = a.M;
    ti.col_lim = a.N;
    return ti.nk > 0;
  }
  __device__ const CUtensorMap* mapA(const TileInfo& ti) const { return &items[ti.item].ma; }
  __device__ const CUtensorMap* mapB(const TileInfo& ti) const { return &items[ti.item].mb64; }
  __device__ void acquire_maps(const CUtensorMap* a, const CUtensorMap* b) const {
    // tensor maps written to global memory by a copy before the launch
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(reinterpret_cast<uint64_t>(a))
                 : "memory");
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(reinterpret_cast<uint64_t>(b))
                 : "memory");
  }
  __device__ const TcGemmArgs& args(const TileInfo& ti) const { return items[ti.item].a; }
  __device__ int* status() const { return st; }
};

template <int KIND, bool F16>
__global__ void __launch_bounds__(192, 1) k_tc_gemm_pair_batch(const TcBatchItem* __restrict__ items, int n,
                                                                int total, int* status) {
  pdl_wait();
  PairBatchSrc src{items, n, total, status};
  tc_gemm_pair_body<KIND, F16>(src);
}

// ------------------------------------------------------------------------------------
// host side

template <int KIND, bool F16>
static cudaError_t set_gemm_pair_attr() {
  cudaError_t e = cudaFuncSetAttribute(k_tc_gemm_pair<KIND, F16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)pair_smem_bytes<KIND>());
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_tc_gemm_pair_batch<KIND, F16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)pair_smem_bytes<KIND>());
}

// Number of CTA pairs the device holds at once (one CTA per SM), cached per kernel.
template <int KIND, bool F16>
static int gemm_pair_clusters() {
  static int n = -1;
  if (n < 0) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2 * 256);
    cfg.blockDim = dim3(192);
    cfg.dynamicSmemBytes = pair_smem_bytes<KIND>();
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int c = 0;
    if (cudaOccupancyMaxActiveClusters(&c, k_tc_gemm_pair<KIND, F16>, &cfg) != cudaSuccess || c <= 0) {
      cudaGetLastError();
      c = 0;
    }
    n = c;
  }
  return n;
}

// Stage 2 on CTA pairs; a.streamk must be > 0.  Returns cudaErrorNotSupported when the
// device holds no CTA pair of this kernel (the caller then takes the one-CTA kernel).
template <int KIND, bool F16>
static cudaError_t launch_gemm_pair(const CUtensorMap& ma, const CUtensorMap& mb64, TcGemmArgs a, dim3 tiles,
                                    cudaStream_t st) {
  a.tm = (int)tiles.x;
  a.tn = (int)tiles.y;
  a.tz = (int)tiles.z;
  const int pairs = gemm_pair_clusters<KIND, F16>();
  if (pairs <= 0 || a.streamk <= 0) return cudaErrorNotSupported;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(2 * pairs);
  cfg.blockDim = dim3(192);
  cfg.dynamicSmemBytes = pair_smem_bytes<KIND>();
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  return cudaLaunchKernelEx(&cfg, k_tc_gemm_pair<KIND, F16>, ma, mb64, a);
}

// The batch's stage 2 on CTA pairs over `total` pair units; cudaErrorNotSupported when the
// device holds no CTA pair of this kernel.
template <int KIND, bool F16>
static cudaError_t launch_gemm_pair_batch(const TcBatchItem* d_items, int n, int total, int* status,
                                          cudaStream_t st) {
  int pairs = gemm_pair_clusters<KIND, F16>();
  if (pairs <= 0) return cudaErrorNotSupported;
  if (pairs > total) pairs = total;
  if (pairs <= 0) return cudaSuccess;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(2 * pairs);
  cfg.blockDim = dim3(192);
  cfg.dynamicSmemBytes = pair_smem_bytes<KIND>();
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_tc_gemm_pair_batch<KIND, F16>, d_items, n, total, status);
}
