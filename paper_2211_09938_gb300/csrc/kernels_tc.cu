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
#include <vector>

#include "tc_fused.cuh"
#include "tc_gemm_pair.cuh"

// ------------------------------------------------------------------------------------
// operand preparation kernels


__global__ void k_tc_scatter(const int32_t* __restrict__ l0, const int32_t* __restrict__ l1,
                             const int32_t* __restrict__ l2, const int32_t* __restrict__ l3,
                             const int32_t* __restrict__ d_counts, TcFlags fl, int H, int W, int Z,
                             int* status) {
  pdl_wait();
  pdl_trigger();
  const int li = blockIdx.y;
  const int32_t* lst = li == 0 ? l0 : li == 1 ? l1 : li == 2 ? l2 : l3;
  const int level = li == 0 ? 3 : li;
  const int hl = H >> level, wl = W >> level;
  const int cnt = clamp_list_count(d_counts[2 * li], Z * hl * wl, blockIdx.x == 0 ? status : nullptr);
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
      // keep the block's 8-pixel bands even when no LLL entry covers them (lists that are
      // not nested, e.g. a truncated LLL list)
      fl.rowband[(size_t)z * (H >> 3) + (by >> (3 - level))] = 1;
      fl.colband[(size_t)z * (W >> 3) + (bx >> (3 - level))] = 1;
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

// Per layer: compacted object rows / columns in 32-pixel bands (a band is kept when one
// of the layer's listed blocks, LLL or detail, lies in it), entries past the object edge
// set to -1, and the
// band of every 32-wide K step: stage-1 A reads fringe columns 32*band directly, and the
// stage-2 A coordinate of K step k of the concatenated layers is the fringe column
// z*H + 32*band (kmap2).
// Contraction order: the "rows" outputs (stage-2 K) take the object rows, or, for a square
// object, the object columns when their sum over the layers is the smaller (or the plan
// asks for columns): H^T = sum_z E_z A^_z^T E_z^T is then computed and written transposed.
// Every CTA counts the kept bands of all layers (for the decision and for its layer's
// offset in the concatenated K); CTA 0 records the decision.
struct CompactArgs {
  TcFlags fl;
  int H, W, Z, order;
  int *rows, *cols, *kr_pad, *kc_pad;
  int ld_rows, ld_cols;
  int *rband, *cband, *kmap2, *orient, *fused_sync;
};

__device__ __forceinline__ void compact_body(const CompactArgs& A, int z) {
  const TcFlags& fl = A.fl;
  const int H = A.H, W = A.W, Z = A.Z, order = A.order, ld_rows = A.ld_rows, ld_cols = A.ld_cols;
  int* const rows = A.rows;
  int* const cols = A.cols;
  int* const kr_pad = A.kr_pad;
  int* const kc_pad = A.kc_pad;
  int* const rband = A.rband;
  int* const cband = A.cband;
  int* const kmap2 = A.kmap2;
  int* const orient = A.orient;
  int* const fused_sync = A.fused_sync;
  __shared__ int s_warp[33];
  __shared__ int s_cnt[2][CGH_MAX_LAYERS];  // kept bands per layer: object rows, object columns
  const int t = threadIdx.x;
  for (int e = t; e < 2 * CGH_MAX_LAYERS; e += blockDim.x) s_cnt[e / CGH_MAX_LAYERS][e % CGH_MAX_LAYERS] = 0;
  __syncthreads();
  for (int axis = 0; axis < 2; ++axis) {
    const int n8 = axis == 0 ? (H >> 3) : (W >> 3), n32 = (n8 + 3) >> 2;
    const uint8_t* band = axis == 0 ? fl.rowband : fl.colband;
    for (int e = t; e < Z * n32; e += blockDim.x) {
      const int zz = e / n32, b = e - (e / n32) * n32;
      int f = 0;
      for (int q = 4 * b; q < 4 * b + 4 && q < n8; ++q) f |= band[(size_t)zz * n8 + q];
      if (f) atomicAdd(&s_cnt[axis][zz], 1);
    }
  }
  __syncthreads();
  int tr = 0;
  if (H == W && order == CGH_CONTRACT_COLS) {
    tr = 1;
  } else if (H == W && order != CGH_CONTRACT_ROWS) {
    int sr = 0, sc = 0;
    for (int q = 0; q < Z; ++q) sr += s_cnt[0][q], sc += s_cnt[1][q];
    tr = sc < sr ? 1 : 0;
  }
  if (z == 0 && t == 0) *orient = tr;
  // the fused GEMM launch's counters (per-layer stage-1 tiles, cleared CTAs) start at zero
  if (z == 0 && fused_sync)
    for (int e = t; e <= CGH_MAX_LAYERS; e += blockDim.x) fused_sync[e] = 0;
  int koff = 0;  // this layer's first K step in the concatenated stage-2 K
  for (int q = 0; q < z; ++q) koff += s_cnt[tr][q];
  for (int axis = 0; axis < 2; ++axis) {
    const int role = axis ^ tr;  // 0: the stage-2 contraction ("rows") outputs, 1: "cols"
    const int n8 = axis == 0 ? (H >> 3) : (W >> 3);
    const int n32 = (n8 + 3) >> 2;
    const int lim = axis == 0 ? H : W;
    const uint8_t* band = axis == 0 ? fl.rowband + (size_t)z * (H >> 3) : fl.colband + (size_t)z * (W >> 3);
    int* out = role == 0 ? rows + (size_t)z * ld_rows : cols + (size_t)z * ld_cols;
    int* bout = role == 0 ? rband + (size_t)z * (ld_rows / 32) : cband + (size_t)z * (ld_cols / 32);
    int f = 0;
    if (t < n32)
      for (int q = 4 * t; q < 4 * t + 4 && q < n8; ++q) f |= band[q];
    int total;
    const int r = block_scan_flags(f ? 1 : 0, s_warp, &total);
    if (f) {
      for (int q = 0; q < 32; ++q) {
        const int v = 32 * t + q;
        out[32 * r + q] = v < lim ? v : -1;
      }
      bout[r] = role == 0 ? t : 32 * t;
      if (role == 0) kmap2[koff + r] = z * H + 32 * t;
    }
    if (t == 0) (role == 0 ? kr_pad : kc_pad)[z] = 32 * total;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(1024) k_tc_compact(const CompactArgs A) {
  pdl_wait();
  pdl_trigger();
  compact_body(A, blockIdx.x);
}

// Batched compaction: blockIdx.y is the scene, blockIdx.x its layer.
__global__ void __launch_bounds__(1024) k_tc_compact_batch(const CompactArgs* __restrict__ scenes) {
  pdl_wait();
  pdl_trigger();
  const CompactArgs& A = scenes[blockIdx.y];
  if ((int)blockIdx.x >= A.Z) return;
  compact_body(A, blockIdx.x);
}

// 64 x A^_z at eight consecutive pixels of one object row (ALONG_Y = false: (y0, x0 + q))
// or one object column (ALONG_Y = true: (y0 + q, x0)), the run starting on a multiple of 8,
// from the Haar coefficients and the selection flags:
// V = LLL + sum_{l=3,2,1} 4^(3-l) [selected] (sx X + sy Y + sx sy D), with sx = -1 for the
// right child column and sy = -1 for the lower child row of the level-l cell.  The run
// shares one LLL block and one level-3 block, and spans two level-2 and four level-1 blocks.
template <bool ALONG_Y>
__device__ __forceinline__ void idwt_run8(const int32_t* __restrict__ P, const TcFlags& fl, int z, int H, int W,
                                          int y0, int x0, int* V) {
  const int h3 = H >> 3, w3 = W >> 3, by3 = y0 >> 3, bx3 = x0 >> 3;
  const size_t f3 = ((size_t)z * h3 + by3) * w3 + bx3;
  if (fl.occ3[f3]) {
    const int LL = P[(size_t)by3 * W + bx3];
#pragma unroll
    for (int q = 0; q < 8; ++q) V[q] = LL;
  }
  if (fl.sel[3][f3]) {
    const int X = P[(size_t)by3 * W + w3 + bx3], Y = P[(size_t)(h3 + by3) * W + bx3],
              D = P[(size_t)(h3 + by3) * W + w3 + bx3];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int y = ALONG_Y ? y0 + q : y0, x = ALONG_Y ? x0 : x0 + q;
      const int sx = ((x >> 2) & 1) ? -1 : 1, sy = ((y >> 2) & 1) ? -1 : 1;
      V[q] += sx * X + sy * Y + sx * sy * D;
    }
  }
  const int h2 = H >> 2, w2 = W >> 2;
#pragma unroll
  for (int g = 0; g < 2; ++g) {
    const int by2 = ALONG_Y ? (y0 >> 2) + g : y0 >> 2, bx2 = ALONG_Y ? x0 >> 2 : (x0 >> 2) + g;
    if (fl.sel[2][((size_t)z * h2 + by2) * w2 + bx2]) {
      const int X = P[(size_t)by2 * W + w2 + bx2], Y = P[(size_t)(h2 + by2) * W + bx2],
                D = P[(size_t)(h2 + by2) * W + w2 + bx2];
#pragma unroll
      for (int q = 4 * g; q < 4 * g + 4; ++q) {
        const int y = ALONG_Y ? y0 + q : y0, x = ALONG_Y ? x0 : x0 + q;
        const int sx = ((x >> 1) & 1) ? -1 : 1, sy = ((y >> 1) & 1) ? -1 : 1;
        V[q] += 4 * (sx * X + sy * Y + sx * sy * D);
      }
    }
  }
  const int h1 = H >> 1, w1 = W >> 1;
#pragma unroll
  for (int g = 0; g < 4; ++g) {
    const int by1 = ALONG_Y ? (y0 >> 1) + g : y0 >> 1, bx1 = ALONG_Y ? x0 >> 1 : (x0 >> 1) + g;
    if (fl.sel[1][((size_t)z * h1 + by1) * w1 + bx1]) {
      const int X = P[(size_t)by1 * W + w1 + bx1], Y = P[(size_t)(h1 + by1) * W + bx1],
                D = P[(size_t)(h1 + by1) * W + w1 + bx1];
#pragma unroll
      for (int q = 2 * g; q < 2 * g + 2; ++q) {
        const int y = ALONG_Y ? y0 + q : y0, x = ALONG_Y ? x0 : x0 + q;
        const int sx = (x & 1) ? -1 : 1, sy = (y & 1) ? -1 : 1;
        V[q] += 16 * (sx * X + sy * Y + sx * sy * D);
      }
    }
  }
}

// Stage-1 B operand: 64 x A^_z at (rows[k], cols[c .. c+7]), or, in the transposed order,
// at (cols[c .. c+7], rows[k]) (the "rows" then hold object columns).  One thread builds the
// eight compacted columns of one 8-pixel band (or of padding).
struct IdwtArgs {
  const int32_t* coef;
  TcFlags fl;
  const int *rows, *cols, *kr_pad, *kc_pad, *orient;
  int H, W, ld_rows, ld_cols;
  uint16_t* B1;
  long long b1_plane;
  int ldb1;
};

template <bool F16>
__device__ __forceinline__ void idwt_body(const IdwtArgs& A, int z, int bxi, int byi) {
  const int32_t* __restrict__ coef = A.coef;
  const TcFlags& fl = A.fl;
  const int* __restrict__ rows = A.rows;
  const int* __restrict__ cols = A.cols;
  const int* __restrict__ kr_pad = A.kr_pad;
  const int* __restrict__ kc_pad = A.kc_pad;
  const int* __restrict__ orient = A.orient;
  const int H = A.H, W = A.W, ld_rows = A.ld_rows, ld_cols = A.ld_cols, ldb1 = A.ldb1;
  uint16_t* __restrict__ B1 = A.B1;
  const long long b1_plane = A.b1_plane;
  __shared__ int s_kr[CGH_MAX_LAYERS];
  // the layers' row counts, loaded in parallel (a per-thread loop of loads would cost a memory
  // latency per earlier layer)
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  if (tid <= z) s_kr[tid] = kr_pad[tid];
  __syncthreads();
  const int c = 8 * (bxi * blockDim.x + threadIdx.x);
  const int k = byi * blockDim.y + threadIdx.y;
  if (k >= s_kr[z] || c >= kc_pad[z]) return;
  int off = 0;
  for (int q = 0; q < z; ++q) off += s_kr[q];
  const int i = rows[(size_t)z * ld_rows + k], j0 = cols[(size_t)z * ld_cols + c];
  int V[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) V[q] = 0;
  if (i >= 0 && j0 >= 0) {
    const int32_t* P = coef + (size_t)z * H * W;
    if (*orient)
      idwt_run8<true>(P, fl, z, H, W, j0, i, V);
    else
      idwt_run8<false>(P, fl, z, H, W, i, j0, V);
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

template <bool F16>
__global__ void k_tc_idwt(const IdwtArgs A) {
  pdl_wait();
  pdl_trigger();
  idwt_body<F16>(A, blockIdx.z, blockIdx.x, blockIdx.y);
}

// Batched inverse DWT: blockIdx.z walks the (scene, layer) items (item.x scene, item.y
// layer); x and y cover the largest scene.
template <bool F16>
__global__ void k_tc_idwt_batch(const IdwtArgs* __restrict__ scenes, const int2* __restrict__ items) {
  pdl_wait();
  pdl_trigger();
  const int2 it = items[blockIdx.z];
  const IdwtArgs& A = scenes[it.x];
  if ((int)blockIdx.x * (int)blockDim.x * 8 >= A.ld_cols || (int)blockIdx.y * (int)blockDim.y >= A.ld_rows) return;
  idwt_body<F16>(A, it.y, blockIdx.x, blockIdx.y);
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
      (e = set_gemm_attr<KIND_CC, EPI_H, true>()) != cudaSuccess ||
      (e = set_gemm_attr<KIND_CR2, EPI_Y, true>()) != cudaSuccess ||
      (e = set_gemm_attr<KIND_CC2, EPI_H, true>()) != cudaSuccess ||
      (e = set_gemm_pair_attr<KIND_CC, false>()) != cudaSuccess ||
      (e = set_gemm_pair_attr<KIND_CC, true>()) != cudaSuccess ||
      (e = set_gemm_pair_attr<KIND_CC2, true>()) != cudaSuccess ||
      (e = set_fused_attr<KIND_CR, KIND_CC, false>()) != cudaSuccess ||
      (e = set_fused_attr<KIND_CR, KIND_CC, true>()) != cudaSuccess ||
      (e = set_fused_attr<KIND_CR2, KIND_CC2, true>()) != cudaSuccess)
    return cgh_cuda_check(e, "tensor-core kernel attributes");
  // how many CTA pairs the device holds, looked up once here (outside any capture)
  gemm_pair_clusters<KIND_CC, false>();
  gemm_pair_clusters<KIND_CC, true>();
  gemm_pair_clusters<KIND_CC2, true>();
  fused_max_ctas<KIND_CR, KIND_CC, false>();
  fused_max_ctas<KIND_CR, KIND_CC, true>();
  fused_max_ctas<KIND_CR2, KIND_CC2, true>();
  return CGH_OK;
}

struct cgh_tc_state {
  int kc_alloc, kr_alloc, ktot_alloc;
  uint8_t* flags;  // one block: occ3 | rowband | colband | sel1 | sel2 | sel3
  size_t flags_bytes, flags_alloc;  // used / allocated (a multiple of 16 bytes)
  int flags_dirty;  // host: flags may hold a previous call's marks (see tc_run)
  TcFlags fl;
  int *rows, *cols, *kr_pad, *kc_pad;
  int *rband, *cband, *kmap2;  // K-step band maps (see k_tc_compact)
  int* orient;                 // device: 1 when the last call contracted over object columns
  uint16_t *B1, *Y;
  long long b1_plane, y_plane;
  CUtensorMap mB1, mY;
  CUtensorMap mY64;  // the stage-1 output with 64-row boxes (stage 2 on CTA pairs)
  int* fused_sync;   // [CGH_MAX_LAYERS + 1] counters of the fused GEMM launch
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
  t->flags_alloc = (t->flags_bytes + 15) & ~(size_t)15;
  TC_TRY(cudaMalloc(&t->flags, t->flags_alloc), "tensor-core scratch: flags");
  TC_TRY(cudaMemset(t->flags, 0, t->flags_alloc), "tensor-core scratch: flags");
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
  TC_TRY(cudaMalloc(&t->rband, (size_t)Z * (t->kr_alloc / 32) * sizeof(int)), "tensor-core scratch: bands");
  TC_TRY(cudaMalloc(&t->cband, (size_t)Z * (t->kc_alloc / 32) * sizeof(int)), "tensor-core scratch: bands");
  TC_TRY(cudaMalloc(&t->kmap2, (size_t)(t->ktot_alloc / 32) * sizeof(int)), "tensor-core scratch: K map");
  TC_TRY(cudaMalloc(&t->fused_sync, (CGH_MAX_LAYERS + 1) * sizeof(int)), "tensor-core scratch: counters");
  TC_TRY(cudaMemset(t->fused_sync, 0, (CGH_MAX_LAYERS + 1) * sizeof(int)), "tensor-core scratch: counters");
  TC_TRY(cudaMalloc(&t->orient, sizeof(int)), "tensor-core scratch: order");
  TC_TRY(cudaMemset(t->orient, 0, sizeof(int)), "tensor-core scratch: order");
  t->b1_plane = (long long)t->ktot_alloc * t->kc_alloc;
  t->y_plane = (long long)p->holo_w * t->ktot_alloc;
  TC_TRY(cudaMalloc(&t->B1, 2 * t->b1_plane * sizeof(uint16_t)), "tensor-core scratch: B1");
  TC_TRY(cudaMalloc(&t->Y, 4 * t->y_plane * sizeof(uint16_t)), "tensor-core scratch: Y");
  if ((rc = make_plane_map(&t->mB1, t->B1, 2, t->ktot_alloc, t->kc_alloc)) != CGH_OK) goto fail;
  if ((rc = make_plane_map(&t->mY, t->Y, 4, p->holo_w, t->ktot_alloc)) != CGH_OK) goto fail;
  if ((rc = make_plane_map(&t->mY64, t->Y, 4, p->holo_w, t->ktot_alloc, 64)) != CGH_OK) goto fail;
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
  cudaFree(t->rband);
  cudaFree(t->cband);
  cudaFree(t->kmap2);
  cudaFree(t->orient);
  cudaFree(t->fused_sync);
  cudaFree(t->B1);
  cudaFree(t->Y);
  free(t);
  p->tc = nullptr;
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

#define TC_CK(expr, what)                                   \
  do {                                                      \
    int _rc = cgh_cuda_check((expr), (what));               \
    if (_rc != CGH_OK) return _rc;                          \
  } while (0)

static CompactArgs compact_args(const cgh_plan* p) {
  cgh_tc_state* t = p->tc;
  return CompactArgs{t->fl,       p->obj_h,    p->obj_w,     p->n_layers, p->contraction, t->rows,
                     t->cols,     t->kr_pad,   t->kc_pad,    t->kr_alloc, t->kc_alloc,    t->rband,
                     t->cband,    t->kmap2,    t->orient,    t->fused_sync};
}

static IdwtArgs idwt_args(const cgh_plan* p, const int32_t* coef) {
  cgh_tc_state* t = p->tc;
  return IdwtArgs{coef,     t->fl,       t->rows,     t->cols,     t->kr_pad,   t->kc_pad,   t->orient,
                  p->obj_h, p->obj_w,    t->kr_alloc, t->kc_alloc, t->B1,       t->b1_plane, t->kc_alloc};
}

// Operands of both GEMM stages for one scene: selection flags, per-layer band compaction,
// the stage-2 K-step map and the inverse-DWT operand (stage-1 B).  The A operands of both
// stages are the plan's fringe planes (eops_get), read band by band through the K maps.
// flags_ready: the selection flags were marked by the fused selection (tc_progressive_step)
// instead of being derived here from the lists.
template <bool F16>
static int tc_prep(const cgh_plan* p, const int32_t* coef, const int32_t* const* lists, const int32_t* d_counts,
                   cudaStream_t st, bool flags_ready = false, cudaEvent_t coef_ready = nullptr) {
  cgh_tc_state* t = p->tc;
  const int H = p->obj_h, W = p->obj_w, Z = p->n_layers;
  if (!flags_ready) {
    // the flags are clear unless a call left them marked (the single-scene path clears them
    // in its stage-1 kernel for the next call)
    if (t->flags_dirty) TC_CK(cudaMemsetAsync(t->flags, 0, t->flags_bytes, st), "tc: clear flags");
    t->flags_dirty = 1;
    TC_CK(launch_pdl(k_tc_scatter, dim3(64, 4), dim3(256), 0, st, lists[0], lists[1], lists[2], lists[3],
                     d_counts, t->fl, H, W, Z, p->d_status),
          "tc: scatter");
  }
  TC_CK(launch_pdl(k_tc_compact, dim3(Z), dim3(1024), 0, st, compact_args(p)), "tc: compact");
  if (coef_ready) TC_CK(cudaStreamWaitEvent(st, coef_ready, 0), "tc: wait for the coefficients");
  {
    dim3 blk(8, 32), grid((t->kc_alloc / 8 + 7) / 8, (t->kr_alloc + 31) / 32, Z);
    TC_CK(launch_pdl(k_tc_idwt<F16>, grid, blk, 0, st, idwt_args(p, coef)), "tc: idwt");
  }

  return CGH_OK;
}

// Stage 1: Y^T = E_z[:, cols] * A^_z[rows, cols]^T / 64 (scaled by a further 2^-4 for fp16
// headroom); units (M tiles, N tiles, layers).
static void stage1_args(const cgh_plan* p, bool f16, TcGemmArgs& a, dim3& tiles) {
  cgh_tc_state* t = p->tc;
  memset(&a, 0, sizeof(a));
  a.mode = 1;
  a.a_rows_per_z = p->holo_w;
  a.kr_pad = t->kr_pad;
  a.kc_pad = t->kc_pad;
  a.n_layers = p->n_layers;
  a.M = p->holo_w;
  a.N = t->ktot_alloc;
  // fp16: a further 2^-4, and 2^-lf_extra for the layer factor's 1/sqrt(z) on each fringe
  a.scale = f16 ? ldexpf(1.0f, -10 - p->lf_extra) : 1.0f / 64.0f;
  a.Y = t->Y;
  a.y_plane = t->y_plane;
  a.ldy = t->ktot_alloc;
  a.y_rows = p->holo_w;
  a.status = p->d_status;
  a.a_kmap = t->cband;
  a.a_kmap_ld = t->kc_alloc / 32;
  tiles = dim3((p->holo_w + TC_BM - 1) / TC_BM, (t->kr_alloc + TC_BN - 1) / TC_BN, p->n_layers);
  a.tm = tiles.x;
  a.tn = tiles.y;
  a.tz = tiles.z;
}

// Stage 2: H += sum_kappa E[m][kappa] Y^T[n][kappa] over the concatenated layer rows,
// K split S ways; units (M tiles, N tiles, S).
static void stage2_args(const cgh_plan* p, bool f16, float2* holo, int S, TcGemmArgs& a, dim3& tiles) {
  cgh_tc_state* t = p->tc;
  memset(&a, 0, sizeof(a));
  a.mode = 2;
  a.kr_pad = t->kr_pad;
  a.n_layers = p->n_layers;
  a.M = p->holo_h;
  a.N = p->holo_w;
  a.scale = f16 ? ldexpf(1.0f, 4 + p->lf_extra) : 1.0f;
  a.H = holo;
  a.ldh = p->holo_w;
  a.h_vec4 = ((p->holo_w & 1) == 0) && (((uintptr_t)holo & 15) == 0);
  a.h_transposed = t->orient;
  a.status = p->d_status;
  a.a_kmap = t->kmap2;
  tiles = dim3((p->holo_h + TC_BM - 1) / TC_BM, (p->holo_w + TC_BN - 1) / TC_BN, S);
  a.tm = tiles.x;
  a.tn = tiles.y;
  a.tz = tiles.z;
}

// X2 (fp16 only): the fringe operand as its hi planes, two products per real product
// (CGH_FORM_TC_FP16X2).
template <bool F16, bool X2 = false>
static int tc_run(const cgh_plan* p, const int32_t* coef, const int32_t* const* lists, const int32_t* d_counts,
                  float2* holo, int accumulate, cudaStream_t st, bool flags_ready = false,
                  cudaEvent_t coef_ready = nullptr) {
  static_assert(F16 || !X2, "the hi-only fringe form is fp16");
  constexpr int K1 = X2 ? KIND_CR2 : KIND_CR, K2 = X2 ? KIND_CC2 : KIND_CC;
  cgh_tc_state* t = p->tc;
  const CUtensorMap *mEZ, *mEZt;
  int rc = X2 ? eops_get_hi(p, 1, &mEZ, &mEZt, st) : eops_get(p, F16 ? 1 : 0, &mEZ, &mEZt, st);
  if (rc != CGH_OK) return rc;
  // H is cleared by the stage-1 kernel's idle warps when it can be cleared in float4 units
  const size_t hpix = (size_t)p->holo_h * p->holo_w;
  const bool h_zero_in_stage1 = !accumulate && (hpix % 2 == 0) && (((uintptr_t)holo & 15) == 0);
  if (!accumulate && !h_zero_in_stage1) TC_CK(cudaMemsetAsync(holo, 0, hpix * sizeof(float2), st), "tc: clear");
  prof_mark(p, CGH_PROF_TC_PREP, 0, st);
  rc = tc_prep<F16>(p, coef, lists, d_counts, st, flags_ready, coef_ready);
  if (rc != CGH_OK) return rc;
  prof_mark(p, CGH_PROF_TC_PREP, 1, st);
  TcGemmArgs a1, a2;
  dim3 tiles1, tiles2;
  stage1_args(p, F16, a1, tiles1);
  a1.zero_ptr[0] = reinterpret_cast<float4*>(t->flags);  // marks of this call, for the next one
  a1.zero_n[0] = (long long)(t->flags_alloc / 16);
  if (h_zero_in_stage1) {
    a1.zero_ptr[1] = reinterpret_cast<float4*>(holo);
    a1.zero_n[1] = (long long)(hpix / 2);
  }
  const int tm = (p->holo_h + TC_BM - 1) / TC_BM, tn = (p->holo_w + TC_BN - 1) / TC_BN;
  // Stream-K over the (tile, K step) space unless the plan asks for single-writer tiles
  // (deterministic).  Chains of at most the plan's cap, else 32 K steps for fp16 hi+lo
  // (whose 1e-5 bar the tensor pipe's chain-length error would otherwise approach) and 128
  // for bf16 hi+lo (whose error is its operand split, far above that of the chains), which
  // halves the partial-sum atomics.
  const int streamk = p->deterministic ? 0 : (p->max_ksteps > 0 ? p->max_ksteps : (F16 && !X2 ? 32 : 128));
  int S = p->deterministic ? 1 : stage2_splits(tm * tn, t->ktot_alloc / TC_BK);
  if (!p->deterministic && p->max_ksteps > 0) {
    // cap the chain length on the actual K: sum of the layers' compacted rows is at most
    // the allocation, so bound it by the allocation's K steps scaled to the occupancy seen
    const int kst = t->ktot_alloc / TC_BK;
    const int need = (kst + p->max_ksteps - 1) / p->max_ksteps;
    if (need > S) S = need;
  }
  stage2_args(p, F16, holo, S, a2, tiles2);
  a2.streamk = streamk;
  cudaError_t e = cudaErrorNotSupported;
  if (streamk > 0 && p->fusion && p->stage2_tiles != CGH_TILES_PAIR) {
    // both stages in one cooperative launch (stage 2 starts on finished layers)
    prof_mark(p, CGH_PROF_TC_FUSED, 0, st);
    e = launch_fused<K1, K2, F16>(*mEZt, t->mB1, t->mY, *mEZ, a1, tiles1, a2, tiles2, t->fused_sync, st);
    prof_mark(p, CGH_PROF_TC_FUSED, 1, st);
    if (e != cudaErrorNotSupported) {
      TC_CK(e, "tc: fused GEMMs");
      t->flags_dirty = 0;
      return CGH_OK;
    }
  }
  // both stages' A operands are the plan's fringe planes and their K sizes and maps come from
  // the compaction, two or more kernels back: their first A loads may start early
  a1.a_early = 1;
  a2.a_early = 1;
  prof_mark(p, CGH_PROF_TC_STAGE1, 0, st);
  e = launch_gemm<K1, EPI_Y, F16>(*mEZt, t->mB1, t->mY, a1, tiles1, st);
  prof_mark(p, CGH_PROF_TC_STAGE1, 1, st);
  TC_CK(e, "tc: stage-1 GEMM");
  t->flags_dirty = 0;
  prof_mark(p, CGH_PROF_TC_STAGE2, 0, st);
  e = cudaErrorNotSupported;
  // CTA pairs when asked, or by default once the hologram has at least 64 128x128 tiles
  // (1024^2 and larger): with both kernels starting early behind stage 1, pairs take the
  // paper-scale step from 0.1312 to 0.1292 ms (2048^2: 2-3% faster); smaller holograms keep
  // one CTA per tile
  const bool pairs = p->stage2_tiles == CGH_TILES_PAIR || (p->stage2_tiles == CGH_TILES_AUTO && tm * tn >= 64);
  const_cast<cgh_plan*>(p)->stage2_used = CGH_TILES_CTA;
  if (streamk > 0 && pairs) {
    e = launch_gemm_pair<K2, F16>(*mEZ, t->mY64, a2, tiles2, st);
    if (e == cudaSuccess) const_cast<cgh_plan*>(p)->stage2_used = CGH_TILES_PAIR;
  }
  if (e == cudaErrorNotSupported) e = launch_gemm<K2, EPI_H, F16>(*mEZ, t->mY, t->mY, a2, tiles2, st);
  prof_mark(p, CGH_PROF_TC_STAGE2, 1, st);
  TC_CK(e, "tc: stage-2 GEMM");
  return CGH_OK;
}

// ------------------------------------------------------------------------------------
// batches: many scenes, each with its own plan, through one persistent launch per stage

__global__ void k_batch_koff(TcBatchItem* __restrict__ a, TcBatchItem* __restrict__ b, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int o = 0;
  a[i].koff[0] = b[i].koff[0] = 0;
  for (int q = 0; q < a[i].a.n_layers; ++q) {
    o += a[i].a.kr_pad[q];
    a[i].koff[q + 1] = b[i].koff[q + 1] = o;
  }
}

// A region the batch clears before its preparation (selection flags, holograms).
struct ZeroRegion {
  float4* p;
  long long n;  // float4 units
};

__global__ void k_zero_regions(const ZeroRegion* __restrict__ regs) {
  const ZeroRegion r = regs[blockIdx.y];
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < r.n; i += (long long)gridDim.x * blockDim.x)
    r.p[i] = make_float4(0.f, 0.f, 0.f, 0.f);
}

struct cgh_batch {
  int n, form, ksteps;
  cgh_plan** plans;
  const uint8_t **I, **L, **S;
  float2** H;
  int thr[3];
  int32_t** coeffs;
  int32_t** lists;  // [n][4]
  int32_t* counts;  // device [n][4][2]
  TcBatchItem *h1, *h2, *d1, *d2;
  int units1, units2, units2p;
  int stage2_tiles;  // CGH_TILES_*: stage 2 on one CTA per tile or on CTA pairs
  // one launch per preparation kernel across the scenes: device tables and scratch
  ZeroRegion* d_zero;
  int n_zero;
  HaarItem* d_haar;
  int n_haar, max_h, max_w;
  SelTaskB* d_sel;
  int n_sel, sel_chunks, sel_scan_blocks;
  int *sel_cnt, *sel_off;
  CompactArgs* d_compact;
  int max_z;
  IdwtArgs* d_idwt;
  int2* d_idwt_items;
  int max_kr, max_kc;
};

// Device tables of the batched preparation (built once per batch: every pointer is fixed).
static int batch_prep_tables(cgh_batch* b) {
  const int n = b->n;
  std::vector<ZeroRegion> zero;
  std::vector<HaarItem> haar;
  std::vector<SelTaskB> sel;
  std::vector<CompactArgs> comp;
  std::vector<IdwtArgs> idw;
  std::vector<int2> items;
  int chunk0 = 0, cnt_off = 0, scan_blocks = 1;
  b->max_h = b->max_w = b->max_z = b->max_kr = b->max_kc = 0;
  for (int i = 0; i < n; ++i) {
    const cgh_plan* p = b->plans[i];
    cgh_tc_state* t = p->tc;
    const int H = p->obj_h, W = p->obj_w, Z = p->n_layers;
    zero.push_back(ZeroRegion{reinterpret_cast<float4*>(t->flags), (long long)(t->flags_alloc / 16)});
    const size_t hb = (size_t)p->holo_h * p->holo_w * sizeof(float2);
    if (hb % 16 || ((uintptr_t)b->H[i] & 15))
      return cgh_fail(CGH_ERR_ARG, "cgh_batch: hologram %d must be 16-byte aligned with an even pixel count", i);
    zero.push_back(ZeroRegion{reinterpret_cast<float4*>(b->H[i]), (long long)(hb / 16)});
    for (int z = 0; z < Z; ++z) {
      haar.push_back(HaarItem{b->I[i], b->L[i], b->coeffs[i], H, W, z});
      items.push_back(make_int2(i, z));
    }
    for (int k = 0; k < 4; ++k) {
      SelTaskB tb;
      memset(&tb, 0, sizeof(tb));
      const int lvl = k == 0 ? CGH_LEVELS : k;
      tb.t.level = lvl;
      tb.t.threshold = k == 0 ? -1 : b->thr[k - 1];
      tb.t.capacity = Z * (H >> lvl) * (W >> lvl);
      tb.t.nchunks = select_num_chunks(H, W, lvl);
      tb.t.chunk0 = chunk0;
      tb.t.cnt_off = cnt_off;
      tb.t.flag_kind = k == 0 ? SEL_FLAGS_LLL : SEL_FLAGS_DETAIL;
      tb.t.list = b->lists[4 * i + k];
      tb.t.count = b->counts + 8 * i + 2 * k;
      tb.sal = k == 0 ? nullptr : b->S[i];
      tb.L = b->L[i];
      tb.H = H;
      tb.W = W;
      tb.Z = Z;
      tb.fl = t->fl;
      chunk0 += tb.t.nchunks;
      cnt_off += Z * tb.t.nchunks;
      const int sb = select_scan_blocks(Z, tb.t.nchunks);
      scan_blocks = sb > scan_blocks ? sb : scan_blocks;
      sel.push_back(tb);
    }
    comp.push_back(compact_args(p));
    idw.push_back(idwt_args(p, b->coeffs[i]));
    b->max_h = H > b->max_h ? H : b->max_h;
    b->max_w = W > b->max_w ? W : b->max_w;
    b->max_z = Z > b->max_z ? Z : b->max_z;
    b->max_kr = t->kr_alloc > b->max_kr ? t->kr_alloc : b->max_kr;
    b->max_kc = t->kc_alloc > b->max_kc ? t->kc_alloc : b->max_kc;
  }
  b->n_zero = (int)zero.size();
  b->n_haar = (int)haar.size();
  b->n_sel = (int)sel.size();
  b->sel_chunks = chunk0;
  b->sel_scan_blocks = scan_blocks;
  if (b->n_haar > 65535) return cgh_fail(CGH_ERR_ARG, "cgh_batch: more than 65535 scene layers");
#define BP_TRY(expr, what)                            \
  do {                                                \
    int _rc = cgh_cuda_check((expr), (what));         \
    if (_rc != CGH_OK) return _rc;                    \
  } while (0)
  BP_TRY(cudaMalloc(&b->d_zero, zero.size() * sizeof(ZeroRegion)), "cgh_batch: tables");
  BP_TRY(cudaMalloc(&b->d_haar, haar.size() * sizeof(HaarItem)), "cgh_batch: tables");
  BP_TRY(cudaMalloc(&b->d_sel, sel.size() * sizeof(SelTaskB)), "cgh_batch: tables");
  BP_TRY(cudaMalloc(&b->d_compact, comp.size() * sizeof(CompactArgs)), "cgh_batch: tables");
  BP_TRY(cudaMalloc(&b->d_idwt, idw.size() * sizeof(IdwtArgs)), "cgh_batch: tables");
  BP_TRY(cudaMalloc(&b->d_idwt_items, items.size() * sizeof(int2)), "cgh_batch: tables");
  BP_TRY(cudaMalloc(&b->sel_cnt, (size_t)cnt_off * sizeof(int)), "cgh_batch: selection scratch");
  BP_TRY(cudaMalloc(&b->sel_off, (size_t)cnt_off * sizeof(int)), "cgh_batch: selection scratch");
  BP_TRY(cudaMemcpy(b->d_zero, zero.data(), zero.size() * sizeof(ZeroRegion), cudaMemcpyHostToDevice), "cgh_batch: tables");
  BP_TRY(cudaMemcpy(b->d_haar, haar.data(), haar.size() * sizeof(HaarItem), cudaMemcpyHostToDevice), "cgh_batch: tables");
  BP_TRY(cudaMemcpy(b->d_sel, sel.data(), sel.size() * sizeof(SelTaskB), cudaMemcpyHostToDevice), "cgh_batch: tables");
  BP_TRY(cudaMemcpy(b->d_compact, comp.data(), comp.size() * sizeof(CompactArgs), cudaMemcpyHostToDevice),
         "cgh_batch: tables");
  BP_TRY(cudaMemcpy(b->d_idwt, idw.data(), idw.size() * sizeof(IdwtArgs), cudaMemcpyHostToDevice), "cgh_batch: tables");
  BP_TRY(cudaMemcpy(b->d_idwt_items, items.data(), items.size() * sizeof(int2), cudaMemcpyHostToDevice),
         "cgh_batch: tables");
#undef BP_TRY
  return CGH_OK;
}

static int batch_upload(cgh_batch* b) {
  const bool f16 = b->form == CGH_FORM_TC_FP16X3;
  int u1 = 0, u2 = 0, u2p = 0;
  for (int i = 0; i < b->n; ++i) {
    const cgh_plan* p = b->plans[i];
    cgh_tc_state* t = p->tc;
    dim3 tiles;
    const CUtensorMap *mEZ, *mEZt;
    const int rc = eops_get(p, f16 ? 1 : 0, &mEZ, &mEZt, 0);
    if (rc != CGH_OK) return rc;
    b->h1[i].ma = *mEZt;
    b->h1[i].mb = t->mB1;
    b->h1[i].mc = t->mY;
    stage1_args(p, f16, b->h1[i].a, tiles);
    b->h1[i].unit0 = u1;
    u1 += tiles.x * tiles.y * tiles.z;
    const int tm = (p->holo_h + TC_BM - 1) / TC_BM, tn = (p->holo_w + TC_BN - 1) / TC_BN;
    const int kst = t->ktot_alloc / TC_BK;
    int S = p->deterministic ? 1 : (kst + b->ksteps - 1) / b->ksteps;
    if (S < 1) S = 1;
    b->h2[i].ma = *mEZ;
    b->h2[i].mb = t->mY;
    b->h2[i].mc = t->mY;
    b->h2[i].mb64 = t->mY64;
    stage2_args(p, f16, b->H[i], S, b->h2[i].a, tiles);
    b->h2[i].unit0 = u2;
    b->h2[i].unit0p = u2p;
    u2 += tiles.x * tiles.y * tiles.z;
    u2p += ((tiles.x + 1) / 2) * tiles.y * tiles.z;
  }
  b->units1 = u1;
  b->units2 = u2;
  b->units2p = u2p;
  TC_CK(cudaMemcpy(b->d1, b->h1, b->n * sizeof(TcBatchItem), cudaMemcpyHostToDevice), "batch: upload");
  TC_CK(cudaMemcpy(b->d2, b->h2, b->n * sizeof(TcBatchItem), cudaMemcpyHostToDevice), "batch: upload");
  return CGH_OK;
}

extern "C" int cgh_batch_destroy(cgh_batch* b) {
  if (!b) return CGH_OK;
  cudaDeviceSynchronize();
  for (int i = 0; i < b->n; ++i) {
    if (b->coeffs) cudaFree(b->coeffs[i]);
    if (b->lists)
      for (int k = 0; k < 4; ++k) cudaFree(b->lists[4 * i + k]);
  }
  cudaFree(b->counts);
  cudaFree(b->d1);
  cudaFree(b->d2);
  cudaFree(b->d_zero);
  cudaFree(b->d_haar);
  cudaFree(b->d_sel);
  cudaFree(b->sel_cnt);
  cudaFree(b->sel_off);
  cudaFree(b->d_compact);
  cudaFree(b->d_idwt);
  cudaFree(b->d_idwt_items);
  free(b->h1);
  free(b->h2);
  free(b->coeffs);
  free(b->lists);
  free(b->plans);
  free(b->I);
  free(b->L);
  free(b->S);
  free(b->H);
  free(b);
  return CGH_OK;
}

extern "C" int cgh_batch_create(cgh_batch** out, cgh_plan* const* plans, int n, const uint8_t* const* intensity,
                                const uint8_t* const* layer_idx, const uint8_t* const* saliency,
                                const int* thresholds, float* const* holos, int form, void* stream) {
  if (!out || !plans || !intensity || !layer_idx || !saliency || !thresholds || !holos)
    return cgh_fail(CGH_ERR_ARG, "cgh_batch_create: NULL argument");
  *out = nullptr;
  if (n < 1 || n > TC_BATCH_MAX) return cgh_fail(CGH_ERR_ARG, "cgh_batch_create: n %d not in 1..%d", n, TC_BATCH_MAX);
  if (form != CGH_FORM_TC_BF16X3 && form != CGH_FORM_TC_FP16X3)
    return cgh_fail(CGH_ERR_UNSUPPORTED, "cgh_batch_create: batches run the tensor-core forms");
  for (int k = 0; k < 3; ++k)
    if (thresholds[k] < -1 || thresholds[k] > 255) return cgh_fail(CGH_ERR_ARG, "cgh_batch_create: bad threshold");
  for (int i = 0; i < n; ++i) {
    if (!plans[i] || !intensity[i] || !layer_idx[i] || !saliency[i] || !holos[i])
      return cgh_fail(CGH_ERR_ARG, "cgh_batch_create: NULL pointer for scene %d", i);
    if (((uintptr_t)intensity[i] & 7) || ((uintptr_t)layer_idx[i] & 7) || ((uintptr_t)saliency[i] & 7) ||
        ((uintptr_t)holos[i] & 7))
      return cgh_fail(CGH_ERR_ARG, "cgh_batch_create: misaligned buffer for scene %d", i);
  }
  cgh_batch* b = (cgh_batch*)calloc(1, sizeof(cgh_batch));
  if (!b) return cgh_fail(CGH_ERR_NOMEM, "cgh_batch_create: host allocation");
  b->n = n;
  b->form = form;
  b->ksteps = 32;
  for (int k = 0; k < 3; ++k) b->thr[k] = thresholds[k];
  b->plans = (cgh_plan**)calloc(n, sizeof(cgh_plan*));
  b->I = (const uint8_t**)calloc(n, sizeof(void*));
  b->L = (const uint8_t**)calloc(n, sizeof(void*));
  b->S = (const uint8_t**)calloc(n, sizeof(void*));
  b->H = (float2**)calloc(n, sizeof(void*));
  b->coeffs = (int32_t**)calloc(n, sizeof(void*));
  b->lists = (int32_t**)calloc(4 * (size_t)n, sizeof(void*));
  b->h1 = (TcBatchItem*)aligned_alloc(128, n * sizeof(TcBatchItem));
  b->h2 = (TcBatchItem*)aligned_alloc(128, n * sizeof(TcBatchItem));
  int rc = CGH_OK;
  if (!b->plans || !b->I || !b->L || !b->S || !b->H || !b->coeffs || !b->lists || !b->h1 || !b->h2) {
    cgh_batch_destroy(b);
    return cgh_fail(CGH_ERR_NOMEM, "cgh_batch_create: host allocation");
  }
  memset(b->h1, 0, n * sizeof(TcBatchItem));
  memset(b->h2, 0, n * sizeof(TcBatchItem));
#define B_TRY(expr, what)                  \
  do {                                     \
    rc = cgh_cuda_check((expr), (what));   \
    if (rc != CGH_OK) {                    \
      cgh_batch_destroy(b);                \
      return rc;                           \
    }                                      \
  } while (0)
  B_TRY(cudaMalloc(&b->counts, (size_t)n * 8 * sizeof(int32_t)), "cgh_batch_create: counts");
  B_TRY(cudaMalloc(&b->d1, n * sizeof(TcBatchItem)), "cgh_batch_create: items");
  B_TRY(cudaMalloc(&b->d2, n * sizeof(TcBatchItem)), "cgh_batch_create: items");
  for (int i = 0; i < n; ++i) {
    cgh_plan* p = plans[i];
    b->plans[i] = p;
    b->I[i] = intensity[i];
    b->L[i] = layer_idx[i];
    b->S[i] = saliency[i];
    b->H[i] = (float2*)holos[i];
    if ((rc = tc_ensure(p)) != CGH_OK) {
      cgh_batch_destroy(b);
      return rc;
    }
    B_TRY(cudaMalloc(&b->coeffs[i], (size_t)p->n_layers * p->obj_h * p->obj_w * sizeof(int32_t)),
          "cgh_batch_create: coefficients");
    for (int k = 0; k < 4; ++k) {
      const int lvl = k == 0 ? 3 : k;
      const size_t cap = (size_t)p->n_layers * (p->obj_h >> lvl) * (p->obj_w >> lvl);
      B_TRY(cudaMalloc(&b->lists[4 * i + k], cap * sizeof(int32_t)), "cgh_batch_create: lists");
    }
  }
#undef B_TRY
  if ((rc = batch_upload(b)) != CGH_OK || (rc = batch_prep_tables(b)) != CGH_OK) {
    cgh_batch_destroy(b);
    return rc;
  }
  (void)stream;
  *out = b;
  return CGH_OK;
}

extern "C" int cgh_batch_set_stage2_tiles(cgh_batch* b, int tiles) {
  if (!b || (tiles != CGH_TILES_CTA && tiles != CGH_TILES_PAIR && tiles != CGH_TILES_AUTO))
    return cgh_fail(CGH_ERR_ARG, "cgh_batch_set_stage2_tiles: bad argument");
  b->stage2_tiles = tiles == CGH_TILES_AUTO ? CGH_TILES_CTA : tiles;
  return CGH_OK;
}

extern "C" int cgh_batch_set_tuning(cgh_batch* b, int ksteps_per_unit) {
  if (!b || ksteps_per_unit < 1) return cgh_fail(CGH_ERR_ARG, "cgh_batch_set_tuning: bad argument");
  cudaDeviceSynchronize();
  b->ksteps = ksteps_per_unit;
  return batch_upload(b);
}

// One launch per preparation kernel across all scenes: clear flags and holograms, DWT,
// the three selection passes (which also mark the tensor-core flags), compaction, inverse
// DWT; then the per-scene K offsets and one persistent launch per GEMM stage.
template <bool F16>
static int batch_run(cgh_batch* b, cudaStream_t st) {
  k_zero_regions<<<dim3(64, b->n_zero), 256, 0, st>>>(b->d_zero);
  TC_CK(cudaGetLastError(), "batch: clear");
  TC_CK(launch_haar_batch(b->d_haar, b->n_haar, b->max_h, b->max_w, st), "batch: DWT");
  TC_CK(launch_select_batch(b->d_sel, b->n_sel, b->sel_chunks, b->sel_scan_blocks, b->sel_cnt, b->sel_off, st),
        "batch: selection");
  TC_CK(launch_pdl(k_tc_compact_batch, dim3(b->max_z, b->n), dim3(1024), 0, st, (const CompactArgs*)b->d_compact),
        "batch: compact");
  {
    dim3 blk(8, 32), grid((b->max_kc / 8 + 7) / 8, (b->max_kr + 31) / 32, b->n_haar);
    TC_CK(launch_pdl(k_tc_idwt_batch<F16>, grid, blk, 0, st, (const IdwtArgs*)b->d_idwt,
                     (const int2*)b->d_idwt_items),
          "batch: idwt");
  }
  for (int i = 0; i < b->n; ++i) b->plans[i]->tc->flags_dirty = 1;
  k_batch_koff<<<(b->n + 127) / 128, 128, 0, st>>>(b->d1, b->d2, b->n);
  TC_CK(cudaGetLastError(), "batch: offsets");
  const int sms = tc_num_sms();
  int* status = b->plans[0]->d_status;
  k_tc_gemm_batch<KIND_CR, EPI_Y, F16><<<b->units1 < sms ? b->units1 : sms, 192, tc_smem_bytes<KIND_CR, EPI_Y>(), st>>>(
      b->d1, b->n, b->units1, status);
  TC_CK(cudaGetLastError(), "batch: stage 1");
  cudaError_t e = cudaErrorNotSupported;
  if (b->stage2_tiles == CGH_TILES_PAIR) e = launch_gemm_pair_batch<KIND_CC, F16>(b->d2, b->n, b->units2p, status, st);
  if (e == cudaErrorNotSupported) {
    k_tc_gemm_batch<KIND_CC, EPI_H, F16><<<b->units2 < sms ? b->units2 : sms, 192, tc_smem_bytes<KIND_CC, EPI_H>(),
                                           st>>>(b->d2, b->n, b->units2, status);
    e = cudaGetLastError();
  }
  TC_CK(e, "batch: stage 2");
  return CGH_OK;
}

extern "C" int cgh_batch_run(cgh_batch* b, void* stream) {
  if (!b) return cgh_fail(CGH_ERR_ARG, "cgh_batch_run: batch is NULL");
  if (b->form == CGH_FORM_TC_FP16X3) return batch_run<true>(b, (cudaStream_t)stream);
  return batch_run<false>(b, (cudaStream_t)stream);
}

extern "C" int cgh_batch_lists(const cgh_batch* b, int scene, int32_t** lists, int32_t** d_counts,
                               int32_t** coeffs) {
  if (!b || scene < 0 || scene >= b->n || !lists || !d_counts || !coeffs)
    return cgh_fail(CGH_ERR_ARG, "cgh_batch_lists: bad argument");
  for (int k = 0; k < 4; ++k) lists[k] = b->lists[4 * scene + k];
  *d_counts = b->counts + 8 * scene;
  *coeffs = b->coeffs[scene];
  return CGH_OK;
}

int tc_progressive(const cgh_plan* p, const int32_t* coef, const int32_t* const* lists, const int32_t* d_counts,
                   float2* holo, int accumulate, int form, cudaStream_t st) {
  if (p->obj_h > 8192 || p->obj_w > 8192)
    return cgh_fail(CGH_ERR_UNSUPPORTED, "tensor-core form: object too large");
  int rc = tc_ensure(p);
  if (rc != CGH_OK) return rc;
  if (form == CGH_FORM_TC_FP16X3) return tc_run<true>(p, coef, lists, d_counts, holo, accumulate, st);
  if (form == CGH_FORM_TC_FP16X2) return tc_run<true, true>(p, coef, lists, d_counts, holo, accumulate, st);
  return tc_run<false>(p, coef, lists, d_counts, holo, accumulate, st);
}

// Selection and superposition in one call: the fused selection writes the lists and marks
// the selection flags itself when its tables are small (else the flags come from the lists).
int tc_progressive_step(const cgh_plan* p, const uint8_t* sal, const uint8_t* L, const int32_t* coef,
                        cudaEvent_t coef_ready, SelTasks T, const int32_t* const* lists, const int32_t* d_counts,
                        float2* holo, int accumulate, int form, cudaStream_t st) {
  if (p->obj_h > 8192 || p->obj_w > 8192)
    return cgh_fail(CGH_ERR_UNSUPPORTED, "tensor-core form: object too large");
  int rc = tc_ensure(p);
  if (rc != CGH_OK) return rc;
  cgh_tc_state* t = p->tc;
  if (t->flags_dirty) TC_CK(cudaMemsetAsync(t->flags, 0, t->flags_bytes, st), "tc: clear flags");
  t->flags_dirty = 1;
  for (int k = 0; k < T.n; ++k) T.t[k].flag_kind = k == 0 ? SEL_FLAGS_LLL : SEL_FLAGS_DETAIL;
  const SelCoop coop = plan_sel_coop(p);
  bool done = false;
  prof_mark(p, CGH_PROF_SELECT, 0, st);
  TC_CK(launch_select_tasks(p->obj_h, p->obj_w, p->n_layers, sal, L, T, p->d_chunk_cnt, p->d_chunk_off, st, &coop,
                            &t->fl, &done),
        "tc: selection");
  prof_mark(p, CGH_PROF_SELECT, 1, st);
  if (!done)
    TC_CK(launch_pdl(k_tc_scatter, dim3(64, 4), dim3(256), 0, st, lists[0], lists[1], lists[2], lists[3], d_counts,
                     t->fl, p->obj_h, p->obj_w, p->n_layers, p->d_status),
          "tc: scatter");
  if (form == CGH_FORM_TC_FP16X3) return tc_run<true>(p, coef, lists, d_counts, holo, accumulate, st, true, coef_ready);
  if (form == CGH_FORM_TC_FP16X2)
    return tc_run<true, true>(p, coef, lists, d_counts, holo, accumulate, st, true, coef_ready);
  return tc_run<false>(p, coef, lists, d_counts, holo, accumulate, st, true, coef_ready);
}

int tc_build_flags(const cgh_plan* p, const int32_t* const* lists, const int32_t* d_counts, TcFlags* out,
                   cudaStream_t st) {
  int rc = tc_ensure(p);
  if (rc != CGH_OK) return rc;
  cgh_tc_state* t = p->tc;
  rc = cgh_cuda_check(cudaMemsetAsync(t->flags, 0, t->flags_bytes, st), "flags: clear");
  t->flags_dirty = 1;
  if (rc != CGH_OK) return rc;
  k_tc_scatter<<<dim3(64, 4), 256, 0, st>>>(lists[0], lists[1], lists[2], lists[3], d_counts, t->fl, p->obj_h,
                                          p->obj_w, p->n_layers, p->d_status);
  rc = cgh_cuda_check(cudaGetLastError(), "flags: scatter");
  if (rc != CGH_OK) return rc;
  *out = t->fl;
  return CGH_OK;
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
  cudaError_t e = is_fp16 ? launch_gemm<KIND_TEST, EPI_C, true>(ma, mb, ma, a, grid, (cudaStream_t)stream)
                          : launch_gemm<KIND_TEST, EPI_C, false>(ma, mb, ma, a, grid, (cudaStream_t)stream);
  return cgh_cuda_check(e, "cgh_tc_selftest_gemm");
}

// Failure-detection self-test: one thread waits, with the same bounded wait as the GEMM
// pipeline, on an mbarrier that nothing ever completes; the wait gives up after limit_ns
// and records CGH_ERR_TIMEOUT in the status word, and the kernel returns normally.
__global__ void k_wait_timeout(int* status, unsigned long long limit_ns) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ volatile int s_abort;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) mbar_wait_bounded(&bar, 0, &s_abort, status, limit_ns);
}

extern "C" int cgh_selftest_timeout(const cgh_plan* p, int limit_us, void* stream) {
  if (!p || limit_us < 1 || limit_us > 1000000)
    return cgh_fail(CGH_ERR_ARG, "cgh_selftest_timeout: plan NULL or limit outside 1..1000000 us");
  k_wait_timeout<<<1, 32, 0, (cudaStream_t)stream>>>(p->d_status, 1000ull * (unsigned long long)limit_us);
  return cgh_cuda_check(cudaGetLastError(), "cgh_selftest_timeout");
}
