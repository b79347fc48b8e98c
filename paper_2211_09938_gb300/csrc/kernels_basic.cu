// Fringe tables, integer Haar DWT, saliency block selection, plain point-wise
// hologram and the detail-basis direct superposition (CUDA cores).
//
// Paper: arXiv 2211.09938, Eq. 1 (point-source fringe, paraxial), Eq. 2 (Haar
// expansion), Eq. 3 (superposition of basis holograms), Section 2 steps 1-5.
#include <stdio.h>
#include <string.h>

#include <cuda_fp16.h>

#include "cgh_internal.h"

#include <type_traits>

// ---------------------------------------------------------------------------
// (A1) fringe tables.  tab[z][l][kind][idx], offset d = idx - tab_off:
//   kind 0: b_l(d) = sum_{t<2^l} f_z(d - s t)
//   kind 1: w_l(d) = sum_{t<2^(l-1)} f_z(d - s t) - sum_{2^(l-1)<=t<2^l} f_z(d - s t)
// f_z(d) = exp(j 2 pi frac(a_z d^2)); the product a_z*d^2 and its reduction are FP64
// with d^2 an exact integer (Eq. 1 under the paraxial approximation).
__global__ void k_fringe_f64(double2* __restrict__ F, const double* __restrict__ a_frac, int f_len, int f_off,
                             const double2* __restrict__ lf_half) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= f_len) return;
  const int z = blockIdx.y;
  const long long d = (long long)q - f_off;
  double x = a_frac[z] * (double)(d * d);
  x -= rint(x);  // exact: |x| < 2^53 and x - rint(x) is representable
  double sn, cs;
  sincospi(2.0 * x, &sn, &cs);
  if (lf_half) {  // the square root of the layer factor, on each axis's fringe
    const double2 c = lf_half[z];
    const double re = c.x * cs - c.y * sn, im = c.x * sn + c.y * cs;
    cs = re;
    sn = im;
  }
  F[(size_t)z * f_len + q] = make_double2(cs, sn);
}

// F[z][q] = f_z(q - f_off) with f_off = tab_off + 7s, so entry idx of a table needs
// F[z][idx + 7s - s t] for the shifts t < 8.
__global__ void k_build_tables(float2* __restrict__ tab, const double2* __restrict__ F, int f_len,
                               int tab_len, int s) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= tab_len) return;
  const int z = blockIdx.y;
  const double2* Fz = F + (size_t)z * f_len + idx + 7 * s;
  double2 v[8];
#pragma unroll
  for (int t = 0; t < 8; ++t) v[t] = Fz[-s * t];
  float2* T = tab + (size_t)z * 8 * tab_len + idx;
#pragma unroll
  for (int l = 0; l < 4; ++l) {
    const int n = 1 << l, half = n >> 1;
    double br = 0.0, bi = 0.0, wr = 0.0, wi = 0.0;
#pragma unroll
    for (int t = 0; t < n; ++t) {
      br += v[t].x;
      bi += v[t].y;
      if (t < half) {
        wr += v[t].x;
        wi += v[t].y;
      } else {
        wr -= v[t].x;
        wi -= v[t].y;
      }
    }
    if (l == 0) wr = wi = 0.0;
    T[(size_t)(2 * l) * tab_len] = make_float2((float)br, (float)bi);
    T[(size_t)(2 * l + 1) * tab_len] = make_float2((float)wr, (float)wi);
  }
}

cudaError_t launch_build_tables(const cgh_plan* p, cudaStream_t st) {
  k_fringe_f64<<<dim3((p->f_len + 255) / 256, p->n_layers), 256, 0, st>>>(p->d_f64, p->d_a_frac, p->f_len,
                                                                        p->tab_off + 7 * p->s, p->d_lf_half);
  k_build_tables<<<dim3((p->tab_len + 255) / 256, p->n_layers), 256, 0, st>>>(p->d_tab, p->d_f64, p->f_len,
                                                                            p->tab_len, p->s);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// (A2) three-level integer Haar DWT of every layer plane (Eq. 2, Section 2 step 1).
// One thread per (8x8 block, layer).  The 2x2 cell [a b; c d] gives
// S = a+b+c+d, X = a-b+c-d, Y = a+b-c-d, D = a-b-c+d; Mallat output.
// The block's rows of intensity (iv) and layer index (lv).
__device__ __forceinline__ void haar3_load(const uint8_t* __restrict__ I, const uint8_t* __restrict__ L, int W,
                                           int bx, int by, uint2 (&iv)[8], uint2 (&lv)[8]) {
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const size_t o = (size_t)(8 * by + r) * W + 8 * bx;
    iv[r] = *reinterpret_cast<const uint2*>(I + o);
    lv[r] = *reinterpret_cast<const uint2*>(L + o);
  }
}

// The three levels of layer z of one 8x8 block, from its loaded rows.
__device__ __forceinline__ void haar3_layer(const uint2 (&iv)[8], const uint2 (&lv)[8], int32_t* __restrict__ coef,
                                            int H, int W, int z, int bx, int by) {
  // the layer's intensities: bytes of other layers cleared word by word (carry-free test of
  // byte == z on bit 7 of each byte, widened to a byte mask), then unpacked
  const unsigned zz = 0x01010101u * (unsigned)z;
  int a[8][8];
#pragma unroll
  for (int r = 0; r < 8; ++r) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const unsigned x = (h ? lv[r].y : lv[r].x) ^ zz;
      const unsigned eq = ~(((x & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | x) & 0x80808080u;
      const unsigned w = (h ? iv[r].y : iv[r].x) & ((eq >> 7) * 0xFFu);
#pragma unroll
      for (int c = 0; c < 4; ++c) a[r][4 * h + c] = (int)((w >> (8 * c)) & 0xFFu);
    }
  }
  int s1[4][4], x1[4][4], y1[4][4], d1[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int A = a[2 * r][2 * c], B = a[2 * r][2 * c + 1], C = a[2 * r + 1][2 * c],
                D = a[2 * r + 1][2 * c + 1];
      s1[r][c] = A + B + C + D;
      x1[r][c] = A - B + C - D;
      y1[r][c] = A + B - C - D;
      d1[r][c] = A - B - C + D;
    }
  int s2[2][2], x2[2][2], y2[2][2], d2[2][2];
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int A = s1[2 * r][2 * c], B = s1[2 * r][2 * c + 1], C = s1[2 * r + 1][2 * c],
                D = s1[2 * r + 1][2 * c + 1];
      s2[r][c] = A + B + C + D;
      x2[r][c] = A - B + C - D;
      y2[r][c] = A + B - C - D;
      d2[r][c] = A - B - C + D;
    }
  const int A = s2[0][0], B = s2[0][1], C = s2[1][0], D = s2[1][1];
  int32_t* P = coef + (size_t)z * H * W;
  const int h1 = H >> 1, w1 = W >> 1, h2 = H >> 2, w2 = W >> 2, h3 = H >> 3, w3 = W >> 3;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    *reinterpret_cast<int4*>(P + (size_t)(4 * by + r) * W + w1 + 4 * bx) =
        make_int4(x1[r][0], x1[r][1], x1[r][2], x1[r][3]);
    *reinterpret_cast<int4*>(P + (size_t)(h1 + 4 * by + r) * W + 4 * bx) =
        make_int4(y1[r][0], y1[r][1], y1[r][2], y1[r][3]);
    *reinterpret_cast<int4*>(P + (size_t)(h1 + 4 * by + r) * W + w1 + 4 * bx) =
        make_int4(d1[r][0], d1[r][1], d1[r][2], d1[r][3]);
  }
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    *reinterpret_cast<int2*>(P + (size_t)(2 * by + r) * W + w2 + 2 * bx) = make_int2(x2[r][0], x2[r][1]);
    *reinterpret_cast<int2*>(P + (size_t)(h2 + 2 * by + r) * W + 2 * bx) = make_int2(y2[r][0], y2[r][1]);
    *reinterpret_cast<int2*>(P + (size_t)(h2 + 2 * by + r) * W + w2 + 2 * bx) =
        make_int2(d2[r][0], d2[r][1]);
  }
  P[(size_t)by * W + bx] = A + B + C + D;
  P[(size_t)by * W + w3 + bx] = A - B + C - D;
  P[(size_t)(h3 + by) * W + bx] = A + B - C - D;
  P[(size_t)(h3 + by) * W + w3 + bx] = A - B - C + D;
}

__device__ __forceinline__ void haar3_block(const uint8_t* __restrict__ I, const uint8_t* __restrict__ L,
                                            int32_t* __restrict__ coef, int H, int W, int z, int bx, int by) {
  uint2 iv[8], lv[8];
  haar3_load(I, L, W, bx, by, iv, lv);
  haar3_layer(iv, lv, coef, H, W, z, bx, by);
}

// One layer per CTA, the layer fastest in the grid (blockIdx.x): the CTAs of all layers of a
// tile run next to each other, so the tile's input rows come from HBM once and from L2 for the
// other layers (with the layer slowest, an 8192^2 object with 4 layers re-read its 128 MB of
// inputs from HBM for every layer: 537 MB read for 1 GB of coefficients written).
__global__ void __launch_bounds__(128) k_haar3(const uint8_t* __restrict__ I,
                                               const uint8_t* __restrict__ L,
                                               int32_t* __restrict__ coef, int H, int W) {
  const int bx = blockIdx.y * blockDim.x + threadIdx.x;
  const int by = blockIdx.z * blockDim.y + threadIdx.y;
  if (bx >= (W >> 3) || by >= (H >> 3)) return;
  haar3_block(I, L, coef, H, W, blockIdx.x, bx, by);
}

// Batched DWT: grid.z walks the (scene, layer) items; x and y cover the largest scene.
__global__ void __launch_bounds__(128) k_haar3_batch(const HaarItem* __restrict__ items) {
  const HaarItem it = items[blockIdx.z];
  const int bx = blockIdx.x * blockDim.x + threadIdx.x;
  const int by = blockIdx.y * blockDim.y + threadIdx.y;
  if (bx >= (it.W >> 3) || by >= (it.H >> 3)) return;
  haar3_block(it.I, it.L, it.coef, it.H, it.W, it.z, bx, by);
}

cudaError_t launch_haar_batch(const HaarItem* d_items, int n_items, int max_h, int max_w, cudaStream_t st) {
  if (n_items <= 0) return cudaSuccess;
  dim3 block(32, 4);
  dim3 grid(((max_w >> 3) + 31) / 32, ((max_h >> 3) + 3) / 4, n_items);
  k_haar3_batch<<<grid, block, 0, st>>>(d_items);
  return cudaGetLastError();
}

cudaError_t launch_haar(const cgh_plan* p, const uint8_t* I, const uint8_t* L, int32_t* coef,
                        cudaStream_t st) {
  dim3 block(32, 4);
  dim3 grid(p->n_layers, ((p->obj_w >> 3) + 31) / 32, ((p->obj_h >> 3) + 3) / 4);
  k_haar3<<<grid, block, 0, st>>>(I, L, coef, p->obj_h, p->obj_w);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// (A3) saliency block maximum, selection and ordered compaction (Section 2 steps 1-5).
// A block is summarised by the bit mask of the layers it may contribute to: the layers
// owning one of its pixels, cleared when the block maximum of the saliency does not
// exceed the threshold.
// The k x k block (k = 2^LEVEL) is read one row at a time as a k-byte vector (rows start on
// multiples of k bytes because the object width is a multiple of 8), so a thread issues 2k
// independent loads instead of 2k^2 dependent byte loads.
template <int LEVEL>
__device__ __forceinline__ unsigned long long block_layer_mask_k(const uint8_t* __restrict__ sal,
                                                                 const uint8_t* __restrict__ L, int W, int by,
                                                                 int bx, int threshold, int Z) {
  constexpr int k = 1 << LEVEL;
  using V = typename std::conditional<k == 8, uint2, typename std::conditional<k == 4, unsigned, unsigned short>::type>::type;
  unsigned long long occ = 0ull;
  int mx = 0;
  V lv[k], sv[k];
#pragma unroll
  for (int r = 0; r < k; ++r) {
    const size_t o = (size_t)(by * k + r) * W + (size_t)bx * k;
    lv[r] = *reinterpret_cast<const V*>(L + o);
    if (sal) sv[r] = *reinterpret_cast<const V*>(sal + o);
  }
#pragma unroll
  for (int r = 0; r < k; ++r) {
    uint8_t lb[k], sb[k];
    memcpy(lb, &lv[r], k);
    if (sal) memcpy(sb, &sv[r], k);
#pragma unroll
    for (int c = 0; c < k; ++c) {
      const int lz = lb[c];
      if (lz < Z) occ |= 1ull << lz;
      if (sal) mx = max(mx, (int)sb[c]);
    }
  }
  if (threshold >= 0 && mx <= threshold) occ = 0ull;
  return occ;
}

__device__ __forceinline__ unsigned long long block_layer_mask(const uint8_t* __restrict__ sal,
                                                               const uint8_t* __restrict__ L, int W, int level,
                                                               int by, int bx, int threshold, int Z) {
  switch (level) {
    case 1: return block_layer_mask_k<1>(sal, L, W, by, bx, threshold, Z);
    case 2: return block_layer_mask_k<2>(sal, L, W, by, bx, threshold, Z);
    default: return block_layer_mask_k<3>(sal, L, W, by, bx, threshold, Z);
  }
}

int select_num_chunks(int obj_h, int obj_w, int level) {
  const long long nb = (long long)(obj_h >> level) * (obj_w >> level);
  return (int)((nb + CGH_SEL_CHUNK - 1) / CGH_SEL_CHUNK);
}

// A launch may serve up to four selections (the LLL list and the three detail levels);
// each owns a contiguous range of the grid's chunks and of the count scratch.
__device__ __forceinline__ int sel_task_of(const SelTasks& T, int chunk) {
  int k = 0;
  for (int q = 1; q < T.n; ++q)
    if (chunk >= T.t[q].chunk0) k = q;
  return k;
}

// Pass 1: per (task, layer, chunk) counts; one thread per block of the chunk.
__device__ __forceinline__ void select_count_body(const uint8_t* __restrict__ sal, const uint8_t* __restrict__ L,
                                                  int H, int W, int Z, const SelTask& tk, int chunk,
                                                  int* __restrict__ chunk_cnt) {
  __shared__ int s_cnt[CGH_MAX_LAYERS];
  const int level = tk.level, nbx = W >> level, nb = (H >> level) * nbx;
  for (int t = threadIdx.x; t < Z; t += blockDim.x) s_cnt[t] = 0;
  if (chunk == 0 && threadIdx.x == 0) tk.count[1] = 0;  // the scan's CTA counter
  __syncthreads();
  const int b = chunk * CGH_SEL_CHUNK + threadIdx.x;
  unsigned long long m =
      b < nb ? block_layer_mask(sal, L, W, level, b / nbx, b % nbx, tk.threshold, Z) : 0ull;
  while (m) {
    atomicAdd(&s_cnt[__ffsll((long long)m) - 1], 1);
    m &= m - 1ull;
  }
  __syncthreads();
  for (int z = threadIdx.x; z < Z; z += blockDim.x) chunk_cnt[tk.cnt_off + z * tk.nchunks + chunk] = s_cnt[z];
}

__global__ void __launch_bounds__(CGH_SEL_CHUNK) k_select_count(const uint8_t* __restrict__ sal,
                                                                const uint8_t* __restrict__ L, int H, int W,
                                                                int Z, const SelTasks T,
                                                                int* __restrict__ chunk_cnt) {
  pdl_wait();
  pdl_trigger();
  const SelTask& tk = T.t[sel_task_of(T, blockIdx.x)];
  select_count_body(sal, L, H, W, Z, tk, blockIdx.x - tk.chunk0, chunk_cnt);
}

// Pass 2: per task, exclusive scan of its counts in (layer, chunk) order, in blocks of
// SEL_SCAN_BLOCK entries (1024 threads x 4 consecutive entries; grid: blocks x tasks).  Each
// CTA writes the offsets within its block and leaves the block's total in the count table
// at the block's first entry (which it has read by then).  The task's last CTA to finish
// (counted on count[1], zeroed by pass 1) replaces the totals by their exclusive prefix
// and writes the list length; the scatter adds the prefix of its block.
#define SEL_SCAN_BLOCK 4096

// Exclusive scan of one int per thread over a 1024-thread CTA; returns the CTA total too.
__device__ __forceinline__ int cta_exclusive_scan(int x, int* s_warp, int& total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) s_warp[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    const int w = s_warp[lane];
    int wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += t;
    }
    s_warp[lane] = wi - w;
    if (lane == 31) s_warp[32] = wi;
  }
  __syncthreads();
  total = s_warp[32];
  const int r = s_warp[warp] + inc - x;
  __syncthreads();  // s_warp may be reused
  return r;
}

__device__ __forceinline__ void select_scan_body(int* chunk_cnt, int* __restrict__ chunk_off, int Z,
                                                 const SelTask& tk, int blk) {
  __shared__ int s_warp[33];
  __shared__ int s_last;
  const int n = Z * tk.nchunks, nblk = (n + SEL_SCAN_BLOCK - 1) / SEL_SCAN_BLOCK;
  const int b0 = blk * SEL_SCAN_BLOCK;
  if (b0 >= n) return;
  int* cnt = chunk_cnt + tk.cnt_off;
  int* off = chunk_off + tk.cnt_off;
  const int i0 = b0 + 4 * threadIdx.x;
  int v[4], sum = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    v[q] = i0 + q < n ? cnt[i0 + q] : 0;
    sum += v[q];
  }
  int block_total;
  int run = cta_exclusive_scan(sum, s_warp, block_total);
#pragma unroll
  for (int q = 0; q < 4; ++q)
    if (i0 + q < n) {
      off[i0 + q] = run;
      run += v[q];
    }
  if (threadIdx.x == 0) {  // every count of the block was read before the scan's barriers
    cnt[b0] = block_total;
    __threadfence();
    s_last = atomicAdd(&tk.count[1], 1) == nblk - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  int carry = 0;
  for (int r0 = 0; r0 < nblk; r0 += 1024) {
    const int b = r0 + threadIdx.x;
    const int t = b < nblk ? __ldcg(cnt + (size_t)b * SEL_SCAN_BLOCK) : 0;
    int round_total;
    const int e = cta_exclusive_scan(t, s_warp, round_total);
    if (b < nblk) cnt[(size_t)b * SEL_SCAN_BLOCK] = carry + e;
    carry += round_total;
  }
  if (threadIdx.x == 0) {
    tk.count[0] = min(carry, tk.capacity);
    tk.count[1] = carry;
  }
}

__global__ void __launch_bounds__(1024) k_select_scan(int* chunk_cnt, int* __restrict__ chunk_off,
                                                      int Z, const SelTasks T) {
  pdl_wait();
  pdl_trigger();
  select_scan_body(chunk_cnt, chunk_off, Z, T.t[blockIdx.y], blockIdx.x);
}

// Pass 3: ordered scatter.  Per layer, warp ballots give every warp's count and every
// thread's rank inside its warp; one shared exclusive scan over the warps (per layer) gives
// the warp offsets.  Two barriers per CTA whatever the number of layers.
// FLAGS: also mark the tensor-core selection flags of every written entry (as the fused
// selection does; fl is then the scene's flag block).
template <bool FLAGS>
__device__ __forceinline__ void select_scatter_body(const uint8_t* __restrict__ sal, const uint8_t* __restrict__ L,
                                                    int H, int W, int Z, const SelTask& tk, int chunk,
                                                    const int* __restrict__ chunk_cnt,
                                                    const int* __restrict__ chunk_off, const TcFlags& fl) {
  constexpr int NW = CGH_SEL_CHUNK / 32;
  __shared__ int s_wcnt[NW][CGH_MAX_LAYERS];
  __shared__ int s_pre[CGH_MAX_LAYERS];
  const int level = tk.level, nbx = W >> level, nb = (H >> level) * nbx;
  const int b = chunk * CGH_SEL_CHUNK + threadIdx.x;
  const int by = b / nbx, bx = b - by * nbx;
  const unsigned long long m =
      b < nb ? block_layer_mask(sal, L, W, level, by, bx, tk.threshold, Z) : 0ull;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned below = (1u << lane) - 1u;
  for (int z = 0; z < Z; ++z) {
    const unsigned bal = __ballot_sync(0xffffffffu, (m >> z) & 1ull);
    if (lane == 0) s_wcnt[warp][z] = __popc(bal);
  }
  __syncthreads();
  if (threadIdx.x < Z) {
    int run = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
      const int c = s_wcnt[w][threadIdx.x];
      s_wcnt[w][threadIdx.x] = run;
      run += c;
    }
    // this layer's first position: the prefix of the scan block holding its entry plus the
    // entry's offset in the block (loaded here, off the ballot loop below)
    const int e = threadIdx.x * tk.nchunks + chunk;
    s_pre[threadIdx.x] = chunk_cnt[tk.cnt_off + (e / SEL_SCAN_BLOCK) * SEL_SCAN_BLOCK] + chunk_off[tk.cnt_off + e];
  }
  __syncthreads();
  const int hl = H >> level, wl = W >> level;
  for (int z = 0; z < Z; ++z) {
    const bool f = (m >> z) & 1ull;
    const unsigned bal = __ballot_sync(0xffffffffu, f);
    if (f) {
      const int pos = s_pre[z] + s_wcnt[warp][z] + __popc(bal & below);
      if (pos < tk.capacity) {
        tk.list[pos] = (z << 24) | (by << 12) | bx;
        if (FLAGS) {
          if (tk.flag_kind == SEL_FLAGS_LLL) {
            fl.occ3[((size_t)z * hl + by) * wl + bx] = 1;
            fl.rowband[(size_t)z * hl + by] = 1;
            fl.colband[(size_t)z * wl + bx] = 1;
          } else if (tk.flag_kind == SEL_FLAGS_DETAIL) {
            uint8_t* sel = level == 1 ? fl.sel[1] : level == 2 ? fl.sel[2] : fl.sel[3];
            sel[((size_t)z * hl + by) * wl + bx] = 1;
            fl.rowband[(size_t)z * (H >> 3) + (by >> (3 - level))] = 1;
            fl.colband[(size_t)z * (W >> 3) + (bx >> (3 - level))] = 1;
          }
        }
      }
    }
  }
}

__global__ void __launch_bounds__(CGH_SEL_CHUNK) k_select_scatter(
    const uint8_t* __restrict__ sal, const uint8_t* __restrict__ L, int H, int W, int Z, const SelTasks T,
    const int* __restrict__ chunk_cnt, const int* __restrict__ chunk_off) {
  pdl_wait();
  pdl_trigger();
  const SelTask& tk = T.t[sel_task_of(T, blockIdx.x)];
  select_scatter_body<false>(sal, L, H, W, Z, tk, blockIdx.x - tk.chunk0, chunk_cnt, chunk_off, TcFlags{});
}

// Batched three-pass selection: every task carries its scene; chunks of all tasks form one
// grid (a task's chunk0 and cnt_off are global), found by binary search.
__device__ __forceinline__ int sel_task_of_batch(const SelTaskB* __restrict__ tasks, int n, int chunk) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tasks[mid].t.chunk0 <= chunk)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

__global__ void __launch_bounds__(CGH_SEL_CHUNK) k_select_count_batch(const SelTaskB* __restrict__ tasks, int n,
                                                                      int* __restrict__ chunk_cnt) {
  pdl_wait();
  pdl_trigger();
  const SelTaskB& tb = tasks[sel_task_of_batch(tasks, n, blockIdx.x)];
  select_count_body(tb.sal, tb.L, tb.H, tb.W, tb.Z, tb.t, blockIdx.x - tb.t.chunk0, chunk_cnt);
}

__global__ void __launch_bounds__(1024) k_select_scan_batch(const SelTaskB* __restrict__ tasks, int* chunk_cnt,
                                                            int* __restrict__ chunk_off) {
  pdl_wait();
  pdl_trigger();
  const SelTaskB& tb = tasks[blockIdx.y];
  select_scan_body(chunk_cnt, chunk_off, tb.Z, tb.t, blockIdx.x);
}

__global__ void __launch_bounds__(CGH_SEL_CHUNK) k_select_scatter_batch(const SelTaskB* __restrict__ tasks, int n,
                                                                        const int* __restrict__ chunk_cnt,
                                                                        const int* __restrict__ chunk_off) {
  pdl_wait();
  pdl_trigger();
  const SelTaskB& tb = tasks[sel_task_of_batch(tasks, n, blockIdx.x)];
  select_scatter_body<true>(tb.sal, tb.L, tb.H, tb.W, tb.Z, tb.t, blockIdx.x - tb.t.chunk0, chunk_cnt, chunk_off,
                            tb.fl);
}

// The three passes over all tasks of a batch (the tasks' chunk0 / cnt_off / nchunks set by
// the caller): lists, counts and, for tasks with a flag kind, the tensor-core flags.
cudaError_t launch_select_batch(const SelTaskB* d_tasks, int n_tasks, int total_chunks, int max_scan_blocks,
                                int* chunk_cnt, int* chunk_off, cudaStream_t st) {
  if (n_tasks <= 0) return cudaSuccess;
  cudaError_t e = launch_pdl(k_select_count_batch, dim3(total_chunks), dim3(CGH_SEL_CHUNK), 0, st, d_tasks, n_tasks,
                             chunk_cnt);
  if (e == cudaSuccess)
    e = launch_pdl(k_select_scan_batch, dim3(max_scan_blocks, n_tasks), dim3(1024), 0, st, d_tasks, chunk_cnt,
                   chunk_off);
  if (e == cudaSuccess)
    e = launch_pdl(k_select_scatter_batch, dim3(total_chunks), dim3(CGH_SEL_CHUNK), 0, st, d_tasks, n_tasks,
                   (const int*)chunk_cnt, (const int*)chunk_off);
  return e != cudaSuccess ? e : cudaGetLastError();
}

int select_scan_blocks(int n_layers, int nchunks) {
  return (n_layers * nchunks + SEL_SCAN_BLOCK - 1) / SEL_SCAN_BLOCK;
}

// ---------------------------------------------------------------------------
// Multi-level selection for large objects (width a multiple of 2048): the four lists of a
// progressive hologram (LLL = every occupied 8x8 block, and the detail blocks of levels 3,
// 2, 1 above their thresholds) in two passes over the 8x8 blocks.  One thread owns one 8x8
// block; one CTA owns a segment of 256 consecutive 8x8 blocks of one row of them.  The count
// table of a list holds, per layer, one entry per (row of that level's blocks, segment): 1
// row of level-3 blocks, 2 rows of level-2 and 4 rows of level-1 blocks per segment.  In the
// order (layer, row, segment) these are the list's own order (layer, block row, block
// column), so the blocked exclusive scan of the three-pass selection gives every segment row
// its first position, and the scatter ranks the blocks inside it.
//   count:   reads the block's 64 saliency and layer bytes, writes a 64-bit record of the block
//            and adds its per-layer row counts into the CTA's table (warp reductions);
//   scatter: reads the records instead of the inputs (the layer map again only for blocks
//            with points in three or more layers), ranks the blocks and writes the entries.
// Byte-wise work uses 32-bit integer and paired fp16 operations: the block maxima of the
// saliency as fp16 pairs 1024 + s (exact: integers up to 2048 are fp16 numbers), layer
// equality and range tests as carry-free byte arithmetic.  Bit-exact with the per-level
// selection.
#define SEL_ML_SEG 256

// Record of one 8x8 block, two words.  Each word describes one layer of the block: bits 0-15
// its level-1 entries (the 2x2 blocks, 4r+c), bits 16-19 its level-2 entries (the 4x4 blocks,
// 2r+c), bit 20 its level-3 entry, bit 21 its LLL entry (the block holds a point of that
// layer), bits 22-27 the layer; 0 = no layer.  A block with points in three or more layers
// sets ML_MULTI in word 1 and keeps its threshold tests in word 0 (bits 0-20 as above: a
// sub-block passes when the maximum of its saliency is above its level's threshold, or the
// level has none); the scatter reads its layer map again.
#define ML_MULTI 0x80000000u
#define ML_BITS 0x3FFFFFu
#define ML_B7 0x80808080u
#define ML_LO7 0x7F7F7F7Fu

__device__ __forceinline__ __half2 ml_as_h2(unsigned u) { return *reinterpret_cast<const __half2*>(&u); }
__device__ __forceinline__ unsigned ml_as_u(__half2 h) { return *reinterpret_cast<const unsigned*>(&h); }
// Bytes 0 and 2 (SEL 0x4240) or 1 and 3 (0x4341) of w as the fp16 pair (1024 + b, 1024 + b').
__device__ __forceinline__ __half2 ml_pair(unsigned w, unsigned sel) { return ml_as_h2(__byte_perm(w, 0x64u, sel)); }
// A level's threshold t as the fp16 pair 1024 + t, clamped so that "above" stays exact: no
// threshold (t < 0) passes every block, t >= 255 none.
__device__ __forceinline__ __half2 ml_threshold(int t) {
  return __float2half2_rn(1024.f + (float)(t < 0 ? -1 : t > 255 ? 255 : t));
}
// Bits of the low and high halves of a paired mask (0xFFFF per true half).
__device__ __forceinline__ unsigned ml_two(unsigned g) { return (g & 1u) | ((g >> 15) & 2u); }

// Threshold tests of the block (record bits 0-20) from its saliency rows.
__device__ __forceinline__ unsigned ml_tests(const uint2 (&sv)[8], __half2 t1, __half2 t2, __half2 t3) {
  __half2 m[4][2];  // [row pair][half]: maxima of the 2x2 blocks 4p + 2h (low) and 4p + 2h + 1 (high)
  unsigned tests = 0u;
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const unsigned a = h ? sv[2 * p].y : sv[2 * p].x, b = h ? sv[2 * p + 1].y : sv[2 * p + 1].x;
      m[p][h] = __hmax2(__hmax2(ml_pair(a, 0x4240u), ml_pair(a, 0x4341u)),
                        __hmax2(ml_pair(b, 0x4240u), ml_pair(b, 0x4341u)));
      tests |= ml_two(__hgt2_mask(m[p][h], t1)) << (4 * p + 2 * h);
    }
  // 4x4 blocks of row r2: low = column 0, high = column 1
  __half2 x[2];
#pragma unroll
  for (int r2 = 0; r2 < 2; ++r2) {
    const unsigned c0 = ml_as_u(__hmax2(m[2 * r2][0], m[2 * r2 + 1][0]));
    const unsigned c1 = ml_as_u(__hmax2(m[2 * r2][1], m[2 * r2 + 1][1]));
    x[r2] = __hmax2(ml_as_h2(__byte_perm(c0, c1, 0x5410u)), ml_as_h2(__byte_perm(c0, c1, 0x7632u)));
    tests |= ml_two(__hgt2_mask(x[r2], t2)) << (16 + 2 * r2);
  }
  const __half2 y = __hmax2(x[0], x[1]);
  const unsigned yu = ml_as_u(y);
  tests |= (__hgt2_mask(__hmax2(y, ml_as_h2(__byte_perm(yu, yu, 0x1032u))), t3) & 1u) << 20;
  return tests;
}

// Carry-free byte tests (bit 7 of every byte): byte == 0, and byte >= Z (Z <= 128).
__device__ __forceinline__ unsigned ml_zero_bytes(unsigned x) { return ~(((x & ML_LO7) + ML_LO7) | x) & ML_B7; }
__device__ __forceinline__ unsigned ml_absent_bytes(unsigned w, unsigned kz) { return (((w & ML_LO7) + kz) | w) & ML_B7; }

// The 2x2 blocks (4r+c) holding a marked pixel, from per-row byte marks (bit 7 of every byte).
__device__ __forceinline__ unsigned ml_gather(const uint2 (&mk)[8]) {
  unsigned bits = 0u;
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      unsigned t = h ? (mk[2 * p].y | mk[2 * p + 1].y) : (mk[2 * p].x | mk[2 * p + 1].x);
      t |= t << 8;  // bit 15: columns 0-1, bit 31: columns 2-3
      bits |= (((t >> 15) & 1u) | ((t >> 30) & 2u)) << (4 * p + 2 * h);
    }
  return bits;
}
// The 2x2 blocks holding a pixel of layer z.
__device__ __forceinline__ unsigned ml_pres_layer(const uint2 (&lv)[8], unsigned z) {
  const unsigned zz = 0x01010101u * z;
  uint2 mk[8];
#pragma unroll
  for (int r = 0; r < 8; ++r) mk[r] = make_uint2(ml_zero_bytes(lv[r].x ^ zz), ml_zero_bytes(lv[r].y ^ zz));
  return ml_gather(mk);
}

// Record bits 0-21 of one layer from the 2x2 blocks holding its points (pres, 4r+c) and the
// threshold tests: a block of any level is an entry when it holds a point and passes.
__device__ __forceinline__ unsigned ml_layer_bits(unsigned pres, unsigned tests) {
  if (!pres) return 0u;
  const unsigned p2 = ((pres & 0x0033u) ? 1u : 0u) | ((pres & 0x00CCu) ? 2u : 0u) | ((pres & 0x3300u) ? 4u : 0u) |
                      ((pres & 0xCC00u) ? 8u : 0u);
  return (pres & tests & 0xFFFFu) | ((p2 & (tests >> 16) & 0xFu) << 16) | (tests & (1u << 20)) | (1u << 21);
}

// The layers present in a block (bit z: a pixel of layer z < Z).
__device__ __forceinline__ unsigned long long ml_layer_mask(const uint2 (&lv)[8], int Z) {
  unsigned long long m = 0ull;
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const unsigned w = h ? lv[r].y : lv[r].x;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int lz = (w >> (8 * c)) & 0xFF;
        if (lz < Z) m |= 1ull << lz;
      }
    }
  return m;
}

__device__ __forceinline__ unsigned ml_layer_of(unsigned w) { return (w >> 22) & 63u; }
// Layers of a record (bit z), for blocks with at most two layers.
__device__ __forceinline__ unsigned long long ml_rec_layers(uint2 r) {
  return ((r.x >> 21) & 1u ? 1ull << ml_layer_of(r.x) : 0ull) | ((r.y >> 21) & 1u ? 1ull << ml_layer_of(r.y) : 0ull);
}
// Bits 0-21 of layer z for a thread's block: from its record, or, for a block with points in
// three or more layers, from its layer rows (lv) and the tests kept in the record.
__device__ __forceinline__ unsigned ml_bits_of(uint2 r, const uint2 (&lv)[8], unsigned long long lmask, int z) {
  if (!(r.y & ML_MULTI))
    return ((int)ml_layer_of(r.x) == z ? (r.x & ML_BITS) : 0u) | ((int)ml_layer_of(r.y) == z ? (r.y & ML_BITS) : 0u);
  if (!((lmask >> z) & 1ull)) return 0u;
  return ml_layer_bits(ml_pres_layer(lv, (unsigned)z), r.x);
}

// Record of the block from its rows of layers (lv) and its threshold tests.
__device__ __forceinline__ uint2 ml_record(const uint2 (&lv)[8], int Z, unsigned tests) {
  const unsigned l0 = 0x01010101u * (lv[0].x & 0xFFu);
  unsigned d = 0u;
#pragma unroll
  for (int r = 0; r < 8; ++r) d |= (lv[r].x ^ l0) | (lv[r].y ^ l0);
  if (!d) {  // one value throughout: one layer, or no point
    const unsigned z = l0 & 0xFFu;
    return make_uint2((int)z < Z ? (z << 22) | ml_layer_bits(0xFFFFu, tests) : 0u, 0u);
  }
  const unsigned kz = 0x01010101u * (unsigned)(128 - Z);
  // a layer of the block: its first pixel's, or else the first point's
  unsigned za = l0 & 0xFFu;
  if ((int)za >= Z) {
    za = 0xFFu;
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const unsigned w = h ? lv[r].y : lv[r].x, pr = ~ml_absent_bytes(w, kz) & ML_B7;
        if (za == 0xFFu && pr) za = (w >> (__ffs(pr) - 8)) & 0xFFu;
      }
    if (za == 0xFFu) return make_uint2(0u, 0u);
  }
  // pixels of layer za, and the first pixel of another value
  uint2 ea[8];
  unsigned zb = 0xFFu;
  const unsigned zza = 0x01010101u * za;
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    ea[r] = make_uint2(ml_zero_bytes(lv[r].x ^ zza), ml_zero_bytes(lv[r].y ^ zza));
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const unsigned w = h ? lv[r].y : lv[r].x, o = ~(h ? ea[r].y : ea[r].x) & ML_B7;
      if (zb == 0xFFu && o) zb = (w >> (__ffs(o) - 8)) & 0xFFu;
    }
  }
  const unsigned wa = (za << 22) | ml_layer_bits(ml_gather(ea), tests);
  if ((int)zb < Z) {  // the common case: two layers and a point in every pixel
    const unsigned zzb = 0x01010101u * zb;
    uint2 eb[8];
    unsigned other = 0u;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      eb[r] = make_uint2(ml_zero_bytes(lv[r].x ^ zzb), ml_zero_bytes(lv[r].y ^ zzb));
      other |= ~(ea[r].x | eb[r].x) | ~(ea[r].y | eb[r].y);
    }
    if (!(other & ML_B7)) return make_uint2(wa, (zb << 22) | ml_layer_bits(ml_gather(eb), tests));
  }
  // otherwise: points of layers other than za (pixels without a point left out)
  unsigned rest = 0u;
  zb = 0xFFu;
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const unsigned w = h ? lv[r].y : lv[r].x;
      const unsigned o = ~ml_absent_bytes(w, kz) & ML_B7 & ~(h ? ea[r].y : ea[r].x);
      if (zb == 0xFFu && o) zb = (w >> (__ffs(o) - 8)) & 0xFFu;
      rest |= o;
    }
  if (!rest) return make_uint2(wa, 0u);
  // a second layer: the block is described when no point lies in a third
  const unsigned zzb = 0x01010101u * zb;
  uint2 eb[8];
  unsigned third = 0u;
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    eb[r] = make_uint2(ml_zero_bytes(lv[r].x ^ zzb), ml_zero_bytes(lv[r].y ^ zzb));
    third |= (~ml_absent_bytes(lv[r].x, kz) & ~(ea[r].x | eb[r].x)) | (~ml_absent_bytes(lv[r].y, kz) & ~(ea[r].y | eb[r].y));
  }
  if (third & ML_B7) return make_uint2(tests, ML_MULTI);
  return make_uint2(wa, (zb << 22) | ml_layer_bits(ml_gather(eb), tests));
}

// The eight rows of a segment: 0 LLL, 1 level 3, 2-3 level 2, 4-7 level 1.  A thread's count of
// entries in each row, packed as 16-bit fields, two rows per word (a row of a segment has at
// most 1024 blocks, so no field overflows in the CTA-wide sums).
__device__ __forceinline__ void ml_pack(unsigned b, unsigned (&w)[4]) {
  w[0] = ((b >> 21) & 1u) | (((b >> 20) & 1u) << 16);
  w[1] = __popc((b >> 16) & 3u) | (__popc((b >> 18) & 3u) << 16);
  unsigned x = b & 0xFFFFu;
  x = (x & 0x5555u) + ((x >> 1) & 0x5555u);
  x = (x & 0x3333u) + ((x >> 2) & 0x3333u);  // nibble q: the count of level-1 row q
  w[2] = (x & 0xFu) | (((x >> 4) & 0xFu) << 16);
  w[3] = ((x >> 8) & 0xFu) | (((x >> 12) & 0xFu) << 16);
}
__host__ __device__ __forceinline__ int ml_rows(int k) { return k == 1 ? 4 : k == 2 ? 2 : 1; }
// Row r of the eight -> (list k, row q within the segment).
__host__ __device__ __forceinline__ int ml_row_list(int r) { return r == 0 ? 0 : r == 1 ? 3 : r < 4 ? 2 : 1; }
__host__ __device__ __forceinline__ int ml_row_q(int r) { return r < 2 ? 0 : r < 4 ? r - 2 : r - 4; }

__device__ __forceinline__ unsigned long long ml_warp_or(unsigned long long v) {
  return ((unsigned long long)__reduce_or_sync(0xffffffffu, (unsigned)(v >> 32)) << 32) |
         __reduce_or_sync(0xffffffffu, (unsigned)v);
}

// Pass 1: the blocks' records and the per (list, layer, segment row) counts.  CTA = (row of
// 8x8 blocks, segment).
__global__ void __launch_bounds__(SEL_ML_SEG, 4) k_select_ml_count(const uint8_t* __restrict__ sal,
                                                                const uint8_t* __restrict__ L, int H, int W, int Z,
                                                                const SelTasks T, int* __restrict__ chunk_cnt,
                                                                uint2* __restrict__ rec, uint4* __restrict__ wt) {
  __shared__ unsigned s_cnt[CGH_MAX_LAYERS][4];
  pdl_wait();
  pdl_trigger();
  const int nseg = (W >> 3) / SEL_ML_SEG, R = blockIdx.x / nseg, sg = blockIdx.x - R * nseg;
  const int bx3 = sg * SEL_ML_SEG + threadIdx.x, lane = threadIdx.x & 31;
  uint2 lv[8], sv[8];
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const size_t o = (size_t)(8 * R + r) * W + 8 * bx3;
    lv[r] = *reinterpret_cast<const uint2*>(L + o);
    sv[r] = *reinterpret_cast<const uint2*>(sal + o);
  }
  if (blockIdx.x == 0 && threadIdx.x < 4) T.t[threadIdx.x].count[1] = 0;  // the scan's CTA counters
  for (int e = threadIdx.x; e < 4 * Z; e += blockDim.x) (&s_cnt[0][0])[e] = 0u;
  // threshold tests; a block of one saliency value (common) takes them directly
  const int t1 = T.t[1].threshold, t2 = T.t[2].threshold, t3 = T.t[3].threshold;
  const unsigned s0 = 0x01010101u * (sv[0].x & 0xFFu);
  unsigned ds = 0u;
#pragma unroll
  for (int r = 0; r < 8; ++r) ds |= (sv[r].x ^ s0) | (sv[r].y ^ s0);
  unsigned tests;
  if (!ds) {
    const int s = (int)(s0 & 0xFFu);
    tests = (t1 < 0 || s > t1 ? 0xFFFFu : 0u) | (t2 < 0 || s > t2 ? 0xF0000u : 0u) | (t3 < 0 || s > t3 ? 0x100000u : 0u);
  } else {
    tests = ml_tests(sv, ml_threshold(t1), ml_threshold(t2), ml_threshold(t3));
  }
  const uint2 r = ml_record(lv, Z, tests);
  rec[(size_t)R * (W >> 3) + bx3] = r;
  const unsigned long long lmask = (r.y & ML_MULTI) ? ml_layer_mask(lv, Z) : ml_rec_layers(r);
  __syncthreads();  // s_cnt cleared
  // per layer of the warp: its row totals, kept for the scatter (zero for the other layers)
  // and added into the CTA's table
  const unsigned long long uw = ml_warp_or(lmask);
  uint4* const wtw = wt + ((size_t)blockIdx.x * (SEL_ML_SEG / 32) + (threadIdx.x >> 5)) * Z;
  for (unsigned long long u = uw; u; u &= u - 1ull) {
    const int z = __ffsll((long long)u) - 1;
    unsigned w[4];
    ml_pack(ml_bits_of(r, lv, lmask, z), w);
#pragma unroll
    for (int j = 0; j < 4; ++j) w[j] = __reduce_add_sync(0xffffffffu, w[j]);
    if (lane == 0) {
      wtw[z] = make_uint4(w[0], w[1], w[2], w[3]);
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (w[j]) atomicAdd(&s_cnt[z][j], w[j]);
    }
  }
  for (int z = lane; z < Z; z += 32)
    if (!((uw >> z) & 1ull)) wtw[z] = make_uint4(0u, 0u, 0u, 0u);
  __syncthreads();
  for (int e = threadIdx.x; e < 8 * Z; e += blockDim.x) {
    const int z = e >> 3, r8 = e & 7, k = ml_row_list(r8);
    const SelTask& tk = T.t[k];
    const int row = R * ml_rows(k) + ml_row_q(r8);
    chunk_cnt[tk.cnt_off + z * tk.nchunks + row * nseg + sg] = (int)((s_cnt[z][r8 >> 1] >> (16 * (r8 & 1))) & 0xFFFFu);
  }
}

// Entries of one block in one layer z (bits b, record layout) from the first positions of the
// warp's rows (pos0[r8]) and the lane's exclusive counts within the warp (bytes of e[0] for
// rows 0-3, e[1] for rows 4-7).  FLAGS: also the tensor-core flags.
template <bool FLAGS>
__device__ __forceinline__ void ml_write(unsigned b, int z, const unsigned (&e)[2], const int* pos0, int R, int bx3,
                                         int H, int W, const SelTasks& T, const TcFlags& fl) {
#pragma unroll
  for (int r8 = 0; r8 < 8; ++r8) {
    const int k = ml_row_list(r8), q = ml_row_q(r8);
    const int cols = k == 1 ? 4 : k == 2 ? 2 : 1;
    const int sh = k == 0 ? 21 : k == 3 ? 20 : k == 2 ? 16 + 2 * q : 4 * q;
    const int bits = (int)((b >> sh) & ((1u << cols) - 1u));
    if (!bits) continue;
    const SelTask& tk = T.t[k];
    int pos = pos0[r8] + (int)((e[r8 >> 2] >> (8 * (r8 & 3))) & 0xFFu);
    const int by = R * ml_rows(k) + q, v0 = (z << 24) | (by << 12) | (bx3 * cols);
    if (!FLAGS && pos + __popc(bits) <= tk.capacity) {  // the whole run fits
#pragma unroll
      for (int cc = 0; cc < cols; ++cc)
        if ((bits >> cc) & 1) tk.list[pos++] = v0 + cc;
      continue;
    }
    const int level = tk.level, hl = H >> level, wl = W >> level;
    for (int cc = 0; cc < cols; ++cc) {
      if (!((bits >> cc) & 1)) continue;
      const int bx = bx3 * cols + cc;
      if (pos < tk.capacity) {
        tk.list[pos] = v0 + cc;
        if (FLAGS) {
          if (k == 0) {
            fl.occ3[((size_t)z * hl + by) * wl + bx] = 1;
            fl.rowband[(size_t)z * hl + by] = 1;
            fl.colband[(size_t)z * wl + bx] = 1;
          } else {
            uint8_t* sel = level == 1 ? fl.sel[1] : level == 2 ? fl.sel[2] : fl.sel[3];
            sel[((size_t)z * hl + by) * wl + bx] = 1;
            fl.rowband[(size_t)z * (H >> 3) + (by >> (3 - level))] = 1;
            fl.colband[(size_t)z * (W >> 3) + (bx >> (3 - level))] = 1;
          }
        }
      }
      ++pos;
    }
  }
}

// Pass 3: ordered scatter of all four lists from the records (FLAGS: also the tensor-core
// flags).  Per CTA: the warps' per-layer row totals, their prefix over the warps added to the
// rows' first positions (one table per warp, layer and row), then per layer of the warp an
// exclusive scan of the lanes' row counts (bytes: at most 4 a lane, 128 a warp).  A lane keeps
// the scans of its record's one or two layers and writes its entries once per layer.
template <bool FLAGS>
__global__ void __launch_bounds__(SEL_ML_SEG) k_select_ml_scatter(const uint8_t* __restrict__ L, int H, int W, int Z,
                                                                  const SelTasks T, const int* __restrict__ chunk_cnt,
                                                                  const int* __restrict__ chunk_off,
                                                                  const uint2* __restrict__ rec,
                                                                  const uint4* __restrict__ wt, TcFlags fl) {
  constexpr int NW = SEL_ML_SEG / 32;
  __shared__ int s_base[CGH_MAX_LAYERS][8];
  __shared__ uint4 s_wt[NW * CGH_MAX_LAYERS];  // the count pass's row totals, [warp][layer]
  __shared__ int s_pos[NW][CGH_MAX_LAYERS][8];
  pdl_wait();
  pdl_trigger();
  const int nseg = (W >> 3) / SEL_ML_SEG, R = blockIdx.x / nseg, sg = blockIdx.x - R * nseg;
  const int bx3 = sg * SEL_ML_SEG + threadIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint2 r = rec[(size_t)R * (W >> 3) + bx3];
  const bool multi = (r.y & ML_MULTI) != 0u;
  uint2 lv[8];
  unsigned long long lmask;
  if (multi) {
#pragma unroll
    for (int q = 0; q < 8; ++q) lv[q] = *reinterpret_cast<const uint2*>(L + (size_t)(8 * R + q) * W + 8 * bx3);
    lmask = ml_layer_mask(lv, Z);
  } else {
#pragma unroll
    for (int q = 0; q < 8; ++q) lv[q] = make_uint2(0u, 0u);
    lmask = ml_rec_layers(r);
  }
  // every row's first position per layer: the prefix of its scan block plus its offset
  for (int e = threadIdx.x; e < 8 * Z; e += blockDim.x) {
    const int z = e >> 3, r8 = e & 7, k = ml_row_list(r8);
    const SelTask& tk = T.t[k];
    const int row = R * ml_rows(k) + ml_row_q(r8);
    const int idx = z * tk.nchunks + row * nseg + sg;
    s_base[z][r8] = chunk_cnt[tk.cnt_off + (idx / SEL_SCAN_BLOCK) * SEL_SCAN_BLOCK] + chunk_off[tk.cnt_off + idx];
  }
  // every warp's row totals per layer, as the count pass left them
  for (int e = threadIdx.x; e < NW * Z; e += blockDim.x) s_wt[e] = wt[(size_t)blockIdx.x * NW * Z + e];
  const unsigned long long uw = ml_warp_or(lmask);
  __syncthreads();
  // first position of every (warp, layer, row)
  for (int e = threadIdx.x; e < 8 * Z; e += blockDim.x) {
    const int z = e >> 3, r8 = e & 7;
    int acc = s_base[z][r8];
#pragma unroll
    for (int v = 0; v < NW; ++v) {
      s_pos[v][z][r8] = acc;
      const uint4 t = s_wt[v * Z + z];
      const unsigned wj = (r8 >> 1) == 0 ? t.x : (r8 >> 1) == 1 ? t.y : (r8 >> 1) == 2 ? t.z : t.w;
      acc += (int)((wj >> (16 * (r8 & 1))) & 0xFFFFu);
    }
  }
  __syncthreads();
  const int za = (int)ml_layer_of(r.x), zb = (int)ml_layer_of(r.y);
  unsigned ea[2] = {0u, 0u}, eb[2] = {0u, 0u};
  for (unsigned long long u = uw; u; u &= u - 1ull) {
    const int z = __ffsll((long long)u) - 1;
    const unsigned b = ml_bits_of(r, lv, lmask, z);
    // the lane's row counts as bytes, rows 0-3 and 4-7, and the warp's inclusive scan
    unsigned nb = b & 0xFFFFu;
    nb = (nb & 0x5555u) + ((nb >> 1) & 0x5555u);
    nb = (nb & 0x3333u) + ((nb >> 2) & 0x3333u);  // nibble q: level-1 row q
    nb = ((nb & 0xFF00u) << 8) | (nb & 0xFFu);
    const unsigned c[2] = {((b >> 21) & 1u) | (((b >> 20) & 1u) << 8) | ((unsigned)__popc((b >> 16) & 3u) << 16) |
                               ((unsigned)__popc((b >> 18) & 3u) << 24),
                           (nb | (nb << 4)) & 0x0F0F0F0Fu};
    unsigned x[2] = {c[0], c[1]};
#pragma unroll
    for (int o = 1; o < 32; o <<= 1)
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const unsigned y = __shfl_up_sync(0xffffffffu, x[j], o);
        if (lane >= o) x[j] += y;
      }
    const unsigned ex[2] = {x[0] - c[0], x[1] - c[1]};
    if (multi) {
      if (b) ml_write<FLAGS>(b, z, ex, s_pos[warp][z], R, bx3, H, W, T, fl);
    } else {
      if (z == za) ea[0] = ex[0], ea[1] = ex[1];
      if (z == zb) eb[0] = ex[0], eb[1] = ex[1];
    }
  }
  if (!multi) {
    if ((r.x >> 21) & 1u) ml_write<FLAGS>(r.x & ML_BITS, za, ea, s_pos[warp][za], R, bx3, H, W, T, fl);
    if ((r.y >> 21) & 1u) ml_write<FLAGS>(r.y & ML_BITS, zb, eb, s_pos[warp][zb], R, bx3, H, W, T, fl);
  }
}

// The four lists of a progressive hologram through the multi-level passes, when the tasks
// are exactly that set (T.t[0]: level 3, no threshold; T.t[l]: level l) and the object
// width is a multiple of 8 x SEL_ML_SEG.  Returns false (nothing launched) otherwise.
static bool select_ml_applies(int obj_h, int obj_w, const SelTasks& T) {
  if (T.n != 4 || (obj_w >> 3) % SEL_ML_SEG || obj_h % 8 || obj_w % 8) return false;
  if (T.t[0].level != 3 || T.t[0].threshold >= 0) return false;
  for (int l = 1; l <= 3; ++l)
    if (T.t[l].level != l) return false;
  return true;
}

static cudaError_t launch_select_ml(int obj_h, int obj_w, int n_layers, const uint8_t* sal, const uint8_t* L,
                                    SelTasks T, int* chunk_cnt, int* chunk_off, uint2* rec, uint4* wt,
                                    cudaStream_t st, const TcFlags* fl) {
  const int nseg = (obj_w >> 3) / SEL_ML_SEG, h3 = obj_h >> 3;
  int off = 0, nblk = 1;
  for (int k = 0; k < 4; ++k) {
    const int rows = ml_rows(k) * h3;
    T.t[k].nchunks = rows * nseg;
    T.t[k].chunk0 = 0;
    T.t[k].cnt_off = off;
    off += n_layers * T.t[k].nchunks;
    const int b = (n_layers * T.t[k].nchunks + SEL_SCAN_BLOCK - 1) / SEL_SCAN_BLOCK;
    nblk = b > nblk ? b : nblk;
  }
  const int grid = h3 * nseg;
  cudaError_t e = launch_pdl(k_select_ml_count, dim3(grid), dim3(SEL_ML_SEG), 0, st, sal, L, obj_h, obj_w, n_layers,
                             T, chunk_cnt, rec, wt);
  if (e == cudaSuccess)
    e = launch_pdl(k_select_scan, dim3(nblk, T.n), dim3(1024), 0, st, chunk_cnt, chunk_off, n_layers, T);
  if (e == cudaSuccess) {
    const TcFlags f = fl ? *fl : TcFlags{};
    e = fl ? launch_pdl(k_select_ml_scatter<true>, dim3(grid), dim3(SEL_ML_SEG), 0, st, L, obj_h, obj_w, n_layers, T,
                        (const int*)chunk_cnt, (const int*)chunk_off, (const uint2*)rec, (const uint4*)wt, f)
           : launch_pdl(k_select_ml_scatter<false>, dim3(grid), dim3(SEL_ML_SEG), 0, st, L, obj_h, obj_w, n_layers, T,
                        (const int*)chunk_cnt, (const int*)chunk_off, (const uint2*)rec, (const uint4*)wt, f);
  }
  return e != cudaSuccess ? e : cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Single-launch selection for small count tables: one CTA per chunk, all co-resident
// (cooperative launch), one grid barrier between the counts and the scatter.
//   1. each CTA computes its blocks' layer masks (kept in registers), its per-layer warp
//      counts and chunk counts, and stores the chunk counts;
//   2. grid barrier;
//   3. each CTA reads its task's whole count table (at most SEL_FUSED_MAX_TABLE entries)
//      and forms, per layer, the task's total and the count of the chunks before its own;
//      an exclusive scan of the totals over the layers gives each layer's first position;
//   4. ordered scatter as in pass 3, optionally marking the selection flags of the
//      tensor-core operands (exactly the marks the written list entries would give).
// The barrier is a sense-reversing counter: CTA 0 adds 2^31 - (G - 1) and the others 1, so
// the top bit flips when the last CTA arrives and the low bits return to their value; it
// needs no reset between launches.  Its wait is bounded (CGH_ERR_TIMEOUT in *status).
#define SEL_FUSED_MAX_TABLE 8192
#define SEL_WAIT_NS 2000000000ull

__device__ __forceinline__ unsigned long long sel_timer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ bool sel_grid_barrier(unsigned* bar, int* status, unsigned long long limit_ns = SEL_WAIT_NS) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned add = blockIdx.x == 0 ? 0x80000000u - (gridDim.x - 1u) : 1u;
    __threadfence();
    const unsigned old = atomicAdd(bar, add);
    const unsigned long long t0 = sel_timer();
    int ok = 1;
    while (((ld_acquire_u32(bar) ^ old) & 0x80000000u) == 0u) {
      if (sel_timer() - t0 > limit_ns) {
        ok = 0;
        if (status) atomicExch(status, CGH_ERR_TIMEOUT);
        break;
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Self-test of the grid barrier's bounded wait: every CTA but `absent` crosses the barrier
// (absent < 0: all of them).  With one CTA absent the barrier never completes, so every
// waiting CTA gives up after limit_ns, records CGH_ERR_TIMEOUT and returns.
__global__ void k_grid_barrier_selftest(unsigned* bar, int* status, unsigned long long limit_ns, int absent,
                                        int* crossed) {
  if ((int)blockIdx.x == absent) return;
  if (sel_grid_barrier(bar, status, limit_ns) && threadIdx.x == 0) atomicAdd(crossed, 1);
}

cudaError_t launch_grid_barrier_selftest(unsigned* bar, int* status, int* crossed, int ctas,
                                         unsigned long long limit_ns, int absent, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(bar, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(ctas);
  cfg.blockDim = dim3(32);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, k_grid_barrier_selftest, bar, status, limit_ns, absent, crossed);
  return e != cudaSuccess ? e : cudaGetLastError();
}

template <bool FLAGS>
__global__ void __launch_bounds__(CGH_SEL_CHUNK) k_select_fused(const uint8_t* __restrict__ sal,
                                                                const uint8_t* __restrict__ L, int H, int W,
                                                                int Z, const SelTasks T, int* cnt_tab,
                                                                unsigned* bar, int* status, TcFlags fl) {
  constexpr int NW = CGH_SEL_CHUNK / 32;
  __shared__ int s_wcnt[NW][CGH_MAX_LAYERS];
  __shared__ int s_tot[CGH_MAX_LAYERS], s_pre[CGH_MAX_LAYERS];
  pdl_wait();
  pdl_trigger();
  const SelTask& tk = T.t[sel_task_of(T, blockIdx.x)];
  const int chunk = blockIdx.x - tk.chunk0, nch = tk.nchunks;
  const int level = tk.level, nbx = W >> level, nb = (H >> level) * nbx;
  const int b = chunk * CGH_SEL_CHUNK + threadIdx.x;
  const int by = b / nbx, bx = b - by * nbx;
  const unsigned long long m = b < nb ? block_layer_mask(sal, L, W, level, by, bx, tk.threshold, Z) : 0ull;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned below = (1u << lane) - 1u;
  for (int z = 0; z < Z; ++z) {
    const unsigned bal = __ballot_sync(0xffffffffu, (m >> z) & 1ull);
    if (lane == 0) s_wcnt[warp][z] = __popc(bal);
  }
  __syncthreads();
  int* cnt = cnt_tab + tk.cnt_off;
  if (threadIdx.x < Z) {
    int run = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
      const int c = s_wcnt[w][threadIdx.x];
      s_wcnt[w][threadIdx.x] = run;
      run += c;
    }
    cnt[threadIdx.x * nch + chunk] = run;
  }
  if (!sel_grid_barrier(bar, status)) return;
  for (int z = warp; z < Z; z += NW) {
    int tot = 0, bef = 0;
#pragma unroll 4
    for (int c = lane; c < nch; c += 32) {
      const int v = __ldcg(cnt + z * nch + c);
      tot += v;
      bef += c < chunk ? v : 0;
    }
    tot = __reduce_add_sync(0xffffffffu, tot);
    bef = __reduce_add_sync(0xffffffffu, bef);
    if (lane == 0) {
      s_tot[z] = tot;
      s_pre[z] = bef;
    }
  }
  __syncthreads();
  if (warp == 0) {  // exclusive scan of the layer totals, two layers per lane
    const int z0 = 2 * lane, z1 = z0 + 1;
    const int a0 = z0 < Z ? s_tot[z0] : 0, a1 = z1 < Z ? s_tot[z1] : 0;
    int inc = a0 + a1;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += t;
    }
    const int ex = inc - a0 - a1;
    if (z0 < Z) s_pre[z0] += ex;
    if (z1 < Z) s_pre[z1] += ex + a0;
    if (chunk == 0 && lane == 31) {
      tk.count[0] = min(inc, tk.capacity);
      tk.count[1] = inc;
    }
  }
  __syncthreads();
  const int hl = H >> level, wl = W >> level;
  for (int z = 0; z < Z; ++z) {
    const bool f = (m >> z) & 1ull;
    const unsigned bal = __ballot_sync(0xffffffffu, f);
    if (f) {
      const int pos = s_pre[z] + s_wcnt[warp][z] + __popc(bal & below);
      if (pos < tk.capacity) {
        tk.list[pos] = (z << 24) | (by << 12) | bx;
        if (FLAGS) {
          if (tk.flag_kind == SEL_FLAGS_LLL) {
            fl.occ3[((size_t)z * hl + by) * wl + bx] = 1;
            fl.rowband[(size_t)z * hl + by] = 1;
            fl.colband[(size_t)z * wl + bx] = 1;
          } else if (tk.flag_kind == SEL_FLAGS_DETAIL) {
            uint8_t* sel = level == 1 ? fl.sel[1] : level == 2 ? fl.sel[2] : fl.sel[3];  // no local copy of fl
            sel[((size_t)z * hl + by) * wl + bx] = 1;
            // the block's 8-pixel bands are kept even when no LLL entry covers them
            fl.rowband[(size_t)z * (H >> 3) + (by >> (3 - level))] = 1;
            fl.colband[(size_t)z * (W >> 3) + (bx >> (3 - level))] = 1;
          }
        }
      }
    }
  }
}

// CTAs of the fused selection that one SM holds at once (the smaller of the two variants).
int select_fused_ctas_per_sm() {
  int a = 0, b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_select_fused<false>, CGH_SEL_CHUNK, 0) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_select_fused<true>, CGH_SEL_CHUNK, 0) != cudaSuccess)
    return 0;
  return a < b ? a : b;
}

int select_tasks_chunks(const SelTasks& T) {
  int n = 0;
  for (int k = 0; k < T.n; ++k) n += T.t[k].nchunks;
  return n;
}

// Fills chunk0 / cnt_off of the tasks and launches the fused selection when its grid fits
// on the device at once and every count table is small, else the three passes.  With `fl`
// the fused kernel also marks the tensor-core selection flags; *flags_done says whether it
// did (the caller derives them from the lists otherwise).
cudaError_t launch_select_tasks(int obj_h, int obj_w, int n_layers, const uint8_t* sal, const uint8_t* L,
                                SelTasks T, int* chunk_cnt, int* chunk_off, cudaStream_t st, const SelCoop* coop,
                                const TcFlags* fl, bool* flags_done) {
  if (flags_done) *flags_done = false;
  int c0 = 0;
  bool small = true;
  for (int k = 0; k < T.n; ++k) {
    T.t[k].nchunks = select_num_chunks(obj_h, obj_w, T.t[k].level);
    T.t[k].chunk0 = c0;
    T.t[k].cnt_off = c0 * n_layers;
    c0 += T.t[k].nchunks;
    small = small && (long long)n_layers * T.t[k].nchunks <= SEL_FUSED_MAX_TABLE;
  }
  if (coop && coop->bar && small && c0 <= coop->max_ctas) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(c0);
    cfg.blockDim = dim3(CGH_SEL_CHUNK);
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    const TcFlags f = fl ? *fl : TcFlags{};
    cudaError_t e = fl ? cudaLaunchKernelEx(&cfg, k_select_fused<true>, sal, L, obj_h, obj_w, n_layers, T, chunk_cnt,
                                            coop->bar, coop->status, f)
                       : cudaLaunchKernelEx(&cfg, k_select_fused<false>, sal, L, obj_h, obj_w, n_layers, T, chunk_cnt,
                                            coop->bar, coop->status, f);
    if (e == cudaSuccess && flags_done) *flags_done = fl != nullptr;
    return e != cudaSuccess ? e : cudaGetLastError();
  }
  if (sal && coop && coop->ml_rec && coop->ml_wt && select_ml_applies(obj_h, obj_w, T)) {
    // the four lists of a large object: one read of the inputs for all levels, then the
    // blocks' records
    const cudaError_t e = launch_select_ml(obj_h, obj_w, n_layers, sal, L, T, chunk_cnt, chunk_off, coop->ml_rec,
                                           coop->ml_wt, st, fl);
    if (e == cudaSuccess && flags_done) *flags_done = fl != nullptr;
    return e;
  }
  cudaError_t e = launch_pdl(k_select_count, dim3(c0), dim3(CGH_SEL_CHUNK), 0, st, sal, L, obj_h, obj_w, n_layers,
                             T, chunk_cnt);
  int nblk = 1;
  for (int k = 0; k < T.n; ++k) {
    const int b = (n_layers * T.t[k].nchunks + SEL_SCAN_BLOCK - 1) / SEL_SCAN_BLOCK;
    nblk = b > nblk ? b : nblk;
  }
  if (e == cudaSuccess)
    e = launch_pdl(k_select_scan, dim3(nblk, T.n), dim3(1024), 0, st, chunk_cnt, chunk_off, n_layers, T);
  if (e == cudaSuccess)
    e = launch_pdl(k_select_scatter, dim3(c0), dim3(CGH_SEL_CHUNK), 0, st, sal, L, obj_h, obj_w, n_layers, T,
                   (const int*)chunk_cnt, (const int*)chunk_off);
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_select(int obj_h, int obj_w, int n_layers, const uint8_t* sal, const uint8_t* L,
                          int threshold, int level, int32_t* list, int32_t* d_count, int capacity,
                          int* chunk_cnt, int* chunk_off, cudaStream_t st, const SelCoop* coop) {
  SelTasks T;
  memset(&T, 0, sizeof(T));
  T.n = 1;
  T.t[0].level = level;
  T.t[0].threshold = threshold;
  T.t[0].capacity = capacity;
  T.t[0].list = list;
  T.t[0].count = d_count;
  return launch_select_tasks(obj_h, obj_w, n_layers, sal, L, T, chunk_cnt, chunk_off, st, coop);
}

// ---------------------------------------------------------------------------
// (A5) plain point-wise hologram (Eq. 1): one SFU sine/cosine per (point, pixel).
// The phase a*(dm^2 + dn^2) mod 1 is exact in 64-bit fixed point: with
// A = round(frac(a) 2^64) and q = dm^2 + dn^2 < 2^31, the top 32 bits of A*q mod 2^64
// are umulhi(A_lo, q) + A_hi*q (mod 2^32).  Their top 23 bits (rounded) become a float
// in [-1/2, 1/2) cycles through the exponent trick (no int-to-float conversion).
// Layered (DEPTH = false): a point takes its layer's rate.  Per-point depth (DEPTH = true,
// the 3-D extension at the end of Section 2 without depth layers): a pixel with a finite
// depth z > 0 takes a = p^2 / (2 lambda z), formed in FP64 with the same operations and
// rounding as the plan's per-layer rates (so a depth map equal to the layer distances
// gives the layered result bit for bit); other pixels are no point.
#define PD_TM 32
#define PD_TN 64
#define PD_CHUNK 256

// LF (the plan's layer factor): each point's amplitude is complex, intensity times
// exp(j 2 pi frac(z/lambda)) / z of its layer or of its own depth.
template <bool DEPTH, bool LF>
__global__ void __launch_bounds__(256) k_plain_direct(const uint8_t* __restrict__ I,
                                                      const uint8_t* __restrict__ L,
                                                      const float* __restrict__ depth, int H, int W,
                                                      int Z, int s, const unsigned long long* a_fixed,
                                                      const float2* __restrict__ lf_full,
                                                      double pitch, double wavelength,
                                                      float2* __restrict__ holo, int HH, int HW,
                                                      int accumulate) {
  __shared__ int4 s_pt[PD_CHUNK];      // (s*i, s*j, amp bits (real part), low word of the rate)
  __shared__ unsigned s_ph[PD_CHUNK];  // high word of the rate
  __shared__ float s_ai[LF ? PD_CHUNK : 1];  // imaginary part of the amplitude
  __shared__ unsigned long long s_a[CGH_MAX_LAYERS];
  __shared__ float2 s_lf[LF && !DEPTH ? CGH_MAX_LAYERS : 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int m0 = blockIdx.y * PD_TM, n0 = blockIdx.x * PD_TN;
  if (!DEPTH && threadIdx.x < Z) s_a[threadIdx.x] = a_fixed[threadIdx.x];
  if constexpr (LF && !DEPTH) {
    if (threadIdx.x < Z) s_lf[threadIdx.x] = lf_full[threadIdx.x];
  }
  int mm[2], nn[4];
#pragma unroll
  for (int r = 0; r < 2; ++r) mm[r] = m0 + ty + 16 * r;
#pragma unroll
  for (int c = 0; c < 4; ++c) nn[c] = n0 + tx + 16 * c;
  float re[2][4], im[2][4];
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) re[r][c] = im[r][c] = 0.f;
  const int npts = H * W;
  for (int base = 0; base < npts; base += PD_CHUNK) {
    __syncthreads();
    {
      const int p = base + threadIdx.x;
      int4 v = make_int4(0, 0, 0, 0);
      unsigned long long af = 0;
      float ai = 0.f;
      if (p < npts) {
        const int i = p / W, j = p - (p / W) * W;
        float amp;
        if constexpr (DEPTH) {
          const float zf = depth[p];
          const bool ok = zf > 0.f && isfinite(zf);
          amp = ok ? (float)I[p] : 0.f;
          if (ok) {
            const double a = pitch * pitch / (2.0 * wavelength * (double)zf);
            const double x = floor((a - floor(a)) * 18446744073709551616.0 + 0.5);
            af = x >= 18446744073709551616.0 ? 0ull : (unsigned long long)x;
            if constexpr (LF) {  // exp(j 2 pi frac(z/lambda)) / z of the point's own depth
              const double zl = (double)zf / wavelength;
              double sn, cs;
              sincospi(2.0 * (zl - floor(zl)), &sn, &cs);
              ai = (float)(amp * sn / (double)zf);
              amp = (float)(amp * cs / (double)zf);
            }
          }
        } else {
          const int lz = L[p];
          amp = lz < Z ? (float)I[p] : 0.f;
          af = s_a[lz < Z ? lz : 0];
          if constexpr (LF) {
            const float2 c = s_lf[lz < Z ? lz : 0];
            ai = amp * c.y;
            amp = amp * c.x;
          }
        }
        v = make_int4(s * i, s * j, __float_as_int(amp), (int)(unsigned)(af & 0xffffffffull));
      }
      s_pt[threadIdx.x] = v;
      s_ph[threadIdx.x] = (unsigned)(af >> 32);
      if constexpr (LF) s_ai[threadIdx.x] = ai;
    }
    __syncthreads();
    const int cnt = min(PD_CHUNK, npts - base);
    // Two-level accumulation: a chunk of points is summed in fresh registers and then
    // added to the running total, which keeps the FP32 rounding error near
    // u*(sqrt(chunk) + sqrt(points/chunk)) instead of u*sqrt(points).
    float cre[2][4], cim[2][4];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) cre[r][c] = cim[r][c] = 0.f;
#pragma unroll 2
    for (int k = 0; k < cnt; ++k) {
      const int4 pt = s_pt[k];
      const float amp = __int_as_float(pt.z);
      const float amp_i = LF ? s_ai[k] : 0.f;
      const unsigned alo = (unsigned)pt.w, ahi = s_ph[k];
      unsigned dx2[2], dy2[4];
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        const int d = mm[r] - pt.x;
        dx2[r] = (unsigned)(d * d);
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int d = nn[c] - pt.y;
        dy2[c] = (unsigned)(d * d);
      }
#pragma unroll
      for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const unsigned q = dx2[r] + dy2[c];
          const unsigned ph = __umulhi(alo, q) + ahi * q + 256u;  // +half LSB of the 23-bit cut
          const float cyc = __int_as_float(((ph >> 9) ^ 0x400000u) | 0x3f800000u) - 1.5f;
          float sn, cs;
          __sincosf(cyc * 6.28318530717958647692f, &sn, &cs);
          if constexpr (LF) {
            cre[r][c] = fmaf(amp, cs, fmaf(-amp_i, sn, cre[r][c]));
            cim[r][c] = fmaf(amp, sn, fmaf(amp_i, cs, cim[r][c]));
          } else {
            cre[r][c] = fmaf(amp, cs, cre[r][c]);
            cim[r][c] = fmaf(amp, sn, cim[r][c]);
          }
        }
    }
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        re[r][c] += cre[r][c];
        im[r][c] += cim[r][c];
      }
  }
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c)
      if (mm[r] < HH && nn[c] < HW) {
        float2* o = holo + (size_t)mm[r] * HW + nn[c];
        if (accumulate) {
          const float2 prev = *o;
          *o = make_float2(prev.x + re[r][c], prev.y + im[r][c]);
        } else {
          *o = make_float2(re[r][c], im[r][c]);
        }
      }
}

cudaError_t launch_plain_direct(const cgh_plan* p, const uint8_t* I, const uint8_t* L, float2* holo,
                                cudaStream_t st) {
  dim3 grid((p->holo_w + PD_TN - 1) / PD_TN, (p->holo_h + PD_TM - 1) / PD_TM);
  if (p->layer_factor)
    k_plain_direct<false, true><<<grid, 256, 0, st>>>(I, L, nullptr, p->obj_h, p->obj_w, p->n_layers, p->s,
                                                      p->d_a_fixed, p->d_lf_full, p->pitch, p->wavelength, holo,
                                                      p->holo_h, p->holo_w, 0);
  else
    k_plain_direct<false, false><<<grid, 256, 0, st>>>(I, L, nullptr, p->obj_h, p->obj_w, p->n_layers, p->s,
                                                       p->d_a_fixed, nullptr, p->pitch, p->wavelength, holo,
                                                       p->holo_h, p->holo_w, 0);
  return cudaGetLastError();
}

cudaError_t launch_pointcloud_direct(const cgh_plan* p, const uint8_t* I, const float* depth, float2* holo,
                                     int accumulate, cudaStream_t st) {
  dim3 grid((p->holo_w + PD_TN - 1) / PD_TN, (p->holo_h + PD_TM - 1) / PD_TM);
  if (p->layer_factor)
    k_plain_direct<true, true><<<grid, 256, 0, st>>>(I, nullptr, depth, p->obj_h, p->obj_w, p->n_layers, p->s,
                                                     nullptr, nullptr, p->pitch, p->wavelength, holo, p->holo_h,
                                                     p->holo_w, accumulate);
  else
    k_plain_direct<true, false><<<grid, 256, 0, st>>>(I, nullptr, depth, p->obj_h, p->obj_w, p->n_layers, p->s,
                                                      nullptr, nullptr, p->pitch, p->wavelength, holo, p->holo_h,
                                                      p->holo_w, accumulate);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// (A4, direct form) detail-basis superposition on CUDA cores (Eq. 3, Section 2 steps 2-5).
// Every LLL block adds the rank-1 term  b_3(m-u) x (LLL/64) b_3(n-v); every selected
// detail block of level l adds the rank-2 update
//     b_l(m-u) x 4^-l X w_l(n-v)  +  w_l(m-u) x 4^-l (Y b_l(n-v) + D w_l(n-v)),
// (X pairs with the column difference, Y with the row difference).  A CTA owns a
// 128x128 hologram tile and a 1/S share of every list (split over the grid's z),
// stages 32 rank-1 terms at a time in shared memory as row and column factors and
// accumulates 8x8 complex pixels per thread in registers (two packed FP32x2 FMAs, i.e. 4
// fused multiply-adds, per term and pixel).
#define DL_TM 128
#define DL_TN 128
#define DL_KC 32

struct DlTerm {
  int row_base;  // table index of (row factor) at m = 0
  int col_b;     // table index of b_l at n = 0
  int col_w;     // table index of w_l at n = 0
  float cb, cw;  // column factor = cb*b_l + cw*w_l
};

__global__ void __launch_bounds__(256, 1) k_direct_lut(
    const float2* __restrict__ tab, int tab_len, int tab_off, const int32_t* __restrict__ coef,
    const int32_t* __restrict__ l0, const int32_t* __restrict__ l1, const int32_t* __restrict__ l2,
    const int32_t* __restrict__ l3, const int32_t* __restrict__ d_counts, int H, int W, int Z, int s,
    float2* __restrict__ holo, int HH, int HW, int use_atomic, int* status) {
  // Row factors staged as (x, x, -y, y) and column factors as (x, y, y, x): a complex
  // multiply-accumulate is then two packed FP32x2 FMAs, (x,x)*(cx,cy) + (-y,y)*(cy,cx).
  extern __shared__ float4 dl_smem[];
  float4* Rs = dl_smem;                  // [DL_KC][DL_TM]
  float4* Cs = dl_smem + DL_KC * DL_TM;  // [DL_KC][DL_TN]
  __shared__ DlTerm s_term[DL_KC];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int m0 = blockIdx.y * DL_TM, n0 = blockIdx.x * DL_TN;
  const int split = blockIdx.z, nsplit = gridDim.z;
  float2 acc[8][8];
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[r][c] = make_float2(0.f, 0.f);

  const int32_t* lists[4] = {l0, l1, l2, l3};
  for (int li = 0; li < 4; ++li) {
    const int level = li == 0 ? 3 : li;
    const bool lll = li == 0;
    const int cnt = clamp_list_count(d_counts[2 * li], Z * (H >> level) * (W >> level),
                                     blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 ? status : nullptr);
    const int e0 = (int)((long long)cnt * split / nsplit);
    const int e1 = (int)((long long)cnt * (split + 1) / nsplit);
    const int per = lll ? DL_KC : DL_KC / 2;  // entries per chunk
    const int hl = H >> level, wl = W >> level;
    const float kappa = 1.0f / (float)(1 << (2 * level));
    const int32_t* lst = lists[li];
    for (int e = e0; e < e1; e += per) {
      const int ne = min(per, e1 - e);
      const int nt = lll ? ne : 2 * ne;
      __syncthreads();  // previous chunk fully consumed
      if (threadIdx.x < ne) {
        const int ent = lst[e + threadIdx.x];
        int z = (ent >> 24) & 0x7F, by = (ent >> 12) & 0xFFF, bx = ent & 0xFFF;
        // An entry outside the plan (corrupt list) adds nothing instead of reading out of bounds.
        const bool ok = z < Z && by < hl && bx < wl;
        if (!ok) z = by = bx = 0;
        const int32_t* P = coef + (size_t)z * H * W;
        const int u = s * (by << level), v = s * (bx << level);
        const int tb = ((z * 4 + level) * 2 + 0) * tab_len + tab_off;
        const int tw = ((z * 4 + level) * 2 + 1) * tab_len + tab_off;
        if (lll) {
          const float S3 = ok ? (float)P[(size_t)by * W + bx] : 0.f;
          s_term[threadIdx.x] = DlTerm{tb - u, tb - v, tw - v, kappa * S3, 0.f};
        } else {
          const float X = ok ? (float)P[(size_t)by * W + wl + bx] : 0.f;
          const float Y = ok ? (float)P[(size_t)(hl + by) * W + bx] : 0.f;
          const float D = ok ? (float)P[(size_t)(hl + by) * W + wl + bx] : 0.f;
          s_term[2 * threadIdx.x] = DlTerm{tb - u, tb - v, tw - v, 0.f, kappa * X};
          s_term[2 * threadIdx.x + 1] = DlTerm{tw - u, tb - v, tw - v, kappa * Y, kappa * D};
        }
      }
      __syncthreads();
      for (int q = threadIdx.x; q < nt * DL_TM; q += 256) {
        const int k = q / DL_TM, r = q - k * DL_TM;
        const DlTerm t = s_term[k];
        const int m = m0 + r, n = n0 + r;
        float2 rv = make_float2(0.f, 0.f), cv = make_float2(0.f, 0.f);
        if (m < HH) rv = tab[t.row_base + m];
        if (n < HW) {
          const float2 b = tab[t.col_b + n], w = tab[t.col_w + n];
          cv = make_float2(t.cb * b.x + t.cw * w.x, t.cb * b.y + t.cw * w.y);
        }
        Rs[k * DL_TM + r] = make_float4(rv.x, rv.x, -rv.y, rv.y);
        Cs[k * DL_TN + r] = make_float4(cv.x, cv.y, cv.y, cv.x);
      }
      __syncthreads();
#pragma unroll 2
      for (int k = 0; k < nt; ++k) {
        float4 rv[8], cv[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) rv[r] = Rs[k * DL_TM + ty + 16 * r];
#pragma unroll
        for (int c = 0; c < 8; ++c) cv[c] = Cs[k * DL_TN + tx + 16 * c];
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            acc[r][c] = __ffma2_rn(make_float2(rv[r].x, rv[r].y), make_float2(cv[c].x, cv[c].y), acc[r][c]);
            acc[r][c] = __ffma2_rn(make_float2(rv[r].z, rv[r].w), make_float2(cv[c].z, cv[c].w), acc[r][c]);
          }
      }
    }
  }
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int m = m0 + ty + 16 * r, n = n0 + tx + 16 * c;
      if (m < HH && n < HW) {
        float2* dst = holo + (size_t)m * HW + n;
        if (use_atomic)
          atomicAdd(dst, acc[r][c]);
        else
          *dst = acc[r][c];
      }
    }
}

static int g_num_sms = 0;

static int num_sms() {
  if (!g_num_sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_num_sms <= 0) g_num_sms = 148;
  }
  return g_num_sms;
}

// Number of term splits: the smallest S (<= 64) whose CTA count S*tiles fills at least
// two waves of one CTA per SM with a tail under 5%, else the best found.
static int direct_lut_splits(int tiles) {
  const int sms = num_sms();
  int best = 1;
  double best_eff = 0.0;
  for (int S = 1; S <= 64; ++S) {
    const long long ctas = (long long)S * tiles;
    const double waves = (double)ctas / sms;
    const double eff = waves / ceil(waves);
    if (ctas >= 2LL * sms && eff >= 0.95) return S;
    if (eff > best_eff + 1e-9) {
      best_eff = eff;
      best = S;
    }
  }
  return best;
}

#define DL_SMEM ((size_t)DL_KC * (DL_TM + DL_TN) * sizeof(float4))

cudaError_t basic_init_attributes() {
  return cudaFuncSetAttribute(k_direct_lut, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)DL_SMEM);
}

cudaError_t launch_direct_lut(const cgh_plan* p, const int32_t* coef, const int32_t* const* lists,
                              const int32_t* d_counts, float2* holo, cudaStream_t st) {
  const int tn = (p->holo_w + DL_TN - 1) / DL_TN, tm = (p->holo_h + DL_TM - 1) / DL_TM;
  const int S = p->deterministic ? 1 : direct_lut_splits(tn * tm);
  const size_t smem = DL_SMEM;
  dim3 grid(tn, tm, S);
  // holo must be zero (or hold the previous hologram) when S > 1: atomics accumulate.
  k_direct_lut<<<grid, 256, smem, st>>>(p->d_tab, p->tab_len, p->tab_off, coef, lists[0], lists[1],
                                        lists[2], lists[3], d_counts, p->obj_h, p->obj_w, p->n_layers, p->s, holo,
                                        p->holo_h, p->holo_w, 1, p->d_status);
  return cudaGetLastError();
}
