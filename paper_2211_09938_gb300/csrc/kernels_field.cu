// Layer fields on the tensor cores: Fresnel back-propagation (reconstruction), its
// adjoint (propagation of complex layer fields to the hologram) and the adjoint of the
// progressive operator with respect to the object.
//
// With E_z[m][i] = f_z(m - s*i) (Eq. 1, paraxial, one axis) and square geometry:
//   reconstruct:  R_z = E_z^H H conj(E_z)             (stages R1: T_z = E_z^H H, R2: T_z conj(E_z))
//   propagate:    H  += sum_z E_z F_z E_z^T            (stages P1: Y_z^T = E_z F_z^T, P2: sum over z)
// The three fringe operands (conj(E_z) by rows i, E_z by rows m, E_z by rows n) depend only
// on the geometry and are built once per plan in bf16 hi+lo planes.  Data operands (the
// hologram, its intermediate T_z, the fields, Y^T) are split into bf16 hi+lo planes, and
// every complex product is 3 x 4 real MMAs with FP32 accumulation (tc_gemm.cuh).
#include "tc_gemm.cuh"

// ------------------------------------------------------------------------------------
// operand builders

// Fringe planes out[p][r][c], 8 columns per thread (C a multiple of 8), hi+lo in bf16 or fp16:
//   MODE 0 (conj rows):  r = z*div + i, c = m         -> conj(f_z(m - s*i))   (div = obj edge)
//   MODE 1 (E by m):     r = m,         c = z*div + i -> f_z(m - s*i)         (div = obj_h)
//   MODE 2 (E by n):     r = z*div + n, c = j         -> f_z(n - s*j)         (div = holo_w)
template <int MODE, bool F16>
__global__ void k_fe_build(const float2* __restrict__ tab, int tab_len, int tab_off, int s, int div, int R, int C,
                           uint16_t* __restrict__ out, long long plane) {
  const int c = 8 * (blockIdx.x * blockDim.x + threadIdx.x);
  const int r = blockIdx.y * blockDim.y + threadIdx.y;
  if (r >= R || c >= C) return;
  uint32_t w[4][4];
#pragma unroll
  for (int q = 0; q < 8; q += 2) {
    uint16_t h[2][4];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int cc = c + q + u;
      int z, d;
      if (MODE == 0) {
        z = r / div;
        d = cc - s * (r - z * div);
      } else if (MODE == 1) {
        z = cc / div;
        d = r - s * (cc - z * div);
      } else {
        z = r / div;
        d = (r - z * div) - s * cc;
      }
      float2 v = tab[(size_t)(z * 4 + 0) * 2 * tab_len + tab_off + d];
      if (MODE == 0) v.y = -v.y;
      split_hi_lo<F16>(v.x, h[u][0], h[u][1]);
      split_hi_lo<F16>(v.y, h[u][2], h[u][3]);
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) w[p][q / 2] = (uint32_t)h[0][p] | ((uint32_t)h[1][p] << 16);
  }
  uint16_t* dst = out + (size_t)r * C + c;
#pragma unroll
  for (int p = 0; p < 4; ++p)
    *reinterpret_cast<uint4*>(dst + p * plane) = make_uint4(w[p][0], w[p][1], w[p][2], w[p][3]);
}

// Complex matrix -> bf16 hi+lo planes, transposed: out[p][c][r] from in[r][c] (n x n tiles
// of 32 through shared memory).
__global__ void k_split_transpose(const float2* __restrict__ in, int rows, int cols, uint16_t* __restrict__ out,
                                  long long plane, float scale) {
  __shared__ float2 tile[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int r = r0 + y, c = c0 + threadIdx.x;
    tile[y][threadIdx.x] = (r < rows && c < cols) ? in[(size_t)r * cols + c] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int c = c0 + y, r = r0 + threadIdx.x;  // output row c, column r
    if (c < cols && r < rows) {
      const float2 v = tile[threadIdx.x][y];
      uint16_t rh, rl, ih, il;
      split_hi_lo<false>(v.x * scale, rh, rl);
      split_hi_lo<false>(v.y * scale, ih, il);
      uint16_t* d = out + (size_t)c * rows + r;
      d[0] = rh;
      d[plane] = rl;
      d[2 * plane] = ih;
      d[3 * plane] = il;
    }
  }
}

// Complex matrix -> bf16 hi+lo planes, same layout (8 columns per thread, cols % 8 == 0).
__global__ void k_split_rows(const float2* __restrict__ in, long long rows, int cols, uint16_t* __restrict__ out,
                             long long plane) {
  const int c = 8 * (blockIdx.x * blockDim.x + threadIdx.x);
  const long long r = (long long)blockIdx.y * blockDim.y + threadIdx.y;
  if (r >= rows || c >= cols) return;
  uint32_t w[4][4];
#pragma unroll
  for (int q = 0; q < 8; q += 2) {
    uint16_t h[2][4];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const float2 v = in[r * cols + c + q + u];
      split_hi_lo<false>(v.x, h[u][0], h[u][1]);
      split_hi_lo<false>(v.y, h[u][2], h[u][3]);
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) w[p][q / 2] = (uint32_t)h[0][p] | ((uint32_t)h[1][p] << 16);
  }
  uint16_t* dst = out + r * cols + c;
#pragma unroll
  for (int p = 0; p < 4; ++p)
    *reinterpret_cast<uint4*>(dst + p * plane) = make_uint4(w[p][0], w[p][1], w[p][2], w[p][3]);
}

// amplitude(i,j) = |R_{layer(i,j)}(i,j)| (0 where the pixel owns no layer)
__global__ void k_amplitude(const float2* __restrict__ F, const uint8_t* __restrict__ L, int n, int Z,
                            float* __restrict__ amp) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const int z = L[p];
  float a = 0.f;
  if (z < Z) {
    const float2 v = F[(size_t)z * n + p];
    a = sqrtf(v.x * v.x + v.y * v.y);
  }
  amp[p] = a;
}

// d amplitude -> d fields: for z = layer(i,j): g * R / |R| (0 at R = 0); 0 elsewhere.
__global__ void k_amplitude_backward(const float2* __restrict__ F, const uint8_t* __restrict__ L, int n, int Z,
                                     const float* __restrict__ g, float2* __restrict__ gF) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  const int z = blockIdx.y;
  if (p >= n) return;
  float2 out = make_float2(0.f, 0.f);
  if (L[p] == z) {
    const float2 v = F[(size_t)z * n + p];
    const float a = sqrtf(v.x * v.x + v.y * v.y);
    if (a > 0.f) out = make_float2(g[p] * v.x / a, g[p] * v.y / a);
  }
  gF[(size_t)z * n + p] = out;
}

// The progressive approximation P_z of one 8x8 block of layer z, in place: 3-level Haar,
// LLL and detail coefficients of blocks outside the layer's lists set to zero (flags),
// inverse Haar.  It is an orthogonal projection in the Haar basis, hence self-adjoint.
__device__ __forceinline__ void haar_project_block(float (&a)[8][8], const TcFlags& fl, int H, int W, int z,
                                                   int by, int bx) {
  // forward: levels 1..3 in place on the low band, detail kept or dropped per flags
  float s1[4][4], x1[4][4], y1[4][4], d1[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const float A = a[2 * r][2 * c], B = a[2 * r][2 * c + 1], C = a[2 * r + 1][2 * c], D = a[2 * r + 1][2 * c + 1];
      const bool k = fl.sel[1][((size_t)z * (H >> 1) + 4 * by + r) * (W >> 1) + 4 * bx + c] != 0;
      s1[r][c] = A + B + C + D;
      x1[r][c] = k ? A - B + C - D : 0.f;
      y1[r][c] = k ? A + B - C - D : 0.f;
      d1[r][c] = k ? A - B - C + D : 0.f;
    }
  float s2[2][2], x2[2][2], y2[2][2], d2[2][2];
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const float A = s1[2 * r][2 * c], B = s1[2 * r][2 * c + 1], C = s1[2 * r + 1][2 * c], D = s1[2 * r + 1][2 * c + 1];
      const bool k = fl.sel[2][((size_t)z * (H >> 2) + 2 * by + r) * (W >> 2) + 2 * bx + c] != 0;
      s2[r][c] = A + B + C + D;
      x2[r][c] = k ? A - B + C - D : 0.f;
      y2[r][c] = k ? A + B - C - D : 0.f;
      d2[r][c] = k ? A - B - C + D : 0.f;
    }
  const size_t f3 = ((size_t)z * (H >> 3) + by) * (W >> 3) + bx;
  const bool k3 = fl.sel[3][f3] != 0;
  const float A = s2[0][0], B = s2[0][1], C = s2[1][0], D = s2[1][1];
  const float S3 = fl.occ3[f3] ? A + B + C + D : 0.f;
  const float X3 = k3 ? A - B + C - D : 0.f, Y3 = k3 ? A + B - C - D : 0.f, D3 = k3 ? A - B - C + D : 0.f;
  // inverse: child (r, c) of a cell gets (S + sx X + sy Y + sx sy D) / 4
  float t2[2][2];
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const float sx = c ? -1.f : 1.f, sy = r ? -1.f : 1.f;
      t2[r][c] = 0.25f * (S3 + sx * X3 + sy * Y3 + sx * sy * D3);
    }
  float t1[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int pr = r >> 1, pc = c >> 1;
      const float sx = (c & 1) ? -1.f : 1.f, sy = (r & 1) ? -1.f : 1.f;
      t1[r][c] = 0.25f * (t2[pr][pc] + sx * x2[pr][pc] + sy * y2[pr][pc] + sx * sy * d2[pr][pc]);
    }
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int pr = r >> 1, pc = c >> 1;
      const float sx = (c & 1) ? -1.f : 1.f, sy = (r & 1) ? -1.f : 1.f;
      a[r][c] = 0.25f * (t1[pr][pc] + sx * x1[pr][pc] + sy * y1[pr][pc] + sx * sy * d1[pr][pc]);
    }
}

// Adjoint of the progressive operator on one 8x8 block of one layer: x = Re R_z, then the
// layer's progressive approximation, kept where the pixel belongs to layer z.
__global__ void k_adjoint_project(const float2* __restrict__ F, const uint8_t* __restrict__ L, TcFlags fl, int H,
                                  int W, int Z, float* __restrict__ grad) {
  const int bx = blockIdx.x * blockDim.x + threadIdx.x, by = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (bx >= (W >> 3) || by >= (H >> 3)) return;
  float a[8][8];
  const float2* Fz = F + (size_t)z * H * W;
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = 0; c < 8; ++c) a[r][c] = Fz[(size_t)(8 * by + r) * W + 8 * bx + c].x;
  haar_project_block(a, fl, H, W, z, by, bx);
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const size_t o = (size_t)(8 * by + r) * W + 8 * bx + c;
      if (L[o] == z) grad[o] = a[r][c];
    }
}

// The progressive operator's object side for a real object x (its transpose is
// k_adjoint_project): the layer plane x [layer = z], projected by P_z, written as the
// complex layer field F_z (imaginary part 0) over the whole block.
__global__ void k_forward_project(const float* __restrict__ x, const uint8_t* __restrict__ L, TcFlags fl, int H,
                                  int W, int Z, float2* __restrict__ F) {
  const int bx = blockIdx.x * blockDim.x + threadIdx.x, by = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (bx >= (W >> 3) || by >= (H >> 3)) return;
  float a[8][8];
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const size_t o = (size_t)(8 * by + r) * W + 8 * bx + c;
      a[r][c] = L[o] == z ? x[o] : 0.f;
    }
  haar_project_block(a, fl, H, W, z, by, bx);
  float2* Fz = F + (size_t)z * H * W;
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = 0; c < 8; ++c) Fz[(size_t)(8 * by + r) * W + 8 * bx + c] = make_float2(a[r][c], 0.f);
}

__global__ void k_phase_to_field(const float* __restrict__ phase, float2* __restrict__ field, long long n) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  float sn, cs;
  sincosf(phase[p], &sn, &cs);
  field[p] = make_float2(cs, sn);
}

// dL/dphi = Im(g * conj(H)) for H = exp(j phi) and the real-pair gradient g of L wrt H.
__global__ void k_phase_grad(const float2* __restrict__ field, const float2* __restrict__ g,
                             float* __restrict__ gphi, long long n) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const float2 h = field[p], q = g[p];
  gphi[p] = q.y * h.x - q.x * h.y;
}

// ------------------------------------------------------------------------------------
// host side

// Geometry operands shared by the progressive tensor form and the field stages, built once
// per plan and dtype: EZ[p][m][z*obj_h + i] = f_z(m - s*i) and EZt[p][z*holo_w + n][j] =
// f_z(n - s*j) as hi+lo planes (index 0 bf16, 1 fp16).
struct cgh_eops {
  int built[2];
  uint16_t* EZ[2];
  uint16_t* EZt[2];
  long long ez_plane, ezt_plane;
  CUtensorMap mEZ[2], mEZt[2];
  CUtensorMap mEZh[2], mEZth[2];  // the hi planes only (re_hi, im_hi) of the same memory
};

void eops_destroy(cgh_plan* p) {
  cgh_eops* e = p->eops;
  if (!e) return;
  for (int k = 0; k < 2; ++k) {
    cudaFree(e->EZ[k]);
    cudaFree(e->EZt[k]);
  }
  free(e);
  p->eops = nullptr;
}

int eops_get(const cgh_plan* pc, int f16, const CUtensorMap** mEZ, const CUtensorMap** mEZt, cudaStream_t st) {
  cgh_plan* p = const_cast<cgh_plan*>(pc);
  if (!p->eops) {
    p->eops = (cgh_eops*)calloc(1, sizeof(cgh_eops));
    if (!p->eops) return cgh_fail(CGH_ERR_NOMEM, "fringe operands: host allocation");
    p->eops->ez_plane = (long long)p->holo_h * p->n_layers * p->obj_h;
    p->eops->ezt_plane = (long long)p->n_layers * p->holo_w * p->obj_w;
  }
  cgh_eops* e = p->eops;
  const int k = f16 ? 1 : 0;
  if (!e->built[k]) {
    const int Z = p->n_layers;
    int rc = cgh_cuda_check(cudaMalloc(&e->EZ[k], 4 * e->ez_plane * 2), "fringe operands: EZ");
    if (rc == CGH_OK) rc = cgh_cuda_check(cudaMalloc(&e->EZt[k], 4 * e->ezt_plane * 2), "fringe operands: EZt");
    if (rc == CGH_OK) rc = make_plane_map(&e->mEZ[k], e->EZ[k], 4, p->holo_h, (long long)Z * p->obj_h);
    if (rc == CGH_OK) rc = make_plane_map(&e->mEZt[k], e->EZt[k], 4, (long long)Z * p->holo_w, p->obj_w);
    if (rc == CGH_OK) rc = make_hi_plane_map(&e->mEZh[k], e->EZ[k], p->holo_h, (long long)Z * p->obj_h);
    if (rc == CGH_OK) rc = make_hi_plane_map(&e->mEZth[k], e->EZt[k], (long long)Z * p->holo_w, p->obj_w);
    if (rc != CGH_OK) {
      cudaFree(e->EZ[k]);
      cudaFree(e->EZt[k]);
      e->EZ[k] = e->EZt[k] = nullptr;
      return rc;
    }
    dim3 blk(8, 32);
    const int C1 = Z * p->obj_h, R2 = Z * p->holo_w;
    if (f16) {
      k_fe_build<1, true><<<dim3((C1 / 8 + 7) / 8, (p->holo_h + 31) / 32), blk, 0, st>>>(
          p->d_tab, p->tab_len, p->tab_off, p->s, p->obj_h, p->holo_h, C1, e->EZ[k], e->ez_plane);
      k_fe_build<2, true><<<dim3((p->obj_w / 8 + 7) / 8, (R2 + 31) / 32), blk, 0, st>>>(
          p->d_tab, p->tab_len, p->tab_off, p->s, p->holo_w, R2, p->obj_w, e->EZt[k], e->ezt_plane);
    } else {
      k_fe_build<1, false><<<dim3((C1 / 8 + 7) / 8, (p->holo_h + 31) / 32), blk, 0, st>>>(
          p->d_tab, p->tab_len, p->tab_off, p->s, p->obj_h, p->holo_h, C1, e->EZ[k], e->ez_plane);
      k_fe_build<2, false><<<dim3((p->obj_w / 8 + 7) / 8, (R2 + 31) / 32), blk, 0, st>>>(
          p->d_tab, p->tab_len, p->tab_off, p->s, p->holo_w, R2, p->obj_w, e->EZt[k], e->ezt_plane);
    }
    rc = cgh_cuda_check(cudaGetLastError(), "fringe operands: build");
    if (rc != CGH_OK) return rc;
    e->built[k] = 1;
  }
  if (mEZ) *mEZ = &e->mEZ[k];
  if (mEZt) *mEZt = &e->mEZt[k];
  return CGH_OK;
}

int eops_get_hi(const cgh_plan* p, int f16, const CUtensorMap** mEZh, const CUtensorMap** mEZth, cudaStream_t st) {
  const int rc = eops_get(p, f16, nullptr, nullptr, st);
  if (rc != CGH_OK) return rc;
  const int k = f16 ? 1 : 0;
  *mEZh = &p->eops->mEZh[k];
  *mEZth = &p->eops->mEZth[k];
  return CGH_OK;
}

// Reconstruction and propagation scratch for batches of up to `cap` holograms: the data
// planes stack the holograms (Ht rows b*Nh + n, T and Fp rows (b*Z + z)*No + i, Yp columns
// (b*Z + z)*No + i), so that one launch per GEMM stage covers the batch (units (b, z) decoded
// by the stacked-problem fields of mode 3); the propagation's last stage runs per hologram on
// a view of Yp (mYpb[b]).
#define FIELD_MAX_BATCH 64
struct cgh_field_state {
  int No, Nh, Z, cap;
  uint16_t* GZ;                // conj(E_z) by rows i (built once)
  uint16_t *Ht, *T, *Fp, *Yp;  // data planes, for `cap` holograms
  float2* F;                   // fields scratch [cap][Z][No][No]
  long long gz_plane, ht_plane, t_plane, fp_plane, yp_plane;
  CUtensorMap mGZ, mHt, mT, mFp, mYp;
  CUtensorMap mYpb[FIELD_MAX_BATCH];  // hologram b's columns of Yp
  const CUtensorMap *mEZ, *mEZt;      // bf16 geometry operands (cgh_eops)
  int built;
};

int field_init_attributes() {
  cudaError_t e;
  if ((e = set_gemm_attr<KIND_CC, EPI_Y, false>()) != cudaSuccess ||
      (e = set_gemm_attr<KIND_CC, EPI_F, false>()) != cudaSuccess ||
      (e = set_gemm_attr<KIND_CC, EPI_H, false>()) != cudaSuccess)
    return cgh_cuda_check(e, "field kernel attributes");
  return CGH_OK;
}

static void field_free_data(cgh_field_state* f) {
  cudaFree(f->Ht);
  cudaFree(f->T);
  cudaFree(f->Fp);
  cudaFree(f->Yp);
  cudaFree(f->F);
  f->Ht = f->T = f->Fp = f->Yp = nullptr;
  f->F = nullptr;
  f->cap = 0;
}

void field_destroy(cgh_plan* p) {
  cgh_field_state* f = p->fs;
  if (!f) return;
  cudaFree(f->GZ);
  field_free_data(f);
  free(f);
  p->fs = nullptr;
}

// A 4-plane hi+lo map over a column range of a wider row-major array: rows x cols from
// `base`, ld elements between rows, plane_stride elements between planes.
static int make_plane_view(CUtensorMap* map, const void* base, long long rows, long long cols, long long ld,
                           long long plane_stride) {
  if (get_encoder() != CGH_OK) return CGH_ERR_CUDA;
  if (((uintptr_t)base & 15) || (ld * 2) % 16 || (cols * 2) % 16)
    return cgh_fail(CGH_ERR_ARG, "tensor map: base must be 16-byte aligned and rows a multiple of 16 bytes");
  cuuint64_t dims[3] = {(cuuint64_t)cols, (cuuint64_t)rows, 4};
  cuuint64_t strides[2] = {(cuuint64_t)(ld * 2), (cuuint64_t)(plane_stride * 2)};
  cuuint32_t box[3] = {TC_BK, 128, 4};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_UINT16, 3, const_cast<void*>(base), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return cgh_fail(CGH_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return CGH_OK;
}

// The plan's field state with room for n holograms: the geometry operand once, the data planes
// (re)allocated when n exceeds the capacity (outside stream capture: the first call with the
// largest batch must run eagerly).
static int field_ensure(const cgh_plan* pc, cudaStream_t st, int n = 1) {
  cgh_plan* p = const_cast<cgh_plan*>(pc);
  if (n < 1 || n > FIELD_MAX_BATCH) return cgh_fail(CGH_ERR_ARG, "fields: batch %d not in [1, %d]", n, FIELD_MAX_BATCH);
  if (p->fs && p->fs->built && p->fs->cap >= n) return CGH_OK;
  if (p->obj_h != p->obj_w || p->holo_h != p->holo_w)
    return cgh_fail(CGH_ERR_UNSUPPORTED, "fields: square object and hologram required");
  const int No = p->obj_h, Nh = p->holo_h, Z = p->n_layers;
  if (No % 32) return cgh_fail(CGH_ERR_UNSUPPORTED, "fields: object edge must be a multiple of 32");
  int rc = eops_get(p, 0, nullptr, nullptr, st);
  if (rc != CGH_OK) return rc;
  cgh_field_state* f = p->fs ? p->fs : (cgh_field_state*)calloc(1, sizeof(cgh_field_state));
  if (!f) return cgh_fail(CGH_ERR_NOMEM, "fields: host allocation");
  p->fs = f;
#define FS_TRY(expr, what)                     \
  do {                                         \
    rc = cgh_cuda_check((expr), (what));       \
    if (rc != CGH_OK) goto fail;               \
  } while (0)
  if (!f->GZ) {
    f->No = No;
    f->Nh = Nh;
    f->Z = Z;
    f->mEZ = &p->eops->mEZ[0];
    f->mEZt = &p->eops->mEZt[0];
    f->gz_plane = (long long)Z * No * Nh;
    FS_TRY(cudaMalloc(&f->GZ, 4 * f->gz_plane * 2), "fields: GZ");
    if ((rc = make_plane_map(&f->mGZ, f->GZ, 4, (long long)Z * No, Nh)) != CGH_OK) goto fail;
    dim3 blk(8, 32);
    k_fe_build<0, false><<<dim3((Nh / 8 + 7) / 8, (Z * No + 31) / 32), blk, 0, st>>>(
        p->d_tab, p->tab_len, p->tab_off, p->s, No, Z * No, Nh, f->GZ, f->gz_plane);
    FS_TRY(cudaGetLastError(), "fields: operand build");
  }
  if (f->cap < n) {
    // the kernels of a previous call may still read the old planes
    FS_TRY(cudaStreamSynchronize(st), "fields: grow");
    field_free_data(f);
    const long long c = n;
    f->ht_plane = c * Nh * Nh;
    f->t_plane = c * Z * No * Nh;
    f->fp_plane = c * Z * No * No;
    f->yp_plane = (long long)Nh * c * Z * No;
    FS_TRY(cudaMalloc(&f->Ht, 4 * f->ht_plane * 2), "fields: Ht");
    FS_TRY(cudaMalloc(&f->T, 4 * f->t_plane * 2), "fields: T");
    FS_TRY(cudaMalloc(&f->Fp, 4 * f->fp_plane * 2), "fields: Fp");
    FS_TRY(cudaMalloc(&f->Yp, 4 * f->yp_plane * 2), "fields: Yp");
    FS_TRY(cudaMalloc(&f->F, (size_t)c * Z * No * No * sizeof(float2)), "fields: F");
    if ((rc = make_plane_map(&f->mHt, f->Ht, 4, c * Nh, Nh)) != CGH_OK) goto fail;
    if ((rc = make_plane_map(&f->mT, f->T, 4, c * Z * No, Nh)) != CGH_OK) goto fail;
    if ((rc = make_plane_map(&f->mFp, f->Fp, 4, c * Z * No, No)) != CGH_OK) goto fail;
    if ((rc = make_plane_map(&f->mYp, f->Yp, 4, Nh, c * Z * No)) != CGH_OK) goto fail;
    for (int b = 0; b < n; ++b)
      if ((rc = make_plane_view(&f->mYpb[b], f->Yp + (size_t)b * Z * No, Nh, (long long)Z * No, c * Z * No,
                                f->yp_plane)) != CGH_OK)
        goto fail;
    f->cap = n;
  }
#undef FS_TRY
  f->built = 1;
  return CGH_OK;
fail:
  field_destroy(p);
  return rc;
}

// R_{b,z} = E_z^H H_b conj(E_z) for n holograms (holo [n][Nh][Nh]) and every layer, into
// fields [n][Z][No][No].  One launch per GEMM stage over the (hologram, layer) units.
static int field_reconstruct_into(const cgh_plan* p, const float2* holo, int n, float2* fields, cudaStream_t st) {
  cgh_field_state* f = p->fs;
  const int No = f->No, Nh = f->Nh, Z = f->Z;
  for (int b = 0; b < n; ++b)
    k_split_transpose<<<dim3((Nh + 31) / 32, (Nh + 31) / 32), dim3(32, 8), 0, st>>>(
        holo + (size_t)b * Nh * Nh, Nh, Nh, f->Ht + (size_t)b * Nh * Nh, f->ht_plane, 1.0f);
  int rc = cgh_cuda_check(cudaGetLastError(), "reconstruct: transpose");
  if (rc != CGH_OK) return rc;
  TcGemmArgs a;
  memset(&a, 0, sizeof(a));
  a.mode = 3;
  a.n_layers = Z;
  a.status = p->d_status;
  a.scale = 1.0f;
  // R1: T_{b,z}[i][n] = sum_m conj(E_z[m][i]) H_b[m][n]; unit zz = b Z + z
  a.a_rows_per_z = No;
  a.a_zmod = Z;
  a.b_rows_per_z = Nh;
  a.b_zdiv = Z;
  a.out_rows_per_z = No;
  a.out_cols_per_z = 0;
  a.M = No;
  a.N = Nh;
  a.K = Nh;
  a.Y = f->T;
  a.y_plane = f->t_plane;
  a.ldy = Nh;
  a.y_rows = f->cap * Z * No;  // the store map's extent
  rc = cgh_cuda_check(launch_gemm<KIND_CC, EPI_Y, false>(f->mGZ, f->mHt, f->mT, a,
                                                         dim3((No + 127) / 128, (Nh + 127) / 128, n * Z), st),
                      "reconstruct: R1");
  if (rc != CGH_OK) return rc;
  // R2: R_{b,z}[i][j] = sum_n T_{b,z}[i][n] conj(E_z[n][j])
  a.a_zmod = 0;
  a.b_zdiv = 0;
  a.b_zmod = Z;
  a.b_rows_per_z = No;
  a.M = No;
  a.N = No;
  a.K = Nh;
  a.F = fields;
  a.ldf = No;
  a.h_vec4 = ((No & 1) == 0) && (((uintptr_t)fields & 15) == 0);
  return cgh_cuda_check(launch_gemm<KIND_CC, EPI_F, false>(f->mT, f->mGZ, f->mGZ, a,
                                                           dim3((No + 127) / 128, (No + 127) / 128, n * Z), st),
                        "reconstruct: R2");
}

// H_b (+)= sum_z E_z F_{b,z} E_z^T for n field stacks (fields [n][Z][No][No]) into holo
// [n][Nh][Nh]: the first stage over the (hologram, layer) units in one launch, the second per
// hologram (a split-K GEMM over its layers' stacked rows).
int field_propagate(const cgh_plan* p, const float2* fields, int n, float2* holo, int accumulate, cudaStream_t st) {
  int rc = field_ensure(p, st, n);
  if (rc != CGH_OK) return rc;
  cgh_field_state* f = p->fs;
  const int No = f->No, Nh = f->Nh, Z = f->Z;
  prof_mark(p, CGH_PROF_PROPAGATE, 0, st);
  k_split_rows<<<dim3((No / 8 + 7) / 8, (n * Z * No + 31) / 32), dim3(8, 32), 0, st>>>(
      fields, (long long)n * Z * No, No, f->Fp, f->fp_plane);
  rc = cgh_cuda_check(cudaGetLastError(), "propagate: split");
  if (rc != CGH_OK) return rc;
  TcGemmArgs a;
  memset(&a, 0, sizeof(a));
  a.mode = 3;
  a.n_layers = Z;
  a.status = p->d_status;
  a.scale = 1.0f;
  // P1: Y^T[n][(b Z + z) No + i] = sum_j E_z[n][j] F_{b,z}[i][j]
  a.a_rows_per_z = Nh;
  a.a_zmod = Z;
  a.b_rows_per_z = No;
  a.out_rows_per_z = 0;
  a.out_cols_per_z = No;
  a.M = Nh;
  a.N = No;
  a.K = No;
  a.Y = f->Yp;
  a.y_plane = f->yp_plane;
  a.ldy = f->cap * Z * No;
  a.y_rows = Nh;
  rc = cgh_cuda_check(launch_gemm<KIND_CC, EPI_Y, false>(*f->mEZt, f->mFp, f->mYp, a,
                                                         dim3((Nh + 127) / 128, (No + 127) / 128, n * Z), st),
                      "propagate: P1");
  if (rc != CGH_OK) return rc;
  // P2: H_b[m][n] += sum_kappa E[m][kappa] Y^T[n][b Z No + kappa], kappa = z No + i
  const int tm = (Nh + 127) / 128;
  int S = 1;
  if (!p->deterministic) {
    const int sms = tc_num_sms(), kst = Z * No / TC_BK;
    double best = 0;
    for (int q = 1; q <= 32 && q * 4 <= kst; ++q) {
      const double rounds = (double)q * tm * tm / sms, eff = rounds / ceil(rounds);
      if (q * tm * tm >= sms && eff >= 0.9) {
        S = q;
        break;
      }
      if (eff > best + 1e-9) best = eff, S = q;
    }
  }
  for (int bh = 0; bh < n; ++bh) {
    float2* H = holo + (size_t)bh * Nh * Nh;
    if (!accumulate) {
      rc = cgh_cuda_check(cudaMemsetAsync(H, 0, (size_t)Nh * Nh * sizeof(float2), st), "propagate: clear");
      if (rc != CGH_OK) return rc;
    }
    TcGemmArgs c;
    memset(&c, 0, sizeof(c));
    c.mode = 2;
    c.n_layers = Z;
    c.K = Z * No;
    c.M = Nh;
    c.N = Nh;
    c.scale = 1.0f;
    c.H = H;
    c.ldh = Nh;
    c.h_vec4 = ((Nh & 1) == 0) && (((uintptr_t)H & 15) == 0);
    c.status = p->d_status;
    rc = cgh_cuda_check(launch_gemm<KIND_CC, EPI_H, false>(*f->mEZ, f->mYpb[bh], f->mYpb[bh], c, dim3(tm, tm, S), st),
                        "propagate: P2");
    if (rc != CGH_OK) return rc;
  }
  prof_mark(p, CGH_PROF_PROPAGATE, 1, st);
  return CGH_OK;
}

int tc_reconstruct(const cgh_plan* p, const float2* holo, int n, float2* fields, const uint8_t* L, float* amp,
                   cudaStream_t st) {
  int rc = field_ensure(p, st, n);
  if (rc != CGH_OK) return rc;
  cgh_field_state* f = p->fs;
  float2* out = fields ? fields : f->F;
  prof_mark(p, CGH_PROF_RECON, 0, st);
  rc = field_reconstruct_into(p, holo, n, out, st);
  if (rc != CGH_OK) return rc;
  if (amp) {
    const int np = f->No * f->No;
    for (int b = 0; b < n; ++b)
      k_amplitude<<<(np + 255) / 256, 256, 0, st>>>(out + (size_t)b * f->Z * np, L, np, f->Z, amp + (size_t)b * np);
    rc = cgh_cuda_check(cudaGetLastError(), "reconstruct: amplitude");
  }
  prof_mark(p, CGH_PROF_RECON, 1, st);
  return rc;
}

int field_amplitude_backward(const cgh_plan* p, const float2* fields, int n, const uint8_t* L, const float* grad_amp,
                             float2* grad_fields, cudaStream_t st) {
  const int np = p->obj_h * p->obj_w, Z = p->n_layers;
  for (int b = 0; b < n; ++b)
    k_amplitude_backward<<<dim3((np + 255) / 256, Z), 256, 0, st>>>(
        fields + (size_t)b * Z * np, L, np, Z, grad_amp + (size_t)b * np, grad_fields + (size_t)b * Z * np);
  return cgh_cuda_check(cudaGetLastError(), "amplitude backward");
}

int field_adjoint(const cgh_plan* p, const float2* grad_holo, const int32_t* const* lists, const int32_t* d_counts,
                  const uint8_t* L, float* grad_obj, cudaStream_t st) {
  int rc = field_ensure(p, st);
  if (rc != CGH_OK) return rc;
  cgh_field_state* f = p->fs;
  TcFlags fl;
  rc = tc_build_flags(p, lists, d_counts, &fl, st);
  if (rc != CGH_OK) return rc;
  rc = field_reconstruct_into(p, grad_holo, 1, f->F, st);
  if (rc != CGH_OK) return rc;
  rc = cgh_cuda_check(cudaMemsetAsync(grad_obj, 0, (size_t)f->No * f->No * sizeof(float), st), "adjoint: clear");
  if (rc != CGH_OK) return rc;
  dim3 blk(32, 4), grid((f->No / 8 + 31) / 32, (f->No / 8 + 3) / 4, f->Z);
  k_adjoint_project<<<grid, blk, 0, st>>>(f->F, L, fl, f->No, f->No, f->Z, grad_obj);
  return cgh_cuda_check(cudaGetLastError(), "adjoint: projection");
}

int field_forward(const cgh_plan* p, const float* obj, const int32_t* const* lists, const int32_t* d_counts,
                  const uint8_t* L, float2* holo, int accumulate, cudaStream_t st) {
  int rc = field_ensure(p, st);
  if (rc != CGH_OK) return rc;
  cgh_field_state* f = p->fs;
  TcFlags fl;
  rc = tc_build_flags(p, lists, d_counts, &fl, st);
  if (rc != CGH_OK) return rc;
  dim3 blk(32, 4), grid((f->No / 8 + 31) / 32, (f->No / 8 + 3) / 4, f->Z);
  k_forward_project<<<grid, blk, 0, st>>>(obj, L, fl, f->No, f->No, f->Z, f->F);
  rc = cgh_cuda_check(cudaGetLastError(), "progressive apply: projection");
  if (rc != CGH_OK) return rc;
  return field_propagate(p, f->F, 1, holo, accumulate, st);
}

extern "C" int cgh_phase_to_field(const float* phase, float* field, long long n, void* stream) {
  if (!phase || !field || n < 0) return cgh_fail(CGH_ERR_ARG, "cgh_phase_to_field: bad argument");
  if (n == 0) return CGH_OK;
  k_phase_to_field<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(phase, (float2*)field, n);
  return cgh_cuda_check(cudaGetLastError(), "cgh_phase_to_field");
}

extern "C" int cgh_phase_grad(const float* field, const float* grad_field, float* grad_phase, long long n,
                              void* stream) {
  if (!field || !grad_field || !grad_phase || n < 0) return cgh_fail(CGH_ERR_ARG, "cgh_phase_grad: bad argument");
  if (n == 0) return CGH_OK;
  k_phase_grad<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>((const float2*)field,
                                                                             (const float2*)grad_field, grad_phase, n);
  return cgh_cuda_check(cudaGetLastError(), "cgh_phase_grad");
}
