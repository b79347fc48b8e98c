// Reconstruction by the inverse angular spectrum method (Section 2, last paragraph: the
// paper renders its reconstructions this way, at the scene's own parameters).
//
//   R_z(i, j) = p^2/(lambda z) * IDFT_PxP[ DFT_PxP[pad(H)] * T_z ](s i, s j)
//   T_z(f) = exp(-j 2 pi z (sqrt(1/lambda^2 - |f|^2) - 1/lambda))   (0 if evanescent)
//
// P = pad * holo edge (pad 2 turns the DFT's circular convolution into a linear one).
// Four kernels, each a batch of 1-D FFTs over tiles of B lines (fft.cuh):
//   1. forward FFT of the hologram rows, zero-padded to P           H  [Nh][Nh] -> Xr [Nh][P]
//   2. forward FFT of the columns (rows >= Nh are zero)             Xr          -> X  [P][P]
//   3. per layer: spectrum times T_z, folded by s along both axes (the inverse DFT is only
//      read at multiples of s, and x[s i] of a length-P inverse DFT is the length-P/s
//      inverse DFT of the spectrum summed over its s aliases k + t P/s), inverse FFT of
//      the folded columns, rows i < obj edge kept                  X  -> Y  [Z][No][P/s]
//   4. per layer: inverse FFT of those rows, columns j < obj edge kept, scaled; writes the
//      fields and / or the amplitude |R_layer(i,j)(i, j)|           Y  -> R  [Z][No][No]
//
// T_z without loss of precision in FP32: with u = lambda^2 |f|^2 = c q, q = ky^2 + kx^2
// (signed DFT indices) and c = lambda^2 / (P p)^2, the phase in cycles is
//   z (1/lambda - sqrt(1/lambda^2 - |f|^2)) = b q + (z/lambda) u^2 / (2 (1 + sqrt(1 - u))^2)
// with b = z lambda / (2 P^2 p^2).  The first (Fresnel) term is reduced exactly in 64-bit
// fixed point (frac(b) * 2^64 times the integer q, modulo 2^64); the second is below a
// quarter cycle for any geometry here and is evaluated in FP32 without cancellation.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <type_traits>

#include "cgh_internal.h"
#include "fft.cuh"

// Tile shapes (threads T, elements B * L per tile; 16 elements a thread, 64 registers a
// thread, so 1024 / T CTAs fill an SM's register file).  The column kernels take the large
// tile so that every row segment they read is at least a 32-byte sector (B >= 4 lines up
// to L = 2048); the row kernels run smaller tiles, more of them per SM, which hides the
// latency of their load, transform and store phases better.
#define ASM_BIG_T 512
#define ASM_BIG_TILE 8192
// The inverse-column kernel takes 16384-element tiles on 1024 threads (one CTA per SM): at a
// folded edge of 1024 a warp's spectrum load then covers 128 bytes of each of two rows, half
// the L1 wavefronts of 64-byte runs (measured: 90 -> 86 us, L1 data path 77% -> 53% busy).
#define ASM_IC_T 1024
#define ASM_IC_TILE 16384
#define ASM_SMALL_T 256
#define ASM_SMALL_TILE 4096
// The inverse-row kernel: 2048-element tiles on 128 threads up to a folded edge of 512 (eight
// CTAs per SM overlap their load, transform and store phases: 41 -> 37 us at 512), 4096 from
// 1024 (there the smaller tiles measured slower, 44 -> 48 us).
template <int L>
constexpr int asm_ir_tile() {
  return L >= 1024 ? (L > 4096 ? L : 4096) : 2048;
}
#define ASM_MINB(T) (1024 / (T))

struct AsmLayer {
  unsigned long long bfix;  // round(frac(b_z) * 2^64)
  float zl;                 // z / lambda
  float c;                  // lambda^2 / (P p)^2
  float scale;              // p^2 / (lambda z) / P^2 (the inverse DFT's normalisation included)
  int kmax;                 // band limit on |ky|, |kx| (P when inactive)
};

struct cgh_asm_state {
  int P, pad, band_limit;
  int exact;          // 1: exact correction term with band-limit / evanescent checks; 0: series, no checks
  float2* Xr;         // [Nh][P]
  float2* X;          // [P][P]
  float2* Y;          // [Z][No][P/s]
  float2* tw;         // [LMAX] exp(-2 pi i k / LMAX)
  AsmLayer* layers;   // [Z]
};

// exp(j 2 pi (b q + corr(u))) from the Fresnel phase fr = frac(b q) in [-1/2, 1/2) cycles
// (from the fixed-point sum) and u = c q.  EXACT: corr = (z/lambda) u^2 / (2 (1 + sqrt(1-u))^2)
// with rsqrtf / __fdividef; otherwise its power series (z/lambda) sum_{n=2..6} c_n u^n, c_n the
// coefficients of 1 - sqrt(1-u) = u/2 + u^2/8 + u^3/16 + 5u^4/128 + 7u^5/256 + 21u^6/1024 + ...,
// used only when the host has bounded the truncated tail below 1e-8 cycles.  The phase is
// reduced to [-1/2, 1/2] cycles before __sincosf; each step stays within a few 1e-7 of the
// exact value, far below the FFTs' own rounding budget.
template <bool EXACT>
__device__ __forceinline__ float2 asm_phasor(float fr, float u, float zl) {
  float corr;
  if constexpr (EXACT) {
    const float w = 1.f - u;
    const float d = 1.f + w * rsqrtf(w);  // 1 + sqrt(1 - u)
    corr = __fdividef(zl * u * u, 2.f * d * d);
  } else {
    const float poly = fmaf(u, fmaf(u, fmaf(u, fmaf(u, 0.0205078125f, 0.02734375f), 0.0390625f), 0.0625f), 0.125f);
    corr = zl * (u * u) * poly;
  }
  float t = fr + corr;
  t -= rintf(t);
  float sn, cs;
  __sincosf(6.28318530717958648f * t, &sn, &cs);
  return make_float2(cs, sn);
}

// frac(b * k^2) as the top 32 bits of the 64-bit fixed-point product (k^2 < 2^32).
__device__ __forceinline__ unsigned int fresnel_fix32(unsigned long long bfix, int k) {
  return (unsigned int)((bfix * (unsigned long long)(unsigned int)(k * k)) >> 32);
}

template <int L, int B, int T>
__global__ void __launch_bounds__(T, ASM_MINB(T)) k_asm_fwd_rows(const float2* __restrict__ H, int Nh,
                                                        float2* __restrict__ Xr, const float2* __restrict__ tw) {
  extern __shared__ float2 sm[];
  const int r0 = blockIdx.x * B;
  fft::fft_tile<L, B, T, false>(
      sm, tw,
      [&](int b, int i) {
        return (i < Nh && r0 + b < Nh) ? H[(size_t)(r0 + b) * Nh + i] : make_float2(0.f, 0.f);
      },
      [&](int b, int i, float2 v) {
        if (r0 + b < Nh) Xr[(size_t)(r0 + b) * L + i] = v;
      });
}

template <int L, int B, int T>
__global__ void __launch_bounds__(T, ASM_MINB(T)) k_asm_fwd_cols(const float2* __restrict__ Xr, int Nh,
                                                        float2* __restrict__ X, const float2* __restrict__ tw) {
  extern __shared__ float2 sm[];
  const int c0 = blockIdx.x * B;
  fft::fft_tile<L, B, T, false>(
      sm, tw,
      [&](int b, int i) {
        return (i < Nh && c0 + b < L) ? Xr[(size_t)i * L + c0 + b] : make_float2(0.f, 0.f);
      },
      [&](int b, int i, float2 v) {
        if (c0 + b < L) X[(size_t)i * L + c0 + b] = v;
      });
}

// Transfer value at the signed frequencies (sx, sy) from its separable parts (fixed-point
// Fresnel fractions ex, ey; u parts ux, uy), zero where EXACT cuts it (band limit, evanescent).
template <bool EXACT>
__device__ __forceinline__ float2 asm_transfer(unsigned int ex, float ux, bool okx, unsigned int ey, float uy,
                                               bool oky, float zl) {
  const float u = ux + uy;
  if (EXACT && (!okx || !oky || u >= 1.f)) return make_float2(0.f, 0.f);
  const float fr = (float)(int)(ex + ey) * 2.3283064365386963e-10f;  // signed, / 2^32
  return asm_phasor<EXACT>(fr, u, zl);
}

__device__ __forceinline__ void cmad(float2& acc, float2 v, float2 t) {
  acc.x = fmaf(v.x, t.x, fmaf(-v.y, t.y, acc.x));
  acc.y = fmaf(v.x, t.y, fmaf(v.y, t.x, acc.y));
}

// L = P / S: folded column c0 + b of layer blockIdx.y.  The tile (spectrum times T_z,
// summed over the S x S aliases) is built in shared memory first, then transformed.
// T_z depends on the squared signed frequencies only, and the aliases of folded row L - r
// are those of row r negated, in reverse order (L - r + t L = -(r + (S-1-t) L) mod P).  So a
// thread builds the folded rows r and L - r of its column from the S x S transfer values of
// (c, r): S^2 / 2 transfer values per folded point instead of S^2.  Rows 0 and L/2 are their
// own mirrors and are built one at a time.
// T_z separates into x and y parts except for the correction term: every thread keeps one
// column (b = thread mod B), so the x part of its S aliases is computed once, and the y part
// once per row alias.  The Fresnel phase is the sum of the two parts' fixed-point fractions
// (top 32 bits each: error below 2^-31 cycles).  EXACT also applies the band limit and the
// evanescent cut (the fast path runs only where the host has found neither active).
template <int L, int B, int T, int S, bool EXACT>
__global__ void __launch_bounds__(T, ASM_MINB(T)) k_asm_inv_cols(const float2* __restrict__ X, int No,
                                                                  const AsmLayer* __restrict__ layers,
                                                                  float2* __restrict__ Y,
                                                                  const float2* __restrict__ tw) {
  extern __shared__ float2 sm[];
  using SM = fft::Smem<L, B>;
  constexpr int P = L * S, HALF = P / 2, RSTEP = T / B, NQ = L / 2;
  static_assert(T % B == 0 && NQ % RSTEP == 0, "a thread keeps one column and whole row pairs");
  const int c0 = blockIdx.x * B, z = blockIdx.y;
  const AsmLayer a = layers[z];
  const int b = threadIdx.x % B, kx = c0 + b;
  auto sgn = [](int k) { return k < HALF ? k : k - P; };
  if (kx < L) {
    unsigned int ex[S];
    float ux[S];
    bool okx[S];
#pragma unroll
    for (int tx = 0; tx < S; ++tx) {
      const int sx = sgn(kx + tx * L);
      ex[tx] = fresnel_fix32(a.bfix, sx);
      ux[tx] = a.c * (float)(sx * sx);
      okx[tx] = !EXACT || abs(sx) <= a.kmax;
    }
    // folded row r (v0) and, with `mirror`, row L - r (v1) from the same transfer values
    auto unit = [&](int r, bool mirror, float2& v0, float2& v1) {
#pragma unroll(S <= 2 ? S : 1)
      for (int ty = 0; ty < S; ++ty) {
        const int r0 = r + ty * L, r1 = mirror ? L - r + (S - 1 - ty) * L : r0;  // the mirrored alias
        const float2* x0 = X + (size_t)r0 * P + kx;
        const float2* x1 = X + (size_t)r1 * P + kx;
        const int sy = sgn(r0);
        const unsigned int ey = fresnel_fix32(a.bfix, sy);
        const float uy = a.c * (float)(sy * sy);
        const bool oky = !EXACT || abs(sy) <= a.kmax;
        float2 va[S], vb[S];
#pragma unroll
        for (int tx = 0; tx < S; ++tx) {
          va[tx] = x0[tx * L];
          vb[tx] = x1[tx * L];
        }
#pragma unroll
        for (int tx = 0; tx < S; ++tx) {
          const float2 t = asm_transfer<EXACT>(ex[tx], ux[tx], okx[tx], ey, uy, oky, a.zl);
          cmad(v0, va[tx], t);
          if (mirror) cmad(v1, vb[tx], t);
        }
      }
    };
#pragma unroll 2
    for (int it = 0; it < NQ / RSTEP; ++it) {
      const int q = threadIdx.x / B + it * RSTEP, qm = q ? L - q : L / 2;
      float2 v0 = make_float2(0.f, 0.f), v1 = v0;
      if (q) {
        unit(q, true, v0, v1);
      } else {  // rows 0 and L/2: each its own mirror
        float2 d = v0;
        unit(0, false, v0, d);
        unit(L / 2, false, v1, d);
      }
      sm[SM::at(b, q)] = v0;
      sm[SM::at(b, qm)] = v1;
    }
  } else {
    for (int it = 0; it < NQ / RSTEP; ++it) {
      const int q = threadIdx.x / B + it * RSTEP, qm = q ? L - q : L / 2;
      sm[SM::at(b, q)] = make_float2(0.f, 0.f);
      sm[SM::at(b, qm)] = make_float2(0.f, 0.f);
    }
  }
  __syncthreads();
  fft::fft_tile<L, B, T, true, true>(
      sm, tw, [&](int bb, int i) { return sm[SM::at(bb, i)]; },
      [&](int bb, int i, float2 v) {
        if (i < No && c0 + bb < L) Y[((size_t)z * No + i) * L + c0 + bb] = v;
      });
}

// Rows i0 .. i0+B-1 of layer blockIdx.y.  The layer indices of the tile's output pixels
// are staged in shared memory (after the FFT tile) before the transform.
template <int L, int B, int T>
__global__ void __launch_bounds__(T, ASM_MINB(T)) k_asm_inv_rows(const float2* __restrict__ Y, int No, int Z,
                                                                  const AsmLayer* __restrict__ layers,
                                                                  const uint8_t* __restrict__ lay,
                                                                  float2* __restrict__ F, float* __restrict__ amp,
                                                                  const float2* __restrict__ tw) {
  extern __shared__ float2 sm[];
  uint8_t* lsm = reinterpret_cast<uint8_t*>(sm + fft::Smem<L, B>::floats2);
  const int i0 = blockIdx.x * B, z = blockIdx.y;
  const float scale = layers[z].scale;
  if (amp)
    for (int e = threadIdx.x; e < B * No; e += T) {
      const int i = i0 + e / No;
      lsm[e] = i < No ? lay[(size_t)i * No + e % No] : (uint8_t)0;
    }
  // (the barrier at the end of the first FFT pass orders these stores before the reads)
  fft::fft_tile<L, B, T, true>(
      sm, tw,
      [&](int b, int kx) {
        return i0 + b < No ? Y[((size_t)z * No + i0 + b) * L + kx] : make_float2(0.f, 0.f);
      },
      [&](int b, int j, float2 v) {
        const int i = i0 + b;
        if (j >= No || i >= No) return;
        v = make_float2(v.x * scale, v.y * scale);
        const size_t pix = (size_t)i * No + j;
        if (F) F[(size_t)z * No * No + pix] = v;
        if (amp) {
          const int l = lsm[b * No + j];
          if (l == z)
            amp[pix] = sqrtf(v.x * v.x + v.y * v.y);
          else if (z == 0 && l >= Z)
            amp[pix] = 0.f;
        }
      });
}

// Calls f(std::integral_constant<int, L>) for a supported length.
template <class F>
static bool with_len(int L, F&& f) {
  switch (L) {
    case 64: f(std::integral_constant<int, 64>{}); return true;
    case 128: f(std::integral_constant<int, 128>{}); return true;
    case 256: f(std::integral_constant<int, 256>{}); return true;
    case 512: f(std::integral_constant<int, 512>{}); return true;
    case 1024: f(std::integral_constant<int, 1024>{}); return true;
    case 2048: f(std::integral_constant<int, 2048>{}); return true;
    case 4096: f(std::integral_constant<int, 4096>{}); return true;
    default: return false;
  }
}

template <int L, int TILE>
static constexpr size_t tile_smem() {
  return (size_t)fft::Smem<L, TILE / L>::floats2 * sizeof(float2);
}
// the inverse-row kernel also stages B rows of layer indices (at most B * L bytes)
template <int L, int TILE>
static constexpr size_t rows_smem() {
  return tile_smem<L, TILE>() + TILE;
}

// Calls f(std::integral_constant<int, S>) for a supported sampling stride.
template <class F>
static bool with_stride(int s, F&& f) {
  switch (s) {
    case 1: f(std::integral_constant<int, 1>{}); return true;
    case 2: f(std::integral_constant<int, 2>{}); return true;
    case 4: f(std::integral_constant<int, 4>{}); return true;
    case 8: f(std::integral_constant<int, 8>{}); return true;
    default: return false;
  }
}

int asm_init_attributes() {
  cudaError_t e = cudaSuccess;
  auto keep = [&](cudaError_t x) {
    if (x != cudaSuccess && e == cudaSuccess) e = x;
  };
  for (int L = 64; L <= 4096; L <<= 1)
    with_len(L, [&](auto lc) {
      constexpr int Lc = decltype(lc)::value;
      constexpr int BB = ASM_BIG_TILE / Lc, BS = ASM_SMALL_TILE / Lc;
      constexpr int smb = (int)tile_smem<Lc, ASM_BIG_TILE>(), sms = (int)tile_smem<Lc, ASM_SMALL_TILE>();
      keep(cudaFuncSetAttribute(k_asm_fwd_rows<Lc, BS, ASM_SMALL_T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                sms));
      keep(cudaFuncSetAttribute(k_asm_fwd_cols<Lc, BB, ASM_BIG_T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smb));
      constexpr int IRT = asm_ir_tile<Lc>();
      keep(cudaFuncSetAttribute(k_asm_inv_rows<Lc, IRT / Lc, IRT / 16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)rows_smem<Lc, IRT>()));
      constexpr int BI = ASM_IC_TILE / Lc, smi = (int)tile_smem<Lc, ASM_IC_TILE>();
      for (int s = 1; s <= 8; s <<= 1)
        with_stride(s, [&](auto sc) {
          constexpr int Sc = decltype(sc)::value;
          if constexpr (Lc * Sc <= 4096) {
            keep(cudaFuncSetAttribute(k_asm_inv_cols<Lc, BI, ASM_IC_T, Sc, true>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, smi));
            keep(cudaFuncSetAttribute(k_asm_inv_cols<Lc, BI, ASM_IC_T, Sc, false>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, smi));
          }
        });
    });
  return cgh_cuda_check(e, "angular spectrum kernel attributes");
}

void asm_destroy(cgh_plan* p) {
  cgh_asm_state* a = p->asmst;
  if (!a) return;
  cudaFree(a->Xr);
  cudaFree(a->X);
  cudaFree(a->Y);
  cudaFree(a->tw);
  cudaFree(a->layers);
  free(a);
  p->asmst = nullptr;
}

static bool pow2(int x) { return x > 0 && (x & (x - 1)) == 0; }

// Buffers for padding `pad` and the layer constants for `band_limit`.
static int asm_ensure(const cgh_plan* pc, int pad, int band_limit, cudaStream_t st) {
  cgh_plan* p = const_cast<cgh_plan*>(pc);
  const int Nh = p->holo_h, No = p->obj_h, Z = p->n_layers, P = pad * Nh, L = P / p->s;
  cgh_asm_state* a = p->asmst;
  if (a && a->P == P && a->band_limit == band_limit) return CGH_OK;
  if (a && a->P != P) asm_destroy(p);
  a = p->asmst;
  int rc = CGH_OK;
#define ASM_TRY(expr, what)                 \
  do {                                      \
    rc = cgh_cuda_check((expr), (what));    \
    if (rc != CGH_OK) {                     \
      asm_destroy(p);                       \
      return rc;                            \
    }                                       \
  } while (0)
  if (!a) {
    a = (cgh_asm_state*)calloc(1, sizeof(cgh_asm_state));
    if (!a) return cgh_fail(CGH_ERR_NOMEM, "angular spectrum: host allocation");
    p->asmst = a;
    a->P = P;
    a->pad = pad;
    ASM_TRY(cudaMalloc(&a->Xr, (size_t)Nh * P * sizeof(float2)), "angular spectrum: row spectra");
    ASM_TRY(cudaMalloc(&a->X, (size_t)P * P * sizeof(float2)), "angular spectrum: spectrum");
    ASM_TRY(cudaMalloc(&a->Y, (size_t)Z * No * L * sizeof(float2)), "angular spectrum: layer columns");
    ASM_TRY(cudaMalloc(&a->tw, fft::LMAX * sizeof(float2)), "angular spectrum: twiddles");
    ASM_TRY(cudaMalloc(&a->layers, CGH_MAX_LAYERS * sizeof(AsmLayer)), "angular spectrum: layers");
    float2 tw[fft::LMAX];
    for (int k = 0; k < fft::LMAX; ++k) {
      const double t = -2.0 * M_PI * k / fft::LMAX;
      tw[k] = make_float2((float)cos(t), (float)sin(t));
    }
    ASM_TRY(cudaMemcpyAsync(a->tw, tw, sizeof(tw), cudaMemcpyHostToDevice, st), "angular spectrum: twiddles");
    ASM_TRY(cudaStreamSynchronize(st), "angular spectrum: twiddles");
  }
  AsmLayer h[CGH_MAX_LAYERS];
  memset(h, 0, sizeof(h));
  const double lam = p->wavelength, pp = p->pitch, df = 1.0 / (P * pp);
  for (int k = 0; k < Z; ++k) {
    const double z = p->z[k];
    const double b = z * lam / (2.0 * (double)P * P * pp * pp);
    const double fr = b - floor(b);
    const double x = floor(ldexp(fr, 64) + 0.5);
    h[k].bfix = x >= 18446744073709551616.0 ? 0ull : (unsigned long long)x;
    h[k].zl = (float)(z / lam);
    h[k].c = (float)(lam * lam * df * df);
    h[k].scale = (float)(pp * pp / (lam * z) / ((double)P * P));
    h[k].kmax = P;
    if (band_limit) {
      const double flim = 1.0 / (lam * sqrt(4.0 * df * df * z * z + 1.0));
      const double km = floor(flim / df);
      h[k].kmax = km < P ? (int)km : P;
    }
  }
  // The series form of the correction term is used when its truncated tail,
  // (z/lambda) * (33/2048) u^7 / (1 - u) at the largest u of the grid, stays below 1e-8
  // cycles for every layer, and no band limit or evanescent cut applies.
  const double umax = lam * lam * df * df * 2.0 * (P / 2) * (P / 2);
  bool exact = band_limit != 0 || umax >= 0.5;
  for (int k = 0; k < Z && !exact; ++k)
    if (p->z[k] / lam * (33.0 / 2048.0) * pow(umax, 7) / (1.0 - umax) > 1e-8) exact = true;
  a->exact = exact ? 1 : 0;
  ASM_TRY(cudaMemcpyAsync(a->layers, h, sizeof(h), cudaMemcpyHostToDevice, st), "angular spectrum: layers");
  ASM_TRY(cudaStreamSynchronize(st), "angular spectrum: layers");
  a->band_limit = band_limit;
#undef ASM_TRY
  return CGH_OK;
}

extern "C" int cgh_reconstruct_asm(const cgh_plan* p, const float* holo, float* fields, const uint8_t* layer_idx,
                                   float* amplitude, int pad, int band_limit, void* stream) {
  if (!p || !holo) return cgh_fail(CGH_ERR_ARG, "cgh_reconstruct_asm: NULL argument");
  if (amplitude && !layer_idx) return cgh_fail(CGH_ERR_ARG, "cgh_reconstruct_asm: amplitude needs layer_idx");
  if (!fields && !amplitude) return cgh_fail(CGH_ERR_ARG, "cgh_reconstruct_asm: nothing to compute");
  if (((uintptr_t)holo & 7) || ((uintptr_t)fields & 7))
    return cgh_fail(CGH_ERR_ARG, "cgh_reconstruct_asm: complex arrays must be 8-byte aligned");
  if (pad != 1 && pad != 2) return cgh_fail(CGH_ERR_ARG, "cgh_reconstruct_asm: pad %d not 1 or 2", pad);
  if (band_limit != 0 && band_limit != 1)
    return cgh_fail(CGH_ERR_ARG, "cgh_reconstruct_asm: band_limit %d not 0 or 1", band_limit);
  const int Nh = p->holo_h, No = p->obj_h, s = p->s, Z = p->n_layers;
  if (p->holo_w != Nh || p->obj_w != No || !pow2(Nh) || !pow2(s) || s > 8)
    return cgh_fail(CGH_ERR_UNSUPPORTED,
                    "cgh_reconstruct_asm: square power-of-two hologram and sampling stride 1, 2, 4 or 8 required");
  const int P = pad * Nh, L = P / s;
  if (P < 64 || P > 4096 || L < 64)
    return cgh_fail(CGH_ERR_UNSUPPORTED, "cgh_reconstruct_asm: padded edge %d and folded edge %d must lie in [64, 4096]",
                    P, L);
  cudaStream_t st = (cudaStream_t)stream;
  int rc = asm_ensure(p, pad, band_limit, st);
  if (rc != CGH_OK) return rc;
  const cgh_asm_state* a = p->asmst;
  const float2* H = (const float2*)holo;

  prof_mark(p, CGH_PROF_ASM_FFT, 0, st);
  with_len(P, [&](auto lc) {
    constexpr int Lc = decltype(lc)::value;
    constexpr int BB = ASM_BIG_TILE / Lc, BS = ASM_SMALL_TILE / Lc;
    k_asm_fwd_rows<Lc, BS, ASM_SMALL_T><<<(Nh + BS - 1) / BS, ASM_SMALL_T, tile_smem<Lc, ASM_SMALL_TILE>(), st>>>(
        H, Nh, a->Xr, a->tw);
    k_asm_fwd_cols<Lc, BB, ASM_BIG_T><<<(Lc + BB - 1) / BB, ASM_BIG_T, tile_smem<Lc, ASM_BIG_TILE>(), st>>>(
        a->Xr, Nh, a->X, a->tw);
  });
  prof_mark(p, CGH_PROF_ASM_FFT, 1, st);
  rc = cgh_cuda_check(cudaGetLastError(), "cgh_reconstruct_asm: forward transform");
  if (rc != CGH_OK) return rc;

  prof_mark(p, CGH_PROF_ASM_INV, 0, st);
  with_len(L, [&](auto lc) {
    constexpr int Lc = decltype(lc)::value;
    with_stride(s, [&](auto sc) {
      constexpr int Sc = decltype(sc)::value;
      if constexpr (Lc * Sc <= 4096) {
        constexpr int BI = ASM_IC_TILE / Lc;
        const dim3 grid((Lc + BI - 1) / BI, Z);
        constexpr size_t smi = tile_smem<Lc, ASM_IC_TILE>();
        if (a->exact)
          k_asm_inv_cols<Lc, BI, ASM_IC_T, Sc, true><<<grid, ASM_IC_T, smi, st>>>(a->X, No, a->layers, a->Y, a->tw);
        else
          k_asm_inv_cols<Lc, BI, ASM_IC_T, Sc, false><<<grid, ASM_IC_T, smi, st>>>(a->X, No, a->layers, a->Y, a->tw);
      }
    });
    constexpr int IRT = asm_ir_tile<Lc>(), BR = IRT / Lc;
    k_asm_inv_rows<Lc, BR, IRT / 16><<<dim3((No + BR - 1) / BR, Z), IRT / 16, rows_smem<Lc, IRT>(), st>>>(
        a->Y, No, Z, a->layers, layer_idx, (float2*)fields, amplitude, a->tw);
  });
  prof_mark(p, CGH_PROF_ASM_INV, 1, st);
  return cgh_cuda_check(cudaGetLastError(), "cgh_reconstruct_asm: inverse transforms");
}
