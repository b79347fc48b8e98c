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

#define ASM_T 256       // threads per CTA
#define ASM_TILE 8192   // elements per tile: B lines of length L with B * L = ASM_TILE

struct AsmLayer {
  unsigned long long bfix;  // round(frac(b_z) * 2^64)
  float zl;                 // z / lambda
  float c;                  // lambda^2 / (P p)^2
  float scale;              // p^2 / (lambda z) / P^2 (the inverse DFT's normalisation included)
  int kmax;                 // band limit on |ky|, |kx| (P when inactive)
};

struct cgh_asm_state {
  int P, pad, band_limit;
  float2* Xr;         // [Nh][P]
  float2* X;          // [P][P]
  float2* Y;          // [Z][No][P/s]
  float2* tw;         // [LMAX] exp(-2 pi i k / LMAX)
  AsmLayer* layers;   // [Z]
};

__device__ __forceinline__ float2 asm_transfer(const AsmLayer& a, int ky, int kx, int P) {
  const int sy = ky < (P >> 1) ? ky : ky - P;
  const int sx = kx < (P >> 1) ? kx : kx - P;
  if (abs(sy) > a.kmax || abs(sx) > a.kmax) return make_float2(0.f, 0.f);
  const unsigned int q = (unsigned int)(sy * sy + sx * sx);
  const float u = a.c * (float)q;
  if (u >= 1.f) return make_float2(0.f, 0.f);  // evanescent
  const unsigned long long ph = a.bfix * (unsigned long long)q;  // frac(b q) in units of 2^-64
  const float fres = (float)(unsigned int)(ph >> 40) * 5.9604644775390625e-8f;  // top 24 bits / 2^24
  const float d = 1.f + sqrtf(1.f - u);
  const float corr = a.zl * u * u / (2.f * d * d);
  float sn, cs;
  sincospif(2.f * (fres + corr), &sn, &cs);
  return make_float2(cs, sn);
}

template <int L, int B>
__global__ void __launch_bounds__(ASM_T) k_asm_fwd_rows(const float2* __restrict__ H, int Nh,
                                                        float2* __restrict__ Xr, const float2* __restrict__ tw) {
  extern __shared__ float2 sm[];
  const int r0 = blockIdx.x * B;
  fft::fft_tile<L, B, ASM_T, false>(
      sm, tw,
      [&](int b, int i) {
        return (i < Nh && r0 + b < Nh) ? H[(size_t)(r0 + b) * Nh + i] : make_float2(0.f, 0.f);
      },
      [&](int b, int i, float2 v) {
        if (r0 + b < Nh) Xr[(size_t)(r0 + b) * L + i] = v;
      });
}

template <int L, int B>
__global__ void __launch_bounds__(ASM_T) k_asm_fwd_cols(const float2* __restrict__ Xr, int Nh,
                                                        float2* __restrict__ X, const float2* __restrict__ tw) {
  extern __shared__ float2 sm[];
  const int c0 = blockIdx.x * B;
  fft::fft_tile<L, B, ASM_T, false>(
      sm, tw,
      [&](int b, int i) {
        return (i < Nh && c0 + b < L) ? Xr[(size_t)i * L + c0 + b] : make_float2(0.f, 0.f);
      },
      [&](int b, int i, float2 v) {
        if (c0 + b < L) X[(size_t)i * L + c0 + b] = v;
      });
}

// L = P / s: folded column c0 + b of layer blockIdx.y.
template <int L, int B>
__global__ void __launch_bounds__(ASM_T) k_asm_inv_cols(const float2* __restrict__ X, int P, int s, int No,
                                                        const AsmLayer* __restrict__ layers,
                                                        float2* __restrict__ Y, const float2* __restrict__ tw) {
  extern __shared__ float2 sm[];
  const int c0 = blockIdx.x * B, z = blockIdx.y;
  const AsmLayer a = layers[z];
  fft::fft_tile<L, B, ASM_T, true>(
      sm, tw,
      [&](int b, int ky) {
        float2 acc = make_float2(0.f, 0.f);
        if (c0 + b < L) {
          for (int ty = 0; ty < s; ++ty)
            for (int tx = 0; tx < s; ++tx) {
              const int kyf = ky + ty * L, kxf = c0 + b + tx * L;
              const float2 v = fft::cmul(X[(size_t)kyf * P + kxf], asm_transfer(a, kyf, kxf, P));
              acc = fft::cadd(acc, v);
            }
        }
        return acc;
      },
      [&](int b, int i, float2 v) {
        if (i < No && c0 + b < L) Y[((size_t)z * No + i) * L + c0 + b] = v;
      });
}

template <int L, int B>
__global__ void __launch_bounds__(ASM_T) k_asm_inv_rows(const float2* __restrict__ Y, int No, int Z,
                                                        const AsmLayer* __restrict__ layers,
                                                        const uint8_t* __restrict__ lay, float2* __restrict__ F,
                                                        float* __restrict__ amp, const float2* __restrict__ tw) {
  extern __shared__ float2 sm[];
  const int i0 = blockIdx.x * B, z = blockIdx.y;
  const float scale = layers[z].scale;
  fft::fft_tile<L, B, ASM_T, true>(
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
          const int l = lay[pix];
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

template <int L>
static constexpr size_t tile_smem() {
  return (size_t)fft::Smem<L, ASM_TILE / L>::floats2 * sizeof(float2);
}

int asm_init_attributes() {
  cudaError_t e = cudaSuccess;
  for (int L = 64; L <= 4096; L <<= 1)
    with_len(L, [&](auto lc) {
      constexpr int Lc = decltype(lc)::value, B = ASM_TILE / Lc;
      const int sm = (int)tile_smem<Lc>();
      cudaError_t r[4] = {
          cudaFuncSetAttribute(k_asm_fwd_rows<Lc, B>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm),
          cudaFuncSetAttribute(k_asm_fwd_cols<Lc, B>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm),
          cudaFuncSetAttribute(k_asm_inv_cols<Lc, B>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm),
          cudaFuncSetAttribute(k_asm_inv_rows<Lc, B>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm)};
      for (cudaError_t x : r)
        if (x != cudaSuccess && e == cudaSuccess) e = x;
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
  if (p->holo_w != Nh || p->obj_w != No || !pow2(Nh) || !pow2(s))
    return cgh_fail(CGH_ERR_UNSUPPORTED,
                    "cgh_reconstruct_asm: square power-of-two hologram and power-of-two sampling stride required");
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
    constexpr int Lc = decltype(lc)::value, B = ASM_TILE / Lc;
    k_asm_fwd_rows<Lc, B><<<(Nh + B - 1) / B, ASM_T, tile_smem<Lc>(), st>>>(H, Nh, a->Xr, a->tw);
    k_asm_fwd_cols<Lc, B><<<(Lc + B - 1) / B, ASM_T, tile_smem<Lc>(), st>>>(a->Xr, Nh, a->X, a->tw);
  });
  prof_mark(p, CGH_PROF_ASM_FFT, 1, st);
  rc = cgh_cuda_check(cudaGetLastError(), "cgh_reconstruct_asm: forward transform");
  if (rc != CGH_OK) return rc;

  prof_mark(p, CGH_PROF_ASM_INV, 0, st);
  with_len(L, [&](auto lc) {
    constexpr int Lc = decltype(lc)::value, B = ASM_TILE / Lc;
    k_asm_inv_cols<Lc, B><<<dim3((Lc + B - 1) / B, Z), ASM_T, tile_smem<Lc>(), st>>>(a->X, P, s, No, a->layers,
                                                                                    a->Y, a->tw);
    k_asm_inv_rows<Lc, B><<<dim3((No + B - 1) / B, Z), ASM_T, tile_smem<Lc>(), st>>>(
        a->Y, No, Z, a->layers, layer_idx, (float2*)fields, amplitude, a->tw);
  });
  prof_mark(p, CGH_PROF_ASM_INV, 1, st);
  return cgh_cuda_check(cudaGetLastError(), "cgh_reconstruct_asm: inverse transforms");
}
