// Shared-memory complex FP32 FFT of power-of-two lengths 64..4096, used by the
// angular-spectrum reconstruction.
//
// Algorithm: Stockham auto-sort FFT (Stockham 1966; the GPU formulation of Govindaraju et
// al., SC 2008): pass p combines R-point DFTs of the sub-transforms of length Ns = 16^p
// already computed; group j reads the R elements j + r*L/R, multiplies element r by the
// twiddle W_{Ns*R}^{(j mod Ns)*r}, takes an R-point DFT in registers and writes element r
// to (j div Ns)*Ns*R + (j mod Ns) + r*Ns.  Radix 16 for every pass but possibly the last
// (radix 2, 4 or 8), so 1024 = 16*16*4 takes three passes and two trips through shared
// memory, and a thread holding 16 elements takes one whole group per pass.  Output in
// natural order.
// Forward: X[k] = sum_n x[n] exp(-2 pi i n k / L); inverse: exp(+...), unnormalised.
//
// A CTA transforms B lines of length L at once (a tile of rows or of columns).  Thread
// mapping: group index g -> line b = g mod B, group j = g div B, so that a warp touches
// 32/B consecutive elements of each of B lines (coalesced for both row and column tiles).
// The first pass reads its inputs through a loader functor and the last pass writes its
// outputs through a storer functor (both see (line, index)); the passes in between work
// in shared memory, padded by one element every 16 and with a line stride chosen so that
// the strided accesses of the early passes spread over the banks.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

namespace fft {

constexpr int LMAX = 4096;  // twiddle table length: tw[k] = exp(-2 pi i k / LMAX)

__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ float2 cmulc(float2 a, float2 b) {  // a * conj(b)
  return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
// a * (-i) forward, a * (+i) inverse
template <bool INV>
__host__ __device__ __forceinline__ float2 rot(float2 a) {
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

template <bool INV>
__host__ __device__ __forceinline__ void dft2(float2* v) {
  const float2 a = v[0];
  v[0] = cadd(a, v[1]);
  v[1] = csub(a, v[1]);
}

// 4-point DFT of (a0, a1, a2, a3) in natural order.
template <bool INV>
__host__ __device__ __forceinline__ void dft4(float2& a0, float2& a1, float2& a2, float2& a3) {
  const float2 s02 = cadd(a0, a2), d02 = csub(a0, a2);
  const float2 s13 = cadd(a1, a3), d13 = rot<INV>(csub(a1, a3));
  a0 = cadd(s02, s13);
  a2 = csub(s02, s13);
  a1 = cadd(d02, d13);
  a3 = csub(d02, d13);
}

// 8-point DFT: 4-point DFTs of the even and odd samples, odd half times W_8^k, then one
// radix-2 combination.
template <bool INV>
__host__ __device__ __forceinline__ void dft8(float2* v) {
  constexpr float h = 0.70710678118654752440f;  // 1/sqrt(2)
  float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  float2 o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  dft4<INV>(e0, e1, e2, e3);
  dft4<INV>(o0, o1, o2, o3);
  // W_8^1 = (1 - i)/sqrt(2) forward, (1 + i)/sqrt(2) inverse; W_8^2 = -+i; W_8^3 = (-1 -+ i)/sqrt(2)
  o1 = INV ? make_float2(h * (o1.x - o1.y), h * (o1.x + o1.y)) : make_float2(h * (o1.x + o1.y), h * (o1.y - o1.x));
  o2 = rot<INV>(o2);
  o3 = INV ? make_float2(-h * (o3.x + o3.y), h * (o3.x - o3.y)) : make_float2(h * (o3.y - o3.x), -h * (o3.x + o3.y));
  v[0] = cadd(e0, o0);
  v[4] = csub(e0, o0);
  v[1] = cadd(e1, o1);
  v[5] = csub(e1, o1);
  v[2] = cadd(e2, o2);
  v[6] = csub(e2, o2);
  v[3] = cadd(e3, o3);
  v[7] = csub(e3, o3);
}

// 16-point DFT as 4 x 4: 4-point DFTs over the stride-4 samples, twiddles W_16^(n2 k1),
// 4-point DFTs across, and the 4 x 4 transpose back to natural order.
template <bool INV>
__host__ __device__ __forceinline__ void dft16(float2* v) {
  constexpr float c = 0.92387953251128675613f;  // cos(pi/8)
  constexpr float s = 0.38268343236508977173f;  // sin(pi/8)
  constexpr float h = 0.70710678118654752440f;  // 1/sqrt(2)
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) dft4<INV>(v[n2], v[4 + n2], v[8 + n2], v[12 + n2]);
  // slot 4 k1 + n2 times W_16^(n2 k1); forward W_16^m = exp(-2 pi i m / 16), inverse its conjugate
  const float sg = INV ? 1.f : -1.f;
  v[5] = cmul(v[5], make_float2(c, sg * s));       // W^1
  v[6] = cmul(v[6], make_float2(h, sg * h));       // W^2
  v[7] = cmul(v[7], make_float2(s, sg * c));       // W^3
  v[9] = cmul(v[9], make_float2(h, sg * h));       // W^2
  v[10] = rot<INV>(v[10]);                         // W^4
  v[11] = cmul(v[11], make_float2(-h, sg * h));    // W^6
  v[13] = cmul(v[13], make_float2(s, sg * c));     // W^3
  v[14] = cmul(v[14], make_float2(-h, sg * h));    // W^6
  v[15] = cmul(v[15], make_float2(-c, -sg * s));   // W^9
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) dft4<INV>(v[4 * k1], v[4 * k1 + 1], v[4 * k1 + 2], v[4 * k1 + 3]);
  // X[k1 + 4 k2] sits in slot 4 k1 + k2
  float2 t[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) t[k] = v[4 * (k & 3) + (k >> 2)];
#pragma unroll
  for (int k = 0; k < 16; ++k) v[k] = t[k];
}

template <int R, bool INV>
__host__ __device__ __forceinline__ void dft(float2* v) {
  if constexpr (R == 16) {
    dft16<INV>(v);
  } else if constexpr (R == 8) {
    dft8<INV>(v);
  } else if constexpr (R == 4) {
    dft4<INV>(v[0], v[1], v[2], v[3]);
  } else {
    static_assert(R == 2, "radix 2, 4, 8 or 16");
    dft2<INV>(v);
  }
}

// Radix 16 for every pass but possibly the last (radix 2, 4 or 8).
constexpr int LR = 4;  // log2 of the radix
__host__ __device__ constexpr int ilog2(int x) { return x <= 1 ? 0 : 1 + ilog2(x >> 1); }
__host__ __device__ constexpr int n_passes(int L) { return ilog2(L) / LR + (ilog2(L) % LR ? 1 : 0); }
__host__ __device__ constexpr int pass_radix(int L, int p) {
  return p < ilog2(L) / LR ? (1 << LR) : (1 << (ilog2(L) % LR));
}
__host__ __device__ constexpr int pass_ns(int p) { return 1 << (LR * p); }  // only the last pass may have a smaller radix

// Twiddle and DFT of one group of pass (R, NS): v[r] *= W_{NS*R}^{(j mod NS) r}.
template <int R, int NS, bool INV>
__host__ __device__ __forceinline__ void group_dft(float2* v, int j, const float2* __restrict__ tw) {
  if constexpr (NS > 1) {
    const int k = j % NS;
    constexpr int step = LMAX / (NS * R);
#pragma unroll
    for (int r = 1; r < R; ++r) {
      const float2 w = tw[k * r * step];
      v[r] = INV ? cmulc(v[r], w) : cmul(v[r], w);
    }
  }
  dft<R, INV>(v);
}

// Destination of element r of group j in pass (R, NS) is out_base(j) + r * NS.
template <int R, int NS>
__host__ __device__ __forceinline__ int out_base(int j) {
  return (j / NS) * NS * R + (j % NS);
}

// Shared-memory layout of B lines of length L: line stride LS floats2, one pad element
// after every 16 (the first pass writes each group's 16 outputs contiguously, so padded
// groups start 17 elements apart and the threads of a half-warp hit distinct banks).
// LS = L + L/16 + 16/min(B,16): the last term is the bank offset that separates the B lines
// a half-warp touches.
template <int L, int B>
struct Smem {
  static constexpr int bo = 16 / (B < 16 ? B : 16);
  static constexpr int LS = L + L / 16 + (bo == 16 ? 1 : bo);
  static constexpr int floats2 = B * LS;
  __host__ __device__ static __forceinline__ int at(int b, int i) { return b * LS + i + (i >> 4); }
};

#ifdef __CUDACC__
// Transforms the B lines of one tile.  T threads; B * L / T elements live in each thread's
// registers during a pass.  ld(b, i) -> float2 gives input element i of line b; st(b, i, v)
// receives output element i.  s must hold Smem<L, B>::floats2 float2 values.  LD_SMEM:
// the loader reads the tile from s itself (filled by the caller, followed by a barrier),
// so pass 0 waits for every thread's loads before it overwrites s.
template <int L, int B, int T, bool INV, bool LD_SMEM = false, class Ld, class St>
__device__ __forceinline__ void fft_tile(float2* s, const float2* __restrict__ tw, Ld&& ld, St&& st) {
  using S = Smem<L, B>;
  constexpr int NP = n_passes(L);
  static_assert(NP >= 2 && NP <= 3, "L in [64, 4096]");
  static_assert(L <= LMAX, "L too large");

  // pass 0 (NS = 1): global -> registers -> shared
  {
    constexpr int R = pass_radix(L, 0), G = L / R, NG = B * G / T;
    static_assert((B * G) % T == 0, "tile does not divide among the threads");
    float2 v[NG][R];
#pragma unroll
    for (int g = 0; g < NG; ++g) {
      const int gi = threadIdx.x + g * T, b = gi % B, j = gi / B;
#pragma unroll
      for (int r = 0; r < R; ++r) v[g][r] = ld(b, j + r * G);
    }
    if constexpr (LD_SMEM) __syncthreads();
#pragma unroll
    for (int g = 0; g < NG; ++g) {
      const int gi = threadIdx.x + g * T, b = gi % B, j = gi / B;
      group_dft<R, 1, INV>(v[g], j, tw);
      const int o = out_base<R, 1>(j);
#pragma unroll
      for (int r = 0; r < R; ++r) s[S::at(b, o + r)] = v[g][r];
    }
    __syncthreads();
  }
  // middle passes: shared -> registers -> shared
  auto middle = [&](auto pc) {
    constexpr int p = decltype(pc)::value;
    constexpr int R = pass_radix(L, p), NS = pass_ns(p), G = L / R, NG = B * G / T;
    float2 v[NG][R];
#pragma unroll
    for (int g = 0; g < NG; ++g) {
      const int gi = threadIdx.x + g * T, b = gi % B, j = gi / B;
#pragma unroll
      for (int r = 0; r < R; ++r) v[g][r] = s[S::at(b, j + r * G)];
    }
    __syncthreads();
#pragma unroll
    for (int g = 0; g < NG; ++g) {
      const int gi = threadIdx.x + g * T, b = gi % B, j = gi / B;
      group_dft<R, NS, INV>(v[g], j, tw);
      const int o = out_base<R, NS>(j);
#pragma unroll
      for (int r = 0; r < R; ++r) s[S::at(b, o + r * NS)] = v[g][r];
    }
    __syncthreads();
  };
  if constexpr (NP > 2) middle(std::integral_constant<int, 1>{});
  // last pass: shared -> registers -> global (NS * R = L, so group j writes j + r * NS)
  {
    constexpr int p = NP - 1;
    constexpr int R = pass_radix(L, p), NS = pass_ns(p), G = L / R, NG = B * G / T;
    static_assert(NS * R == L, "pass schedule");
    float2 v[NG][R];
#pragma unroll
    for (int g = 0; g < NG; ++g) {
      const int gi = threadIdx.x + g * T, b = gi % B, j = gi / B;
#pragma unroll
      for (int r = 0; r < R; ++r) v[g][r] = s[S::at(b, j + r * G)];
    }
#pragma unroll
    for (int g = 0; g < NG; ++g) {
      const int gi = threadIdx.x + g * T, b = gi % B, j = gi / B;
      group_dft<R, NS, INV>(v[g], j, tw);
#pragma unroll
      for (int r = 0; r < R; ++r) st(b, j + r * NS, v[g][r]);
    }
  }
}
#endif

}  // namespace fft
