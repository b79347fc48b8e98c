// Microbenchmarks for the roofline peaks of the direct kernels (the paper has no
// counterpart): the rate of SFU sine-cosine pairs, which bounds the point-wise kernels,
// and of FP32 fused multiply-adds, which bounds the detail-basis direct form.  Each thread
// runs independent dependency chains so that the unit, not latency, sets the rate; one
// value per thread goes to `sink` so that nothing is optimised away.
#include "cgh_internal.h"

#define PROBE_T 256

__global__ void __launch_bounds__(PROBE_T) k_probe_sfu(float* __restrict__ sink, long long iters) {
  float x[8], acc[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    x[q] = 0.1f * (float)(threadIdx.x + q);
    acc[q] = 0.f;
  }
#pragma unroll 4
  for (long long it = 0; it < iters; ++it) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      float sn, cs;
      __sincosf(x[q], &sn, &cs);
      acc[q] += sn + cs;
      x[q] = fmaf(x[q], 0.999f, 1e-3f);  // stays in (0, 1.1): no range reduction
    }
  }
  float t = 0.f;
#pragma unroll
  for (int q = 0; q < 8; ++q) t += acc[q];
  sink[(size_t)blockIdx.x * PROBE_T + threadIdx.x] = t;
}

__global__ void __launch_bounds__(PROBE_T) k_probe_ffma(float* __restrict__ sink, long long iters) {
  float2 a[16];
  const float2 m = make_float2(0.9999f, 0.9998f), c = make_float2(1e-4f, 2e-4f);
#pragma unroll
  for (int q = 0; q < 16; ++q) a[q] = make_float2(0.01f * (float)(threadIdx.x + q), 0.02f * (float)q);
#pragma unroll 8  // keeps the loop counter's share of the issue slots small
  for (long long it = 0; it < iters; ++it) {
#pragma unroll
    for (int q = 0; q < 16; ++q) a[q] = __ffma2_rn(a[q], m, c);  // two FMAs per instruction
  }
  float t = 0.f;
#pragma unroll
  for (int q = 0; q < 16; ++q) t += a[q].x + a[q].y;
  sink[(size_t)blockIdx.x * PROBE_T + threadIdx.x] = t;
}

static int probe_args(const float* sink, int grid, long long iters, const char* name) {
  if (!sink || grid < 1 || grid > (1 << 20) || iters < 1 || iters > (1ll << 32))
    return cgh_fail(CGH_ERR_ARG, "%s: NULL sink, grid outside 1..2^20 or iters outside 1..2^32", name);
  return CGH_OK;
}

extern "C" int cgh_probe_sfu(float* sink, int grid, long long iters, void* stream) {
  int rc = probe_args(sink, grid, iters, "cgh_probe_sfu");
  if (rc != CGH_OK) return rc;
  k_probe_sfu<<<grid, PROBE_T, 0, (cudaStream_t)stream>>>(sink, iters);
  return cgh_cuda_check(cudaGetLastError(), "cgh_probe_sfu");
}

extern "C" int cgh_probe_ffma(float* sink, int grid, long long iters, void* stream) {
  int rc = probe_args(sink, grid, iters, "cgh_probe_ffma");
  if (rc != CGH_OK) return rc;
  k_probe_ffma<<<grid, PROBE_T, 0, (cudaStream_t)stream>>>(sink, iters);
  return cgh_cuda_check(cudaGetLastError(), "cgh_probe_ffma");
}
