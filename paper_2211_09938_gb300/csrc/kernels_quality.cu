// Reconstruction quality: mean SSIM of two images (the paper compares every progressive
// level with the fully point-wise reconstruction by SSIM, Section 3 / Table 3).
//
// SSIM after Wang et al. 2004: 11x11 Gaussian window (sigma 1.5) over the valid region,
// K1 = 0.01, K2 = 0.03, data range 1; with normalisation each image is first divided by
// its own maximum (the amplitudes of different holograms differ in scale).
#include "cgh_internal.h"

#define SSIM_WIN 11

struct SsimTaps {  // normalised 1-D Gaussian taps, passed by value with the launch
  float g[SSIM_WIN];
};

// max over a non-negative float image (bit patterns of non-negative floats order as ints)
__global__ void k_max_nonneg(const float* __restrict__ x, long long n, unsigned int* __restrict__ out) {
  unsigned int m = 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    m = max(m, __float_as_uint(fmaxf(x[i], 0.f)));
  m = __reduce_max_sync(0xffffffffu, m);
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

// One thread per valid window position: the five Gaussian-weighted moments, the local SSIM,
// and a block sum added in FP64 to out[0].
__global__ void __launch_bounds__(256) k_ssim(const float* __restrict__ x, const float* __restrict__ y, int H, int W,
                                              const unsigned int* __restrict__ maxes, int normalize,
                                              const SsimTaps taps, double* __restrict__ out) {
  __shared__ double s_sum[8];
  const int oh = H - SSIM_WIN + 1, ow = W - SSIM_WIN + 1;
  const int c = blockIdx.x * 32 + (threadIdx.x & 31);
  const int r = blockIdx.y * 8 + (threadIdx.x >> 5);
  float sx = 1.f, sy = 1.f;
  if (normalize) {
    const float mx = __uint_as_float(maxes[0]), my = __uint_as_float(maxes[1]);
    sx = mx > 0.f ? 1.f / mx : 1.f;
    sy = my > 0.f ? 1.f / my : 1.f;
  }
  double v = 0.0;
  if (r < oh && c < ow) {
    // Moments of the values minus the window's centre value: (co)variances are shift
    // invariant, and the smaller magnitudes keep E[x^2] - E[x]^2 from cancelling in FP32.
    const int ctr = (SSIM_WIN - 1) / 2;
    const float x0 = x[(size_t)(r + ctr) * W + c + ctr] * sx, y0 = y[(size_t)(r + ctr) * W + c + ctr] * sy;
    float mx = 0.f, my = 0.f, xx = 0.f, yy = 0.f, xy = 0.f;
    for (int a = 0; a < SSIM_WIN; ++a) {
      const float* xr = x + (size_t)(r + a) * W + c;
      const float* yr = y + (size_t)(r + a) * W + c;
      for (int b = 0; b < SSIM_WIN; ++b) {
        const float g = taps.g[a] * taps.g[b];
        const float xv = fmaf(xr[b], sx, -x0), yv = fmaf(yr[b], sy, -y0);
        mx = fmaf(g, xv, mx);
        my = fmaf(g, yv, my);
        xx = fmaf(g, xv * xv, xx);
        yy = fmaf(g, yv * yv, yy);
        xy = fmaf(g, xv * yv, xy);
      }
    }
    const float c1 = 1e-4f, c2 = 9e-4f;  // (0.01 * 1)^2, (0.03 * 1)^2
    const float vx = xx - mx * mx, vy = yy - my * my, cxy = xy - mx * my;
    const float ux = mx + x0, uy = my + y0;  // the local means themselves
    v = (double)((2.f * ux * uy + c1) * (2.f * cxy + c2)) / (double)((ux * ux + uy * uy + c1) * (vx + vy + c2));
  }
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) s_sum[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < 8; ++k) t += s_sum[k];
    atomicAdd(out, t / ((double)oh * ow));
  }
}

extern "C" int cgh_ssim(const float* x, const float* y, int h, int w, int normalize, double* out_mean,
                        void* scratch, void* stream) {
  if (!x || !y || !out_mean || (normalize && !scratch))
    return cgh_fail(CGH_ERR_ARG, "cgh_ssim: NULL argument");
  if (h < SSIM_WIN || w < SSIM_WIN || h > 65536 || w > 65536)
    return cgh_fail(CGH_ERR_ARG, "cgh_ssim: image %dx%d outside [11, 65536]", h, w);
  cudaStream_t st = (cudaStream_t)stream;
  SsimTaps taps;
  {
    double s = 0.0, d[SSIM_WIN];
    for (int k = 0; k < SSIM_WIN; ++k) {
      const double t = k - (SSIM_WIN - 1) / 2.0;
      d[k] = exp(-t * t / (2.0 * 1.5 * 1.5));
      s += d[k];
    }
    for (int k = 0; k < SSIM_WIN; ++k) taps.g[k] = (float)(d[k] / s);
  }
  int rc = cgh_cuda_check(cudaMemsetAsync(out_mean, 0, sizeof(double), st), "cgh_ssim: clear");
  if (rc != CGH_OK) return rc;
  unsigned int* maxes = (unsigned int*)scratch;
  if (normalize) {
    rc = cgh_cuda_check(cudaMemsetAsync(maxes, 0, 2 * sizeof(unsigned int), st), "cgh_ssim: clear");
    if (rc != CGH_OK) return rc;
    const long long n = (long long)h * w;
    k_max_nonneg<<<152, 256, 0, st>>>(x, n, maxes);
    k_max_nonneg<<<152, 256, 0, st>>>(y, n, maxes + 1);
  }
  dim3 grid((w - SSIM_WIN + 1 + 31) / 32, (h - SSIM_WIN + 1 + 7) / 8);
  k_ssim<<<grid, 256, 0, st>>>(x, y, h, w, maxes, normalize, taps, out_mean);
  return cgh_cuda_check(cudaGetLastError(), "cgh_ssim");
}
