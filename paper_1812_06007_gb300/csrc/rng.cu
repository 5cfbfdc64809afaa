// rng.cu -- the Gaussian start matrix G of PowerURV (Section 3: "a Gaussian
// random matrix G in R^{n x n} is drawn").  The paper names no generator;
// this library uses the counter-based Philox4x64-10 (Salmon, Moraes, Dror,
// Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11) so that every
// element is a pure function of (seed, stream, position) and the draw is
// embarrassingly parallel, then Box-Muller for the normal deviates.
#include "common.cuh"
#include "profile.cuh"
#include "rng.cuh"

namespace purl {

namespace {

__device__ __forceinline__ double u53(uint64_t x) {
  return (static_cast<double>(x >> 11) + 0.5) * 0x1.0p-53;
}

// One thread per Philox block: 4 consecutive (column-major) elements.  F32:
// the same words through the FP32 Box-Muller of gaussian_block_f32 (stored as
// FP64), for the paths whose first use of G rounds it to 16 bits.
template <bool F32>
__global__ void __launch_bounds__(256) gaussian_kernel(uint64_t seed, uint64_t stream_id,
                                                       int rows, long long count, double *G,
                                                       long long ldg) {
  const double two_pi = 6.283185307179586476925286766559;
  long long nblk = (count + 3) / 4;
  for (long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x; b < nblk;
       b += (long long)gridDim.x * blockDim.x) {
    double z[4];
    if constexpr (F32) {
      float zf[4];
      gaussian_block_f32(seed, stream_id, (uint64_t)b, zf);
#pragma unroll
      for (int t = 0; t < 4; ++t) z[t] = zf[t];
    } else {
      uint64_t c[4] = {static_cast<uint64_t>(b), 0, 0, 0};
      philox4x64_10(c, seed, stream_id);
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        double r = sqrt(-2.0 * log(u53(c[2 * p])));
        double s, co;
        sincos(two_pi * u53(c[2 * p + 1]), &s, &co);
        z[2 * p] = r * co;
        z[2 * p + 1] = r * s;
      }
    }
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      long long e = 4 * b + t;
      if (e < count) G[(e % rows) + (e / rows) * ldg] = z[t];
    }
  }
}

}  // namespace

int launch_gaussian(uint64_t seed, uint64_t stream_id, int rows, int cols, double *G, int ldg,
                    cudaStream_t stream, bool fp32_math) {
  long long count = (long long)rows * cols;
  if (count == 0) return PURL_OK;
  const DeviceInfo *di = device_info();
  if (!di) return PURL_ERR_CUDA;
  long long nblk = (count + 3) / 4;
  long long want = (nblk + 255) / 256;
  int grid = (int)(want < (long long)di->num_sms * 8 ? want : (long long)di->num_sms * 8);
  LaunchScope ls(KC_OTHER, stream, 0.0, 8.0 * count, "gaussian_kernel");
  if (fp32_math) gaussian_kernel<true><<<grid, 256, 0, stream>>>(seed, stream_id, rows, count, G, ldg);
  else gaussian_kernel<false><<<grid, 256, 0, stream>>>(seed, stream_id, rows, count, G, ldg);
  return cudaGetLastError() == cudaSuccess ? PURL_OK : PURL_ERR_CUDA;
}

}  // namespace purl
