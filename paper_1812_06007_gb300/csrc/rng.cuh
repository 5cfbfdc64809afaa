// rng.cuh -- Philox4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
// numbers: as easy as 1, 2, 3", SC'11), the counter-based generator behind
// the Gaussian start matrix G of Section 3.  Ten rounds of the 4x64 Philox
// S-box with the published multipliers and Weyl key increments; the block
// (c[0..3]) is encrypted in place under the key (k0, k1).
#pragma once

#include <stdint.h>

namespace purl {

__device__ __forceinline__ void philox4x64_10(uint64_t c[4], uint64_t k0, uint64_t k1) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
  const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint64_t hi0 = __umul64hi(M0, c[0]), lo0 = M0 * c[0];
    uint64_t hi1 = __umul64hi(M1, c[2]), lo1 = M1 * c[2];
    uint64_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
    k0 += W0; k1 += W1;  // the bump after the last round is unused
  }
}

// FP32 normal deviates of one Philox block: the 53-bit uniform
// ((w >> 11) + 0.5) 2^-53 of the FP64 generator, rounded once to FP32, then
// Box-Muller with FP32 logf / sincospif.
__device__ __forceinline__ float u53_f32(uint64_t w) {
  return __ull2float_rn(2ull * (w >> 11) + 1ull) * 0x1.0p-54f;
}

__device__ __forceinline__ void gaussian_block_f32(uint64_t seed, uint64_t stream_id, uint64_t b, float z[4]) {
  uint64_t c[4] = {b, 0, 0, 0};
  philox4x64_10(c, seed, stream_id);
#pragma unroll
  for (int p = 0; p < 2; ++p) {
    const float r = sqrtf(-2.f * logf(u53_f32(c[2 * p])));
    float s, co;
    sincospif(2.f * u53_f32(c[2 * p + 1]), &s, &co);
    z[2 * p] = r * co;
    z[2 * p + 1] = r * s;
  }
}

}  // namespace purl
