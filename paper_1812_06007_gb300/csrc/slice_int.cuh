// slice_int.cuh -- fixed-point BF16 slicing of FP64 values with integer arithmetic only.
//
// GB300's FP64 pipe does about two operations per clock per SM, so slicing
// with FP64 arithmetic (scale, round, subtract per slice) made the slicing
// passes slower than the products they feed.  Here an FP64 value x with
// |x| < 2^e becomes the integer N = round(x 2^(P-e)), P = 7 + 8(S-1),
// straight from its IEEE bits, and N is cut into S balanced digits
//   N = d_0 2^(8(S-1)) + d_1 2^(8(S-2)) + ... + d_{S-1},
//   d_1..d_{S-1} in [-128, 127], d_0 in [-128, 128],
// each of which is written as an exact BF16 (at most 8 significant bits) by
// assembling its bit pattern.  x is then carried to 2^(e-P-1) (half a unit
// of the last digit), i.e. 2^-8S of the scale 2^e.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace purl {

// Exponent e with |x| < 2^e for the largest |x| given as its IEEE bits with the
// sign cleared (0 for zero or subnormal maxima).
__device__ __forceinline__ int exp_above_bits(unsigned long long absbits) {
  const int E = (int)(absbits >> 52);
  return E == 0 ? 0 : E - 1022;
}

__device__ __forceinline__ unsigned long long abs_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFULL;
}

// round(x 2^(P - e)) for |x| < 2^e (ties away from zero), from the bits of x.
__device__ __forceinline__ long long fixed_point(double x, int e, int P) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int E = (int)((b >> 52) & 0x7FF);
  if (E == 0) return 0;  // zero or subnormal: below every scale used here
  const unsigned long long mant = (b & 0xFFFFFFFFFFFFFULL) | (1ULL << 52);
  const int sh = E - 1075 + P - e;  // x = mant 2^(E-1075)
  long long n;
  if (sh >= 0) {
    n = sh < 11 ? (long long)(mant << sh) : 0;  // |x| < 2^e keeps this below 2^P
  } else {
    const int r = -sh;
    n = r > 54 ? 0 : (long long)((mant + (1ULL << (r - 1))) >> r);
  }
  return (b >> 63) ? -n : n;
}

// BF16 bit pattern of a small integer |d| <= 255: its FP32 conversion is
// exact and has no significant bits below the top 8, so the upper half of the
// FP32 bits is the BF16 value.
__device__ __forceinline__ unsigned short bf16_bits_small(int d) {
  return (unsigned short)(__float_as_uint(__int2float_rn(d)) >> 16);
}

// Write the S digits of x (|x| < 2^e) as BF16 slices: slice s at dst[s * plane],
// from N = round(x 2^(P - e)) (write_int_slices takes N itself, |N| <= 2^P),
// S <= 8 (P = 7 + 8(S-1) <= 63 keeps N in a 64-bit integer).  The balanced
// base-256 digits of N are read off M = N + 128 (1 + 2^8 + ... + 2^(8(S-2))):
// byte j of M minus 128 is the digit of weight 2^(8j) for j < S-1, and M
// shifted right (arithmetically) by 8(S-1) is the top digit -- the same
// digits as peeling them off one at a time from the bottom.  M is formed
// modulo 2^64 (for S = 8 it can pass 2^63), so the top digit t in [-128, 128]
// is read from its byte, which leaves only t = +-128 ambiguous; N's sign
// settles that.
__device__ __forceinline__ void write_int_slices(long long n, __nv_bfloat16 *dst, long long plane, int S) {
  const unsigned long long bias = 0x0080808080808080ULL >> (8 * (8 - S));
  const unsigned long long M = (unsigned long long)n + bias;
  unsigned short *out = reinterpret_cast<unsigned short *>(dst);
  int t = (int)((M >> (8 * (S - 1))) & 255u);
  t = t >= 128 ? t - 256 : t;
  if (t == -128 && n > 0) t = 128;
  out[0] = bf16_bits_small(t);
  for (int s = 1; s < S; ++s) {
    const int j = S - 1 - s;  // byte of M that holds slice s
    out[s * plane] = bf16_bits_small((int)((M >> (8 * j)) & 255u) - 128);
  }
}

__device__ __forceinline__ void write_fixed_slices(double x, int e, __nv_bfloat16 *dst, long long plane, int S) {
  write_int_slices(fixed_point(x, e, 7 + 8 * (S - 1)), dst, plane, S);
}

// The same digits as write_fixed_slices for a compile-time S, returned as BF16
// bit patterns (d[0] the top digit).
template <int S>
__device__ __forceinline__ void fixed_digits(double x, int e, unsigned short (&d)[S]) {
  const long long n = fixed_point(x, e, 7 + 8 * (S - 1));
  const unsigned long long M = (unsigned long long)n + (0x0080808080808080ULL >> (8 * (8 - S)));
  int t = (int)((M >> (8 * (S - 1))) & 255u);
  t = t >= 128 ? t - 256 : t;
  if (t == -128 && n > 0) t = 128;
  d[0] = bf16_bits_small(t);
#pragma unroll
  for (int s = 1; s < S; ++s) d[s] = bf16_bits_small((int)((M >> (8 * (S - 1 - s))) & 255u) - 128);
}

// round(x 2^(P - e)) for an FP32 x with |x| < 2^e (ties away from zero),
// from the bits of x; P <= 31.
__device__ __forceinline__ int fixed_point_f32(float x, int e, int P) {
  const unsigned b = __float_as_uint(x);
  const int E = (int)((b >> 23) & 0xFFu);
  if (E == 0) return 0;
  const unsigned mant = (b & 0x7FFFFFu) | 0x800000u;
  const int sh = E - 150 + P - e;  // x = mant 2^(E-150)
  int n;
  if (sh >= 0) {
    n = sh < 8 ? (int)(mant << sh) : 0;  // |x| < 2^e keeps this within P + 1 bits
  } else {
    const int r = -sh;
    n = r > 25 ? 0 : (int)((mant + (1u << (r - 1))) >> r);
  }
  return (b >> 31) ? -n : n;
}

// The FP32 value nearest to x 2^k (ties away from zero) for a finite FP64 x,
// from its bits (no FP64-pipe instruction); zero where the result would be
// below FP32's normal range.  The caller keeps |x 2^k| below 2^127.
__device__ __forceinline__ float double_to_scaled_float(double x, int k) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int E = (int)((b >> 52) & 0x7FF);
  if (E == 0) return 0.0f;
  unsigned long long m = ((b & 0xFFFFFFFFFFFFFULL) | (1ULL << 52));
  m = (m + (1ULL << 28)) >> 29;  // 24 bits, or 2^24 after a carry
  int e8 = E - 1023 + k + 127;
  if (m >> 24) {
    m >>= 1;
    ++e8;
  }
  if (e8 <= 0) return 0.0f;
  return __uint_as_float((unsigned)((b >> 63) << 31) | ((unsigned)e8 << 23) | ((unsigned)m & 0x7FFFFFu));
}

// The FP64 value of f * 2^k for a finite FP32 f, assembled from the bits of f
// with integer operations (no FP64-pipe instruction).  Zero and FP32
// subnormals (|f| < 2^-126, far below every value these kernels produce)
// give zero.
__device__ __forceinline__ double scaled_float_to_double(float f, int k) {
  const unsigned b = __float_as_uint(f);
  const unsigned e8 = (b >> 23) & 0xFFu;
  if (e8 == 0) return 0.0;
  const unsigned long long sign = (unsigned long long)(b >> 31) << 63;
  const unsigned long long e11 = (unsigned long long)(int)(e8 + 896 + k);
  const unsigned long long m = (unsigned long long)(b & 0x7FFFFFu) << 29;
  return __longlong_as_double((long long)(sign | (e11 << 52) | m));
}

// f 2^k as an FP64 value for any k: zero below FP64's normal range, an
// infinity above it; otherwise exact.
__device__ __forceinline__ double scaled_float_to_double_any(float f, int k) {
  const unsigned b = __float_as_uint(f);
  const int e11 = (int)((b >> 23) & 0xFFu) + 896 + k;
  if (((b >> 23) & 0xFFu) == 0 || e11 <= 0) return 0.0;
  if (e11 >= 2047) return __longlong_as_double((long long)(((unsigned long long)(b >> 31) << 63) | 0x7FF0000000000000ULL));
  return scaled_float_to_double(f, k);
}

// The FP64 value nearest to x * 2^k (ties away from zero) for |x| < 2^62,
// assembled with integer operations only; zero for x == 0 and for results
// below the normal FP64 range.
__device__ __forceinline__ double int64_scaled_to_double(long long x, int k) {
  if (x == 0) return 0.0;
  const unsigned long long sign = x < 0 ? (1ULL << 63) : 0ULL;
  const unsigned long long a = x < 0 ? (unsigned long long)(-x) : (unsigned long long)x;
  int msb = 63 - __clzll((long long)a);
  unsigned long long mant;
  if (msb <= 52) {
    mant = a << (52 - msb);
  } else {
    const int r = msb - 52;
    mant = (a + (1ULL << (r - 1))) >> r;
    if (mant >> 53) {
      mant >>= 1;
      ++msb;
    }
  }
  const int E = msb + k + 1023;
  if (E <= 0) return 0.0;
  return __longlong_as_double((long long)(sign | ((unsigned long long)E << 52) | (mant & 0xFFFFFFFFFFFFFULL)));
}

}  // namespace purl
