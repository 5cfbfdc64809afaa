// tc.cuh -- BF16 tensor-core product engine (tcgen05 + TMEM + TMA), internal interface.
//
// Operands are stacks of S BF16 "slices" of an FP64 matrix X:
//   X ~= X_0 + X_1 + ... + X_{S-1},  X_0 = bf16(X), X_1 = bf16(X - X_0), ...
// (each slice carries the next ~8 bits of every entry).  A product of two
// sliced operands keeps the slice pairs (s, t) with s + t < S, i.e. 1, 3 or 6
// BF16 products for S = 1, 2, 3, accumulated in FP32 in tensor memory.
//
// Storage: slice s of an R x Cc matrix is column-major with leading dimension
// `ld` (a multiple of 64 elements) at base + s * plane.  As a tcgen05 operand
// ("K-major"), its columns are the operand's rows (M or N) and its rows are
// the reduction index K.
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"

namespace purl {

struct Slices {
  __nv_bfloat16 *base = nullptr;
  int *scale = nullptr;  // exact (fixed-point) slices: exponent per operand row (column of X)
  int rows = 0;         // R (the reduction extent when used as an operand)
  int cols = 0;         // Cc (the M or N extent when used as an operand)
  long long ld = 0;     // elements, multiple of 64
  long long plane = 0;  // elements between slices
  int S = 1;            // slices present
  int f16 = 0;          // element type of plain slices: 0 BF16, 1 FP16 (same 16-bit storage)
};

// Leading dimension of a slice plane: rows rounded up to 64 elements, plus 64
// more when that is a multiple of 512 (1 KB): the rows of a TMA box are then
// not a large power of two apart, which would map them onto the same L2 sets.
inline long long slice_ld(int rows) {
  const long long ld = ((long long)(rows > 0 ? rows : 1) + 63) / 64 * 64;
  return (ld % 512) == 0 ? ld + 64 : ld;
}
inline size_t slice_elems(int rows, int cols, int S) {
  return (size_t)slice_ld(rows) * (size_t)(cols > 0 ? cols : 1) * (size_t)S;
}
inline Slices make_slices(__nv_bfloat16 *base, int rows, int cols, int S) {
  Slices x;
  x.base = base; x.rows = rows; x.cols = cols; x.S = S;
  x.ld = slice_ld(rows);
  x.plane = x.ld * (long long)(cols > 0 ? cols : 1);
  return x;
}

// Epilogue of one product D = sum_{s+t<S} A_s B_t^T (M x N, FP32 in TMEM):
//   mode 0:  C = alpha D + beta C   (FP64, column-major, ldc; beta == 0: C not read)
//            and, if out.base, the S_out slices of the new C (column-major)
//   mode 1:  P_z = D_z for split z (FP32, column-major M x N, at P + z*M*N)
struct TcEpilogue {
  int mode = 0;
  double alpha = 1.0, beta = 0.0;
  double *C = nullptr;
  long long ldc = 0;
  float *P = nullptr;
  double *Pd = nullptr;  // mode 2: FP64 partials
  Slices out;  // optional
  const char *tag = nullptr;  // host-side name for the launch profiler
};

// Exact-accumulation slices (Ozaki-style splitting): every column c of X
// (= one operand row) gets an exponent e_c with |X(:,c)| < 2^e_c, and
//   X(r,c) ~= 2^e_c * sum_s alpha_s(r,c) * 2^(-7-8s),  alpha_s integers, |alpha_s| <= 128,
// stored exactly in BF16.  Products of such slices are integers below 2^14 and
// sums of up to 256 of them per slice-pair class stay below 2^24, so the FP32
// tensor-core accumulator never rounds; tcx_gemm drains it every 256 of K.
// `scale_from` (optional, length Cc): use these exponents instead of the
// column maxima (for matrices whose column norms bound every later entry).
int split_exact(int R, int Cc, const double *X, long long ldx, Slices dst, const int *scale_from,
                cudaStream_t s);
// Column exponents e_c = exponent of (1 + 2^-20) * ||X(:,c)||_2 (so |X(r,c)| < 2^e_c).
int column_norm_exponents(int R, int Cc, const double *X, long long ldx, int *e, cudaStream_t s);
// Slices of the FP64-emulation configuration of the exact engine: 8 digits of
// 8 bits (every operand row carried to 2^-63 of its scale), pairs s + t < 8.
constexpr int kTcxEmuSlices = 8;

// D = A B^T (M x N) with exact accumulation over exact slices (A.scale, B.scale
// required), S = 1..4 or kTcxEmuSlices (K <= 2^20).  Epilogue mode 0 (FP64 C = alpha D + beta C, optional
// slices out) or mode 2 (FP64 split-K partials at Pd + z*M*N).
int tcx_gemm_view(const Slices &A, int a_r0, int a_c0, const Slices &B, int b_r0, int b_c0, int M, int N,
                  int K, int S, const TcEpilogue &ep, int splits, int k_chunk, cudaStream_t s);
// Same with every slice pair (s, t), s, t < S (2S - 1 exact classes, N tile
// 32): the exact product of the two sliced matrices, up to FP64 rounding of
// the result.  Used for Gram matrices that must match the sliced operands.
int tcx_gemm_all_pairs(const Slices &A, int a_r0, int a_c0, const Slices &B, int b_r0, int b_c0, int M, int N,
                       int K, int S, const TcEpilogue &ep, int splits, int k_chunk, cudaStream_t s);

// C = alpha op(A) op(B) + beta C (FP64 operands, column-major) on the exact
// engine with S slices per operand (1..4 or kTcxEmuSlices), the operand slices
// and the FP64 staging of a transposed operand carved from `scratch`
// (gemm_exact_bytes(m, n, k, S) bytes, 256-byte aligned).  k == 0 scales C.
size_t gemm_exact_bytes(int m, int n, int k, int S);
int gemm_exact(bool ta, bool tb, int m, int n, int k, double alpha, const double *A, int lda, const double *B,
               int ldb, double beta, double *C, int ldc, int S, void *scratch, size_t scratch_bytes,
               cudaStream_t s);

// FP64 -> S BF16 slices.  split_slices: same orientation (dst is R x Cc);
// split_slices_t: transposed (dst is Cc x R).
int split_slices(int R, int Cc, const double *X, long long ldx, Slices dst, cudaStream_t s);
int split_slices_t(int R, int Cc, const double *X, long long ldx, Slices dst, cudaStream_t s);

// One plain slice (BF16, or FP16 when dst.f16) of 2^s X, with the power of two
// 2^s chosen on the device from the largest exponent in X so that the largest
// entry lands just below 2^15 (FP16) or 2 (BF16): the 16-bit formats' range
// then holds X whatever its magnitude.  The scale is not undone -- callers
// use it where only the span of the product matters (the power iterates are
// orthonormalised afterwards).  `e_ws`: one device int of scratch.
int split_scaled(int R, int Cc, const double *X, long long ldx, Slices dst, int *e_ws, bool transposed,
                 cudaStream_t s);

// D(M x N) = sum over slice pairs of A_s (M x K) B_t^T (N x K).  A: slices with
// cols = M, rows = K; B: cols = N, rows = K.  Split-K: `splits` chunks of
// `k_chunk` (a multiple of 64); mode 1 writes one FP32 partial per chunk.
int tc_gemm(const Slices &A, const Slices &B, int M, int N, int K, int S, const TcEpilogue &ep,
            int splits, int k_chunk, cudaStream_t s);
int tc_gemm_view(const Slices &A, int a_r0, int a_c0, const Slices &B, int b_r0, int b_c0, int M, int N, int K,
                 int S, const TcEpilogue &ep, int splits, int k_chunk, cudaStream_t s);

// Split count for a tall reduction producing an M x N output (chunks >= 256).
void tc_choose_splits(int M, int N, int K, int num_sms, int max_splits, int *splits, int *k_chunk);

}  // namespace purl
