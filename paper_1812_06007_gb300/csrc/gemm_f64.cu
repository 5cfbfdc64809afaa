// gemm_f64.cu -- FP64 level-3 product engine (the "efficient matrix-matrix
// multiplication routine" PowerURV is built on, Section 3), for the FP64 path.
//
// GB300's FP64 rate is a DFMA pipe of about two fused multiply-adds per clock
// per SM (1.2 TFLOP/s measured; the f64 mma.sync shapes measured slower, 1.05),
// so this kernel is bound by the DFMA pipe, not by memory: a 64x64x16 step does
// 65536 DFMAs (~32K SM clocks) against 16 KB of operand loads.  What matters is
// (a) a grid with enough tiles for all 152 SMs -- split-K covers the tall
// reductions of the QR trailing updates -- and (b) enough independent DFMAs per
// warp (4x4 accumulators per thread).
#include "common.cuh"
#include "profile.cuh"

namespace purl {

namespace {

constexpr int BK = 16;
constexpr int NT = 256;

template <int BM, int BN, int TM, int TN, bool TA, bool TB>
__global__ void __launch_bounds__(NT) gemm_f64_kernel(int m, int n, int k, int k_chunk,
                                                      double alpha, const double *__restrict__ A,
                                                      long long lda, const double *__restrict__ B,
                                                      long long ldb, double beta, double *C,
                                                      long long ldc, long long split_stride) {
  static_assert((BM / TM) * (BN / TN) == NT, "thread layout");
  constexpr int LA = BM * BK / NT;  // A elements loaded per thread
  constexpr int LB = BK * BN / NT;
  __shared__ double As[2][BK][BM + 1];
  __shared__ double Bs[2][BK][BN + 1];

  const int tid = threadIdx.x;
  const int tx = tid % (BM / TM);  // row group: rows tx + r*(BM/TM)
  const int ty = tid / (BM / TM);  // column group: cols ty + c*(BN/TN)
  const int m0 = blockIdx.x * BM;
  const int n0 = blockIdx.y * BN;
  const int kb = blockIdx.z * k_chunk;
  const int ke = min(k, kb + k_chunk);
  double *Cz = C + (long long)blockIdx.z * split_stride;

  double ra[LA], rb[LB];
  auto load = [&](int k0) {
#pragma unroll
    for (int s = 0; s < LA; ++s) {
      int e = tid + s * NT;
      int i, kk;
      if (TA) { kk = e % BK; i = e / BK; } else { i = e % BM; kk = e / BM; }
      int gi = m0 + i, gk = k0 + kk;
      ra[s] = (gi < m && gk < ke) ? (TA ? A[gk + gi * lda] : A[gi + gk * lda]) : 0.0;
    }
#pragma unroll
    for (int s = 0; s < LB; ++s) {
      int e = tid + s * NT;
      int j, kk;
      if (TB) { j = e % BN; kk = e / BN; } else { kk = e % BK; j = e / BK; }
      int gj = n0 + j, gk = k0 + kk;
      rb[s] = (gj < n && gk < ke) ? (TB ? B[gj + gk * ldb] : B[gk + gj * ldb]) : 0.0;
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int s = 0; s < LA; ++s) {
      int e = tid + s * NT;
      int i, kk;
      if (TA) { kk = e % BK; i = e / BK; } else { i = e % BM; kk = e / BM; }
      As[buf][kk][i] = ra[s];
    }
#pragma unroll
    for (int s = 0; s < LB; ++s) {
      int e = tid + s * NT;
      int j, kk;
      if (TB) { j = e % BN; kk = e / BN; } else { kk = e % BK; j = e / BK; }
      Bs[buf][kk][j] = rb[s];
    }
  };

  double acc[TM][TN];
#pragma unroll
  for (int r = 0; r < TM; ++r)
#pragma unroll
    for (int c = 0; c < TN; ++c) acc[r][c] = 0.0;

  int buf = 0;
  if (kb < ke) {
    load(kb);
    store(0);
  }
  __syncthreads();
  for (int k0 = kb; k0 < ke; k0 += BK) {
    bool more = k0 + BK < ke;
    if (more) load(k0 + BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double a[TM], b[TN];
#pragma unroll
      for (int r = 0; r < TM; ++r) a[r] = As[buf][kk][tx + r * (BM / TM)];
#pragma unroll
      for (int c = 0; c < TN; ++c) b[c] = Bs[buf][kk][ty + c * (BN / TN)];
#pragma unroll
      for (int r = 0; r < TM; ++r)
#pragma unroll
        for (int c = 0; c < TN; ++c) acc[r][c] = fma(a[r], b[c], acc[r][c]);
    }
    if (more) store(buf ^ 1);
    __syncthreads();
    buf ^= 1;
  }

#pragma unroll
  for (int c = 0; c < TN; ++c) {
    int gj = n0 + ty + c * (BN / TN);
    if (gj >= n) continue;
#pragma unroll
    for (int r = 0; r < TM; ++r) {
      int gi = m0 + tx + r * (BM / TM);
      if (gi >= m) continue;
      double *p = Cz + gi + gj * ldc;
      *p = (beta == 0.0) ? alpha * acc[r][c] : fma(alpha, acc[r][c], beta * *p);
    }
  }
}

template <int BM, int BN, int TM, int TN>
int launch_cfg(bool ta, bool tb, int m, int n, int k, int splits, int k_chunk, double alpha,
               const double *A, int lda, const double *B, int ldb, double beta, double *C,
               long long ldc, long long split_stride, cudaStream_t s) {
  dim3 grid(ceil_div(m, BM), ceil_div(n, BN), splits);
  if (grid.y > 65535 || grid.z > 65535) return PURL_ERR_UNSUPPORTED;
  double flops = 2.0 * m * n * (double)k;
  double bytes = 8.0 * ((double)m * k + (double)k * n + (double)m * n * (beta != 0.0 ? 2 : 1));
  LaunchScope ls(KC_GEMM_F64, s, flops, bytes, "gemm_f64_kernel");
#define PURL_GEMM_CASE(TA_, TB_)                                                               \
  if (ta == TA_ && tb == TB_) {                                                                \
    gemm_f64_kernel<BM, BN, TM, TN, TA_, TB_><<<grid, NT, 0, s>>>(                              \
        m, n, k, k_chunk, alpha, A, lda, B, ldb, beta, C, ldc, split_stride);                  \
  }
  PURL_GEMM_CASE(false, false)
  PURL_GEMM_CASE(true, false)
  PURL_GEMM_CASE(false, true)
  PURL_GEMM_CASE(true, true)
#undef PURL_GEMM_CASE
  return cudaGetLastError() == cudaSuccess ? PURL_OK : PURL_ERR_CUDA;
}

int launch_any(bool ta, bool tb, int m, int n, int k, int splits, int k_chunk, double alpha,
               const double *A, int lda, const double *B, int ldb, double beta, double *C,
               long long ldc, long long split_stride, cudaStream_t s) {
  if (m <= 32)
    return launch_cfg<32, 128, 4, 4>(ta, tb, m, n, k, splits, k_chunk, alpha, A, lda, B, ldb,
                                     beta, C, ldc, split_stride, s);
  if (n <= 32)
    return launch_cfg<128, 32, 4, 4>(ta, tb, m, n, k, splits, k_chunk, alpha, A, lda, B, ldb,
                                     beta, C, ldc, split_stride, s);
  return launch_cfg<64, 64, 4, 4>(ta, tb, m, n, k, splits, k_chunk, alpha, A, lda, B, ldb, beta,
                                  C, ldc, split_stride, s);
}

}  // namespace

// C = alpha op(A) op(B) + beta C (beta == 0: C is not read).
int gemm_f64(bool ta, bool tb, int m, int n, int k, double alpha, const double *A, int lda,
             const double *B, int ldb, double beta, double *C, int ldc, cudaStream_t s) {
  if (m == 0 || n == 0) return PURL_OK;
  if (k == 0) {
    // C = beta C
    return launch_any(ta, tb, m, n, 0, 1, 0, 0.0, A, lda, B, ldb, beta, C, ldc, 0, s);
  }
  return launch_any(ta, tb, m, n, k, 1, k, alpha, A, lda, B, ldb, beta, C, ldc, 0, s);
}

// Split-K partial products: P_z = op(A)(:, Kz) op(B)(Kz, :), z < splits, each
// m x n with leading dimension m, stored at P + z*m*n; K chunks of k_chunk.
int gemm_f64_splitk(bool ta, bool tb, int m, int n, int k, int splits, int k_chunk,
                    const double *A, int lda, const double *B, int ldb, double *P,
                    cudaStream_t s) {
  if (m == 0 || n == 0) return PURL_OK;
  return launch_any(ta, tb, m, n, k, splits, k_chunk, 1.0, A, lda, B, ldb, 0.0, P, m,
                    (long long)m * n, s);
}

// Split count for a reduction of length k producing an m x n output: enough
// tiles for every SM to hold a few, chunks no shorter than 256.
void choose_splits(int m, int n, int k, int num_sms, int *splits, int *k_chunk) {
  long long tiles = (long long)ceil_div(m, 64) * ceil_div(n, 64);
  long long want = (4LL * num_sms + tiles - 1) / tiles;
  long long maxs = (k + 255) / 256;
  long long sp = want < maxs ? want : maxs;
  if (sp < 1) sp = 1;
  if (sp > 64) sp = 64;
  int chunk = ceil_div(k, (int)sp);
  chunk = ceil_div(chunk, BK) * BK;
  *k_chunk = chunk > 0 ? chunk : BK;
  *splits = k > 0 ? ceil_div(k, *k_chunk) : 1;
}

}  // namespace purl
