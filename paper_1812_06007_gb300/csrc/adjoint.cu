// adjoint.cu -- hand-written reverse mode of the PowerURV map A -> (U, R, V)
// with the Gaussian G held fixed (FP64).
//
// Forward (Section 3):  Y_0 = G;  for i = 1..q:  P_i = A Y_{i-1},  (Z_i, S_i) = QR(P_i)  [reorth]
//                                               W_i = A^T Z_i,      (Y_i, T_i) = QR(W_i)  [reorth, i < q]
//                       (V, Z') = QR(Y_q)   (Eq. 5),   C = A V,   (U, R) = QR(C)   (Eq. 6)
// Without re-orthonormalisation Z_i = P_i and Y_i = W_i.
//
// Reverse sweep, given Ubar, Rbar, Vbar:
//   Cbar = qrbar(U, R; Ubar, Rbar);      Abar = Cbar V^T;   Vbar += A^T Cbar
//   Ybar_q = qrbar(V, Z'; Vbar, 0)
//   for i = q..1:  Wbar = Ybar_i (through qrbar(Y_i, T_i; ., 0) when re-orthonormalised and i < q)
//                  Abar += Z_i Wbar^T;  Zbar = A Wbar
//                  Pbar = Zbar (through qrbar(Z_i, S_i; ., 0) when re-orthonormalised)
//                  Abar += Pbar Y_{i-1}^T;  Ybar_{i-1} = A^T Pbar
// with the QR reverse rule (thin QR, full column rank, any fixed sign convention)
//   qrbar(Q, R; Qbar, Rbar) = (Qbar + Q copyltu(M)) R^{-T},   M = R Rbar^T - Qbar^T Q,
//   copyltu(M) = tril(M) + tril(M, -1)^T.
// The iterates are recomputed from A and the seed at the start of the call
// (nothing is kept from the forward call).
#include "common.cuh"
#include "profile.cuh"
#include "qr.cuh"
#include "qr_mixed.cuh"
#include "tc.cuh"

namespace purl {

int launch_gaussian(uint64_t seed, uint64_t stream_id, int rows, int cols, double *G, int ldg, cudaStream_t stream,
                    bool fp32_math = false);
int gemm_f64(bool ta, bool tb, int m, int n, int k, double alpha, const double *A, int lda, const double *B, int ldb,
             double beta, double *C, int ldc, cudaStream_t s);

namespace {

constexpr int kInvBlock = 32;

// Arithmetic of the products and QRs of one backward call: S = 0 is the FP64
// path (DFMA products, FP64 Householder QR); S > 0 runs every product on the
// exact tensor-core engine with S fixed-point slices per operand (8: FP64
// emulated, 4: FP32 precision) and every QR as the tensor-core QR of the same
// slice count, so the recomputed forward pass is the forward mode's own.
struct Eng {
  int S = 0;
  void *scr = nullptr;  // gemm_exact scratch
  size_t scr_bytes = 0;
  QrWork *qw = nullptr;
  QrMixWork *qm = nullptr;
};

int egemm(const Eng &e, bool ta, bool tb, int m, int n, int k, double alpha, const double *A, int lda,
          const double *B, int ldb, double beta, double *C, int ldc, cudaStream_t s) {
  if (e.S == 0) return gemm_f64(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, s);
  return gemm_exact(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, e.S, e.scr, e.scr_bytes, s);
}

// Inverses of the diagonal blocks of an upper-triangular n x n matrix: block
// b (one CTA of 256 threads) inverts rows/columns [32b, min(32b + 32, n)) by
// column back-substitution in shared memory and writes it into X.
__global__ void __launch_bounds__(256) tri_inv_diag_kernel(int n, const double *__restrict__ R, long long ldr,
                                                           double *X, long long ldx) {
  __shared__ double Rs[kInvBlock][kInvBlock + 1];
  __shared__ double Xs[kInvBlock][kInvBlock + 1];
  __shared__ double dinv[kInvBlock];
  const int o = blockIdx.x * kInvBlock;
  const int nb = min(kInvBlock, n - o);
  const double *Rb = R + o + (long long)o * ldr;
  for (int e = threadIdx.x; e < kInvBlock * kInvBlock; e += blockDim.x) {
    const int i = e % kInvBlock, j = e / kInvBlock;
    Rs[i][j] = (i < nb && j < nb && i <= j) ? Rb[i + j * ldr] : 0.0;
    Xs[i][j] = 0.0;
  }
  __syncthreads();
  if (threadIdx.x < nb) dinv[threadIdx.x] = 1.0 / Rs[threadIdx.x][threadIdx.x];
  __syncthreads();
  const int j = threadIdx.x;  // column j of the block inverse: R^{-1} e_j
  if (j < nb) {
    Xs[j][j] = dinv[j];
    for (int i = j - 1; i >= 0; --i) {
      double acc = 0.0;
      for (int l = i + 1; l <= j; ++l) acc = fma(Rs[i][l], Xs[l][j], acc);
      Xs[i][j] = -acc * dinv[i];
    }
  }
  __syncthreads();
  double *Xb = X + o + (long long)o * ldx;
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    const int i = e % nb, jj = e / nb;
    Xb[i + jj * ldx] = Xs[i][jj];
  }
}

// copyltu(M) = tril(M) + tril(M, -1)^T, in place into S (n x n).
__global__ void copyltu_kernel(int n, const double *__restrict__ M, long long ldm, double *S, long long lds) {
  const long long total = (long long)n * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e % n), j = (int)(e / n);
    S[i + j * lds] = (i >= j) ? M[i + j * ldm] : M[j + i * ldm];
  }
}

// Y = upper triangle of X (n x n), zeros below the diagonal.
__global__ void triu_copy_kernel(int n, const double *__restrict__ X, long long ldx, double *Y, long long ldy) {
  const long long total = (long long)n * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e % n), j = (int)(e / n);
    Y[i + j * ldy] = (i <= j) ? X[i + j * ldx] : 0.0;
  }
}

int grid_of(long long total) {
  const DeviceInfo *di = device_info();
  long long g = (total + 255) / 256;
  const long long cap = (long long)di->num_sms * 16;
  return (int)(g > cap ? cap : (g < 1 ? 1 : g));
}

// Off-diagonal blocks of X = R^{-1} once the 32-aligned diagonal blocks hold
// their inverses: X12 = -X11 R12 X22 on the split n1 (a multiple of 32), and
// X21 = 0.  Every sub-problem starts on a multiple of 32, so its leaves are
// exactly the diagonal blocks.  `tmp` holds n1 x n2 doubles.
int tri_inv_combine(const Eng &e, int n, const double *R, int ldr, double *X, int ldx, double *tmp, cudaStream_t s) {
  if (n <= kInvBlock) return PURL_OK;
  const int n1 = (n / 2 + kInvBlock - 1) / kInvBlock * kInvBlock, n2 = n - n1;
  PURL_TRY(tri_inv_combine(e, n1, R, ldr, X, ldx, tmp, s));
  PURL_TRY(tri_inv_combine(e, n2, R + n1 + (size_t)n1 * ldr, ldr, X + n1 + (size_t)n1 * ldx, ldx, tmp, s));
  PURL_TRY(egemm(e, false, false, n1, n2, n2, 1.0, R + (size_t)n1 * ldr, ldr, X + n1 + (size_t)n1 * ldx, ldx, 0.0,
                 tmp, n1, s));                                                               // R12 X22
  PURL_TRY(egemm(e, false, false, n1, n2, n1, -1.0, X, ldx, tmp, n1, 0.0, X + (size_t)n1 * ldx, ldx, s));
  // X21 = 0: a product with an empty reduction and beta = 0 writes zeros
  return gemm_f64(false, false, n2, n1, 0, 0.0, X, ldx, X, ldx, 0.0, X + n1, ldx, s);
}

// X = R^{-1} for an upper-triangular n x n R with nonzero diagonal.
int tri_inv_upper(const Eng &e, int n, const double *R, int ldr, double *X, int ldx, double *tmp, cudaStream_t s) {
  if (n <= 0) return PURL_OK;
  { LaunchScope ls(KC_OTHER, s, (double)n * kInvBlock * kInvBlock / 3.0, 16.0 * n * kInvBlock, "tri_inv_diag_kernel");
    tri_inv_diag_kernel<<<ceil_div(n, kInvBlock), 256, 0, s>>>(n, R, ldr, X, ldx); }
  PURL_CUDA_TRY(cudaGetLastError());
  return tri_inv_combine(e, n, R, ldr, X, ldx, tmp, s);
}

struct AdjWork {
  double *M = nullptr, *Sy = nullptr, *Rinv = nullptr, *tmp = nullptr;  // n x n each
  double *X = nullptr;  // m x n
};

// Abar_out (m x n) = qrbar(Q, R; Qbar, Rbar); Rbar may be null (zero).
int qr_backward(const Eng &e, int m, int n, const double *Q, int ldq, const double *R, int ldr, const double *Qbar,
                int ldqb, const double *Rbar, int ldrb, double *out, int ldo, AdjWork &w, cudaStream_t s) {
  // M = R Rbar^T - Qbar^T Q
  if (Rbar) PURL_TRY(egemm(e, false, true, n, n, n, 1.0, R, ldr, Rbar, ldrb, 0.0, w.M, n, s));
  PURL_TRY(egemm(e, true, false, n, n, m, -1.0, Qbar, ldqb, Q, ldq, Rbar ? 1.0 : 0.0, w.M, n, s));
  { LaunchScope ls(KC_OTHER, s, 0.0, 16.0 * n * (double)n, "copyltu_kernel");
    copyltu_kernel<<<grid_of((long long)n * n), 256, 0, s>>>(n, w.M, n, w.Sy, n); }
  PURL_CUDA_TRY(cudaGetLastError());
  // X = Qbar + Q copyltu(M)
  PURL_TRY(copy_matrix(m, n, Qbar, ldqb, w.X, m, s));
  PURL_TRY(egemm(e, false, false, m, n, n, 1.0, Q, ldq, w.Sy, n, 1.0, w.X, m, s));
  // out = X R^{-T}
  PURL_TRY(tri_inv_upper(e, n, R, ldr, w.Rinv, n, w.tmp, s));
  return egemm(e, false, true, m, n, n, 1.0, w.X, m, w.Rinv, n, 0.0, out, ldo, s);
}

// QR with explicit Q and diag(R) >= 0: F holds the matrix on entry.
int qr_full(const Eng &e, int rows, int n, double *F, int ldf, double *Q, int ldq, double *R, int ldr, cudaStream_t s) {
  if (e.S == 0) return qr_explicit(rows, n, F, ldf, Q, ldq, R, ldr, PURL_MODE_FP64, *e.qw, s);
  PURL_TRY(qr_mixed_factor(rows, n, F, ldf, *e.qm, s));
  PURL_TRY(qr_mixed_form_q(rows, n, F, ldf, *e.qm, Q, ldq, s));
  return qr_sign_fix(rows, n, F, ldf, Q, ldq, R, ldr, s);
}

struct BwdPlan {
  double *Yprev = nullptr;  // (q+1) Y iterates, n x n each (Y_0 = G, ..., Y_q)
  double *Z = nullptr;      // q Z_i (m x n), the (re-orthonormalised) A Y_{i-1}
  double *S = nullptr;      // q R factors of QR(P_i) (n x n)
  double *T = nullptr;      // q R factors of QR(W_i) (n x n), i < q
  double *Zp = nullptr;     // R factor of QR(Y_q) (n x n)
  double *Vr = nullptr, *Ur = nullptr, *Rr = nullptr;  // recomputed V, U, R
  double *F = nullptr;      // m x n scratch for factorizations and products
  double *Cb = nullptr, *Vb = nullptr, *Wb = nullptr, *Pb = nullptr, *Yb = nullptr;
  double *Rbu = nullptr;    // upper triangle of Rbar
  int *finite = nullptr;    // non-finite input flag
  AdjWork aw;
  QrWork qw;                // FP64 QR (S = 0)
  QrMixWork qm;             // tensor-core QR (S > 0)
  int slices = 0;           // slices of the tensor-core products (0: FP64)
  void *scr = nullptr;      // gemm_exact scratch
  size_t scr_bytes = 0;
};

// Slices of the tensor-core backward modes (0 for the FP64 mode, -1 for an
// unsupported mode).
int bwd_slices(int mode) {
  if (mode == PURL_MODE_FP64) return 0;
  if (mode == PURL_MODE_FP64_EMU) return kTcxEmuSlices;
  if (mode == PURL_MODE_FP32) return 4;
  return -1;
}

int bwd_plan(Arena &ar, int m, int n, int q, int mode, BwdPlan *p) {
  const size_t nn = (size_t)n * n, mn = (size_t)m * n;
  p->finite = ar.take<int>(1);
  p->Yprev = ar.take<double>(nn * (q + 1));
  p->Z = ar.take<double>(mn * (q > 0 ? q : 1));
  p->S = ar.take<double>(nn * (q > 0 ? q : 1));
  p->T = ar.take<double>(nn * (q > 0 ? q : 1));
  p->Zp = ar.take<double>(nn);
  p->Vr = ar.take<double>(nn);
  p->Ur = ar.take<double>(mn);
  p->Rr = ar.take<double>(nn);
  p->F = ar.take<double>(mn);
  p->Cb = ar.take<double>(mn);
  p->Vb = ar.take<double>(nn);
  p->Wb = ar.take<double>(nn);
  p->Pb = ar.take<double>(mn);
  p->Yb = ar.take<double>(nn);
  p->Rbu = ar.take<double>(nn);
  p->aw.M = ar.take<double>(nn);
  p->aw.Sy = ar.take<double>(nn);
  p->aw.Rinv = ar.take<double>(nn);
  p->aw.tmp = ar.take<double>(nn);
  p->aw.X = ar.take<double>(mn);
  p->slices = bwd_slices(mode);
  if (p->slices < 0) return PURL_ERR_UNSUPPORTED;
  if (p->slices == 0) return qr_plan(ar, m, n, PURL_MODE_FP64, &p->qw);
  // the largest products: m x n x n (A Y, A V, ...) and n x n x m (A^T Z, ...)
  const size_t b1 = gemm_exact_bytes(m, n, n, p->slices), b2 = gemm_exact_bytes(n, n, m, p->slices);
  p->scr_bytes = b1 > b2 ? b1 : b2;
  p->scr = ar.take<char>(p->scr_bytes);
  PURL_TRY(qr_mixed_plan(ar, m, n, p->slices, &p->qm));
  p->qw = p->qm.base;
  return PURL_OK;
}

int urv_backward_run(int m, int n, const double *A, int lda, int q, int reorth, uint64_t seed, const double *Ubar,
                     int ldub, const double *Rbar, int ldrb, const double *Vbar, int ldvb, double *Abar, int ldab,
                     BwdPlan &p, cudaStream_t s) {
  const size_t nn = (size_t)n * n, mn = (size_t)m * n;
  Eng e;
  e.S = p.slices;
  e.scr = p.scr;
  e.scr_bytes = p.scr_bytes;
  e.qw = &p.qw;
  e.qm = &p.qm;
  // ---- recompute the forward pass, keeping every iterate ----
  PURL_TRY(launch_gaussian(seed, 0, n, n, p.Yprev, n, s));
  for (int i = 1; i <= q; ++i) {
    double *Yi1 = p.Yprev + (i - 1) * nn, *Yi = p.Yprev + i * nn;
    double *Zi = p.Z + (i - 1) * mn, *Si = p.S + (i - 1) * nn, *Ti = p.T + (i - 1) * nn;
    PURL_TRY(egemm(e, false, false, m, n, n, 1.0, A, lda, Yi1, n, 0.0, p.F, m, s));  // P_i
    if (reorth) PURL_TRY(qr_full(e, m, n, p.F, m, Zi, m, Si, n, s));
    else PURL_TRY(copy_matrix(m, n, p.F, m, Zi, m, s));
    PURL_TRY(egemm(e, true, false, n, n, m, 1.0, A, lda, Zi, m, 0.0, p.F, n, s));  // W_i
    if (reorth && i < q) PURL_TRY(qr_full(e, n, n, p.F, n, Yi, n, Ti, n, s));
    else PURL_TRY(copy_matrix(n, n, p.F, n, Yi, n, s));
  }
  PURL_TRY(copy_matrix(n, n, p.Yprev + q * nn, n, p.F, n, s));
  PURL_TRY(qr_full(e, n, n, p.F, n, p.Vr, n, p.Zp, n, s));                           // Eq. 5
  PURL_TRY(egemm(e, false, false, m, n, n, 1.0, A, lda, p.Vr, n, 0.0, p.F, m, s));     // C = A V
  PURL_TRY(qr_full(e, m, n, p.F, m, p.Ur, m, p.Rr, n, s));                           // Eq. 6
  // ---- reverse sweep ----
  // R's strictly lower triangle is the constant zero: its cotangent is dropped.
  { LaunchScope ls(KC_OTHER, s, 0.0, 16.0 * n * (double)n, "triu_copy_kernel");
    triu_copy_kernel<<<grid_of((long long)n * n), 256, 0, s>>>(n, Rbar, ldrb, p.Rbu, n); }
  PURL_CUDA_TRY(cudaGetLastError());
  PURL_TRY(qr_backward(e, m, n, p.Ur, m, p.Rr, n, Ubar, ldub, p.Rbu, n, p.Cb, m, p.aw, s));   // Cbar
  PURL_TRY(egemm(e, false, true, m, n, n, 1.0, p.Cb, m, p.Vr, n, 0.0, Abar, ldab, s));        // Abar = Cbar V^T
  PURL_TRY(copy_matrix(n, n, Vbar, ldvb, p.Vb, n, s));
  PURL_TRY(egemm(e, true, false, n, n, m, 1.0, A, lda, p.Cb, m, 1.0, p.Vb, n, s));             // Vbar += A^T Cbar
  PURL_TRY(qr_backward(e, n, n, p.Vr, n, p.Zp, n, p.Vb, n, nullptr, 0, p.Yb, n, p.aw, s));       // Ybar_q
  for (int i = q; i >= 1; --i) {
    double *Yi1 = p.Yprev + (i - 1) * nn, *Yi = p.Yprev + i * nn;
    double *Zi = p.Z + (i - 1) * mn, *Si = p.S + (i - 1) * nn, *Ti = p.T + (i - 1) * nn;
    if (reorth && i < q) PURL_TRY(qr_backward(e, n, n, Yi, n, Ti, n, p.Yb, n, nullptr, 0, p.Wb, n, p.aw, s));
    else PURL_TRY(copy_matrix(n, n, p.Yb, n, p.Wb, n, s));
    PURL_TRY(egemm(e, false, true, m, n, n, 1.0, Zi, m, p.Wb, n, 1.0, Abar, ldab, s));   // Abar += Z Wbar^T
    PURL_TRY(egemm(e, false, false, m, n, n, 1.0, A, lda, p.Wb, n, 0.0, p.F, m, s));     // Zbar = A Wbar
    if (reorth) PURL_TRY(qr_backward(e, m, n, Zi, m, Si, n, p.F, m, nullptr, 0, p.Pb, m, p.aw, s));
    else PURL_TRY(copy_matrix(m, n, p.F, m, p.Pb, m, s));
    PURL_TRY(egemm(e, false, true, m, n, n, 1.0, p.Pb, m, Yi1, n, 1.0, Abar, ldab, s));  // Abar += Pbar Y^T
    PURL_TRY(egemm(e, true, false, n, n, m, 1.0, A, lda, p.Pb, m, 0.0, p.Yb, n, s));     // Ybar_{i-1}
  }
  return PURL_OK;
}

}  // namespace

}  // namespace purl

using namespace purl;

extern "C" {

size_t purl_urv_backward_ex_workspace_bytes(int m, int n, int q, int mode) {
  if (m < 0 || n < 0 || m < n || q < 0 || bwd_slices(mode) < 0) return 0;
  if (mode == PURL_MODE_FP64_EMU && m > (1 << 20)) return 0;
  if (!device_info()) return 0;
  Arena ar;
  BwdPlan p;
  if (bwd_plan(ar, m, n, q, mode, &p) != PURL_OK) return 0;
  return ar.used;
}

size_t purl_urv_backward_workspace_bytes(int m, int n, int q) {
  return purl_urv_backward_ex_workspace_bytes(m, n, q, PURL_MODE_FP64);
}

int purl_urv_backward_ex(int m, int n, const double *A, int lda, int q, int reorth, uint64_t seed, const double *Ubar,
                         int ldub, const double *Rbar, int ldrb, const double *Vbar, int ldvb, double *Abar, int ldab,
                         int mode, void *workspace, size_t workspace_bytes, cudaStream_t stream) {
  if (m < 0) return -1;
  if (n < 0) return -2;
  if (m < n) return PURL_ERR_SHAPE;
  if (!A && (long long)m * n > 0) return -3;
  if (lda < (m > 1 ? m : 1)) return -4;
  if (q < 0) return -5;
  if (!Ubar && (long long)m * n > 0) return -8;
  if (ldub < (m > 1 ? m : 1)) return -9;
  if (!Rbar && n > 0) return -10;
  if (ldrb < (n > 1 ? n : 1)) return -11;
  if (!Vbar && n > 0) return -12;
  if (ldvb < (n > 1 ? n : 1)) return -13;
  if (!Abar && (long long)m * n > 0) return -14;
  if (ldab < (m > 1 ? m : 1)) return -15;
  if (bwd_slices(mode) < 0) return -16;
  if (mode == PURL_MODE_FP64_EMU && m > (1 << 20)) return PURL_ERR_UNSUPPORTED;
  if ((long long)m * n == 0) return PURL_OK;
  if (!device_info()) return PURL_ERR_CUDA;
  const size_t need = purl_urv_backward_ex_workspace_bytes(m, n, q, mode);
  void *ptr = workspace;
  bool owned = false;
  if (!ptr) {
    if (cudaMallocAsync(&ptr, need, stream) != cudaSuccess) return PURL_ERR_NOMEM;
    owned = true;
  } else if (workspace_bytes < need || ((uintptr_t)workspace & 255) != 0) {
    return PURL_ERR_NOMEM;
  }
  Arena ar;
  ar.base = static_cast<char *>(ptr);
  ar.size = owned ? need : workspace_bytes;
  BwdPlan p;
  int st = bwd_plan(ar, m, n, q, mode, &p);
  if (st == PURL_OK && !ar.ok) st = PURL_ERR_NOMEM;
  if (st == PURL_OK) st = finite_check(m, n, A, lda, p.finite, stream);
  if (st == PURL_OK)
    st = urv_backward_run(m, n, A, lda, q, reorth, seed, Ubar, ldub, Rbar, ldrb, Vbar, ldvb, Abar, ldab, p, stream);
  if (st == PURL_OK) st = finite_poison(p.finite, m, n, Abar, ldab, stream);
  if (owned) cudaFreeAsync(ptr, stream);
  return st;
}

int purl_urv_backward(int m, int n, const double *A, int lda, int q, int reorth, uint64_t seed, const double *Ubar,
                      int ldub, const double *Rbar, int ldrb, const double *Vbar, int ldvb, double *Abar, int ldab,
                      void *workspace, size_t workspace_bytes, cudaStream_t stream) {
  return purl_urv_backward_ex(m, n, A, lda, q, reorth, seed, Ubar, ldub, Rbar, ldrb, Vbar, ldvb, Abar, ldab,
                              PURL_MODE_FP64, workspace, workspace_bytes, stream);
}

}  // extern "C"
