/*
 * purl_oracle.c -- FP64 CPU oracle for the PowerURV factorization
 * (Gopal & Martinsson, "The PowerURV algorithm for computing rank-revealing
 * full factorizations", arXiv:1812.06007).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * GPU library is checked against.  Only the test-suite, the smoke check and
 * the CPU-baseline leg of the benchmark may load it.  It shares no code,
 * header, table or helper with the CUDA library, and the CUDA library never
 * calls it.
 *
 * Everything is column-major double precision.  No blocking, no fusion: every
 * routine is the textbook definition written out so that it can be checked
 * against the paper by eye.  Loops over independent output columns are
 * OpenMP-parallel; that changes no arithmetic (each column is computed by one
 * thread in a fixed order).
 *
 * Built with -ffp-contract=off so that x86-64 and AArch64 produce the same
 * bits (no fused multiply-add is formed behind our back).
 *
 * Paper map:
 *   orc_gaussian          Section 3: "Gaussian random matrix G in R^{n x n}".
 *                         The paper names no generator; this oracle uses
 *                         Philox4x64-10 (Salmon et al., SC'11) + Box-Muller.
 *   orc_householder_qr    Section 2.2: unpivoted QR by Householder reflectors.
 *   orc_form_q            explicit orthonormal factor of that QR.
 *   orc_qr_explicit       QR with the diagonal of R made nonnegative (the
 *                         sign convention of the footnote in Section 2.2).
 *   orc_urv_factor        Section 3, Eq. (5) (A*A)^q G = V Z and Eq. (6)
 *                         A V = U R, with re-orthonormalisation after each
 *                         application of A or A* (Section 3, third paragraph).
 *   orc_truncate          Section 5: A_k = U(:,1:k) R(1:k,:) V*.
 *   orc_jacobi_svd        one-sided Jacobi SVD (Hestenes), used by the tests
 *                         as a brute-force reference on tiny inputs.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define IDX(i, j, ld) ((size_t)(i) + (size_t)(j) * (size_t)(ld))

/* ------------------------------------------------------------------------ */
/* Philox4x64-10 counter-based generator (Salmon, Moraes, Dror, Shaw,       */
/* "Parallel random numbers: as easy as 1, 2, 3", SC'11).  One round maps   */
/* (c0,c1,c2,c3) with key (k0,k1) through two 64x64->128 multiplications;  */
/* the key is bumped by the Weyl constants between rounds.                  */
/* ------------------------------------------------------------------------ */
static const uint64_t PHILOX_M0 = 0xD2E7470EE14C6C93ULL;
static const uint64_t PHILOX_M1 = 0xCA5A826395121157ULL;
static const uint64_t PHILOX_W0 = 0x9E3779B97F4A7C15ULL;
static const uint64_t PHILOX_W1 = 0xBB67AE8584CAA73BULL;

static void mul_hilo64(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo) {
  /* schoolbook 64x64 -> 128 with 32-bit halves (no compiler extensions) */
  uint64_t a0 = a & 0xffffffffULL, a1 = a >> 32;
  uint64_t b0 = b & 0xffffffffULL, b1 = b >> 32;
  uint64_t p00 = a0 * b0, p01 = a0 * b1, p10 = a1 * b0, p11 = a1 * b1;
  uint64_t mid = (p00 >> 32) + (p01 & 0xffffffffULL) + (p10 & 0xffffffffULL);
  *lo = (p00 & 0xffffffffULL) | (mid << 32);
  *hi = p11 + (p01 >> 32) + (p10 >> 32) + (mid >> 32);
}

void orc_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]) {
  uint64_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint64_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    uint64_t hi0, lo0, hi1, lo1;
    mul_hilo64(PHILOX_M0, c0, &hi0, &lo0);
    mul_hilo64(PHILOX_M1, c2, &hi1, &lo1);
    uint64_t n0 = hi1 ^ c1 ^ k0;
    uint64_t n1 = lo1;
    uint64_t n2 = hi0 ^ c3 ^ k1;
    uint64_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    if (r < 9) { k0 += PHILOX_W0; k1 += PHILOX_W1; }
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* 64 random bits -> uniform in the open interval (0,1): the top 53 bits,
 * centred in their cell, so 0 and 1 are never produced. */
static double u53(uint64_t x) { return ((double)(x >> 11) + 0.5) * 0x1.0p-53; }

/* Uniform stream: element e (column-major linear index over rows x cols) of
 * the matrix drawn with (seed, stream) is word e%4 of block e/4, where block
 * b is Philox4x64-10 with counter (b,0,0,0) and key (seed, stream). */
void orc_uniforms(uint64_t seed, uint64_t stream, int64_t count, double *u) {
  const uint64_t key[2] = {seed, stream};
  int64_t nblk = (count + 3) / 4;
#pragma omp parallel for schedule(static)
  for (int64_t b = 0; b < nblk; ++b) {
    uint64_t ctr[4] = {(uint64_t)b, 0, 0, 0}, w[4];
    orc_philox4x64_10(ctr, key, w);
    for (int t = 0; t < 4; ++t)
      if (4 * b + t < count) u[4 * b + t] = u53(w[t]);
  }
}

/* Standard normal matrix G (rows x cols, column-major, leading dim ldg).
 * Block b gives uniforms (u0,u1,u2,u3); Box-Muller turns (u0,u1) into the
 * normals at linear positions 4b, 4b+1 and (u2,u3) into 4b+2, 4b+3:
 *   z_even = sqrt(-2 ln u_even) cos(2 pi u_odd),
 *   z_odd  = sqrt(-2 ln u_even) sin(2 pi u_odd). */
void orc_gaussian(uint64_t seed, uint64_t stream, int64_t rows, int64_t cols,
                  double *G, int64_t ldg) {
  const uint64_t key[2] = {seed, stream};
  const double two_pi = 6.283185307179586476925286766559;
  int64_t count = rows * cols, nblk = (count + 3) / 4;
#pragma omp parallel for schedule(static)
  for (int64_t b = 0; b < nblk; ++b) {
    uint64_t ctr[4] = {(uint64_t)b, 0, 0, 0}, w[4];
    orc_philox4x64_10(ctr, key, w);
    double z[4];
    for (int p = 0; p < 2; ++p) {
      double u1 = u53(w[2 * p]), u2 = u53(w[2 * p + 1]);
      double r = sqrt(-2.0 * log(u1));
      z[2 * p] = r * cos(two_pi * u2);
      z[2 * p + 1] = r * sin(two_pi * u2);
    }
    for (int t = 0; t < 4; ++t) {
      int64_t e = 4 * b + t;
      if (e < count) G[IDX(e % rows, e / rows, ldg)] = z[t];
    }
  }
}

/* ------------------------------------------------------------------------ */
/* GEMM by definition: C = alpha * op(A) op(B) + beta * C,                  */
/* op(X) = X ('N') or X^T ('T').  Each C(i,j) is one dot product summed in  */
/* increasing l.                                                            */
/* ------------------------------------------------------------------------ */
void orc_gemm(char ta, char tb, int64_t m, int64_t n, int64_t k, double alpha,
              const double *A, int64_t lda, const double *B, int64_t ldb,
              double beta, double *C, int64_t ldc) {
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < n; ++j) {
    for (int64_t i = 0; i < m; ++i) {
      double s = 0.0;
      for (int64_t l = 0; l < k; ++l) {
        double a = (ta == 'N') ? A[IDX(i, l, lda)] : A[IDX(l, i, lda)];
        double b = (tb == 'N') ? B[IDX(l, j, ldb)] : B[IDX(j, l, ldb)];
        s += a * b;
      }
      C[IDX(i, j, ldc)] = (beta == 0.0) ? alpha * s : alpha * s + beta * C[IDX(i, j, ldc)];
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Unpivoted Householder QR, one column at a time (Section 2.2).            */
/* For column j, x = A(j:m-1, j).  The reflector H = I - tau v v^T with     */
/* v(0) = 1 maps x to beta e_1, beta = -sign(x0) ||x|| (sign(0) = +1).      */
/* If x(1:) is zero the column is already reduced: tau = 0, beta = x0.     */
/* On exit R is on and above the diagonal, v(1:) below it, tau[j] beside.  */
/* ------------------------------------------------------------------------ */
void orc_householder_qr(int64_t m, int64_t n, double *A, int64_t lda, double *tau) {
  int64_t kmax = (m < n) ? m : n;
  for (int64_t j = 0; j < kmax; ++j) {
    double x0 = A[IDX(j, j, lda)];
    double sigma = 0.0;
    for (int64_t i = j + 1; i < m; ++i) sigma += A[IDX(i, j, lda)] * A[IDX(i, j, lda)];
    if (sigma == 0.0) {
      tau[j] = 0.0;
      continue;
    }
    double norm = sqrt(x0 * x0 + sigma);
    double beta = (x0 >= 0.0) ? -norm : norm;
    double v0 = x0 - beta;
    tau[j] = (beta - x0) / beta;
    for (int64_t i = j + 1; i < m; ++i) A[IDX(i, j, lda)] /= v0;
    A[IDX(j, j, lda)] = beta;
    /* apply H to the trailing columns: a <- a - tau v (v^T a) */
    const double tj = tau[j];
#pragma omp parallel for schedule(static)
    for (int64_t c = j + 1; c < n; ++c) {
      double w = A[IDX(j, c, lda)];
      for (int64_t i = j + 1; i < m; ++i) w += A[IDX(i, j, lda)] * A[IDX(i, c, lda)];
      w *= tj;
      A[IDX(j, c, lda)] -= w;
      for (int64_t i = j + 1; i < m; ++i) A[IDX(i, c, lda)] -= w * A[IDX(i, j, lda)];
    }
  }
}

/* Explicit Q (m x n) = H_0 H_1 ... H_{n-1} applied to the first n columns of
 * the identity, accumulated from the last reflector to the first. */
void orc_form_q(int64_t m, int64_t n, const double *F, int64_t ldf, const double *tau,
                double *Q, int64_t ldq) {
  for (int64_t c = 0; c < n; ++c)
    for (int64_t i = 0; i < m; ++i) Q[IDX(i, c, ldq)] = (i == c) ? 1.0 : 0.0;
  for (int64_t j = n - 1; j >= 0; --j) {
    const double tj = tau[j];
    if (tj == 0.0) continue;
#pragma omp parallel for schedule(static)
    for (int64_t c = j; c < n; ++c) {
      double w = Q[IDX(j, c, ldq)];
      for (int64_t i = j + 1; i < m; ++i) w += F[IDX(i, j, ldf)] * Q[IDX(i, c, ldq)];
      w *= tj;
      Q[IDX(j, c, ldq)] -= w;
      for (int64_t i = j + 1; i < m; ++i) Q[IDX(i, c, ldq)] -= w * F[IDX(i, j, ldf)];
    }
  }
}

/* QR with diag(R) >= 0: M (m x n, m >= n) = Q R.  Q (m x n) and R (n x n,
 * zeros below the diagonal) are written; either may be NULL.  M is not
 * modified.  The sign of row j of R and column j of Q is flipped when
 * R(j,j) < 0, which makes the factorization unique for full column rank. */
int orc_qr_explicit(int64_t m, int64_t n, const double *M, int64_t ldm, double *Q,
                    int64_t ldq, double *R, int64_t ldr) {
  if (m < n || n < 0) return -1;
  double *F = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1) * (size_t)(n > 0 ? n : 1));
  double *tau = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  if (!F || !tau) { free(F); free(tau); return -4; }
  for (int64_t c = 0; c < n; ++c) memcpy(&F[IDX(0, c, m)], &M[IDX(0, c, ldm)], sizeof(double) * (size_t)m);
  orc_householder_qr(m, n, F, m, tau);
  if (Q) {
    orc_form_q(m, n, F, m, tau, Q, ldq);
    for (int64_t j = 0; j < n; ++j)
      if (F[IDX(j, j, m)] < 0.0)
        for (int64_t i = 0; i < m; ++i) Q[IDX(i, j, ldq)] = -Q[IDX(i, j, ldq)];
  }
  if (R) {
    for (int64_t c = 0; c < n; ++c)
      for (int64_t i = 0; i < n; ++i) R[IDX(i, c, ldr)] = (i <= c) ? F[IDX(i, c, m)] : 0.0;
    for (int64_t j = 0; j < n; ++j)
      if (F[IDX(j, j, m)] < 0.0)
        for (int64_t c = j; c < n; ++c) R[IDX(j, c, ldr)] = -R[IDX(j, c, ldr)];
  }
  free(F);
  free(tau);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* PowerURV (Section 3).                                                    */
/*   Y_0 = G (n x n);  for i = 1..q:  Z = A Y_{i-1}   [Q(Z) if reorth]      */
/*                                    Y_i = A^T Z     [Q(Y_i) if reorth     */
/*                                                     and i < q]           */
/*   Y_q = V Z  (Eq. 5, QR with diag(Z) >= 0; Z is discarded)               */
/*   A V = U R  (Eq. 6, QR with diag(R) >= 0)                               */
/* Q(.) is the orthonormal factor of the QR above.  The last Y needs no     */
/* separate re-orthonormalisation: the QR of Eq. 5 is it.  q = 0 is the     */
/* DDH-URV algorithm of Section 2.2 (V = Q(G)).                             */
/* G is taken as an input (caller draws it with orc_gaussian) so that the   */
/* tests can also feed perturbed copies.                                    */
/* ------------------------------------------------------------------------ */
int orc_urv_factor_g(int64_t m, int64_t n, const double *A, int64_t lda, const double *G,
                     int64_t ldg, int q, int reorth, double *U, int64_t ldu, double *R,
                     int64_t ldr, double *V, int64_t ldv) {
  if (m < n || n < 0 || q < 0) return -1;
  size_t nn = (size_t)(n > 0 ? n : 1) * (size_t)(n > 0 ? n : 1);
  size_t mn = (size_t)(m > 0 ? m : 1) * (size_t)(n > 0 ? n : 1);
  double *Y = (double *)malloc(sizeof(double) * nn);
  double *Z = (double *)malloc(sizeof(double) * mn);
  if (!Y || !Z) { free(Y); free(Z); return -4; }
  for (int64_t c = 0; c < n; ++c) memcpy(&Y[IDX(0, c, n)], &G[IDX(0, c, ldg)], sizeof(double) * (size_t)n);
  for (int i = 1; i <= q; ++i) {
    orc_gemm('N', 'N', m, n, n, 1.0, A, lda, Y, n, 0.0, Z, m);        /* Z = A Y */
    if (reorth) orc_qr_explicit(m, n, Z, m, Z, m, NULL, 0);            /* Z = Q(Z) */
    orc_gemm('T', 'N', n, n, m, 1.0, A, lda, Z, m, 0.0, Y, n);        /* Y = A^T Z */
    if (reorth && i < q) orc_qr_explicit(n, n, Y, n, Y, n, NULL, 0);   /* Y = Q(Y) */
  }
  orc_qr_explicit(n, n, Y, n, V, ldv, NULL, 0);                        /* Eq. 5 */
  orc_gemm('N', 'N', m, n, n, 1.0, A, lda, V, ldv, 0.0, Z, m);        /* A V */
  orc_qr_explicit(m, n, Z, m, U, ldu, R, ldr);                         /* Eq. 6 */
  free(Y);
  free(Z);
  return 0;
}

int orc_urv_factor(int64_t m, int64_t n, const double *A, int64_t lda, int q, int reorth,
                   uint64_t seed, double *U, int64_t ldu, double *R, int64_t ldr, double *V,
                   int64_t ldv) {
  if (m < n || n < 0 || q < 0) return -1;
  double *G = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1) * (size_t)(n > 0 ? n : 1));
  if (!G) return -4;
  orc_gaussian(seed, 0, n, n, G, n);
  int rc = orc_urv_factor_g(m, n, A, lda, G, n, q, reorth, U, ldu, R, ldr, V, ldv);
  free(G);
  return rc;
}

/* Rank-k truncation (Section 5): A_k = U(:,1:k) R(1:k,:) V^T. */
int orc_truncate(int64_t m, int64_t n, int64_t k, const double *U, int64_t ldu,
                 const double *R, int64_t ldr, const double *V, int64_t ldv, double *Ak,
                 int64_t ldak) {
  if (k < 0 || k > n || m < n) return -1;
  double *W = (double *)malloc(sizeof(double) * (size_t)(k > 0 ? k : 1) * (size_t)(n > 0 ? n : 1));
  if (!W) return -4;
  orc_gemm('N', 'T', k, n, n, 1.0, R, ldr, V, ldv, 0.0, W, (k > 0 ? k : 1)); /* R(1:k,:) V^T */
  orc_gemm('N', 'N', m, n, k, 1.0, U, ldu, W, (k > 0 ? k : 1), 0.0, Ak, ldak);
  free(W);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* One-sided Jacobi SVD (Hestenes): rotate column pairs of a copy of A     */
/* until every pair is numerically orthogonal; the singular values are the */
/* column norms.  Written for the tests' brute-force checks on tiny inputs */
/* (sweeps are capped).  Values are returned sorted in decreasing order.   */
/* ------------------------------------------------------------------------ */
int orc_jacobi_svd(int64_t m, int64_t n, const double *A, int64_t lda, double *sigma) {
  double *W = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1) * (size_t)(n > 0 ? n : 1));
  if (!W) return -4;
  for (int64_t c = 0; c < n; ++c) memcpy(&W[IDX(0, c, m)], &A[IDX(0, c, lda)], sizeof(double) * (size_t)m);
  int converged = 0;
  for (int sweep = 0; sweep < 60 && !converged; ++sweep) {
    converged = 1;
    for (int64_t p = 0; p < n - 1; ++p) {
      for (int64_t r = p + 1; r < n; ++r) {
        double alpha = 0.0, beta = 0.0, gamma = 0.0;
        for (int64_t i = 0; i < m; ++i) {
          double wp = W[IDX(i, p, m)], wr = W[IDX(i, r, m)];
          alpha += wp * wp;
          beta += wr * wr;
          gamma += wp * wr;
        }
        if (gamma == 0.0 || fabs(gamma) <= 1e-15 * sqrt(alpha * beta)) continue;
        converged = 0;
        double zeta = (beta - alpha) / (2.0 * gamma);
        double t = ((zeta >= 0.0) ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        double cs = 1.0 / sqrt(1.0 + t * t), sn = cs * t;
        for (int64_t i = 0; i < m; ++i) {
          double wp = W[IDX(i, p, m)], wr = W[IDX(i, r, m)];
          W[IDX(i, p, m)] = cs * wp - sn * wr;
          W[IDX(i, r, m)] = sn * wp + cs * wr;
        }
      }
    }
  }
  for (int64_t c = 0; c < n; ++c) {
    double s = 0.0;
    for (int64_t i = 0; i < m; ++i) s += W[IDX(i, c, m)] * W[IDX(i, c, m)];
    sigma[c] = sqrt(s);
  }
  /* insertion sort, decreasing */
  for (int64_t a = 1; a < n; ++a) {
    double v = sigma[a];
    int64_t b = a - 1;
    while (b >= 0 && sigma[b] < v) { sigma[b + 1] = sigma[b]; --b; }
    sigma[b + 1] = v;
  }
  free(W);
  return converged ? 0 : 1;
}
