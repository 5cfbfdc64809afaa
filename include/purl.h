/*
 * purl.h -- C ABI of libpurl: the PowerURV rank-revealing factorization
 * (Gopal & Martinsson, arXiv:1812.06007) on one NVIDIA GB300 (sm_103a).
 *
 * Given A (m x n, m >= n) the library computes A = U R V^T with
 *   U  m x n, orthonormal columns;  R  n x n upper triangular, diag(R) >= 0;
 *   V  n x n orthogonal,
 * by the PowerURV algorithm of Section 3 of the paper:
 *   1. draw G (n x n) with i.i.d. N(0,1) entries from `seed`;
 *   2. q power steps Y <- A^T (A Y), starting from Y = G, re-orthonormalising
 *      after every product with A or A^T when `reorth` != 0 (Section 3, third
 *      paragraph); Eq. (5): (A^T A)^q G = V Z by an unpivoted Householder QR;
 *   3. Eq. (6): A V = U R by a second unpivoted Householder QR.
 * With q = 0 this is the DDH-URV algorithm (Section 2.2).
 *
 * Conventions shared by every entry point:
 *   - All matrices are column-major FP64 in DEVICE memory with a leading
 *     dimension ld >= rows (ld >= 1 when rows == 0).  The caller owns every
 *     buffer; the library never frees or keeps a caller pointer past the call.
 *   - Outputs must not alias inputs or each other.
 *   - Work is enqueued on `stream` (0 = legacy default stream) and the call
 *     returns without synchronising.  The return value reports argument and
 *     launch errors only.  Errors that can only be seen on the device (a
 *     bounded wait that ran out) are recorded in a per-device status word read
 *     with purl_device_status().
 *   - Argument errors return -i for the i-th argument (LAPACK style, counting
 *     from 1), PURL_ERR_SHAPE when m < n (factor A^T instead: Section 1 notes
 *     that a URV of A^T gives a ULV of A and vice versa).
 *   - Non-finite input: every entry point that takes A (factor, ULV, QR,
 *     RSVD, backward) scans it on the device first.  If any entry is NaN or
 *     infinite, PURL_ERR_NONFINITE is recorded in the device status word
 *     (purl_device_status) and every output of the call is overwritten with
 *     NaN, in every mode (the tensor-core modes' fixed-point slicing would
 *     otherwise turn such an entry into finite but meaningless results).  The
 *     scan reads A once (8 m n bytes).
 *   - Every routine is deterministic: the same inputs on the same GPU give the
 *     same bits.
 */
#ifndef PURL_H_
#define PURL_H_

#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define PURL_OK 0
#define PURL_ERR_SHAPE (-100)  /* m < n */
#define PURL_ERR_NONFINITE 1   /* A held a NaN or an infinity (device status word) */
#define PURL_ERR_TIMEOUT 2     /* a bounded device-side wait ran out */
#define PURL_ERR_CUDA 3        /* a CUDA runtime call failed */
#define PURL_ERR_NOMEM 4       /* workspace allocation failed or too small */
#define PURL_ERR_UNSUPPORTED 5 /* this GPU / build cannot run the request */

/* precision modes for purl_urv_factor_ex / purl_qr */
#define PURL_MODE_FP64 0
/* FP32 precision on the tensor cores: the FP64 mode's algorithm with every
 * product (A Y, A^T Z, A V, every QR trailing update, Gram matrix and Q
 * formation) an exact-accumulation product of 4 fixed-point BF16 slices per
 * operand (every operand row carried to 2^-32 of its scale, so entries down to
 * 2^-8 of their row's largest keep FP32's 24 bits); Householder panels and T
 * factors in FP64.  The precision the
 * FP32 entry points (purl_urv_factor_f32, purl_urv_backward_f32) use by
 * default. */
#define PURL_MODE_FP32 1
/* Power-step products A Y and A^T Z on BF16 tensor cores with FP32
 * accumulation (one plain BF16 slice per operand, scaled as described under
 * PURL_MODE_MIXED_FP16); A V, every QR trailing update,
 * T factor and Q formation as exact-accumulation products of fixed-point BF16
 * slices (2 slices in the power iteration's re-orthonormalisations, 4 in the
 * QRs of Eqs. (5)-(6) and in A V); Householder panels in FP64. */
#define PURL_MODE_MIXED_BF16 2
/* As PURL_MODE_MIXED_BF16 with the power-step products A Y and A^T Z on FP16
 * operands (11-bit significands instead of BF16's 8, FP32 accumulation).  In
 * both mixed modes every power-step operand is sliced as 2^s X, the power of
 * two chosen on the device from X's largest entry (FP16 holds magnitudes up
 * to 65504 only); the scale is never undone because each product is
 * orthonormalised next, or only its span enters the QR of Eq. (5).  purl_qr
 * treats this mode as PURL_MODE_MIXED_BF16 (a QR has no power steps). */
#define PURL_MODE_MIXED_FP16 3
/* FP64 emulated on the BF16 tensor cores: the FP64 mode's algorithm with
 * every product (A Y, A^T Z, A V, every QR trailing update, Gram matrix and
 * Q formation) an exact-accumulation product of 8 fixed-point BF16 slices per
 * operand (every operand row carried to 2^-63 of its scale, slice pairs
 * s + t < 8, integer drains); Householder panels and T factors in FP64.
 * Results agree with the FP64 mode to FP64 rounding.  Every product reduces
 * over at most 2^20 rows: m <= 2^20 for purl_urv_factor_ex and purl_qr,
 * n <= 2^20 for purl_ulv_factor_ex, else PURL_ERR_UNSUPPORTED (workspace
 * queries return 0). */
#define PURL_MODE_FP64_EMU 4

/* Human-readable text for a status code (static storage). */
const char *purl_status_str(int status);

/* Library version string, e.g. "purl 0.1.0 sm_103a". */
const char *purl_version(void);

/*
 * purl_urv_factor -- PowerURV in FP64 (Section 3, Eqs. (5)-(6)).
 *   m, n     A is m x n, m >= n >= 0.
 *   A, lda   input, not modified.
 *   q        number of power steps, q >= 0 (q = 0: DDH-URV, Section 2.2).
 *   reorth   nonzero: orthonormalise (Householder QR, explicit Q with a
 *            nonnegative R diagonal) after every product with A or A^T;
 *            the last one is the QR of Eq. (5) itself.
 *   seed     key of the Gaussian draw (see purl_gaussian, stream 0).
 *   U, ldu   output m x n.   R, ldr  output n x n (zeros below the
 *   diagonal, diag >= 0).    V, ldv  output n x n.
 * Workspace is allocated stream-ordered (cudaMallocAsync) and released on
 * `stream` before the call returns; use purl_urv_factor_ex to pass your own.
 */
int purl_urv_factor(int m, int n, const double *A, int lda, int q, int reorth, uint64_t seed,
                    double *U, int ldu, double *R, int ldr, double *V, int ldv,
                    cudaStream_t stream);

/*
 * purl_urv_factor_ex -- as purl_urv_factor with a precision `mode` and an
 * optional caller workspace (device memory, 256-byte aligned, at least
 * purl_urv_workspace_bytes(m, n, mode) bytes; NULL = allocate on `stream`).
 */
int purl_urv_factor_ex(int m, int n, const double *A, int lda, int q, int reorth, uint64_t seed,
                       double *U, int ldu, double *R, int ldr, double *V, int ldv, int mode,
                       void *workspace, size_t workspace_bytes, cudaStream_t stream);

/* Workspace bytes purl_urv_factor_ex needs for (m, n, mode); 0 on bad args. */
size_t purl_urv_workspace_bytes(int m, int n, int mode);

/*
 * purl_ulv_factor_ex -- the wide case m <= n (Section 1: a URV factorization of
 * A^T gives a ULV factorization of A).  A = U L V^T with U m x m orthogonal,
 * L m x m lower triangular with a nonnegative diagonal, V n x m with
 * orthonormal columns, computed as the PowerURV of A^T (n x m) with the same
 * q, reorth, seed (G is m x m) and mode: A^T = U' R' V'^T gives U = V',
 * L = R'^T, V = U'.  A is not modified.  Workspace as for purl_urv_factor_ex
 * (purl_ulv_workspace_bytes; NULL = allocate on `stream`).  Errors: -i for bad
 * argument i (U = 8, ldu = 9, L = 10, ldl = 11, V = 12, ldv = 13, mode = 14),
 * PURL_ERR_SHAPE for m > n.
 */
int purl_ulv_factor_ex(int m, int n, const double *A, int lda, int q, int reorth, uint64_t seed,
                       double *U, int ldu, double *L, int ldl, double *V, int ldv, int mode,
                       void *workspace, size_t workspace_bytes, cudaStream_t stream);
size_t purl_ulv_workspace_bytes(int m, int n, int mode);

/*
 * purl_rsvd -- the randomized SVD of Section 6 (Eqs. (rsvd1)-(rsvd4)) in FP64,
 * started from the first l columns of PowerURV's Gaussian draw for `seed`
 * (the G_rsvd = G(:, 1:l) of the paper's Lemma, so range(U) equals the
 * range of the first l columns of purl_urv_factor's U for the same seed).
 *   Y = A (A^T A)^q G_rsvd (re-orthonormalised after every product when
 *   `reorth`), Y = Q R, Q^T A = W Sigma V^T, U = Q W.
 *   m, n, A, lda     input (not modified);  1 <= l <= min(m, n, 512).
 *   U (m x l, ldu), S (l, decreasing), V (n x l, ldv): outputs; each pair
 *   (U(:,j), V(:,j)) is signed so that U's entry of largest magnitude is
 *   positive.
 * The small SVD is a one-sided Jacobi iteration on an l x l factor in one
 * thread block (bounded number of sweeps).  Workspace as for
 * purl_urv_factor_ex (purl_rsvd_workspace_bytes).  Errors: -i for bad
 * argument i, PURL_ERR_NOMEM, PURL_ERR_CUDA.
 */
int purl_rsvd(int m, int n, const double *A, int lda, int l, int q, int reorth, uint64_t seed,
              double *U, int ldu, double *S, double *V, int ldv, void *workspace,
              size_t workspace_bytes, cudaStream_t stream);
size_t purl_rsvd_workspace_bytes(int m, int n, int l);

/*
 * purl_urv_backward -- reverse mode of the FP64 map A -> (U, R, V) of
 * purl_urv_factor (Section 3, Eqs. (5)-(6)) with the Gaussian G held fixed:
 * Abar = J^T (Ubar, Rbar, Vbar), the gradient with respect to A of
 * <Ubar, U> + <Rbar, R> + <Vbar, V>.  The paper defines no derivative; this
 * is the chain rule through every product and every QR of the forward pass,
 * with the thin-QR reverse rule (diag(R) > 0)
 *   Mbar = (Qbar + Q copyltu(R Rbar^T - Qbar^T Q)) R^{-T},
 *   copyltu(X) = lower triangle of X mirrored onto the upper one,
 * applied to the QRs of Eqs. (5) and (6) and, when `reorth` is set, to every
 * re-orthonormalisation; power-step products are reversed with transposed
 * products.  The forward iterates are recomputed from A and `seed` inside the
 * call (nothing is kept from a forward call).
 *   m, n, A, lda, q, reorth, seed   as for purl_urv_factor (same G).
 *   Ubar (m x n, ldub), Rbar (n x n, ldrb; only its upper triangle matters,
 *   R's lower triangle being identically zero), Vbar (n x n, ldvb): inputs.
 *   Abar (m x n, ldab): output, overwritten.
 * Requires A V, the power iterates and Y_q to have full column rank (R^{-T}
 * exists); otherwise the result is not finite.  Workspace as for
 * purl_urv_factor_ex (purl_urv_backward_workspace_bytes; NULL = allocate
 * stream-ordered on `stream`).  Errors: -i for bad argument i,
 * PURL_ERR_SHAPE for m < n, PURL_ERR_NOMEM, PURL_ERR_CUDA.
 */
int purl_urv_backward(int m, int n, const double *A, int lda, int q, int reorth, uint64_t seed,
                      const double *Ubar, int ldub, const double *Rbar, int ldrb,
                      const double *Vbar, int ldvb, double *Abar, int ldab, void *workspace,
                      size_t workspace_bytes, cudaStream_t stream);
size_t purl_urv_backward_workspace_bytes(int m, int n, int q);

/*
 * purl_urv_backward_ex -- purl_urv_backward with a precision `mode` for the
 * recomputed forward pass and every product of the reverse sweep (the paper
 * defines no derivative; the chain rule is the one stated above):
 *   PURL_MODE_FP64      FP64 DFMA products, FP64 Householder QRs (as
 *                       purl_urv_backward);
 *   PURL_MODE_FP64_EMU  every product an 8-slice exact tensor-core product and
 *                       every QR that of the FP64-emulation mode (FP64
 *                       accuracy; m <= 2^20, else PURL_ERR_UNSUPPORTED);
 *   PURL_MODE_FP32      the same with 4 slices (FP32 precision).
 * The forward pass it differentiates is purl_urv_factor_ex in the same mode.
 * Workspace: purl_urv_backward_ex_workspace_bytes(m, n, q, mode) bytes, or
 * NULL to allocate on `stream`.  Errors as purl_urv_backward, -16 for a bad
 * mode.
 */
int purl_urv_backward_ex(int m, int n, const double *A, int lda, int q, int reorth, uint64_t seed,
                         const double *Ubar, int ldub, const double *Rbar, int ldrb, const double *Vbar,
                         int ldvb, double *Abar, int ldab, int mode, void *workspace, size_t workspace_bytes,
                         cudaStream_t stream);
size_t purl_urv_backward_ex_workspace_bytes(int m, int n, int q, int mode);

/*
 * FP32 storage.  purl_urv_factor_f32 and purl_urv_backward_f32 take and
 * return column-major FP32 matrices (device memory, same arguments and errors
 * as purl_urv_factor_ex and purl_urv_backward_ex, float in place of double).
 * The inputs are widened to FP64 in the workspace (exactly), the call runs in
 * `mode` -- PURL_MODE_FP32 for FP32 precision; any mode of the FP64 entry
 * point is accepted -- and each result is rounded to FP32 once.  Workspace:
 * the _workspace_bytes query (FP64 copies of the inputs and outputs plus the
 * inner call's workspace), or NULL to allocate on `stream`.  A mode the
 * entry point cannot run returns -14 (factor) or -16 (backward).
 */
int purl_urv_factor_f32(int m, int n, const float *A, int lda, int q, int reorth, uint64_t seed, float *U,
                        int ldu, float *R, int ldr, float *V, int ldv, int mode, void *workspace,
                        size_t workspace_bytes, cudaStream_t stream);
size_t purl_urv_f32_workspace_bytes(int m, int n, int mode);
int purl_urv_backward_f32(int m, int n, const float *A, int lda, int q, int reorth, uint64_t seed,
                          const float *Ubar, int ldub, const float *Rbar, int ldrb, const float *Vbar, int ldvb,
                          float *Abar, int ldab, int mode, void *workspace, size_t workspace_bytes,
                          cudaStream_t stream);
size_t purl_urv_backward_f32_workspace_bytes(int m, int n, int q, int mode);

/*
 * Batched PowerURV in FP32 (Section 3, Eqs. (5)-(6), for many independent
 * small matrices).  The paper factors one matrix at a time; this engine runs
 * thousands in one persistent launch: every CTA takes the next matrix from a
 * queue and carries out the whole algorithm on it (Gaussian G, q power steps
 * with Householder re-orthonormalisation, the QR of Eq. (5), A V, the QR of
 * Eq. (6)), all in FP32 arithmetic with FP32 storage.  Same sign convention
 * as purl_urv_factor: every QR has a nonnegative R diagonal.
 *
 * One descriptor per matrix, in DEVICE memory, column-major FP32 matrices:
 *   m, n      1 <= n <= m <= max_m (<= 1024), n <= max_n (<= 512)
 *   A, lda    input (not modified);  U, ldu (m x n), R, ldr (n x n, zeros
 *             below the diagonal), V, ldv (n x n): outputs, caller-owned,
 *             not aliasing A or each other
 *   seed      key of this matrix's G: element e (column-major) of the n x n
 *             G is drawn as in purl_gaussian (Philox4x64-10, stream 0, the
 *             same 53-bit uniforms) with Box-Muller evaluated in FP32.
 * Matrices are taken in array order; putting the costliest (largest m n^2)
 * first balances the grid.  A descriptor outside the limits is skipped and
 * makes purl_urv_batched_status return PURL_ERR_UNSUPPORTED.
 */
typedef struct purl_batch_item {
  int m, n;
  int lda, ldu, ldr, ldv;
  const float *A;
  float *U, *R, *V;
  uint64_t seed;
} purl_batch_item;

/* Number of kernel variants (panel width x CTAs per SM) of the batched engine. */
int purl_urv_batched_variants(void);

/* Workspace bytes for variant v (0 .. variants-1), or for any variant when
 * v < 0; 0 on bad arguments or when the variant cannot run with max_m. */
size_t purl_urv_batched_workspace_bytes(int max_m, int max_n, int variant);

/*
 * purl_urv_factor_batched -- factor `count` matrices described by `items`
 * (device array) with q power steps (reorth as in purl_urv_factor).
 * variant < 0 uses the variant purl_urv_batched_autotune chose for the same
 * (count, max_m, max_n, q, reorth) on this device, else the first variant
 * that fits.  Workspace: device memory, 256-byte aligned, at least
 * purl_urv_batched_workspace_bytes(max_m, max_n, variant) bytes; its first
 * 256 bytes hold the queue position, reset by a kernel at the start of each
 * call, so one workspace must not serve two calls in flight at once.
 * Enqueues two kernels and nothing else (no allocation, no host sync), so the
 * call can be captured in a CUDA graph once an uncaptured call with the same
 * variant and max_m has run (that first call sets the kernel's shared-memory
 * limit).  Errors: -i for bad argument i, PURL_ERR_NOMEM (workspace),
 * PURL_ERR_UNSUPPORTED, PURL_ERR_CUDA.
 */
int purl_urv_factor_batched(int count, const purl_batch_item *items, int max_m, int max_n, int q,
                            int reorth, int variant, void *workspace, size_t workspace_bytes,
                            cudaStream_t stream);

/* Synchronises `stream` and returns the device-side status of the last
 * batched call on `workspace` (PURL_OK or PURL_ERR_UNSUPPORTED). */
int purl_urv_batched_status(void *workspace, cudaStream_t stream);

/*
 * purl_urv_batched_autotune -- runs every variant whose workspace fits in
 * `workspace_bytes` on the given batch (one warm-up and one timed run each,
 * CUDA events on `stream`; synchronises), remembers the fastest for later
 * calls with variant < 0, and returns it in *variant_out and its time in
 * *ms_out (either may be NULL).  The outputs of the batch are overwritten.
 */
int purl_urv_batched_autotune(int count, const purl_batch_item *items, int max_m, int max_n, int q,
                              int reorth, void *workspace, size_t workspace_bytes, cudaStream_t stream,
                              int *variant_out, float *ms_out);

/*
 * purl_gaussian_f32 -- the FP32 Gaussian draw of the batched engine: the
 * 53-bit uniforms of purl_gaussian rounded once to FP32, then Box-Muller in
 * FP32 (logf, sincospif).  Layout and arguments as purl_gaussian.
 */
int purl_gaussian_f32(uint64_t seed, uint64_t stream_id, int rows, int cols, float *G, int ldg,
                      cudaStream_t stream);

/*
 * purl_wait_probe -- exercises the failure detection (the paper has no
 * counterpart).  Every device-side wait of the library is bounded: when it
 * gives up it records PURL_ERR_TIMEOUT in the per-device status word read by
 * purl_device_status, raises an abort flag that ends the other waits of the
 * same launch, and returns.  The probe launches `blocks` (1..64) cooperative
 * blocks of 32 threads through the library's grid barrier with `polls` polls
 * allowed; with missing = 1 the barrier awaits one block more than exists,
 * so every wait runs out.  Asynchronous on `stream`; read the outcome with
 * purl_device_status (which also clears it).  Nothing faults or hangs.
 */
int purl_wait_probe(int blocks, int missing, long long polls, cudaStream_t stream);

/*
 * purl_wait_probe_noalloc -- the same probe, reporting to the status word that
 * purl_gemm_tc_noalloc keeps in its static device array (setting that array up
 * on this device as the entry point's first call does, which synchronises the
 * device).  Shows that a bounded wait running out inside the allocation-free
 * entry point reaches purl_device_status.  Arguments and errors as
 * purl_wait_probe.
 */
int purl_wait_probe_noalloc(int blocks, int missing, long long polls, cudaStream_t stream);

/*
 * purl_gaussian -- the Gaussian matrix G of Section 3 (the paper fixes no
 * generator; this library's is defined here).  Element e of the rows x cols
 * matrix, e = i + j*rows (column-major linear index), is word e%4 of the
 * Philox4x64-10 block (Salmon et al., SC'11) with counter (e/4, 0, 0, 0) and
 * key (seed, stream_id).  A 64-bit word w becomes u = ((w >> 11) + 0.5) 2^-53
 * in (0,1); Box-Muller turns words (0,1) and (2,3) of a block into
 * sqrt(-2 ln u0) cos(2 pi u1), sqrt(-2 ln u0) sin(2 pi u1), and likewise.
 * purl_urv_factor draws G with stream_id 0.
 */
int purl_gaussian(uint64_t seed, uint64_t stream_id, int rows, int cols, double *G, int ldg,
                  cudaStream_t stream);

/*
 * purl_qr -- unpivoted Householder QR with diag(R) >= 0 (the building block
 * of Eqs. (5) and (6)): M = Q R, M m x n (m >= n), Q m x n with orthonormal
 * columns, R n x n upper triangular.  M is not modified.  Either Q or R may
 * be NULL.  Blocked compact-WY algorithm; `mode` selects FP64 or the mixed
 * precision of PURL_MODE_MIXED_BF16 for trailing updates and Q formation.
 * Workspace as for purl_urv_factor_ex (purl_qr_workspace_bytes).
 */
int purl_qr(int m, int n, const double *M, int ldm, double *Q, int ldq, double *R, int ldr,
            int mode, void *workspace, size_t workspace_bytes, cudaStream_t stream);
size_t purl_qr_workspace_bytes(int m, int n, int mode);

/*
 * purl_gemm_f64 -- C = alpha op(A) op(B) + beta C in FP64 (the level-3 product
 * the paper's Section 3 relies on), op = 'N' or 'T'.  C is m x n, op(A) m x k,
 * op(B) k x n.  Exposed so the product engine can be tested on its own.
 */
int purl_gemm_f64(char transa, char transb, int m, int n, int k, double alpha, const double *A,
                  int lda, const double *B, int ldb, double beta, double *C, int ldc,
                  cudaStream_t stream);

/*
 * purl_gemm_tc -- the same product on the BF16 tensor cores (tcgen05, FP32
 * accumulation in tensor memory) with `slices` in {1, 2, 3} ({1..4} or 8
 * when exact): each FP64
 * operand is split into that many BF16 slices and the slice pairs (s, t) with
 * s + t < slices are multiplied (1, 3, 6, 10 or 36 BF16 products).
 *   exact = 0: floating slices X_0 = bf16(X), X_1 = bf16(X - X_0), ...; the
 *              accumulator's own rounding limits the result to about
 *              (k/16) 2^-23 of sum |a||b| however many slices are used.
 *   exact = 1: Ozaki-style fixed-point slices (a power-of-two scale per row
 *              of op(A) and per column of op(B), slices are integers of at
 *              most 8 bits) whose products sum without any rounding in the
 *              FP32 accumulator; the tensor memory is drained into
 *              double-FP32 sums every 256 of k.  Error about 2^(-8 slices)
 *              of (row scale) x (column scale) x k.  slices = 8 is the FP64
 *              emulation configuration: chunks of 128 of k drained into
 *              exact 64-bit integer sums, k <= 2^20 (PURL_ERR_UNSUPPORTED
 *              beyond), error below 2^-59 of (row max) x (column max) per
 *              term plus the final FP64 rounding.
 * This is the product engine of the mixed-precision mode.  Operand slices are
 * staged in scratch allocated on `stream`.
 */
int purl_gemm_tc(char transa, char transb, int m, int n, int k, double alpha, const double *A,
                 int lda, const double *B, int ldb, double beta, double *C, int ldc, int slices,
                 int exact, cudaStream_t stream);

/*
 * purl_gemm_tc_noalloc -- purl_gemm_tc (exact = 0) that allocates no device
 * memory.  (Library plumbing: the paper has no counterpart.)
 *
 * For callers that cannot call cudaMalloc or cudaMallocAsync at the point of
 * the call: code that runs after a framework has handed all device memory to
 * its own caching allocator, real-time loops that forbid allocation (its
 * latency and the risk of failing mid-run), or hosts that budget device
 * memory up front.  The operand slices are staged in a file-scope device
 * array of 24 MiB that every GPU which loads libpurl holds until the process
 * exits; nothing is allocated or freed per call (no cudaMalloc, cudaFree or
 * allocating library routine).
 *   - Size limit: the BF16 slices of both operands, 2 * slices * (64-rounded
 *     k) * (m + n) bytes plus alignment, must fit in the 24 MiB; larger
 *     requests return PURL_ERR_NOMEM without doing any work.
 *   - The first call on a device sets the array up (resolves its device
 *     address with cudaGetSymbolAddress and clears a status word, which
 *     synchronises the device); make that first call before any stream
 *     capture on that device.
 *   - Every call reuses the same array, which keeps the last call's
 *     contents.  Calls that overlap on the GPU (different streams, or host
 *     threads racing) race on it: serialise them, e.g. on one stream.
 *   - Device-side errors (a bounded wait that ran out) go to a status word at
 *     the start of the array; purl_device_status reads and clears it together
 *     with the library's own word.
 * Arguments, results and return codes are those of purl_gemm_tc with exact = 0.
 */
int purl_gemm_tc_noalloc(char transa, char transb, int m, int n, int k, double alpha, const double *A,
                         int lda, const double *B, int ldb, double beta, double *C, int ldc, int slices,
                         cudaStream_t stream);

/*
 * purl_urv_truncate -- rank-k approximation of Section 5:
 *   A_k = U(:,1:k) R(1:k,:) V^T   (m x n, written to Ak, ldak >= m), 0 <= k <= n.
 * purl_urv_reconstruct is the k = n case (U R V^T).
 */
int purl_urv_truncate(int m, int n, int k, const double *U, int ldu, const double *R, int ldr,
                      const double *V, int ldv, double *Ak, int ldak, cudaStream_t stream);
int purl_urv_reconstruct(int m, int n, const double *U, int ldu, const double *R, int ldr,
                         const double *V, int ldv, double *Ak, int ldak, cudaStream_t stream);

/*
 * purl_device_status -- read and clear the current device's status words
 * (PURL_OK or the first device-side error since the last call): the
 * library's per-device word and, once purl_gemm_tc_noalloc has been set up on
 * the device, the word in that entry point's static array (the library's
 * word is reported first when both are set).  Synchronises `stream`.
 */
int purl_device_status(cudaStream_t stream);

/* ------------------------------------------------------------------------
 * Diagnostics (no counterpart in the paper; used by the benchmark).
 * ------------------------------------------------------------------------ */

/* Number of kernels this library has launched in this process. */
unsigned long long purl_launch_count(void);

/* Opt-in timing: while enabled, every kernel launch is bracketed by two CUDA
 * events recorded on the stream it runs on, and its device time, flops and
 * algorithmic bytes are booked to its class (for the tensor-core classes the
 * flops are those issued: 2 m n k per slice pair multiplied):
 *   0 gemm_f64 (FP64 DFMA products), 1 panel_qr (Householder panels),
 *   2 gemm_tc (BF16 tensor-core products), 3 split (FP64 -> BF16 slicing),
 *   4 other (RNG, T factors, reductions, copies, sign fixes).
 * purl_profile_read synchronises the pending events of all classes and
 * returns the totals since the last purl_profile_reset (-1 for a bad class). */
void purl_profile_enable(int on);
void purl_profile_reset(void);
/* Sampling stride of the timing (default 1: every launch).  With s > 1 the
 * first 8 launches of every kernel name and then every s-th are timed, and a
 * name's (and class's) device time is reported as its timed launches' time
 * scaled by launches / timed launches; launches, flops and bytes count every
 * launch made while timing was on. */
void purl_profile_set_stride(int stride);
int purl_profile_read(int cls, long long *launches, double *ms, double *flops, double *bytes);
const char *purl_profile_class_name(int cls);
/* The same totals per kernel name (index 0, 1, ... until -1 is returned). */
int purl_profile_read_named(int index, char *name, int name_len, long long *launches, double *ms,
                            double *flops, double *bytes);

#ifdef __cplusplus
}
#endif

#endif /* PURL_H_ */
