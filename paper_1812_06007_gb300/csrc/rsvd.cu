// rsvd.cu -- the randomized SVD of Section 6 (Eqs. (rsvd1)-(rsvd4)) on the
// FP64 engine, sharing PowerURV's Gaussian draw: G_rsvd = G(:, 1:l).
//
//   X = G_rsvd;  q times: P = A X [P = Q(P)], X = A^T P [X = Q(X)]    (rsvd1)
//   Y = A X = Q R_y   (Householder QR, diag >= 0)                       (rsvd2)
//   B^T = A^T Q = Q2 R2,  R2^T = W Sigma Vr^T  (one-sided Jacobi)        (rsvd3)
//   so Q^T A = W Sigma (Q2 Vr)^T;  U = Q W,  V = Q2 Vr                  (rsvd4)
// Singular values are sorted in decreasing order and each pair (U(:,j),
// V(:,j)) is signed so that U's entry of largest magnitude is positive.
//
// The l x l SVD is Hestenes' one-sided Jacobi method with the round-robin
// (circle) ordering: each round rotates l/2 disjoint column pairs in
// parallel, one pair per thread block of a cooperative grid, with one grid
// barrier per round; sweeps stop when no pair needs a rotation
// (|a_p . a_q| <= l eps ||a_p|| ||a_q||) or after a fixed number.
#include "common.cuh"
#include "profile.cuh"
#include "qr.cuh"

namespace purl {

int launch_gaussian(uint64_t seed, uint64_t stream_id, int rows, int cols, double *G, int ldg, cudaStream_t stream,
                    bool fp32_math = false);
int gemm_f64(bool ta, bool tb, int m, int n, int k, double alpha, const double *A, int lda, const double *B, int ldb,
             double beta, double *C, int ldc, cudaStream_t s);

namespace {

constexpr int kMaxL = 512;
constexpr int kMaxSweeps = 60;

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// M (l x l, ld l) <- M Vr with orthogonal columns, Vr (l x l) accumulated;
// on exit sig[j] = ||M(:, j)|| and M(:, j) /= sig[j] (the left factor W).
// Cooperative launch, all blocks co-resident: in every round each block
// rotates its column pair(s) with 256 threads, then one bounded grid barrier;
// the number of rotations of a sweep is counted in rot[sweep] and read by
// every block after the sweep's last barrier, so all blocks stop after the
// same sweep.  counter and rot start at zero.
__device__ __forceinline__ void block_sum3(double &a, double &b, double &g, double (*red)[3]) {
  a = warp_sum_d(a);
  b = warp_sum_d(b);
  g = warp_sum_d(g);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) { red[warp][0] = a; red[warp][1] = b; red[warp][2] = g; }
  __syncthreads();
  a = b = g = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { a += red[w][0]; b += red[w][1]; g += red[w][2]; }
  __syncthreads();
}

__global__ void __launch_bounds__(256) jacobi_coop_kernel(int l, double *M, double *Vr, double *sig, unsigned *counter,
                                                          unsigned *rot, int *sweeps_out, DeviceControl *ctrl) {
  __shared__ double red[8][3];
  const int P = gridDim.x, tid = threadIdx.x;
  const int le = l + (l & 1);  // even count: an odd l gets a dummy column that pairs with nothing
  const double tol = (double)l * 2.220446049250313e-16;
  for (long long e = blockIdx.x * 256LL + tid; e < (long long)l * l; e += (long long)P * 256)
    Vr[e] = ((int)(e % l) == (int)(e / l)) ? 1.0 : 0.0;
  unsigned bar = 1;
  if (!grid_barrier(counter, bar * (unsigned)P, ctrl)) return;
  int sweep = 0;
  for (; sweep < kMaxSweeps; ++sweep) {
    for (int r = 0; r < le - 1; ++r) {
      for (int k = blockIdx.x; k < le / 2; k += P) {
        const int x = k, y = le - 1 - k;
        const int p = (x == 0) ? 0 : 1 + (x - 1 + r) % (le - 1);
        const int qq = (y == 0) ? 0 : 1 + (y - 1 + r) % (le - 1);
        if (p >= l || qq >= l) continue;
        double *mp = M + (size_t)p * l, *mq = M + (size_t)qq * l;
        double a = 0.0, b = 0.0, g = 0.0;
        for (int i = tid; i < l; i += 256) {
          const double u = __ldcg(&mp[i]), v = __ldcg(&mq[i]);
          a = fma(u, u, a);
          b = fma(v, v, b);
          g = fma(u, v, g);
        }
        block_sum3(a, b, g, red);
        if (g == 0.0 || fabs(g) <= tol * sqrt(a * b)) continue;
        const double zeta = (b - a) / (2.0 * g);
        const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        const double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
        double *vp = Vr + (size_t)p * l, *vq = Vr + (size_t)qq * l;
        for (int i = tid; i < l; i += 256) {
          const double u = __ldcg(&mp[i]), v = __ldcg(&mq[i]);
          __stcg(&mp[i], c * u - s * v);
          __stcg(&mq[i], s * u + c * v);
          const double uu = __ldcg(&vp[i]), vv = __ldcg(&vq[i]);
          __stcg(&vp[i], c * uu - s * vv);
          __stcg(&vq[i], s * uu + c * vv);
        }
        if (tid == 0) atomicAdd(&rot[sweep], 1u);
      }
      if (!grid_barrier(counter, ++bar * (unsigned)P, ctrl)) return;
    }
    if (__ldcg(&rot[sweep]) == 0u) break;
  }
  for (int j = blockIdx.x; j < l; j += P) {
    double *mj = M + (size_t)j * l;
    double a = 0.0, b = 0.0, g = 0.0;
    for (int i = tid; i < l; i += 256) { const double u = __ldcg(&mj[i]); a = fma(u, u, a); }
    block_sum3(a, b, g, red);
    const double nrm = sqrt(a);
    if (tid == 0) sig[j] = nrm;
    if (nrm > 0.0)
      for (int i = tid; i < l; i += 256) mj[i] = __ldcg(&mj[i]) / nrm;
  }
  if (blockIdx.x == 0 && tid == 0 && sweeps_out) *sweeps_out = sweep;
}

__global__ void zero_u32_kernel(unsigned *x, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) x[i] = 0u;
}

// Sort sigma decreasingly (ties by index) and permute the columns of W and Vr
// accordingly into Ws, Vs.  One block.
__global__ void __launch_bounds__(256) sort_sv_kernel(int l, const double *sig, const double *W, const double *Vr,
                                                      double *sig_out, double *Ws, double *Vs) {
  __shared__ int dest[kMaxL];
  for (int j = threadIdx.x; j < l; j += blockDim.x) {
    int rank = 0;
    const double sj = sig[j];
    for (int i = 0; i < l; ++i) rank += (sig[i] > sj || (sig[i] == sj && i < j)) ? 1 : 0;
    dest[j] = rank;
    sig_out[rank] = sj;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < l * l; e += blockDim.x) {
    const int i = e % l, j = e / l;
    Ws[i + (size_t)dest[j] * l] = W[e];
    Vs[i + (size_t)dest[j] * l] = Vr[e];
  }
}

// Flip U(:, j) and V(:, j) so that U's entry of largest magnitude (the first
// on ties) is positive.  One block per column.
__global__ void __launch_bounds__(256) sign_pairs_kernel(int m, int n, double *U, long long ldu, double *V,
                                                         long long ldv) {
  __shared__ double s_v[8];
  __shared__ int s_i[8];
  const int j = blockIdx.x;
  double *u = U + (long long)j * ldu;
  double best = -1.0;
  int bi = 0;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const double a = fabs(u[i]);
    if (a > best) { best = a; bi = i; }  // ascending i within a thread: first index kept on ties
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double ob = __shfl_xor_sync(0xffffffffu, best, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
  }
  if ((threadIdx.x & 31) == 0) { s_v[threadIdx.x >> 5] = best; s_i[threadIdx.x >> 5] = bi; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < 8; ++w)
      if (s_v[w] > s_v[0] || (s_v[w] == s_v[0] && s_i[w] < s_i[0])) { s_v[0] = s_v[w]; s_i[0] = s_i[w]; }
  }
  __syncthreads();
  if (u[s_i[0]] < 0.0) {
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += blockDim.x) u[i] = -u[i];
    double *v = V + (long long)j * ldv;
    for (int i = threadIdx.x; i < n; i += blockDim.x) v[i] = -v[i];
  }
}

struct RsvdPlan {
  double *X, *P, *Q, *Bt, *Q2, *R2, *M, *Vr, *sig, *Ws, *Vs, *F;
  int *sweeps;
  int *finite;       // non-finite input flag
  unsigned *jcount;  // grid-barrier counter, then one rotation count per sweep
  QrWork qw;
};

int rsvd_plan(Arena &ar, int m, int n, int l, RsvdPlan *p) {
  const size_t ml = (size_t)m * l, nl = (size_t)n * l, ll = (size_t)l * l;
  p->X = ar.take<double>(nl);
  p->P = ar.take<double>(ml);
  p->Q = ar.take<double>(ml);
  p->Bt = ar.take<double>(nl);
  p->Q2 = ar.take<double>(nl);
  p->R2 = ar.take<double>(ll);
  p->M = ar.take<double>(ll);
  p->Vr = ar.take<double>(ll);
  p->sig = ar.take<double>(l);
  p->Ws = ar.take<double>(ll);
  p->Vs = ar.take<double>(ll);
  p->F = ar.take<double>((size_t)(m > n ? m : n) * l);
  p->sweeps = ar.take<int>(1);
  p->finite = ar.take<int>(1);
  p->jcount = ar.take<unsigned>(1 + kMaxSweeps);
  return qr_plan(ar, m > n ? m : n, l, PURL_MODE_FP64, &p->qw);
}

// QR with explicit Q and diag(R) >= 0 of the rows x l matrix X (copied to F first).
int qr_into(int rows, int l, const double *X, int ldx, double *Q, int ldq, double *R, int ldr, RsvdPlan &p,
            cudaStream_t s) {
  PURL_TRY(copy_matrix(rows, l, X, ldx, p.F, rows, s));
  return qr_explicit(rows, l, p.F, rows, Q, ldq, R, ldr, PURL_MODE_FP64, p.qw, s);
}

int rsvd_run(int m, int n, const double *A, int lda, int l, int q, int reorth, uint64_t seed, double *U, int ldu,
             double *S, double *V, int ldv, RsvdPlan &p, cudaStream_t s) {
  PURL_TRY(launch_gaussian(seed, 0, n, l, p.X, n, s));  // G(:, 1:l) of PowerURV's n x n draw
  for (int i = 0; i < q; ++i) {
    PURL_TRY(gemm_f64(false, false, m, l, n, 1.0, A, lda, p.X, n, 0.0, p.P, m, s));  // P = A X
    if (reorth) PURL_TRY(qr_into(m, l, p.P, m, p.P, m, nullptr, 0, p, s));
    PURL_TRY(gemm_f64(true, false, n, l, m, 1.0, A, lda, p.P, m, 0.0, p.X, n, s));   // X = A^T P
    if (reorth) PURL_TRY(qr_into(n, l, p.X, n, p.X, n, nullptr, 0, p, s));
  }
  PURL_TRY(gemm_f64(false, false, m, l, n, 1.0, A, lda, p.X, n, 0.0, p.P, m, s));    // Y = A X  (rsvd1)
  PURL_TRY(qr_into(m, l, p.P, m, p.Q, m, nullptr, 0, p, s));                          // Y = Q R  (rsvd2)
  PURL_TRY(gemm_f64(true, false, n, l, m, 1.0, A, lda, p.Q, m, 0.0, p.Bt, n, s));    // B^T = A^T Q
  PURL_TRY(qr_into(n, l, p.Bt, n, p.Q2, n, p.R2, l, p, s));                           // B^T = Q2 R2
  PURL_TRY(transpose_f64(l, l, p.R2, l, p.M, l, s));                                  // M = R2^T
  {
    // M = W Sigma Vr^T (rsvd3): one column pair per block and round
    const DeviceInfo *di = device_info();
    const int le = l + (l & 1);
    int P = le / 2 < di->num_sms ? le / 2 : di->num_sms;
    if (P < 1) P = 1;
    { LaunchScope ls(KC_OTHER, s, 0.0, 0.0, "zero_u32_kernel");
      zero_u32_kernel<<<1, 128, 0, s>>>(p.jcount, 1 + kMaxSweeps); }
    PURL_CUDA_TRY(cudaGetLastError());
    unsigned *counter = p.jcount, *rot = p.jcount + 1;
    DeviceControl *ctrl = di->ctrl;
    int lv = l;
    void *args[] = {&lv, &p.M, &p.Vr, &p.sig, &counter, &rot, &p.sweeps, &ctrl};
    LaunchScope ls(KC_OTHER, s, 0.0, 0.0, "jacobi_coop_kernel");
    PURL_CUDA_TRY(cudaLaunchCooperativeKernel((const void *)jacobi_coop_kernel, dim3(P), dim3(256), args, 0, s));
  }
  { LaunchScope ls(KC_OTHER, s, 0.0, 0.0, "sort_sv_kernel");
    sort_sv_kernel<<<1, 256, 0, s>>>(l, p.sig, p.M, p.Vr, S, p.Ws, p.Vs); }
  PURL_CUDA_TRY(cudaGetLastError());
  PURL_TRY(gemm_f64(false, false, m, l, l, 1.0, p.Q, m, p.Ws, l, 0.0, U, ldu, s));   // U = Q W  (rsvd4)
  PURL_TRY(gemm_f64(false, false, n, l, l, 1.0, p.Q2, n, p.Vs, l, 0.0, V, ldv, s));  // V = Q2 Vr
  { LaunchScope ls(KC_OTHER, s, 0.0, 0.0, "sign_pairs_kernel");
    sign_pairs_kernel<<<l, 256, 0, s>>>(m, n, U, ldu, V, ldv); }
  return cudaGetLastError() == cudaSuccess ? PURL_OK : PURL_ERR_CUDA;
}

}  // namespace
}  // namespace purl

using namespace purl;

extern "C" {

size_t purl_rsvd_workspace_bytes(int m, int n, int l) {
  if (m < 1 || n < 1 || l < 1 || l > kMaxL || l > m || l > n) return 0;
  if (!device_info()) return 0;
  Arena ar;
  RsvdPlan p;
  if (rsvd_plan(ar, m, n, l, &p) != PURL_OK) return 0;
  return ar.used;
}

int purl_rsvd(int m, int n, const double *A, int lda, int l, int q, int reorth, uint64_t seed, double *U, int ldu,
              double *S, double *V, int ldv, void *workspace, size_t workspace_bytes, cudaStream_t stream) {
  if (m < 0) return -1;
  if (n < 0) return -2;
  if (!A && (long long)m * n > 0) return -3;
  if (lda < (m > 1 ? m : 1)) return -4;
  if (l < 1 || l > kMaxL || l > m || l > n) return -5;
  if (q < 0) return -6;
  if (!U) return -9;
  if (ldu < (m > 1 ? m : 1)) return -10;
  if (!S) return -11;
  if (!V) return -12;
  if (ldv < (n > 1 ? n : 1)) return -13;
  if (!device_info()) return PURL_ERR_CUDA;
  const size_t need = purl_rsvd_workspace_bytes(m, n, l);
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
  RsvdPlan p;
  int st = rsvd_plan(ar, m, n, l, &p);
  if (st == PURL_OK && !ar.ok) st = PURL_ERR_NOMEM;
  if (st == PURL_OK) st = finite_check(m, n, A, lda, p.finite, stream);
  if (st == PURL_OK) st = rsvd_run(m, n, A, lda, l, q, reorth, seed, U, ldu, S, V, ldv, p, stream);
  if (st == PURL_OK) st = finite_poison(p.finite, m, l, U, ldu, stream);
  if (st == PURL_OK) st = finite_poison(p.finite, l, 1, S, l, stream);
  if (st == PURL_OK) st = finite_poison(p.finite, n, l, V, ldv, stream);
  if (owned) cudaFreeAsync(ptr, stream);
  return st;
}

}  // extern "C"
