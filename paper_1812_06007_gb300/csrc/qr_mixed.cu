// qr_mixed.cu -- blocked Householder QR for the mixed-precision mode.
//
// Same algorithm as qr.cu (Section 2.2's blocked unpivoted QR): FP64
// Householder panels, compact-WY blocks, trailing update C <- (I - V T^T V^T) C,
// explicit Q by applying the blocks last to first.  What changes is the
// arithmetic of the level-3 products, which run on the BF16 tensor cores with
// exact accumulation (gemm_tcx.cu) over S fixed-point slices:
//
//   * the matrix being factored (or the Q being formed) keeps FP64 values,
//     read by the panels and rewritten by every trailing update; before each
//     block is applied, its active part is re-sliced with a fresh power-of-two
//     scale per column (the column's current maximum), so each entry is
//     carried to 2^-8S of the largest entry of its column;
//   * V is rounded to a fixed grid (V^) that every slicing of it represents
//     exactly, so V^T C, the update and the Gram matrix all see the same V^;
//     T is built from the FP64 Gram matrix of V^ with tau_k = 2/||v^_k||^2,
//     so every applied block is orthogonal for the vectors it actually uses
//     (the slice pairs the tensor-core products drop would make a tensor-core
//     Gram matrix miss this by ~2^-8S);
//   * W = V^T C comes out as FP64 split-K partials, is multiplied by op(T) in
//     FP64 and re-sliced (per-column scale) for the update C - V W2.
#include "profile.cuh"
#include "qr_mixed.cuh"

namespace purl {

int gemm_f64(bool ta, bool tb, int m, int n, int k, double alpha, const double *A, int lda,
             const double *B, int ldb, double beta, double *C, int ldc, cudaStream_t s);
int gemm_f64_splitk(bool ta, bool tb, int m, int n, int k, int splits, int k_chunk,
                    const double *A, int lda, const double *B, int ldb, double *P, cudaStream_t s);
void choose_splits(int m, int n, int k, int num_sms, int *splits, int *k_chunk);

namespace {

constexpr int kChunkAlign = 256;  // exact-accumulation chunk of the tcx engine

__device__ __forceinline__ void exact_slices(double x, int e, __nv_bfloat16 *dst, long long plane, int S) {
  double t = ldexp(x, -e) * 128.0;
  for (int s = 0; s < S; ++s) {
    const double a = rint(t);
    dst[s * plane] = __double2bfloat16(a);
    t = (t - a) * 256.0;
  }
}

__device__ __forceinline__ int exponent_above(double mx) {
  int e = 0;
  if (mx > 0.0) frexp(mx, &e);
  return e;
}

// Householder vectors with v_k = 1 satisfy |v_i| <= 1 (v = x / (x_0 - beta)
// and |x_0 - beta| >= ||x||).  Each panel's V is rounded once to the grid
// 2^-kVGridBits (V^, written back over V), which every slicing below
// represents exactly: the natural slices use exponent 1 for every column, the
// transposed ones the exponent of each row's largest entry (any exponent
// <= 1 carries the grid).  V^ is then one matrix seen identically by V^T C,
// by the update and by the FP64 Gram matrix that defines T.
constexpr int kVExp = 1;
constexpr int kVGridBits = 30;

__global__ void split_v_kernel(int rows, int bw, double *V, long long ldv, Slices vs, Slices vts) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < rows; i += gridDim.x * blockDim.x) {
    double q[QR_B];
    double mx = 0.0;
#pragma unroll
    for (int t = 0; t < QR_B; ++t) {
      q[t] = 0.0;
      if (t < bw) {
        q[t] = ldexp(rint(ldexp(V[i + t * ldv], kVGridBits)), -kVGridBits);
        V[i + t * ldv] = q[t];
        mx = fmax(mx, fabs(q[t]));
      }
    }
    const int e = exponent_above(mx);
    vts.scale[i] = e;
    if (i < bw) vs.scale[i] = kVExp;
#pragma unroll
    for (int t = 0; t < QR_B; ++t)
      if (t < bw) {
        exact_slices(q[t], kVExp, vs.base + i + (long long)t * vs.ld, vs.plane, vs.S);
        exact_slices(q[t], e, vts.base + t + (long long)i * vts.ld, vts.plane, vts.S);
      }
  }
}

// W2(:, c) = op(T) * sum_z Pd_z(c, :)^T for each trailing column c, then the
// slices of W2(:, c) with its own exponent.  One thread per column.
__global__ void __launch_bounds__(128) reduce_tmul_slices_kernel(int bw, int nc, int splits,
                                                                 const double *__restrict__ Pd,
                                                                 const double *__restrict__ T, bool trans,
                                                                 Slices W2s) {
  __shared__ double Ts[QR_B][QR_B + 1];
  for (int e = threadIdx.x; e < QR_B * QR_B; e += blockDim.x) {
    int i = e % QR_B, j = e / QR_B;
    Ts[i][j] = trans ? T[j + i * QR_B] : T[e];  // Ts = op(T)
  }
  __syncthreads();
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  double w[QR_B];
#pragma unroll
  for (int l = 0; l < QR_B; ++l) {
    double s = 0.0;
    if (l < bw)
      for (int z = 0; z < splits; ++z) s += Pd[(long long)z * nc * bw + c + (long long)l * nc];
    w[l] = s;
  }
  double w2[QR_B];
  double mx = 0.0;
#pragma unroll
  for (int r = 0; r < QR_B; ++r) {
    double t = 0.0;
#pragma unroll
    for (int l = 0; l < QR_B; ++l) t = fma(Ts[r][l], w[l], t);
    w2[r] = t;
    if (r < bw) mx = fmax(mx, fabs(t));
  }
  const int e = exponent_above(mx);
  W2s.scale[c] = e;
#pragma unroll
  for (int r = 0; r < QR_B; ++r)
    if (r < bw) exact_slices(w2[r], e, W2s.base + r + (long long)c * W2s.ld, W2s.plane, W2s.S);
}

void splits_for(int M, int N, int K, int num_sms, int *splits, int *chunk) {
  tc_choose_splits(M, N, K, num_sms, QR_MAX_SPLITS, splits, chunk);
  *chunk = ceil_div(*chunk, kChunkAlign) * kChunkAlign;
  *splits = ceil_div(K, *chunk);
}

// Slices of the panel's V (natural and transposed) from w.base.Vb (rows x bw).
int slice_panel(int rows, int bw, QrMixWork &w, cudaStream_t s) {
  const DeviceInfo *di = device_info();
  int grid = ceil_div(rows, 256);
  if (grid > di->num_sms * 8) grid = di->num_sms * 8;
  { LaunchScope ls(KC_SPLIT, s, 0.0, (8.0 + 4.0 * w.S) * (double)rows * bw);
    split_v_kernel<<<grid, 256, 0, s>>>(rows, bw, w.base.Vb, rows, w.Vs, w.Vts); }
  return cudaGetLastError() == cudaSuccess ? PURL_OK : PURL_ERR_CUDA;
}

// C (rows x nc, FP64 at Cp with ldc) <- (I - V op(T) V^T) C.  The active
// block is first re-sliced into `Cs` at (r0, c0) with a fresh exponent per
// column (its current maximum, written to cexp[c0 + c]): an entry's slicing
// error is then 2^-8S of its column's largest entry, not of the column norm.
int apply_block_mixed(int rows, int bw, int nc, double *Cp, int ldc, const Slices &Cs, int r0, int c0,
                      int *cexp, const double *T, bool trans, QrMixWork &w, cudaStream_t s) {
  if (nc <= 0 || rows <= 0 || bw <= 0) return PURL_OK;
  const DeviceInfo *di = device_info();
  Slices view = Cs;
  view.base = Cs.base + r0 + (long long)c0 * Cs.ld;
  view.scale = cexp + c0;
  PURL_TRY(split_exact(rows, nc, Cp, ldc, view, nullptr, s));
  // W^T = C^T V  (nc x bw), FP64 split-K partials
  int sp, ch;
  splits_for(nc, bw, rows, di->num_sms, &sp, &ch);
  TcEpilogue ep;
  ep.mode = 2;
  ep.Pd = w.Pd;
  PURL_TRY(tcx_gemm_view(Cs, r0, c0, w.Vs, 0, 0, nc, bw, rows, w.S, ep, sp, ch, s));
  // W2 = op(T) W, sliced
  { LaunchScope ls(KC_OTHER, s, 2.0 * bw * bw * (double)nc, 8.0 * sp * (double)nc * bw);
    reduce_tmul_slices_kernel<<<ceil_div(nc, 128), 128, 0, s>>>(bw, nc, sp, w.Pd, T, trans, w.W2s); }
  PURL_CUDA_TRY(cudaGetLastError());
  // C <- C - V W2 (FP64)
  TcEpilogue up;
  up.mode = 0;
  up.alpha = -1.0;
  up.beta = 1.0;
  up.C = Cp;
  up.ldc = ldc;
  return tcx_gemm_view(w.Vts, 0, 0, w.W2s, 0, 0, rows, nc, bw, w.S, up, 1, kChunkAlign, s);
}

}  // namespace

int qr_mixed_plan(Arena &ar, int m, int n, int S, QrMixWork *w) {
  PURL_TRY(qr_plan(ar, m, n, PURL_MODE_FP64, &w->base));
  w->S = S;
  size_t nn = (size_t)(n > 0 ? n : 1), mm = (size_t)(m > 0 ? m : 1);
  w->col_exp = ar.take<int>(nn);
  w->Fs = make_slices(ar.take<__nv_bfloat16>(slice_elems(m, n, S)), m, n, S);
  w->Fs.scale = w->col_exp;
  w->Qs = make_slices(ar.take<__nv_bfloat16>(slice_elems(m, n, S)), m, n, S);
  w->Qs.scale = w->col_exp;
  w->Vs = make_slices(ar.take<__nv_bfloat16>(slice_elems(m, QR_B, S)), m, QR_B, S);
  w->Vs.scale = ar.take<int>(QR_B);
  w->Vts = make_slices(ar.take<__nv_bfloat16>(slice_elems(QR_B, m, S)), QR_B, m, S);
  w->Vts.scale = ar.take<int>(mm);
  w->Pd = ar.take<double>((size_t)QR_MAX_SPLITS * nn * QR_B);
  w->W2s = make_slices(ar.take<__nv_bfloat16>(slice_elems(QR_B, n, S)), QR_B, n, S);
  w->W2s.scale = ar.take<int>(nn);
  return PURL_OK;
}

int qr_mixed_factor(int m, int n, double *F, int ldf, QrMixWork &w, cudaStream_t s) {
  const DeviceInfo *di = device_info();
  if (!di) return PURL_ERR_CUDA;
  if (n == 0) return PURL_OK;
  int npan = ceil_div(n, QR_B);
  PURL_CUDA_TRY(cudaMemsetAsync(w.base.counters, 0, sizeof(unsigned) * npan, s));
  for (int p = 0; p < npan; ++p) {
    const int j0 = p * QR_B, bw = min(QR_B, n - j0), rows = m - j0, nc = n - j0 - bw;
    double *Fp = F + j0 + (size_t)j0 * ldf;
    double *taup = w.base.tau + j0;
    PURL_TRY(panel_factor(rows, bw, Fp, ldf, taup, w.base.counters + p, w.base, s));
    PURL_TRY(slice_panel(rows, bw, w, s));
    // T from the FP64 Gram matrix of the rounded V^ (exact to FP64 rounding)
    int gs, gch;
    choose_splits(bw, bw, rows, di->num_sms, &gs, &gch);
    PURL_TRY(gemm_f64_splitk(true, false, bw, bw, rows, gs, gch, w.base.Vb, rows, w.base.Vb, rows, w.base.Gp, s));
    double *Tp = w.base.T + (size_t)p * QR_B * QR_B;
    PURL_TRY(larft_from_gram(bw, gs, w.base.Gp, taup, Tp, s, true));
    PURL_TRY(apply_block_mixed(rows, bw, nc, Fp + (size_t)bw * ldf, ldf, w.Fs, j0, j0 + bw, w.col_exp, Tp,
                               true, w, s));
  }
  return PURL_OK;
}

int qr_mixed_form_q(int m, int n, const double *F, int ldf, QrMixWork &w, double *Q, int ldq, cudaStream_t s) {
  const DeviceInfo *di = device_info();
  if (!di) return PURL_ERR_CUDA;
  if (m == 0 || n == 0) return PURL_OK;
  PURL_TRY(set_identity(m, n, Q, ldq, s));
  int npan = ceil_div(n, QR_B);
  for (int p = npan - 1; p >= 0; --p) {
    const int j0 = p * QR_B, bw = min(QR_B, n - j0), rows = m - j0;
    PURL_TRY(extract_v(rows, bw, F + j0 + (size_t)j0 * ldf, ldf, w.base.Vb, s));
    PURL_TRY(slice_panel(rows, bw, w, s));
    const double *Tp = w.base.T + (size_t)p * QR_B * QR_B;
    PURL_TRY(apply_block_mixed(rows, bw, n - j0, Q + j0 + (size_t)j0 * ldq, ldq, w.Qs, j0, j0, w.col_exp, Tp,
                               false, w, s));
  }
  return PURL_OK;
}

}  // namespace purl
