// qr_mixed.cu -- blocked Householder QR for the mixed-precision mode.
//
// Same algorithm as qr.cu (Section 2.2's blocked unpivoted QR): Householder
// panels (FP32 arithmetic with FP64 beta and tau at up to 4 slices, FP64 at 8),
// compact-WY blocks, trailing update C <- (I - V T^T V^T) C, explicit Q by
// applying the blocks last to first.  What changes is the arithmetic of the
// level-3 products, which run on the BF16 tensor cores with exact
// accumulation (gemm_tcx.cu) over S fixed-point slices:
//
//   * the matrix being factored (or the Q being formed) keeps FP64 values,
//     read by the panels and rewritten by every trailing update; before each
//     block is applied, its active part is re-sliced with a fresh power-of-two
//     scale per column (the column's current maximum), so each entry is
//     carried to 2^-8S of the largest entry of its column;
//   * V is rounded to a fixed grid (V^) that every slicing of it represents
//     exactly, so V^T C, the update and the Gram matrix all see the same V^;
//     T is built from the Gram matrix of V^ (exact in 64-bit integers at up
//     to 4 slices) with tau_k = 2/||v^_k||^2,
//     so every applied block is orthogonal for the vectors it actually uses
//     (the slice pairs the tensor-core products drop would make a tensor-core
//     Gram matrix miss this by ~2^-8S);
//   * W = V^T C comes out as FP64 split-K partials, is multiplied by op(T) in
//     FP64 and re-sliced (per-column scale) for the update C - V W2;
//   * two levels of blocking: QR_B-column panels are grouped into
//     QR_NB-column outer blocks.  Inside an outer block the panels update only
//     the block's own columns (a slab that stays in L2); the rest of the
//     matrix receives ONE update per outer block with the aggregated
//     I - V T_out V^T, applied as W2^T = C^T V~ with V~ = V op(T_out) and
//     C <- C - V W2, so the trailing matrix is streamed n / QR_NB times
//     instead of n / QR_B times.  T_out is assembled from the panels' T_k and
//     the exact Gram matrix of the rounded V (every slice pair).  Q is formed
//     from the outer blocks only.
#include <map>

#include "profile.cuh"
#include "qr_mixed.cuh"
#include "slice_int.cuh"

namespace purl {

int gemm_f64(bool ta, bool tb, int m, int n, int k, double alpha, const double *A, int lda,
             const double *B, int ldb, double beta, double *C, int ldc, cudaStream_t s);
int gemm_f64_splitk(bool ta, bool tb, int m, int n, int k, int splits, int k_chunk,
                    const double *A, int lda, const double *B, int ldb, double *P, cudaStream_t s);
void choose_splits(int m, int n, int k, int num_sms, int *splits, int *k_chunk);

namespace {

constexpr int kChunkAlign = 256;  // exact-accumulation chunk of the tcx engine
constexpr int kGramParts = 256;   // per-block partials of the panel Gram matrix (>= panel blocks)

// Householder vectors with v_k = 1 satisfy |v_i| <= 1 (v = x / (x_0 - beta)
// and |x_0 - beta| >= ||x||).  Each panel's V is rounded once to the grid
// 2^(kVExp - P), P = 7 + 8(S-1) (V^, inside the panel kernel's fused tail),
// which every slicing below represents exactly: the natural slices use
// exponent kVExp for every column, the transposed ones the exponent of each
// row's largest entry (any exponent <= kVExp carries the grid).  V^ is then
// one matrix seen identically by V^T C, by the update and by the FP64 Gram
// matrix that defines T.
constexpr int kVExp = 1;

// W2(:, c) = op(T) * sum_z Pd_z(c, :)^T for each trailing column c, then the
// slices of W2(:, c) with its own exponent.  Block = 8 columns x 32 rows
// (thread (cx, l) sums the split-K partials of one entry: the inner updates
// have few columns, so the work is spread over rows as well).
constexpr int kTmulCols = 8;
__global__ void __launch_bounds__(256) reduce_tmul_slices_kernel(int bw, int nc, int splits,
                                                                 const double *__restrict__ Pd,
                                                                 const double *__restrict__ T, bool trans,
                                                                 Slices W2s) {
  __shared__ double Ts[QR_B][QR_B + 1];
  __shared__ double ws[QR_B][kTmulCols + 1];
  __shared__ unsigned long long mxs[QR_B][kTmulCols];
  __shared__ int es[kTmulCols];
  const int cx = threadIdx.x % kTmulCols, l = threadIdx.x / kTmulCols;
  const int c = blockIdx.x * kTmulCols + cx;
  for (int e = threadIdx.x; e < QR_B * QR_B; e += blockDim.x) {
    const int i = e % QR_B, j = e / QR_B;
    Ts[i][j] = trans ? T[j + i * QR_B] : T[e];  // Ts = op(T)
  }
  double v0 = 0.0, v1 = 0.0, v2 = 0.0, v3 = 0.0;  // independent loads in flight
  if (c < nc && l < bw) {
    const double *pz = Pd + c + (long long)l * nc;
    const long long st = (long long)nc * bw;
    int z = 0;
    for (; z + 3 < splits; z += 4) {
      v0 += pz[z * st];
      v1 += pz[(z + 1) * st];
      v2 += pz[(z + 2) * st];
      v3 += pz[(z + 3) * st];
    }
    for (; z < splits; ++z) v0 += pz[z * st];
  }
  ws[l][cx] = (v0 + v1) + (v2 + v3);
  __syncthreads();
  // row r = l of W2 for column c
  double t = 0.0;
#pragma unroll 8
  for (int k = 0; k < QR_B; ++k) t = fma(Ts[l][k], ws[k][cx], t);
  mxs[l][cx] = (l < bw) ? abs_bits(t) : 0ull;
  __syncthreads();
  if (l == 0) {
    unsigned long long m = 0;
    for (int y = 0; y < QR_B; ++y) m = max(m, mxs[y][cx]);
    es[cx] = exp_above_bits(m);
    if (c < nc) W2s.scale[c] = es[cx];
  }
  __syncthreads();
  if (c < nc && l < bw) write_fixed_slices(t, es[cx], W2s.base + l + (long long)c * W2s.ld, W2s.plane, W2s.S);
}

// Explicit rounded V of an outer block and its transposed slices, one block
// per 32 rows.  Column t (0 <= t < nbw) of the block is the Householder
// vector of global column J0 + t: 0 above row t, 1 at row t, the stored
// entries below rounded to the grid 2^(kVExp - P) (rows counted from J0).
// Pass 1 writes Vo (lanes along rows) and takes each row's largest entry;
// pass 2 re-reads the block's rows of Vo (from L2) through a 32 x 32 shared
// tile and writes the slices of Vo^T with one exponent per row of Vo, lanes
// along the columns.
__global__ void __launch_bounds__(256) outer_v_kernel(int rows, int nbw, const double *__restrict__ F, long long ldf,
                                                      double *Vo, long long ldv, int P, Slices vts) {
  __shared__ unsigned long long mx_s[8][32];
  __shared__ int es[32];
  __shared__ double tile[32][33];
  const double unit = ldexp(1.0, kVExp - P);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int r0 = blockIdx.x * 32, i = r0 + lane;
  unsigned long long mx = 0;
  for (int t = warp; t < nbw; t += 8) {
    double v = 0.0;
    if (i < rows) {
      if (i == t) v = 1.0;
      else if (i > t) v = (double)fixed_point(F[i + (long long)t * ldf], kVExp, P) * unit;
      Vo[i + (long long)t * ldv] = v;
    }
    mx = max(mx, abs_bits(v));
  }
  mx_s[warp][lane] = mx;
  __syncthreads();
  if (warp == 0) {
    unsigned long long m = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) m = max(m, mx_s[w][lane]);
    es[lane] = exp_above_bits(m);
    if (i < rows) vts.scale[i] = es[lane];
  }
  __syncthreads();
  for (int t0 = 0; t0 < nbw; t0 += 32) {
    for (int j = warp; j < 32; j += 8) {  // tile[j][lane] = Vo(r0 + lane, t0 + j)
      const int t = t0 + j;
      tile[j][lane] = (i < rows && t < nbw) ? Vo[i + (long long)t * ldv] : 0.0;
    }
    __syncthreads();
    for (int j = warp; j < 32; j += 8) {  // row r0 + j of Vo, lanes along its columns
      const int t = t0 + lane, ii = r0 + j;
      if (ii < rows && t < nbw)
        write_fixed_slices(tile[lane][j], es[j], vts.base + t + (long long)ii * vts.ld, vts.plane, vts.S);
    }
    __syncthreads();
  }
}

// W2(:, c) = sum_z Pd_z(c, :)^T (nbw <= QR_NB entries), sliced with its own
// exponent.  Block = 32 columns x 8 row groups; thread (cx, ry) owns rows
// ry, ry + 8, ... of column cx; two passes over the partials (maximum, then
// digits) keep the registers free.
__global__ void __launch_bounds__(256) reduce_slices_kernel(int nbw, int nc, int splits, const double *__restrict__ Pd,
                                                            Slices W2s) {
  __shared__ unsigned long long mxs[8][32];
  const int cx = threadIdx.x & 31, ry = threadIdx.x >> 5;
  const int c = blockIdx.x * 32 + cx;
  unsigned long long mx = 0;
  if (c < nc)
    for (int r = ry; r < nbw; r += 8) {
      double a = 0.0;
      for (int z = 0; z < splits; ++z) a += Pd[(long long)z * nc * nbw + c + (long long)r * nc];
      mx = max(mx, abs_bits(a));
    }
  mxs[ry][cx] = mx;
  __syncthreads();
  __shared__ int es[32];
  __shared__ double tile[32][33];
  if (ry == 0) {
    unsigned long long m = 0;
#pragma unroll
    for (int y = 0; y < 8; ++y) m = max(m, mxs[y][cx]);
    es[cx] = exp_above_bits(m);
    if (c < nc) W2s.scale[c] = es[cx];
  }
  // 32-row chunks: sums read with the lanes along the columns (coalesced
  // partials), digits written with the lanes along the rows (coalesced slices)
  for (int r0 = 0; r0 < nbw; r0 += 32) {
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int r = r0 + ry + 8 * q;
      double a = 0.0;
      if (c < nc && r < nbw)
        for (int z = 0; z < splits; ++z) a += Pd[(long long)z * nc * nbw + c + (long long)r * nc];
      tile[ry + 8 * q][cx] = a;
    }
    __syncthreads();
    const int r = r0 + (threadIdx.x & 31);
    if (r < nbw)
      for (int cc = threadIdx.x >> 5; cc < 32; cc += 8) {
        const int col = blockIdx.x * 32 + cc;
        if (col < nc)
          write_fixed_slices(tile[threadIdx.x & 31][cc], es[cc], W2s.base + r + (long long)col * W2s.ld, W2s.plane,
                             W2s.S);
      }
  }
}

// G = sum of split-K partials (nbw x nbw each) into Gsum (ld nbw).
__global__ void sum_partials_kernel(int count, int splits, const double *__restrict__ P, double *out) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < count; e += gridDim.x * blockDim.x) {
    double v = 0.0;
    for (int z = 0; z < splits; ++z) v += P[(long long)z * count + e];
    out[e] = v;
  }
}

// T_out of an outer block from its panels' T_k (first at Tk, QR_B x QR_B
// each) and the exact Gram matrix G of the block's rounded V (nbw x nbw, ld
// nbw), by recursive doubling: the diagonal 32-blocks are the T_k, and level
// L = 1, 2, ... merges adjacent blocks of h = 32 * 2^(L-1) columns,
//   T(a, b) = -T(a, a) (G(a, b) T(b, b)),
// all merges of a level at once: X = G(a, b) T(b, b), grid barrier,
// T(a, b) = -T(a, a) X, grid barrier.  (The compact-WY T of two reflector
// sets with T1 and T2 and V1^T V2 = G12.)  One cooperative launch; Tout (ld
// QR_NB) is written whole (zeros outside the upper block triangle); X holds
// QR_NB x QR_NB / 2 doubles; `counter` starts at 0.
__device__ __forceinline__ void tout_barrier(unsigned *counter, unsigned &target, DeviceControl *ctrl, bool &ok) {
  target += gridDim.x;
  if (ok) ok = grid_barrier(counter, target, ctrl);
}

__global__ void __launch_bounds__(256) tout_kernel(int nbw, const double *__restrict__ G,
                                                   const double *__restrict__ Tk, double *Tout, double *X,
                                                   unsigned *counter, DeviceControl *ctrl) {
  const long long gt = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long GT = (long long)gridDim.x * blockDim.x;
  const int nk = (nbw + QR_B - 1) / QR_B;
  // level 0: zeros outside the diagonal blocks' upper block triangle, the diagonal blocks
  for (long long e = gt; e < (long long)QR_NB * QR_NB; e += GT) {
    const int i = (int)(e % QR_NB), j = (int)(e / QR_NB);
    const int bi = i / QR_B, bj = j / QR_B;
    double v = 0.0;
    if (i < nbw && j < nbw && bi == bj) v = Tk[(size_t)bi * QR_B * QR_B + (i % QR_B) + (j % QR_B) * QR_B];
    if (!(i < nbw && j < nbw && bi < bj)) Tout[e] = v;  // upper blocks come from the merges
  }
  unsigned target = 0;
  bool ok = true;
  tout_barrier(counter, target, ctrl, ok);
  for (int h = QR_B; h < nk * QR_B && ok; h *= 2) {
    // merges p: a = [2p h, 2p h + h), b = [2p h + h, min(2p h + 2h, nbw)); X_p at X + p h h
    const int npair = (nbw + 2 * h - 1) / (2 * h);
    // X = G(a, b) T(b, b): T(b, b) upper triangular (rows t <= j)
    for (long long e = gt; e < (long long)npair * h * h; e += GT) {
      const int p = (int)(e / ((long long)h * h)), r = (int)(e % ((long long)h * h));
      const int i = r % h, j = r / h, a0 = 2 * p * h, b0 = a0 + h, hb = min(h, nbw - b0);
      if (hb <= 0 || j >= hb) continue;
      const double *gr = G + (a0 + i) + (long long)b0 * nbw;
      const double *tc = Tout + b0 + (long long)(b0 + j) * QR_NB;
      double acc[4] = {0.0, 0.0, 0.0, 0.0};
      int t = 0;
      for (; t + 7 <= j; t += 8) {
        double gv[8], tv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          gv[u] = gr[(long long)(t + u) * nbw];
          tv[u] = __ldcg(&tc[t + u]);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) acc[u & 3] = fma(gv[u], tv[u], acc[u & 3]);
      }
      for (; t <= j; ++t) acc[0] = fma(gr[(long long)t * nbw], __ldcg(&tc[t]), acc[0]);
      __stcg(&X[(size_t)p * h * h + i + (size_t)j * h], (acc[0] + acc[1]) + (acc[2] + acc[3]));
    }
    tout_barrier(counter, target, ctrl, ok);
    if (!ok) break;
    // T(a, b) = -T(a, a) X: T(a, a) upper triangular (columns l >= i)
    for (long long e = gt; e < (long long)npair * h * h; e += GT) {
      const int p = (int)(e / ((long long)h * h)), r = (int)(e % ((long long)h * h));
      const int i = r % h, j = r / h, a0 = 2 * p * h, b0 = a0 + h, hb = min(h, nbw - b0);
      if (hb <= 0 || j >= hb) continue;
      const double *tr = Tout + (a0 + i) + (long long)a0 * QR_NB;
      const double *xc = X + (size_t)p * h * h + (size_t)j * h;
      double acc[4] = {0.0, 0.0, 0.0, 0.0};
      int l = i;
      for (; l + 7 < h; l += 8) {
        double tv[8], xv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          tv[u] = __ldcg(&tr[(long long)(l + u) * QR_NB]);
          xv[u] = __ldcg(&xc[l + u]);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) acc[u & 3] = fma(tv[u], xv[u], acc[u & 3]);
      }
      for (; l < h; ++l) acc[0] = fma(__ldcg(&tr[(long long)l * QR_NB]), __ldcg(&xc[l]), acc[0]);
      __stcg(&Tout[(a0 + i) + (long long)(b0 + j) * QR_NB], -((acc[0] + acc[1]) + (acc[2] + acc[3])));
    }
    tout_barrier(counter, target, ctrl, ok);
  }
}

void splits_for(int M, int N, int K, int num_sms, int *splits, int *chunk) {
  tc_choose_splits(M, N, K, num_sms, QR_MAX_SPLITS, splits, chunk);
  *chunk = ceil_div(*chunk, kChunkAlign) * kChunkAlign;
  *splits = ceil_div(K, *chunk);
}

// Buffers of one inner-block update: the panel's V slices (natural and
// transposed), the split-K partials of W^T = C^T V and the slices of W2.
struct InnerBufs {
  Slices Vs, Vts, W2s;
  double *Pd = nullptr;
};

// C (rows x nc, FP64 at Cp with ldc) <- (I - V op(T) V^T) C.  The active
// block is first re-sliced into `Cs` at (r0, c0) with a fresh exponent per
// column (its current maximum, written to cexp[c0 + c]): an entry's slicing
// error is then 2^-8S of its column's largest entry, not of the column norm.
int apply_block_mixed(int rows, int bw, int nc, double *Cp, int ldc, const Slices &Cs, int r0, int c0,
                      int *cexp, const double *T, bool trans, QrMixWork &w, const InnerBufs &b, cudaStream_t s,
                      cudaEvent_t t_ready) {
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
  ep.Pd = b.Pd;
  ep.tag = "tcx inner V^T C";
  PURL_TRY(tcx_gemm_view(Cs, r0, c0, b.Vs, 0, 0, nc, bw, rows, w.S, ep, sp, ch, s));
  // W2 = op(T) W, sliced (T formed on another stream until t_ready)
  if (t_ready) PURL_CUDA_TRY(cudaStreamWaitEvent(s, t_ready, 0));
  { LaunchScope ls(KC_OTHER, s, 2.0 * bw * bw * (double)nc, 8.0 * sp * (double)nc * bw, "reduce_tmul_slices_kernel");
    reduce_tmul_slices_kernel<<<ceil_div(nc, kTmulCols), 256, 0, s>>>(bw, nc, sp, b.Pd, T, trans, b.W2s); }
  PURL_CUDA_TRY(cudaGetLastError());
  // C <- C - V W2 (FP64)
  TcEpilogue up;
  up.mode = 0;
  up.alpha = -1.0;
  up.beta = 1.0;
  up.C = Cp;
  up.ldc = ldc;
  up.tag = "tcx inner update";
  return tcx_gemm_view(b.Vts, 0, 0, b.W2s, 0, 0, rows, nc, bw, w.S, up, 1, kChunkAlign, s);
}

constexpr int kOuterSplits = 4;

int launch_grid(long long total, int cap) {
  long long g = (total + 255) / 256;
  if (g > cap) g = cap;
  return (int)(g < 1 ? 1 : g);
}

// Build the outer block's rounded V, its slices, its Gram matrix (exact,
// every slice pair) and T_out from the inner T_k:
//   T_out(0:kb, kb:kb+bw) = -T_out(0:kb, 0:kb) G(0:kb, kb:kb+bw) T_k.
int outer_prepare(int rows, int nbw, const double *FJ, int ldf, int m, int first_panel, double *Tout, bool build_t,
                  QrMixWork &w, cudaStream_t s) {
  const DeviceInfo *di = device_info();
  const int P = 7 + 8 * (w.S - 1);
  { LaunchScope ls(KC_SPLIT, s, 0.0, (24.0 + 2.0 * w.S) * rows * (double)nbw, "outer_v_kernel");
    outer_v_kernel<<<ceil_div(rows, 32), 256, 0, s>>>(rows, nbw, FJ, ldf, w.Vo, m, P, w.Vots); }
  PURL_CUDA_TRY(cudaGetLastError());
  if (!build_t) return PURL_OK;
  PURL_TRY(split_exact(rows, nbw, w.Vo, m, w.Vos, nullptr, s));
  // Gram matrix of the rounded V: exact (all slice pairs) for S <= 4; for the
  // FP64-emulation slices the pairs s + t >= S weigh below 2^-59, so the
  // usual product is V^T V^ to FP64 accuracy, as in the FP64 path
  int gs, gch;
  splits_for(nbw, nbw, rows, di->num_sms, &gs, &gch);
  TcEpilogue g;
  g.mode = 2;
  g.Pd = w.Go;
  if (w.S <= 4) {
    g.tag = "tcx outer Gram (all pairs)";
    PURL_TRY(tcx_gemm_all_pairs(w.Vos, 0, 0, w.Vos, 0, 0, nbw, nbw, rows, w.S, g, gs, gch, s));
  } else {
    g.tag = "tcx outer Gram";
    PURL_TRY(tcx_gemm_view(w.Vos, 0, 0, w.Vos, 0, 0, nbw, nbw, rows, w.S, g, gs, gch, s));
  }
  { LaunchScope ls(KC_OTHER, s, 0.0, 0.0, "sum_partials_kernel");
    sum_partials_kernel<<<launch_grid((long long)nbw * nbw, 256), 256, 0, s>>>(nbw * nbw, gs, w.Go, w.Tt); }
  PURL_CUDA_TRY(cudaGetLastError());
  double *G = w.Tt;  // nbw x nbw, ld nbw
  PURL_TRY(zero_async(w.tcount, sizeof(unsigned), s));
  const double *Tk = w.base.T + (size_t)first_panel * QR_B * QR_B;
  double *X = w.Go;  // scratch after the sum: the merges' G(a, b) T(b, b)
  int nbw_ = nbw;
  int grid = di->num_sms;
  void *args[] = {&nbw_, &G, &Tk, &Tout, &X, &w.tcount, (void *)&di->ctrl};
  double fl = 0.0;
  for (int h = QR_B; h < nbw; h *= 2) fl += (double)nbw / (2 * h) * 2.0 * h * h * h;
  LaunchScope ls(KC_OTHER, s, fl, 8.0 * nbw * (double)nbw, "tout_kernel");
  PURL_CUDA_TRY(cudaLaunchCooperativeKernel((const void *)tout_kernel, dim3(grid), dim3(256), args, 0, s));
  return PURL_OK;
}

// C (rows x nc at Cp, ld ldc; slices in Cs at (r0, c0)) <- (I - V op(T_out) V^T) C
// with V = w.Vo (rows x nbw) and its slices already prepared.
int outer_apply(int rows, int nbw, int nc, double *Cp, int ldc, const Slices &Cs, int r0, int c0, int *cexp,
                const double *Tout, bool trans, int m, QrMixWork &w, cudaStream_t s) {
  if (nc <= 0 || rows <= 0) return PURL_OK;
  const DeviceInfo *di = device_info();
  // V~ = V T_out for Q^T C (W2^T = C^T V T_out), V T_out^T for Q C
  const double *Top = Tout;
  if (!trans) {
    PURL_TRY(transpose_f64(nbw, nbw, Tout, QR_NB, w.Tt, QR_NB, s));
    Top = w.Tt;
  }
  PURL_TRY(split_exact(nbw, nbw, Top, QR_NB, w.Ts, nullptr, s));
  TcEpilogue vt;
  vt.mode = 0;
  vt.C = w.Vtl;
  vt.ldc = m;
  vt.tag = "tcx outer V~ = V T";
  PURL_TRY(tcx_gemm_view(w.Vots, 0, 0, w.Ts, 0, 0, rows, nbw, nbw, w.S, vt, 1,
                         ceil_div(nbw, kChunkAlign) * kChunkAlign, s));
  PURL_TRY(split_exact(rows, nbw, w.Vtl, m, w.Vtls, nullptr, s));
  // re-slice the active block with fresh per-column exponents
  Slices view = Cs;
  view.base = Cs.base + r0 + (long long)c0 * Cs.ld;
  view.scale = cexp + c0;
  PURL_TRY(split_exact(rows, nc, Cp, ldc, view, nullptr, s));
  // W2^T = C^T V~  (nc x nbw), FP64 split-K partials
  int sp, ch;
  splits_for(nc, nbw, rows, di->num_sms, &sp, &ch);
  if (sp > kOuterSplits) {
    ch = ceil_div(ceil_div(rows, kOuterSplits), kChunkAlign) * kChunkAlign;
    sp = ceil_div(rows, ch);
  }
  TcEpilogue ep;
  ep.mode = 2;
  ep.Pd = w.Pdo;
  ep.tag = "tcx outer C^T V~";
  PURL_TRY(tcx_gemm_view(Cs, r0, c0, w.Vtls, 0, 0, nc, nbw, rows, w.S, ep, sp, ch, s));
  { LaunchScope ls(KC_SPLIT, s, 0.0, 8.0 * sp * (double)nc * nbw, "reduce_slices_kernel");
    reduce_slices_kernel<<<ceil_div(nc, 32), 256, 0, s>>>(nbw, nc, sp, w.Pdo, w.W2o); }
  PURL_CUDA_TRY(cudaGetLastError());
  // C <- C - V W2
  TcEpilogue up;
  up.mode = 0;
  up.alpha = -1.0;
  up.beta = 1.0;
  up.C = Cp;
  up.ldc = ldc;
  up.tag = "tcx outer update";
  return tcx_gemm_view(w.Vots, 0, 0, w.W2o, 0, 0, rows, nc, nbw, w.S, up, 1, ceil_div(nbw, kChunkAlign) * kChunkAlign, s);
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
  const size_t nout = (size_t)ceil_div(n > 0 ? n : 1, QR_NB);
  w->Tout = ar.take<double>(nout * QR_NB * QR_NB);
  w->Gparts = ar.take<double>((size_t)kGramParts * QR_B * QR_B);
  w->Vo = ar.take<double>(mm * QR_NB);
  w->Vtl = ar.take<double>(mm * QR_NB);
  w->Go = ar.take<double>((size_t)QR_MAX_SPLITS * QR_NB * QR_NB);
  w->Tt = ar.take<double>((size_t)QR_NB * QR_NB);
  w->Pdo = ar.take<double>((size_t)kOuterSplits * nn * QR_NB);
  w->Vos = make_slices(ar.take<__nv_bfloat16>(slice_elems(m, QR_NB, S)), m, QR_NB, S);
  w->Vos.scale = ar.take<int>(QR_NB);
  w->Vots = make_slices(ar.take<__nv_bfloat16>(slice_elems(QR_NB, m, S)), QR_NB, m, S);
  w->Vots.scale = ar.take<int>(mm);
  w->Vtls = make_slices(ar.take<__nv_bfloat16>(slice_elems(m, QR_NB, S)), m, QR_NB, S);
  w->Vtls.scale = ar.take<int>(QR_NB);
  w->Ts = make_slices(ar.take<__nv_bfloat16>(slice_elems(QR_NB, QR_NB, S)), QR_NB, QR_NB, S);
  w->Ts.scale = ar.take<int>(QR_NB);
  w->W2o = make_slices(ar.take<__nv_bfloat16>(slice_elems(QR_NB, n, S)), QR_NB, n, S);
  w->W2o.scale = ar.take<int>(nn);
  w->tcount = ar.take<unsigned>(1);
  return PURL_OK;
}

namespace {

// A second stream of the calling host thread on the current device, with two
// events: the panels' T factors are formed on it beside the first kernels of
// each inner update, which do not need them.
struct SideStream {
  cudaStream_t s = nullptr;
  cudaEvent_t panel_done = nullptr, t_done = nullptr;
};

int side_stream(SideStream **out) {
  thread_local std::map<int, SideStream> per_device;
  int dev = 0;
  PURL_CUDA_TRY(cudaGetDevice(&dev));
  SideStream &ss = per_device[dev];
  if (!ss.s) {
    PURL_CUDA_TRY(cudaStreamCreateWithFlags(&ss.s, cudaStreamNonBlocking));
    PURL_CUDA_TRY(cudaEventCreateWithFlags(&ss.panel_done, cudaEventDisableTiming));
    PURL_CUDA_TRY(cudaEventCreateWithFlags(&ss.t_done, cudaEventDisableTiming));
  }
  *out = &ss;
  return PURL_OK;
}

}  // namespace

int qr_mixed_factor(int m, int n, double *F, int ldf, QrMixWork &w, cudaStream_t s) {
  const DeviceInfo *di = device_info();
  if (!di) return PURL_ERR_CUDA;
  if (n == 0) return PURL_OK;
  const InnerBufs b = {w.Vs, w.Vts, w.W2s, w.Pd};
  const int npan = ceil_div(n, QR_B);
  SideStream *side = nullptr;
  PURL_TRY(side_stream(&side));
  PURL_TRY(zero_async(w.base.counters, sizeof(unsigned) * npan, s));
  // the FP32 panels' tagged partial sums: epoch 0 everywhere, panel p uses 1 + 32 p ...
  PURL_TRY(zero_async(w.base.part, sizeof(double) * 2 * di->num_sms * QR_B, s));
  for (int J0 = 0, ob = 0; J0 < n; J0 += QR_NB, ++ob) {
    const int nbw = min(QR_NB, n - J0), rows = m - J0, nc_out = n - J0 - nbw;
    // inner panels, their updates confined to the outer block's columns
    for (int j0 = J0; j0 < J0 + nbw; j0 += QR_B) {
      const int p = j0 / QR_B, bw = min(QR_B, J0 + nbw - j0), rj = m - j0;
      const int nc_in = J0 + nbw - j0 - bw;
      double *Fp = F + j0 + (size_t)j0 * ldf;
      double *taup = w.base.tau + j0;
      // the panel, with its rounded V^, V^'s slices and V^'s Gram matrix in the
      // same cooperative launch; T_k (tau_k = 2 / ||v^_k||^2) from the Gram
      // matrix on the side stream, waited for just before its first use
      double *Tp = w.base.T + (size_t)p * QR_B * QR_B;
      PanelTail tl;
      tl.vexp = kVExp;
      tl.P = 7 + 8 * (w.S - 1);
      tl.vs = b.Vs;
      tl.vts = b.Vts;
      tl.gpart = w.Gparts;
      tl.G = w.base.Gp;
      tl.T = Tp;
      tl.epoch0 = 1u + 32u * (unsigned)p;
      PURL_TRY(panel_factor_tail(rj, bw, Fp, ldf, taup, w.base.counters + p, w.base, tl, s));
      PURL_CUDA_TRY(cudaEventRecord(side->panel_done, s));
      PURL_CUDA_TRY(cudaStreamWaitEvent(side->s, side->panel_done, 0));
      PURL_TRY(panel_t(rj, bw, taup, tl, side->s));
      PURL_CUDA_TRY(cudaEventRecord(side->t_done, side->s));
      PURL_TRY(apply_block_mixed(rj, bw, nc_in, Fp + (size_t)bw * ldf, ldf, w.Fs, j0, j0 + bw, w.col_exp, Tp, true,
                                 w, b, s, side->t_done));
      // T_k is in place (and the Gram matrix free) before the next panel
      PURL_CUDA_TRY(cudaStreamWaitEvent(s, side->t_done, 0));
    }
    // one aggregated update of everything to the right of the outer block
    double *Tout = w.Tout + (size_t)ob * QR_NB * QR_NB;
    PURL_TRY(outer_prepare(rows, nbw, F + J0 + (size_t)J0 * ldf, ldf, m, J0 / QR_B, Tout, true, w, s));
    if (nc_out > 0)
      PURL_TRY(outer_apply(rows, nbw, nc_out, F + J0 + (size_t)(J0 + nbw) * ldf, ldf, w.Fs, J0, J0 + nbw, w.col_exp,
                           Tout, true, m, w, s));
  }
  return PURL_OK;
}

int qr_mixed_form_q(int m, int n, const double *F, int ldf, QrMixWork &w, double *Q, int ldq, cudaStream_t s) {
  const DeviceInfo *di = device_info();
  if (!di) return PURL_ERR_CUDA;
  if (m == 0 || n == 0) return PURL_OK;
  PURL_TRY(set_identity(m, n, Q, ldq, s));
  const int nout = ceil_div(n, QR_NB);
  for (int ob = nout - 1; ob >= 0; --ob) {
    const int J0 = ob * QR_NB, nbw = min(QR_NB, n - J0), rows = m - J0;
    const double *Tout = w.Tout + (size_t)ob * QR_NB * QR_NB;
    PURL_TRY(outer_prepare(rows, nbw, F + J0 + (size_t)J0 * ldf, ldf, m, J0 / QR_B, nullptr, false, w, s));
    PURL_TRY(outer_apply(rows, nbw, n - J0, Q + J0 + (size_t)J0 * ldq, ldq, w.Qs, J0, J0, w.col_exp, Tout, false, m,
                         w, s));
  }
  return PURL_OK;
}

}  // namespace purl
