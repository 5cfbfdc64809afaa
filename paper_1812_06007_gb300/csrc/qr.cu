// qr.cu -- blocked unpivoted Householder QR with compact-WY reflectors
// (Section 2.2: unpivoted QR "can operate on blocks, accumulate Householder
// reflectors, and then apply the reflectors to the trailing matrix using a
// level-3 BLAS matrix-matrix multiply").  This is the QR behind Eq. (5), Eq. (6)
// and every re-orthonormalisation of the power iteration.
//
// For each panel of b columns starting at j0:
//   1. panel_kernel (cooperative, all blocks co-resident): Householder vectors
//      of the (m-j0) x b panel, one grid barrier per column.  Each block keeps
//      a slab of rows in shared memory; for column k it publishes, in ONE pass,
//      the partial sums  sum_{i>k} x_i^2  and  sum_{i>k} x_i a_it  (t > k), so
//      that after the barrier every block can form beta, tau and the
//      reflector's action on the remaining panel columns without a second
//      round trip (v = (x - beta e_k)/v0 is never needed before the barrier).
//   2. T factor (b x b upper triangular, I - V T V^T = H_0 ... H_{b-1}) from
//      the Gram matrix V^T V (a split-K product) by the column recurrence
//      T(0:k,k) = -tau_k T(0:k,0:k) (V(:,0:k)^T v_k).
//   3. Trailing update C <- (I - V T^T V^T) C as three steps: W = V^T C
//      (split-K), W <- T^T W, C <- C - V W.
// The explicit Q is formed afterwards by applying the blocks, last to first,
// to the first n columns of the identity; the signs are then normalised so
// that diag(R) >= 0 (the convention of the footnote in Section 2.2 that makes
// the factorization unique).
#include <map>
#include <mutex>
#include <type_traits>

#include "common.cuh"
#include "qr.cuh"
#include "profile.cuh"
#include "slice_int.cuh"

namespace purl {

int gemm_f64(bool ta, bool tb, int m, int n, int k, double alpha, const double *A, int lda,
             const double *B, int ldb, double beta, double *C, int ldc, cudaStream_t s);
int gemm_f64_splitk(bool ta, bool tb, int m, int n, int k, int splits, int k_chunk,
                    const double *A, int lda, const double *B, int ldb, double *P, cudaStream_t s);
void choose_splits(int m, int n, int k, int num_sms, int *splits, int *k_chunk);

namespace {

constexpr int PNT = 512;  // panel kernel threads
constexpr int PW = PNT / 32;
constexpr int kPanelMaxBlocks = 160;  // panel grids have at most this many blocks (>= the SM count)

// The FP32 panel's partial sums carry an epoch next to the value (one 64-bit
// word), so a block waits for the data itself instead of for a barrier
// counter: column k of the panel launch with epoch base e0 writes epoch e0 + k.
// The QR zeroes the tagged buffers before its first panel and gives panel p
// the base 1 + 32 p, so no word left by an earlier panel carries the current
// epoch.
__device__ __forceinline__ unsigned long long epoch_tag(unsigned ep, float v) {
  return ((unsigned long long)ep << 32) | __float_as_uint(v);
}
__device__ __forceinline__ unsigned tag_epoch(unsigned long long w) { return (unsigned)(w >> 32); }
__device__ __forceinline__ float tag_value(unsigned long long w) { return __uint_as_float((unsigned)w); }

// ------------------------------------------------------------ panel tail --
// Shared-memory work arrays of larft_core.
struct LarftSmem {
  double Gm[QR_B][QR_B + 1];
  double Ts[QR_B][QR_B + 1];
  double tmp[QR_B * QR_B / 2];
  double tks[QR_B];
};

// T from the Gram matrix already in L.Gm (bw x bw, symmetric), by the whole
// block (256 threads).  Ends with a __syncthreads.
__device__ void larft_core(int bw, LarftSmem &L, const double *tau, double *T, bool tau_from_gram) {
  constexpr int LF = 8;
  for (int e = threadIdx.x; e < QR_B * QR_B; e += blockDim.x) L.Ts[e % QR_B][e / QR_B] = 0.0;
  if (threadIdx.x < bw) {
    const int k = threadIdx.x;
    double tk = tau[k];
    if (tau_from_gram && tk != 0.0) tk = 2.0 / L.Gm[k][k];
    L.tks[k] = tk;
  }
  __syncthreads();
  // diagonal blocks: thread i owns row i of its block
  if (threadIdx.x < bw) {
    const int i = threadIdx.x, a = (i / LF) * LF;
    for (int k = i; k < a + LF && k < bw; ++k) {
      if (k == i) {
        L.Ts[i][k] = L.tks[k];
      } else {
        double s0 = 0.0, s1 = 0.0;
        int l = i;
        for (; l + 1 < k; l += 2) {
          s0 = fma(L.Ts[i][l], L.Gm[l][k], s0);
          s1 = fma(L.Ts[i][l + 1], L.Gm[l + 1][k], s1);
        }
        if (l < k) s0 = fma(L.Ts[i][l], L.Gm[l][k], s0);
        L.Ts[i][k] = -L.tks[k] * (s0 + s1);
      }
    }
  }
  __syncthreads();
  for (int h = LF; h < QR_B; h *= 2) {
    const int outs = (QR_B / (2 * h)) * h * h;
    for (int e = threadIdx.x; e < outs; e += blockDim.x) {  // tmp = G12 T22
      const int pr = e / (h * h), i = (e % (h * h)) / h, j = e % h;
      const int a = pr * 2 * h, b0 = a + h;
      double s0 = 0.0, s1 = 0.0;
      for (int l = 0; l <= j; l += 2) {
        s0 = fma(L.Gm[a + i][b0 + l], L.Ts[b0 + l][b0 + j], s0);
        if (l + 1 <= j) s1 = fma(L.Gm[a + i][b0 + l + 1], L.Ts[b0 + l + 1][b0 + j], s1);
      }
      L.tmp[e] = s0 + s1;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < outs; e += blockDim.x) {  // T12 = -T11 tmp
      const int pr = e / (h * h), i = (e % (h * h)) / h, j = e % h;
      const int a = pr * 2 * h, b0 = a + h;
      double s0 = 0.0, s1 = 0.0;
      for (int l = i; l < h; l += 2) {
        s0 = fma(L.Ts[a + i][a + l], L.tmp[pr * h * h + l * h + j], s0);
        if (l + 1 < h) s1 = fma(L.Ts[a + i][a + l + 1], L.tmp[pr * h * h + (l + 1) * h + j], s1);
      }
      L.Ts[a + i][b0 + j] = -(s0 + s1);
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < QR_B * QR_B; e += blockDim.x) {
    int i = e % QR_B, j = e / QR_B;
    T[e] = (i < bw && j < bw) ? L.Ts[i][j] : 0.0;
  }
  __syncthreads();
}


// V^ as the panel tail keeps it, in place of the factored panel: FP64 values
// for the FP64 panel; for the FP32 panel the integers N = V^ 2^(P - vexp)
// (|N| <= 2^(P - vexp) (1 + 2^-23)).
template <typename Real>
using TailV = typename std::conditional<sizeof(Real) == 4, int, double>::type;

// Entry i of column j of the factored panel, rounded to the grid 2^(vexp - P):
// 0 above the diagonal, 1 on it.
__device__ __forceinline__ double round_entry(double x, int gi, int j, const PanelTail &tl) {
  const double unit = __longlong_as_double((long long)(1023 + tl.vexp - tl.P) << 52);  // 2^(vexp - P)
  return gi < j ? 0.0 : (gi == j ? 1.0 : (double)fixed_point(x, tl.vexp, tl.P) * unit);
}
__device__ __forceinline__ int round_entry(float x, int gi, int j, const PanelTail &tl) {
  return gi < j ? 0 : (gi == j ? 1 << (tl.P - tl.vexp) : fixed_point_f32(x, tl.vexp, tl.P));
}

// Gram entry sum_i a_i b_i over the block's rows: FP64 for the FP64 panel.
// For the FP32 panel every entry of V is at most 1 + 2^-23 in magnitude
// (|v_i| = |x_i| / |v0| with |v0| >= ||x||), so ||v^||^2 <= 2 (1 + 2^-22) and,
// by Cauchy-Schwarz, every partial sum of products of the integers N is below
// 2^(2(P - vexp) + 1) <= 2^61: the Gram matrix of V^ is exact in 64-bit
// integers.
__device__ __forceinline__ double gram_entry(const double *a, const double *b, int nr) {
  double s0 = 0.0, s1 = 0.0;
  int i = 0;
  for (; i + 1 < nr; i += 2) {
    s0 = fma(a[i], b[i], s0);
    s1 = fma(a[i + 1], b[i + 1], s1);
  }
  if (i < nr) s0 = fma(a[i], b[i], s0);
  return s0 + s1;
}
__device__ __forceinline__ long long gram_entry(const int *a, const int *b, int nr) {
  long long s0 = 0, s1 = 0;
  int i = 0;
  for (; i + 1 < nr; i += 2) {
    s0 += (long long)a[i] * b[i];
    s1 += (long long)a[i + 1] * b[i + 1];
  }
  if (i < nr) s0 += (long long)a[i] * b[i];
  return s0 + s1;
}

// Slices and the Gram matrix of a finished panel (see panel_kernel).  Ps holds
// the block's rows of the factored panel (F has been written): below the
// diagonal V itself, or for the FP32 panel x with V = x viv[column]; V^
// replaces them.  `nbar` grid barriers came before.
template <typename Real>
__device__ void panel_tail(int bw, int cs, Real *Ps, const float *viv, int c, int P, int r0, int nr,
                           unsigned *counter, DeviceControl *ctrl, const PanelTail &tl, unsigned nbar) {
  using V = TailV<Real>;
  constexpr bool EXACT = sizeof(Real) == 4;  // integer V^ and Gram matrix
  __shared__ unsigned char pa[QR_B * (QR_B + 1) / 2], pb[QR_B * (QR_B + 1) / 2];
  V *Vh = reinterpret_cast<V *>(Ps);
  int *es = reinterpret_cast<int *>(Vh + (size_t)cs * QR_B);  // the slab's row exponents after V^
  const int tid = threadIdx.x;
  const int npairs = bw * (bw + 1) / 2;
  __syncthreads();
  // (1) V^ in place; the upper-triangle pair table (a <= b), column by column
  for (int e = tid; e < nr * bw; e += PNT) {
    const int i = e % nr, t = e / nr;
    Vh[t * cs + i] = round_entry(viv ? (Real)(Ps[t * cs + i] * viv[t]) : Ps[t * cs + i], r0 + i, t, tl);
  }
  for (int idx = tid; idx < npairs; idx += PNT) {
    int b = 0, rem = idx;
    while (rem > b) { rem -= b + 1; ++b; }
    pa[idx] = (unsigned char)rem;
    pb[idx] = (unsigned char)b;
  }
  __syncthreads();
  // this block's part of the Gram matrix, one thread per entry
  for (int idx = tid; idx < npairs; idx += PNT) {
    auto g = gram_entry(Vh + pa[idx] * cs, Vh + pb[idx] * cs, nr);
    __stcg(reinterpret_cast<decltype(g) *>(tl.gpart) + (size_t)c * npairs + idx, g);
  }
  // (2) natural slices, exponent vexp per column (for the integers N these
  // are N's own digits); (3) row exponents
  for (int e = tid; e < nr * bw; e += PNT) {
    const int i = e % nr, t = e / nr;
    __nv_bfloat16 *dst = tl.vs.base + (r0 + i) + (long long)t * tl.vs.ld;
    if constexpr (EXACT) write_int_slices(Vh[t * cs + i], dst, tl.vs.plane, tl.vs.S);
    else write_fixed_slices(Vh[t * cs + i], tl.vexp, dst, tl.vs.plane, tl.vs.S);
  }
  if (c == 0 && tid < bw) tl.vs.scale[tid] = tl.vexp;
  for (int i = tid; i < nr; i += PNT) {
    if constexpr (EXACT) {
      // |V^| < 2^e for e = msb(max |N|) + 1 + vexp - P (0 for a zero row)
      unsigned mx = 0;
      for (int t = 0; t < bw; ++t) mx = max(mx, (unsigned)abs(Vh[t * cs + i]));
      es[i] = mx == 0 ? 0 : (32 - __clz((int)mx)) + tl.vexp - tl.P;
    } else {
      unsigned long long mx = 0;
      for (int t = 0; t < bw; ++t) mx = max(mx, abs_bits(Vh[t * cs + i]));
      es[i] = exp_above_bits(mx);
    }
    tl.vts.scale[r0 + i] = es[i];
  }
  __syncthreads();
  // transposed slices, the lanes along the columns (for the integers N:
  // N 2^(vexp - e) exactly, e <= vexp)
  for (int e = tid; e < nr * bw; e += PNT) {
    const int t = e % bw, i = e / bw;
    __nv_bfloat16 *dst = tl.vts.base + t + (long long)(r0 + i) * tl.vts.ld;
    if constexpr (EXACT) write_int_slices((long long)Vh[t * cs + i] * (1LL << (tl.vexp - es[i])), dst, tl.vts.plane, tl.vts.S);
    else write_fixed_slices(Vh[t * cs + i], es[i], dst, tl.vts.plane, tl.vts.S);
  }
  if (!grid_barrier(counter, (nbar + 1) * P, ctrl)) return;
  // distributed sum over the blocks in a fixed order: warp w of block c takes
  // entry c + P w, its lanes blocks lane, lane + 32, ... with independent loads
  // (integer sums are exact, then scaled to V^'s unit squared and rounded once)
  const int lane = tid & 31, warp = tid >> 5;
  for (int idx = c + P * warp; idx < npairs; idx += P * PW) {
    constexpr int NZ = (kPanelMaxBlocks + 31) / 32;
    if constexpr (EXACT) {
      const long long *gp = reinterpret_cast<const long long *>(tl.gpart);
      long long v[NZ], sum = 0;
#pragma unroll
      for (int u = 0; u < NZ; ++u) v[u] = lane + 32 * u < P ? __ldcg(&gp[(size_t)(lane + 32 * u) * npairs + idx]) : 0;
#pragma unroll
      for (int u = 0; u < NZ; ++u) sum += v[u];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
      if (lane == 0) __stcg(&tl.G[idx], int64_scaled_to_double(sum, 2 * (tl.vexp - tl.P)));
    } else {
      double v[NZ], sum = 0.0;
#pragma unroll
      for (int u = 0; u < NZ; ++u)
        v[u] = lane + 32 * u < P ? __ldcg(&tl.gpart[(size_t)(lane + 32 * u) * npairs + idx]) : 0.0;
#pragma unroll
      for (int u = 0; u < NZ; ++u) sum += v[u];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
      if (lane == 0) __stcg(&tl.G[idx], sum);
    }
  }
}

// FP32 panel: beta = -sign(x0) ||x|| (R(j,j)) and tau = |v0| / ||x|| of column j
// in FP64 from the FP32 sums sigma and x0 it was formed from.
__device__ __forceinline__ void panel_beta_tau(int j, const float2 *sx, double *s_beta, double *tau) {
  const double sigma = sx[j].x, x0 = sx[j].y;
  double beta = x0, tk = 0.0;
  if (sigma != 0.0) {
    const double norm = sqrt(fma(x0, x0, sigma));
    beta = x0 >= 0.0 ? -norm : norm;
    tk = (fabs(x0) + norm) / norm;
  }
  s_beta[j] = beta;
  if (tau) tau[j] = tk;
}

// ------------------------------------------------------------ panel -------
// F points at F(j0, j0); the panel has `rows` rows and `bw` <= QR_B columns.
// Block c owns panel rows [c*ch, min(rows, (c+1)*ch)).
//
// Real is the arithmetic of the column loop.  Real = double: the FP64 panel.
// Real = float (the tensor-core QR at up to 4 slices): the rows are kept and
// updated in FP32 and the partial sums are FP32, while each reflector's norm,
// sign, beta and tau are formed in FP64 and F(k,k) = beta is written from
// FP64.  Each column is first scaled by a power of two that brings its largest
// entry into [1, 2) (one extra grid barrier), so that FP32's exponent range
// never limits the panel; the reflectors are scale-invariant and R's entries
// are scaled back when written.
//
// TAIL (the tensor-core QR's panel): after the columns, the blocks also round
// the Householder vectors to the grid 2^(vexp - P) (V^), write V^'s fixed-point
// slices (natural, exponent vexp per column; transposed, the exponent of each
// row's largest entry) and form the Gram matrix V^T V^ (per-block partials,
// exact 64-bit integer sums for the FP32 panel, FP64 otherwise; one grid
// barrier and a distributed sum); T follows from it in panel_t_kernel with
// tau_k = 2 / ||v^_k||^2.  Without TAIL the explicit V goes to Vb.
template <bool TAIL, typename Real>
__global__ void __launch_bounds__(PNT) panel_kernel(int rows, int bw, int ch, double *F,
                                                    long long ldf, double *Vb, long long ldv,
                                                    double *tau, double *part, double *rowk,
                                                    unsigned *counter, DeviceControl *ctrl, PanelTail tail) {
  constexpr bool SCALED = sizeof(Real) == 4;
  constexpr unsigned base = SCALED ? 1u : 0u;  // grid barriers before column 0
  extern __shared__ __align__(16) unsigned char p_smem[];
  Real *Ps = reinterpret_cast<Real *>(p_smem);  // the slab, column-major (column t at Ps + t*cs)
  __shared__ Real s_w[QR_B];
  __shared__ double s_par[4];     // beta, -, tau, 1/v0
  __shared__ float s_parf[2];     // FP32 panel: tau, 1/v0 of the current column
  __shared__ float s_iv[QR_B];    // FP32 panel: 1/v0 per column (V = x / v0 below the diagonal)
  __shared__ float2 s_sx[QR_B];   // FP32 panel: sigma and x0 per column
  __shared__ double s_beta[QR_B];
  __shared__ double s_up[QR_B];   // per-column factor back to F's scale (scaled panels) ...
  __shared__ int s_ke[QR_B];      // ... and its exponent
  __shared__ Real s_red[PW][32];
  const int P = gridDim.x;
  const int c = blockIdx.x;
  const int r0 = c * ch;
  const int nr = max(0, min(rows, r0 + ch) - r0);
  const int cs = ch | 1;  // column stride of Ps: odd, so a warp reading one row across columns hits distinct banks
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  Real *parts = reinterpret_cast<Real *>(part);
  Real *rows_k = reinterpret_cast<Real *>(rowk);
  unsigned long long *tparts = reinterpret_cast<unsigned long long *>(part);  // FP32 panel: tagged partials
  unsigned long long *trows = reinterpret_cast<unsigned long long *>(rowk);

  if constexpr (SCALED) {
    // (0) the largest exponent field of each column over all blocks
    __shared__ int s_ex[PW][32];
    int *pe = reinterpret_cast<int *>(part + (size_t)2 * P * QR_B);  // after the two tagged buffers
    for (int t = warp; t < bw; t += PW) {
      unsigned mx = 0;
      for (int i = lane; i < nr; i += 32)
        mx = max(mx, (unsigned)((__double_as_longlong(F[(r0 + i) + t * ldf]) >> 52) & 0x7ff));
      mx = __reduce_max_sync(0xffffffffu, mx);
      if (lane == 0) __stcg(&pe[(size_t)c * QR_B + t], (int)mx);
    }
    if (!grid_barrier(counter, (unsigned)P, ctrl)) return;
    {
      const int t = tid & 31, j = tid >> 5;
      int v[kPanelMaxBlocks / PW];
#pragma unroll
      for (int u = 0; u < kPanelMaxBlocks / PW; ++u) {
        const int b = j + u * PW;
        v[u] = (t < bw && b < P) ? __ldcg(&pe[(size_t)b * QR_B + t]) : 0;
      }
      int mx = 0;
#pragma unroll
      for (int u = 0; u < kPanelMaxBlocks / PW; ++u) mx = max(mx, v[u]);
      s_ex[j][t] = mx;
    }
    __syncthreads();
    if (tid < QR_B) {
      int E = 0;
#pragma unroll
      for (int j = 0; j < PW; ++j) E = max(E, s_ex[j][tid]);
      s_up[tid] = ldexp(1.0, E - 1023);  // largest entry / 2^(E-1023) lies in [1, 2)
      s_ex[0][tid] = E;
      s_ke[tid] = E - 1023;
    }
    __syncthreads();
    for (int e = tid; e < ch * bw; e += PNT) {
      const int i = e % ch, t = e / ch;
      Ps[t * cs + i] = (i < nr) ? double_to_scaled_float(F[(r0 + i) + t * ldf], 1023 - s_ex[0][t]) : Real(0);
    }
  } else {
    for (int e = tid; e < ch * bw; e += PNT) {
      const int i = e % ch, t = e / ch;
      Ps[t * cs + i] = (i < nr) ? (Real)F[(r0 + i) + t * ldf] : Real(0);
    }
  }
  __syncthreads();

  bool fused = false;  // FP32 panel: s_red already holds column k's partial sums
  for (int k = 0; k < bw; ++k) {
    const int buf = k & 1;
    Real *pb = parts + (size_t)buf * P * QR_B;
    Real *rk = rows_k + (size_t)buf * QR_B;
    // rows of this block strictly below row k
    const int i_lo = max(0, k + 1 - r0);
    // (a) partials: t == k gives sum x_i^2, t > k gives sum x_i a_it.  Thread
    // (t = lane, g = warp) sums rows i_lo + g, i_lo + g + 8, ... (the odd
    // column stride keeps the lanes' reads of one row on distinct banks); warp 0
    // adds the 8 row groups in a fixed order and publishes the block's
    // partials and, in the block holding it, row k.
    // (The FP32 panel forms them inside the previous column's update.)
    if (!SCALED || !fused) {
      Real s0 = 0, s1 = 0;
      if (lane >= k && lane < bw) {
        int i = i_lo + warp;
        for (; i + PW < nr; i += 2 * PW) {
          s0 += Ps[k * cs + i] * Ps[lane * cs + i];
          s1 += Ps[k * cs + i + PW] * Ps[lane * cs + i + PW];
        }
        if (i < nr) s0 += Ps[k * cs + i] * Ps[lane * cs + i];
      }
      s_red[warp][lane] = s0 + s1;
      __syncthreads();
    }
    const unsigned ep = tail.epoch0 + (unsigned)k;
    if (warp == 0) {
      Real S = 0;
#pragma unroll
      for (int j = 0; j < PW; ++j) S += s_red[j][lane];
      if (lane >= k && lane < bw) {
        if constexpr (SCALED) {
          __stcg(&tparts[(size_t)buf * P * QR_B + (size_t)c * QR_B + lane], epoch_tag(ep, S));
          if (k >= r0 && k < r0 + nr) __stcg(&trows[buf * QR_B + lane], epoch_tag(ep, Ps[lane * cs + (k - r0)]));
        } else {
          __stcg(&pb[(size_t)c * QR_B + lane], S);
          if (k >= r0 && k < r0 + nr) __stcg(&rk[lane], Ps[lane * cs + (k - r0)]);
        }
      }
    }
    // (b) FP64 panel: one barrier per column, arrived at by warp 0's thread 0
    // once the warp's stores are ordered before it.  FP32 panel: no barrier;
    // (c) waits for the tagged partials themselves.
    if constexpr (!SCALED) {
      if (!grid_barrier(counter, (unsigned)(k + 1 + base) * P, ctrl)) return;
    }
    // (c) every block reduces the partials in the same fixed order; warp 0 adds
    // the 8 partial sums and forms the reflector.
    Real rkt = 0;
    if constexpr (SCALED) {
      // thread (t = lane, j = warp) loads the tagged partials of blocks j,
      // j + 8, ... (and warp 0 row k) and reloads those not yet of epoch ep
      // (bounded, as the grid barrier), then adds them in a fixed order
      const int t = lane, j = warp;
      const unsigned long long *tp = tparts + (size_t)buf * P * QR_B + t;
      Real acc = 0;
      bool fail = false;
      if (t >= k && t < bw) {
        unsigned long long v[kPanelMaxBlocks / PW];
        unsigned long long r = warp == 0 ? __ldcg(&trows[buf * QR_B + t]) : epoch_tag(ep, 0.0f);
#pragma unroll
        for (int u = 0; u < kPanelMaxBlocks / PW; ++u) {
          const int b = j + u * PW;
          v[u] = (b < P) ? __ldcg(tp + (size_t)b * QR_B) : epoch_tag(ep, 0.0f);
        }
        long long polls = 0;
        while (true) {
          bool all = tag_epoch(r) == ep;
#pragma unroll
          for (int u = 0; u < kPanelMaxBlocks / PW; ++u) all &= tag_epoch(v[u]) == ep;
          if (all) break;
          if ((++polls & 63) == 0 && *(volatile int *)&ctrl->abort) { fail = true; break; }
          if (polls > kSpinLimit) {
            atomicCAS(&ctrl->status, PURL_OK, PURL_ERR_TIMEOUT);
            atomicExch(&ctrl->abort, 1);
            fail = true;
            break;
          }
          if (tag_epoch(r) != ep) r = __ldcg(&trows[buf * QR_B + t]);
#pragma unroll
          for (int u = 0; u < kPanelMaxBlocks / PW; ++u)
            if (tag_epoch(v[u]) != ep) v[u] = __ldcg(tp + (size_t)(j + u * PW) * QR_B);
        }
#pragma unroll
        for (int u = 0; u < kPanelMaxBlocks / PW; ++u) acc += tag_value(v[u]);
        rkt = tag_value(r);
      }
      // thread 0 (t = 0 < k, no partials to wait for) forms the previous
      // column's beta and tau in FP64 meanwhile
      if (tid == 0 && k > 0) panel_beta_tau(k - 1, s_sx, s_beta, c == 0 ? tau : nullptr);
      s_red[j][t] = acc;
      if (__syncthreads_or(fail)) return;
    } else {
      // every block reduces the partials in the same fixed order: thread
      // (t = tid % 32, j = tid / 32) sums blocks j, j + 8, ... with independent
      // loads (one L2 round trip, not one per block); row k comes in the same trip
      rkt = (warp == 0 && lane < bw) ? __ldcg(&rk[lane]) : Real(0);
      const int t = tid & 31, j = tid >> 5;
      Real acc = 0;
      if (t >= k && t < bw) {
        Real v[kPanelMaxBlocks / PW];
#pragma unroll
        for (int u = 0; u < kPanelMaxBlocks / PW; ++u) {
          const int b = j + u * PW;
          v[u] = (b < P) ? __ldcg(&pb[(size_t)b * QR_B + t]) : Real(0);
        }
#pragma unroll
        for (int u = 0; u < kPanelMaxBlocks / PW; ++u) acc += v[u];
      }
      s_red[j][t] = acc;
      __syncthreads();
    }
    if constexpr (SCALED) {
      // FP32 panel: the reflector in FP32, by every lane of warp 0 (its inputs
      // are FP32 sums): two independent chains, 1/||x|| and 1/sigma; with
      // |v0| = |x0| + ||x||, tau = |v0| / ||x|| and 1/|v0| = (||x|| - |x0|) / sigma
      // (no cancellation while sigma >= x0^2; otherwise 1/|v0| directly).
      // beta (for R(k,k)) and tau follow in FP64 off the critical path.
      if (warp == 0) {
        Real S = 0;
#pragma unroll
        for (int j = 0; j < PW; ++j) S += s_red[j][lane];  // S(k) = sigma, S(t>k) = dot_t
        const float sigma = __shfl_sync(0xffffffffu, S, k), x0 = __shfl_sync(0xffffffffu, rkt, k);
        float tk = 0.0f, iv = 1.0f;
        if (sigma != 0.0f) {
          const float n2 = fmaf(x0, x0, sigma), ax = fabsf(x0);
          const float rn = rsqrtf(n2), rs = __frcp_rn(sigma);
          const float norm = n2 * rn;
          const float iav0 = sigma >= x0 * x0 ? (norm - ax) * rs : __frcp_rn(ax + norm);
          tk = (ax + norm) * rn;
          iv = x0 >= 0.0f ? iav0 : -iav0;
        }
        // w_t = tau (a_kt + v(k+1:)^T a_t) with v(k+1:) = x(k+1:)/v0
        if (lane > k && lane < bw) s_w[lane] = tk * (rkt + S * iv);
        if (lane == 0) {
          s_parf[0] = tk;
          s_parf[1] = iv;
          s_iv[k] = iv;
          s_sx[k] = make_float2(sigma, x0);
        }
      }
      __syncthreads();
      fused = false;
      if (s_parf[0] != 0.0f) {
        // (d) a_t -= w_t v for t > k, v = x / v0 below row k and 1 at row k:
        // thread (t = lane, g = warp) takes rows i_from + g, i_from + g + PW, ...
        // Column k itself stays unscaled (v is formed where it is used).  The
        // warp shares each updated row, so lane t also accumulates the next
        // column's partial sum x_{k+1,i} a_{t,i} over the rows below k + 1.
        const Real iv = s_parf[1];
        const Real w = (lane > k && lane < bw) ? s_w[lane] : Real(0);
        const int kn = (k + 1) & 31;
        Real s0 = 0;
        for (int i = max(0, k - r0) + warp; i < nr; i += PW) {
          const Real v = (r0 + i == k) ? Real(1) : Ps[k * cs + i] * iv;
          Real a = Ps[lane * cs + i];
          if (lane > k && lane < bw) {
            a -= w * v;
            Ps[lane * cs + i] = a;
          }
          const Real xn = __shfl_sync(0xffffffffu, a, kn);
          if (r0 + i > k + 1) s0 += xn * a;
        }
        s_red[warp][lane] = s0;
        fused = true;
      }
      __syncthreads();
    } else {
      if (warp == 0) {
        Real S = 0;
#pragma unroll
        for (int j = 0; j < PW; ++j) S += s_red[j][lane];  // S(k) = sigma, S(t>k) = dot_t
        const double sigma = (double)__shfl_sync(0xffffffffu, S, k), x0 = (double)__shfl_sync(0xffffffffu, rkt, k);
        double beta, tk, inv_v0;
        if (sigma == 0.0) {
          beta = x0; tk = 0.0; inv_v0 = 1.0;
        } else {
          // one division: r = 1 / (v0 norm) gives 1/v0 = norm r and
          // tau = (beta - x0) / beta = |v0| / norm = |v0| v0 r
          const double norm = sqrt(fma(x0, x0, sigma));
          beta = (x0 >= 0.0) ? -norm : norm;
          const double v0 = x0 - beta;
          const double r = 1.0 / (v0 * norm);
          inv_v0 = norm * r;
          tk = fabs(v0) * v0 * r;
        }
        // w_t = tau (a_kt + v(k+1:)^T a_t) with v(k+1:) = x(k+1:)/v0
        if (lane > k && lane < bw) s_w[lane] = (Real)(tk * ((double)rkt + (double)S * inv_v0));
        if (lane == 0) {
          s_par[0] = beta; s_par[2] = tk; s_par[3] = inv_v0;
          if (c == 0) tau[k] = tk;
        }
      }
      __syncthreads();
      if (s_par[2] != 0.0) {
        // (d) v = x / v0 below row k, 1 at row k (where beta goes), and
        // a_t -= w_t v for t > k: thread (t = lane, g = warp) takes rows
        // i_from + g, i_from + g + 8, ...; lane k writes column k
        const Real iv = (Real)s_par[3];
        const Real beta = (Real)s_par[0];
        const Real w = (lane > k && lane < bw) ? s_w[lane] : Real(0);
        for (int i = max(0, k - r0) + warp; i < nr; i += PW) {
          const bool diag = r0 + i == k;
          const Real x = Ps[k * cs + i];
          const Real v = diag ? Real(1) : x * iv;
          __syncwarp();
          if (lane == k) Ps[k * cs + i] = diag ? beta : v;
          else if (lane > k && lane < bw) Ps[lane * cs + i] -= w * v;
        }
      }
      __syncthreads();
    }
  }
  if constexpr (SCALED) {
    if (tid == 0) panel_beta_tau(bw - 1, s_sx, s_beta, c == 0 ? tau : nullptr);
    __syncthreads();
  }

  for (int e = tid; e < nr * bw; e += PNT) {
    int i = e % nr, t = e / nr;
    int gi = r0 + i;
    double x;
    if constexpr (SCALED) {  // R back to F's scale (beta from FP64); V = x / v0 is scale-free
      const float f = Ps[t * cs + i];
      x = gi == t ? s_beta[t] * s_up[t]
                  : (gi < t ? scaled_float_to_double_any(f, s_ke[t]) : scaled_float_to_double(f * s_iv[t], 0));
    } else {
      x = Ps[t * cs + i];
    }
    F[gi + t * ldf] = x;
    if constexpr (!TAIL) Vb[gi + t * ldv] = (gi < t) ? 0.0 : (gi == t ? 1.0 : x);
  }
  // grid barriers so far: FP32 panel the scale pass only, FP64 panel one per column
  if constexpr (TAIL)
    panel_tail(bw, cs, Ps, SCALED ? s_iv : nullptr, c, P, r0, nr, counter, ctrl, tail, SCALED ? base : (unsigned)bw);
}

// ------------------------------------------------------------ T factor ----
// Sum the split-K partials of the Gram matrix V^T V and form the compact-WY T
// factor (I - V T V^T = H_0 ... H_{b-1}).  One block.  On this GPU a dependent
// FP64 operation costs tens of cycles, so the column recurrence
//   T(0:k,k) = -tau_k T(0:k,0:k) G(0:k,k)
// (a chain of ~b^2/2 dependent FMAs per row) is evaluated blockwise: the
// recurrence inside diagonal blocks of 8 columns, then the standard merge of
// two adjacent blocks, T12 = -T11 (G12 T22), on blocks of 8 and 16 columns,
// all threads working on independent entries.
// With tau_from_gram, tau_k is re-derived as 2 / (v_k^T v_k) from the Gram
// matrix itself, so that each I - tau_k v_k v_k^T is orthogonal for exactly the
// vectors the Gram matrix was formed from (used when the products see a
// rounded copy of V).
__global__ void __launch_bounds__(256) larft_kernel(int bw, int splits, const double *Gp,
                                                    const double *tau, double *T, bool tau_from_gram) {
  __shared__ LarftSmem L;
  for (int e = threadIdx.x; e < QR_B * QR_B; e += blockDim.x) {
    const int i = e % QR_B, j = e / QR_B;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    if (i < bw && j < bw) {
      const int f = i + j * bw;
      int z = 0;
      for (; z + 3 < splits; z += 4) {
        a0 += Gp[(size_t)z * bw * bw + f];
        a1 += Gp[(size_t)(z + 1) * bw * bw + f];
        a2 += Gp[(size_t)(z + 2) * bw * bw + f];
        a3 += Gp[(size_t)(z + 3) * bw * bw + f];
      }
      for (; z < splits; ++z) a0 += Gp[(size_t)z * bw * bw + f];
    }
    L.Gm[i][j] = (a0 + a1) + (a2 + a3);
  }
  __syncthreads();
  larft_core(bw, L, tau, T, tau_from_gram);
}

// T factor of a tensor-core QR panel from the Gram matrix of its rounded
// vectors (upper triangle column by column, as the panel's tail sums it):
// tau_k = 2 / ||v^_k||^2.  One block; it runs beside the next kernels of the QR,
// which do not need T.
__global__ void __launch_bounds__(PNT) panel_t_kernel(int bw, const double *__restrict__ G,
                                                      const double *__restrict__ tau, double *T) {
  __shared__ LarftSmem L;
  const int tid = threadIdx.x;
  const int npairs = bw * (bw + 1) / 2;
  for (int e = tid; e < QR_B * QR_B; e += PNT) L.Gm[e % QR_B][e / QR_B] = 0.0;
  __syncthreads();
  for (int idx = tid; idx < npairs; idx += PNT) {
    int b = 0, a = idx;  // (a, b), a <= b, column by column
    while (a > b) { a -= b + 1; ++b; }
    const double g = __ldcg(&G[idx]);
    L.Gm[a][b] = g;
    L.Gm[b][a] = g;
  }
  __syncthreads();
  larft_core(bw, L, tau, T, true);
}

// W2(:, c) = op(T) * sum_z Wp_z(:, c); op(T) = T^T when trans, else T.
// Block handles 32 columns; T kept in shared memory.
__global__ void __launch_bounds__(256) reduce_tmul_kernel(int bw, int nc, int splits,
                                                          const double *Wp, const double *T,
                                                          bool trans, double *W2) {
  __shared__ double Ts[QR_B][QR_B + 1];
  __shared__ double Ws[32][QR_B + 1];
  const int c0 = blockIdx.x * 32;
  for (int e = threadIdx.x; e < QR_B * QR_B; e += blockDim.x) {
    int i = e % QR_B, j = e / QR_B;
    Ts[i][j] = trans ? T[j + i * QR_B] : T[e];  // Ts = op(T)
  }
  for (int e = threadIdx.x; e < 32 * bw; e += blockDim.x) {
    int r = e % bw, cc = e / bw;
    int col = c0 + cc;
    double s = 0.0;
    if (col < nc)
      for (int z = 0; z < splits; ++z) s += Wp[(size_t)z * bw * nc + r + (size_t)col * bw];
    Ws[cc][r] = s;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 32 * bw; e += blockDim.x) {
    int r = e % bw, cc = e / bw;
    int col = c0 + cc;
    if (col >= nc) continue;
    double s = 0.0;
    for (int l = 0; l < bw; ++l) s += Ts[r][l] * Ws[cc][l];
    W2[r + (size_t)col * bw] = s;
  }
}

// Vb = explicit unit-lower-trapezoidal V of the panel at F(j0, j0).
__global__ void extract_v_kernel(int rows, int bw, const double *F, long long ldf, double *Vb,
                                 long long ldv) {
  long long total = (long long)rows * bw;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    int i = (int)(e % rows), t = (int)(e / rows);
    Vb[i + t * ldv] = (i < t) ? 0.0 : (i == t ? 1.0 : F[i + t * ldf]);
  }
}

__global__ void set_identity_kernel(int m, int n, double *Q, long long ldq) {
  long long total = (long long)m * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    int i = (int)(e % m), j = (int)(e / m);
    Q[i + j * ldq] = (i == j) ? 1.0 : 0.0;
  }
}

// diag(R) >= 0: flip column j of Q and row j of R where F(j,j) < 0; R gets
// zeros below the diagonal.
__global__ void sign_fix_kernel(int m, int n, const double *F, long long ldf, double *Q,
                                long long ldq, double *R, long long ldr) {
  long long totq = Q ? (long long)m * n : 0;
  long long totr = R ? (long long)n * n : 0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < totq + totr;
       e += (long long)gridDim.x * blockDim.x) {
    if (e < totq) {
      int i = (int)(e % m), j = (int)(e / m);
      if (F[j + j * ldf] < 0.0) Q[i + j * ldq] = -Q[i + j * ldq];
    } else {
      long long f = e - totq;
      int i = (int)(f % n), j = (int)(f / n);
      double v = 0.0;
      if (i <= j) {
        v = F[i + j * ldf];
        if (F[i + i * ldf] < 0.0) v = -v;
      }
      R[i + j * ldr] = v;
    }
  }
}

__global__ void copy_kernel(int m, int n, const double *X, long long ldx, double *Y,
                            long long ldy) {
  long long total = (long long)m * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    int i = (int)(e % m), j = (int)(e / m);
    Y[i + j * ldy] = X[i + j * ldx];
  }
}

// Y (Cc x R) = X^T (X is R x Cc), 32 x 32 tiles through shared memory.
__global__ void transpose_kernel(int R, int Cc, const double *__restrict__ X, long long ldx, double *Y,
                                 long long ldy) {
  __shared__ double tile[32][33];
  const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    int r = r0 + threadIdx.x, c = c0 + j;
    tile[j][threadIdx.x] = (r < R && c < Cc) ? X[r + (long long)c * ldx] : 0.0;
  }
  __syncthreads();
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    int c = c0 + threadIdx.x, r = r0 + j;
    if (r < R && c < Cc) Y[c + (long long)r * ldy] = tile[threadIdx.x][j];
  }
}

int grid_for(long long total, const DeviceInfo *di) {
  long long g = (total + 255) / 256;
  long long cap = (long long)di->num_sms * 16;
  if (g > cap) g = cap;
  return (int)(g < 1 ? 1 : g);
}

// Max co-resident blocks for a panel launch with `smem` dynamic bytes.  The
// panel's shared memory changes with every panel (rows shrink), so results
// are cached per 4 KB step of shared memory, computed for the step's upper
// end (capacity only falls as shared memory grows); the kernel's dynamic
// shared-memory limit is only ever raised.  Returns 0 when `smem` does not fit
// beside the kernel's static shared memory.
template <bool TAIL, typename Real>
int panel_capacity(const DeviceInfo *di, size_t smem) {
  static std::mutex mu;
  static std::map<std::pair<int, size_t>, int> cache;
  static std::map<int, size_t> limit;
  std::lock_guard<std::mutex> lock(mu);
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, panel_kernel<TAIL, Real>) != cudaSuccess) return 0;
  const size_t room = (size_t)di->max_smem_optin > fa.sharedSizeBytes ? di->max_smem_optin - fa.sharedSizeBytes : 0;
  if (smem > room) return 0;
  size_t step = (smem + 4095) / 4096 * 4096;
  if (step > room) step = room;
  const auto key = std::make_pair(di->device, step);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  size_t &lim = limit[di->device];
  if (step > 48 * 1024 - fa.sharedSizeBytes && step > lim) {
    if (cudaFuncSetAttribute(panel_kernel<TAIL, Real>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)step) != cudaSuccess)
      return 0;
    lim = step;
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, panel_kernel<TAIL, Real>, PNT, step) != cudaSuccess) return 0;
  const int cap = per_sm * di->num_sms;
  cache[key] = cap;
  return cap;
}

}  // namespace

int panel_blocks(int rows, const DeviceInfo *di) {
  int P = ceil_div(rows, 64);
  if (P > di->num_sms) P = di->num_sms;
  if (P > kPanelMaxBlocks) P = kPanelMaxBlocks;
  return P < 1 ? 1 : P;
}

int qr_plan(Arena &ar, int m, int n, int mode, QrWork *w) {
  (void)mode;
  const DeviceInfo *di = device_info();
  if (!di) return PURL_ERR_CUDA;
  int npan = ceil_div(n, QR_B);
  w->tau = ar.take<double>(n > 0 ? n : 1);
  w->T = ar.take<double>((size_t)(npan > 0 ? npan : 1) * QR_B * QR_B);
  w->Vb = ar.take<double>((size_t)(m > 0 ? m : 1) * QR_B);
  w->Wp = ar.take<double>((size_t)QR_MAX_SPLITS * QR_B * (n > 0 ? n : 1));
  w->W2 = ar.take<double>((size_t)QR_B * (n > 0 ? n : 1));
  w->Gp = ar.take<double>((size_t)QR_MAX_SPLITS * QR_B * QR_B);
  w->part = ar.take<double>((size_t)3 * di->num_sms * QR_B);
  w->rowk = ar.take<double>(2 * QR_B);
  w->counters = ar.take<unsigned>(npan > 0 ? npan : 1);
  return PURL_OK;
}

// Apply the block reflector of one panel (V in w.Vb, T) to C (rows x nc):
// C <- (I - V op(T) V^T) C with op(T) = T^T (trans, i.e. Q^T C) or T.
static int apply_block(int rows, int bw, int nc, double *C, int ldc, const double *T, bool trans,
                       QrWork &w, const DeviceInfo *di, cudaStream_t s) {
  if (nc <= 0 || rows <= 0 || bw <= 0) return PURL_OK;
  int splits, chunk;
  choose_splits(bw, nc, rows, di->num_sms, &splits, &chunk);
  PURL_TRY(gemm_f64_splitk(true, false, bw, nc, rows, splits, chunk, w.Vb, rows, C, ldc, w.Wp, s));
  { LaunchScope ls(KC_OTHER, s, 0.0, 0.0, "reduce_tmul_kernel");
  reduce_tmul_kernel<<<ceil_div(nc, 32), 256, 0, s>>>(bw, nc, splits, w.Wp, T, trans, w.W2); }
  PURL_CUDA_TRY(cudaGetLastError());
  return gemm_f64(false, false, rows, nc, bw, -1.0, w.Vb, rows, w.W2, bw, 1.0, C, ldc, s);
}

// One panel: Householder vectors of F(j0:m, j0:j0+bw) (F points at F(j0, j0)),
// explicit V in w.Vb (ld = rows), tau; `counter` must be 0 on entry.
int panel_factor(int rows, int bw, double *Fp, int ldf, double *taup, unsigned *counter, QrWork &w,
                 cudaStream_t s) {
  const DeviceInfo *di = device_info();
  if (!di) return PURL_ERR_CUDA;
  int P = panel_blocks(rows, di);
  int ch = ceil_div(rows, P);
  size_t smem = (size_t)(ch | 1) * QR_B * sizeof(double);
  int cap = panel_capacity<false, double>(di, smem);
  if (cap < P) return PURL_ERR_UNSUPPORTED;
  int ldv = rows;
  long long ldf_ll = ldf, ldv_ll = ldv;
  PanelTail none;
  void *args[] = {&rows, &bw, &ch, &Fp, &ldf_ll, &w.Vb, &ldv_ll, &taup, &w.part, &w.rowk, &counter,
                  (void *)&di->ctrl, &none};
  LaunchScope ls(KC_PANEL, s, 2.0 * rows * bw * (double)bw, 16.0 * rows * bw, "panel_kernel");
  PURL_CUDA_TRY(cudaLaunchCooperativeKernel((const void *)panel_kernel<false, double>, dim3(P), dim3(PNT), args, smem, s));
  return PURL_OK;
}

template <typename Real>
static int panel_tail_launch(int rows, int bw, double *Fp, int ldf, double *taup, unsigned *counter, QrWork &w,
                             const PanelTail &tail, const DeviceInfo *di, cudaStream_t s) {
  int P = panel_blocks(rows, di);
  int ch = ceil_div(rows, P);
  // the panel's rows (V^ replaces them in the tail), then one int per row (the
  // transposed slices' exponents)
  const size_t es_bytes = align_up((size_t)ch * sizeof(int), 16);
  const size_t cs = (size_t)(ch | 1);  // the kernel's column stride
  const size_t smem = cs * QR_B * sizeof(Real) + es_bytes;
  PanelTail tl = tail;
  int cap = panel_capacity<true, Real>(di, smem);
  if (cap < P) return PURL_ERR_UNSUPPORTED;
  int ldv = rows;
  long long ldf_ll = ldf, ldv_ll = ldv;
  void *args[] = {&rows, &bw, &ch, &Fp, &ldf_ll, &w.Vb, &ldv_ll, &taup, &w.part, &w.rowk, &counter,
                  (void *)&di->ctrl, &tl};
  // panel flops plus the Gram matrix of the rounded vectors
  LaunchScope ls(KC_PANEL, s, 2.0 * rows * bw * (double)bw + (double)rows * bw * (bw + 1), 16.0 * rows * bw,
                 "panel_kernel");
  PURL_CUDA_TRY(cudaLaunchCooperativeKernel((const void *)panel_kernel<true, Real>, dim3(P), dim3(PNT), args, smem, s));
  return PURL_OK;
}

// T of the panel whose tail wrote tail.G, on stream s.
int panel_t(int rows, int bw, const double *taup, const PanelTail &tail, cudaStream_t s) {
  (void)rows;
  LaunchScope ls(KC_OTHER, s, 0.0, 8.0 * bw * (bw + 1) / 2.0, "panel_t_kernel");
  panel_t_kernel<<<1, PNT, 0, s>>>(bw, tail.G, taup, tail.T);
  return cudaGetLastError() == cudaSuccess ? PURL_OK : PURL_ERR_CUDA;
}

// The panel runs in FP32 (FP64 reflector parameters) when V^ carries at most
// 31 bits (up to 4 slices), in FP64 otherwise.
int panel_factor_tail(int rows, int bw, double *Fp, int ldf, double *taup, unsigned *counter, QrWork &w,
                      const PanelTail &tail, cudaStream_t s) {
  const DeviceInfo *di = device_info();
  if (!di) return PURL_ERR_CUDA;
  if (tail.P <= 31) return panel_tail_launch<float>(rows, bw, Fp, ldf, taup, counter, w, tail, di, s);
  return panel_tail_launch<double>(rows, bw, Fp, ldf, taup, counter, w, tail, di, s);
}

// T factor of one panel from split-K partials of its Gram matrix V^T V.
int larft_from_gram(int bw, int splits, const double *Gp, const double *taup, double *Tp, cudaStream_t s,
                    bool tau_from_gram) {
  { LaunchScope ls(KC_OTHER, s, 0.0, 0.0, "larft_kernel"); larft_kernel<<<1, 256, 0, s>>>(bw, splits, Gp, taup, Tp, tau_from_gram); }
  return cudaGetLastError() == cudaSuccess ? PURL_OK : PURL_ERR_CUDA;
}

int extract_v(int rows, int bw, const double *Fp, int ldf, double *Vb, cudaStream_t s) {
  const DeviceInfo *di = device_info();
  if (!di) return PURL_ERR_CUDA;
  { LaunchScope ls(KC_OTHER, s, 0.0, 0.0, "extract_v_kernel");
    extract_v_kernel<<<grid_for((long long)rows * bw, di), 256, 0, s>>>(rows, bw, Fp, ldf, Vb, rows); }
  return cudaGetLastError() == cudaSuccess ? PURL_OK : PURL_ERR_CUDA;
}

int set_identity(int m, int n, double *Q, int ldq, cudaStream_t s) {
  const DeviceInfo *di = device_info();
  if (!di) return PURL_ERR_CUDA;
  { LaunchScope ls(KC_OTHER, s, 0.0, 0.0, "set_identity_kernel"); set_identity_kernel<<<grid_for((long long)m * n, di), 256, 0, s>>>(m, n, Q, ldq); }
  return cudaGetLastError() == cudaSuccess ? PURL_OK : PURL_ERR_CUDA;
}

int qr_factor_f64(int m, int n, double *F, int ldf, QrWork &w, cudaStream_t s) {
  const DeviceInfo *di = device_info();
  if (!di) return PURL_ERR_CUDA;
  if (n == 0) return PURL_OK;
  int npan = ceil_div(n, QR_B);
  PURL_TRY(zero_async(w.counters, sizeof(unsigned) * npan, s));
  for (int p = 0; p < npan; ++p) {
    int j0 = p * QR_B;
    int bw = min(QR_B, n - j0);
    int rows = m - j0;
    double *Fp = F + j0 + (size_t)j0 * ldf;
    double *taup = w.tau + j0;
    PURL_TRY(panel_factor(rows, bw, Fp, ldf, taup, w.counters + p, w, s));
    // T factor from the Gram matrix V^T V
    int gs, gchunk;
    choose_splits(bw, bw, rows, di->num_sms, &gs, &gchunk);
    PURL_TRY(gemm_f64_splitk(true, false, bw, bw, rows, gs, gchunk, w.Vb, rows, w.Vb, rows, w.Gp, s));
    double *Tp = w.T + (size_t)p * QR_B * QR_B;
    PURL_TRY(larft_from_gram(bw, gs, w.Gp, taup, Tp, s));
    // trailing update with Q_p^T
    PURL_TRY(apply_block(rows, bw, n - j0 - bw, Fp + (size_t)bw * ldf, ldf, Tp, true, w, di, s));
  }
  return PURL_OK;
}

int qr_form_q_f64(int m, int n, const double *F, int ldf, QrWork &w, double *Q, int ldq,
                  cudaStream_t s) {
  const DeviceInfo *di = device_info();
  if (!di) return PURL_ERR_CUDA;
  if (m == 0 || n == 0) return PURL_OK;
  PURL_TRY(set_identity(m, n, Q, ldq, s));
  int npan = ceil_div(n, QR_B);
  for (int p = npan - 1; p >= 0; --p) {
    int j0 = p * QR_B;
    int bw = min(QR_B, n - j0);
    int rows = m - j0;
    PURL_TRY(extract_v(rows, bw, F + j0 + (size_t)j0 * ldf, ldf, w.Vb, s));
    const double *Tp = w.T + (size_t)p * QR_B * QR_B;
    PURL_TRY(apply_block(rows, bw, n - j0, Q + j0 + (size_t)j0 * ldq, ldq, Tp, false, w, di, s));
  }
  return PURL_OK;
}

int qr_sign_fix(int m, int n, const double *F, int ldf, double *Q, int ldq, double *R, int ldr,
                cudaStream_t s) {
  const DeviceInfo *di = device_info();
  if (!di) return PURL_ERR_CUDA;
  long long tot = (Q ? (long long)m * n : 0) + (R ? (long long)n * n : 0);
  if (tot == 0) return PURL_OK;
  { LaunchScope ls(KC_OTHER, s, 0.0, 0.0, "sign_fix_kernel"); sign_fix_kernel<<<grid_for(tot, di), 256, 0, s>>>(m, n, F, ldf, Q, ldq, R, ldr); }
  return cudaGetLastError() == cudaSuccess ? PURL_OK : PURL_ERR_CUDA;
}

int copy_matrix(int m, int n, const double *X, int ldx, double *Y, int ldy, cudaStream_t s) {
  const DeviceInfo *di = device_info();
  if (!di) return PURL_ERR_CUDA;
  if ((long long)m * n == 0) return PURL_OK;
  { LaunchScope ls(KC_OTHER, s, 0.0, 0.0, "copy_kernel"); copy_kernel<<<grid_for((long long)m * n, di), 256, 0, s>>>(m, n, X, ldx, Y, ldy); }
  return cudaGetLastError() == cudaSuccess ? PURL_OK : PURL_ERR_CUDA;
}

int transpose_f64(int R, int Cc, const double *X, int ldx, double *Y, int ldy, cudaStream_t s) {
  if ((long long)R * Cc == 0) return PURL_OK;
  dim3 grid(ceil_div(R, 32), ceil_div(Cc, 32));
  if (grid.y > 65535) return PURL_ERR_UNSUPPORTED;
  { LaunchScope ls(KC_OTHER, s, 0.0, 16.0 * (double)R * Cc, "transpose_kernel");
    transpose_kernel<<<grid, dim3(32, 8), 0, s>>>(R, Cc, X, ldx, Y, ldy); }
  return cudaGetLastError() == cudaSuccess ? PURL_OK : PURL_ERR_CUDA;
}

// Full QR with explicit Q and diag(R) >= 0: F holds M on entry (m x n, ld
// ldf) and the packed factor on exit.
int qr_explicit(int m, int n, double *F, int ldf, double *Q, int ldq, double *R, int ldr,
                int mode, QrWork &w, cudaStream_t s) {
  (void)mode;
  PURL_TRY(qr_factor_f64(m, n, F, ldf, w, s));
  if (Q) PURL_TRY(qr_form_q_f64(m, n, F, ldf, w, Q, ldq, s));
  return qr_sign_fix(m, n, F, ldf, Q, ldq, R, ldr, s);
}

}  // namespace purl
