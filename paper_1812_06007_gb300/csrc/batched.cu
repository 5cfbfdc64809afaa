// batched.cu -- PowerURV (Section 3, Eqs. (5)-(6)) on many small independent
// matrices in FP32, in one persistent launch.
//
// Each CTA of a persistent grid takes matrices from an atomic queue (items
// in array order: put the costliest first for load balance) and runs the
// whole factorization of one matrix by itself: Gaussian G, q power steps
// with re-orthonormalisation, the QR of Eq. (5), A V and the QR of Eq. (6).
// Per matrix the data are small (m <= 1024, n <= 512): a CTA's scratch slot
// holds one m x n and one n x n iterate and the T factors (Householder
// vectors stay in place below the factored matrix's diagonal), and nothing
// waits on another CTA -- no grid barrier, no spin-wait.  Building blocks, all CTA-wide:
//   cta_gemm      C = alpha op(A) B + beta C, 64x64 register tiles of FP32 FFMA
//                 staged through shared memory (4x4 outputs per thread)
//   panel_factor  unblocked Householder on an NB-column panel held in shared
//                 memory, one barrier per column
//   T factor      compact-WY T of the panel (Gram of V, then the row-wise
//                 LARFT recurrence in one warp)
//   trailing      C -= V T^T (V^T C) as three cta_gemm calls
//   form Q        backward accumulation of the blocks onto [I; 0]
// The panel width NB and the number of CTAs per SM are the tuning knobs
// (purl_urv_batched_autotune times the variants on the caller's batch).
#include <map>
#include <mutex>
#include <tuple>

#include "common.cuh"
#include "profile.cuh"
#include "rng.cuh"

namespace purl {

namespace {

constexpr int BT = 256;  // threads per CTA
constexpr int GBK = 16, GPAD = 4;
constexpr int kMaxM = 1024, kMaxN = 512;
constexpr int RC = 256;  // rows of V staged at a time by the rank-NB updates

// Row stride (floats) of W staged for a rank update with N columns.
__host__ __device__ inline int rank_ws_ld(int N) { return ((N + 3) / 4) * 4 + GPAD; }

struct Variant {
  int nb;    // panel width
  int rpt;   // panel rows per thread (rows <= 256 rpt)
  int minb;  // CTAs per SM the kernel is compiled for
};
constexpr Variant kVariants[] = {{16, 2, 4}, {16, 2, 2}, {32, 2, 2}, {32, 2, 1}, {16, 4, 2}, {32, 4, 1}};
constexpr int kNumVariants = sizeof(kVariants) / sizeof(kVariants[0]);

struct BatchHeader {
  unsigned next;  // queue position
  int status;
};

struct SlotLayout {
  size_t Sm, Sn, Wg, Wg2, Ts, total;  // offsets in floats
};

__host__ __device__ size_t round64(size_t x) { return (x + 63) / 64 * 64; }

SlotLayout slot_layout(int max_m, int max_n, int nb) {
  SlotLayout L{};
  size_t o = 0;
  L.Sm = o;  o += round64((size_t)max_m * max_n);
  L.Sn = o;  o += round64((size_t)max_n * max_n);
  L.Wg = o;  o += round64((size_t)nb * max_n);
  L.Wg2 = o; o += round64((size_t)nb * max_n);
  L.Ts = o;  o += round64((size_t)((max_n + nb - 1) / nb) * nb * nb);
  L.total = o;
  return L;
}

// Product staging: three ring slots of the largest tile shape (16 x 256), or W and
// a 256-row chunk of V for the rank-nb updates, whichever is larger.
__host__ __device__ inline size_t stage_floats(int nb, int max_n) {
  const size_t gemm = 3 * (size_t)GBK * (16 + 256 + 2 * GPAD);
  const size_t rank = (size_t)nb * rank_ws_ld(max_n) + (size_t)nb * (RC + GPAD);
  return gemm > rank ? gemm : rank;
}

size_t smem_floats(int nb, int max_n) {
  return stage_floats(nb, max_n)           // product staging
         + 2 * (size_t)nb * (nb + 1)       // Gram, T
         + (size_t)nb * nb / 2             // T recursion scratch
         + (size_t)(BT / 32) * nb          // per-warp sums
         + 5 * (size_t)nb + 8;             // row k, coefficients, tau, beta, scale, scalars
}

struct Params {
  int count, max_m, max_n, q, reorth;
  const purl_batch_item *items;
  BatchHeader *hdr;
  float *scratch;
  size_t slot_floats;
  SlotLayout L;
};

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ void cp_async4(float *dst_smem, const float *src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// C (M x N, ldc) = alpha op(A) B + beta C; op(A)(i,k) = A[i + k lda] (TA false)
// or A[k + i lda] (TA true); B(k,j) = B[k + j ldb].  beta == 0: C is not read.
// Tiles of BM x (4096 / BM), 4 x 4 outputs per thread, K in steps of 16
// through a 3-stage shared-memory ring filled by cp.async: two steps are in
// flight while one is multiplied, one barrier per step.  BM = 16 or 32 fits
// the skinny products of the compact-WY updates (M = panel width).  With
// UNITV (TA only), A holds Householder vectors in place below a diagonal:
// op(A)(i, k) = A(k, i) for k > i, 1 for k == i, 0 for k < i.  Ends with a
// barrier, so C is visible to the whole CTA on return.
template <bool TA, int BM, bool UNITV = false>
__device__ __noinline__ void cta_gemm(int M, int N, int K, float alpha, const float *A, int lda, const float *B,
                                      int ldb, float beta, float *C, int ldc, float *stage) {
  constexpr int BN = 4096 / BM;
  constexpr int LA = BM * GBK / BT, LB = BN * GBK / BT;
  constexpr int TXN = BM / 4;
  constexpr int BUF = GBK * (BM + BN + 2 * GPAD);
  constexpr int NSTAGE = 3;
  const int tid = threadIdx.x, tx = tid % TXN, ty = tid / TXN;
  const int tm = (M + BM - 1) / BM, tn = (N + BN - 1) / BN;
  const int nk = (K + GBK - 1) / GBK;
  for (int t = 0; t < tm * tn; ++t) {
    const int m0 = (t % tm) * BM, n0 = (t / tm) * BN;
    float acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[r][c] = 0.f;
    auto issue = [&](int step) {  // step < nk: async copies of K-step `step` into its ring slot
      const int k0 = step * GBK, buf = step % NSTAGE;
      float(*As)[BM + GPAD] = reinterpret_cast<float(*)[BM + GPAD]>(stage + buf * BUF);
      float(*Bs)[BN + GPAD] = reinterpret_cast<float(*)[BN + GPAD]>(stage + buf * BUF + GBK * (BM + GPAD));
#pragma unroll
      for (int s = 0; s < LA; ++s) {
        const int e = tid + s * BT;
        int i, kk;
        if (TA) { kk = e % GBK; i = e / GBK; } else { i = e % BM; kk = e / BM; }
        const int gi = m0 + i, gk = k0 + kk;
        if (gi < M && gk < K && !(UNITV && gk <= gi))
          cp_async4(&As[kk][i], TA ? A + gk + (long long)gi * lda : A + gi + (long long)gk * lda);
        else
          As[kk][i] = (UNITV && gi < M && gk == gi) ? 1.f : 0.f;
      }
#pragma unroll
      for (int s = 0; s < LB; ++s) {
        const int e = tid + s * BT;
        const int kb = e % GBK, j = e / GBK;
        const int gk = k0 + kb, gj = n0 + j;
        if (gk < K && gj < N) cp_async4(&Bs[kb][j], B + gk + (long long)gj * ldb);
        else Bs[kb][j] = 0.f;
      }
    };
    // prologue: steps 0 and 1 in flight (a group is committed even when empty)
    if (nk > 0) issue(0);
    cp_async_commit();
    if (nk > 1) issue(1);
    cp_async_commit();
    for (int step = 0; step < nk; ++step) {
      cp_async_wait<1>();  // this thread's copies of `step` have landed
      __syncthreads();     // ... and everyone's; slot (step + 2) % 3 was last read at step - 1
      if (step + 2 < nk) issue(step + 2);
      cp_async_commit();
      const int buf = step % NSTAGE;
      const float(*As)[BM + GPAD] = reinterpret_cast<const float(*)[BM + GPAD]>(stage + buf * BUF);
      const float(*Bs)[BN + GPAD] = reinterpret_cast<const float(*)[BN + GPAD]>(stage + buf * BUF + GBK * (BM + GPAD));
#pragma unroll
      for (int kk = 0; kk < GBK; ++kk) {
        const float4 a = *reinterpret_cast<const float4 *>(&As[kk][4 * tx]);
        const float4 b = *reinterpret_cast<const float4 *>(&Bs[kk][4 * ty]);
        const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(av[r], bv[c], acc[r][c]);
      }
    }
    cp_async_wait<0>();
    __syncthreads();  // every slot is free before the next tile's prologue
    // epilogue: all old values of C are read before any is written
    float old[4][4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int gj = n0 + 4 * ty + c;
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int gi = m0 + 4 * tx + r;
        old[r][c] = (beta != 0.f && gi < M && gj < N) ? C[gi + (long long)gj * ldc] : 0.f;
      }
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int gj = n0 + 4 * ty + c;
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int gi = m0 + 4 * tx + r;
        if (gi < M && gj < N) C[gi + (long long)gj * ldc] = fmaf(alpha, acc[r][c], beta * old[r][c]);
      }
    }
  }
  __syncthreads();
}

// C(0:M, 0:N) += alpha V(0:M, 0:K) W(0:K, 0:N) for K <= NB (the rank-NB
// updates of the compact-WY blocks; with UNITV, V is read as Householder
// vectors stored in place: 1 on its diagonal, 0 above).  W and a chunk of RC rows of V are staged
// in shared memory once; every 64 x 64 tile of the chunk is then computed from
// shared memory without further barriers.
template <int NB, bool UNITV = false>
__device__ __noinline__ void cta_rank_update(int M, int N, int K, float alpha, const float *V, int ldv,
                                             const float *W, int ldw, float *C, int ldc, float *stage) {
  const int wld = rank_ws_ld(N);
  float *Ws = stage;                   // NB x wld, row k = W(k, :)
  float *Vs = stage + NB * wld;        // NB x (RC + GPAD), row k = V(chunk rows, k)
  constexpr int VLD = RC + GPAD;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  for (int e = tid; e < NB * N; e += BT) {
    const int k = e % NB, c = e / NB;
    Ws[k * wld + c] = (k < K) ? W[k + (long long)c * ldw] : 0.f;
  }
  for (int r0 = 0; r0 < M; r0 += RC) {
    const int rows = min(RC, M - r0);
    __syncthreads();  // W staged / the previous chunk is done with Vs
    for (int e = tid; e < NB * RC; e += BT) {
      const int r = e % RC, k = e / RC;
      const int gr = r0 + r;  // with UNITV, V(gr, k) is 1 on the diagonal and 0 above it
      Vs[k * VLD + r] = (k < K && r < rows)
                            ? ((!UNITV || gr > k) ? V[gr + (long long)k * ldv] : (gr == k ? 1.f : 0.f))
                            : 0.f;
    }
    __syncthreads();
    const int tm = (rows + 63) / 64, tn = (N + 63) / 64;
    // the old C of tile t + 1 is loaded while tile t is multiplied
    float nxt[4][4];
    auto load_c = [&](int t) {
      const int m0 = (t % tm) * 64, n0 = (t / tm) * 64;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int gj = n0 + 4 * ty + c;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const int gi = m0 + 4 * tx + r;
          nxt[r][c] = (gi < rows && gj < N) ? C[(r0 + gi) + (long long)gj * ldc] : 0.f;
        }
      }
    };
    if (tm * tn > 0) load_c(0);
    for (int t = 0; t < tm * tn; ++t) {
      const int m0 = (t % tm) * 64, n0 = (t / tm) * 64;
      float old[4][4];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) old[r][c] = nxt[r][c];
      if (t + 1 < tm * tn) load_c(t + 1);
      float acc[4][4];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = 0.f;
#pragma unroll
      for (int k = 0; k < NB; ++k) {
        const float4 a = *reinterpret_cast<const float4 *>(&Vs[k * VLD + m0 + 4 * tx]);
        const float4 b = *reinterpret_cast<const float4 *>(&Ws[k * wld + n0 + 4 * ty]);
        const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(av[r], bv[c], acc[r][c]);
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int gj = n0 + 4 * ty + c;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const int gi = m0 + 4 * tx + r;
          if (gi < rows && gj < N) C[(r0 + gi) + (long long)gj * ldc] = fmaf(alpha, acc[r][c], old[r][c]);
        }
      }
    }
  }
  __syncthreads();
}

struct Smem {
  float *stage;  // product staging
  float *Gm;     // Gram of the panel's V (strict upper part), NB x (NB+1)
  float *Tt;     // T, row-major NB x (NB+1)
  float *tmp;    // T recursion scratch, NB * NB / 2
  float *part;   // per-warp column sums, NW x NB
  float *rowk;   // row k of the panel, NB
  float *fv;     // reflector coefficients of the trailing panel columns, NB
  float *tau, *beta, *scale;
  int *scal;
};

// Sum of p[c] over the 32 lanes of a warp, scattered: the returned value on
// lane L is the warp sum of column L % NB (NB = 16 or 32).  Each halving
// step sends half of the remaining columns to the partner lane and keeps the
// other half (31 shuffles for NB = 32 instead of 32 x 5).
template <int NB>
__device__ __forceinline__ float reduce_scatter(float (&p)[NB], int lane) {
#pragma unroll
  for (int o = NB / 2; o >= 1; o >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int j = 0; j < o; ++j) {
      const float send = up ? p[j] : p[j + o];
      const float keep = up ? p[j + o] : p[j];
      p[j] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  float v = p[0];
#pragma unroll
  for (int o = NB; o < 32; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Compact-WY T of a panel (LARFT) from the strict upper Gram g[l][k] = v_l.v_k
// and tau: leaves of 8 columns by the forward recurrence
//   T[i][k] = -tau_k sum_{i<=l<k} T[i][l] g[l][k],  T[k][k] = tau_k,
// then T12 = -T11 (G12 T22) on blocks of 8, 16, ... columns.  Writes T to
// shared memory (row-major) and to Tp (column-major, NB x NB).
template <int NB>
__device__ void build_T(int bw, const Smem &sm, float *Tp) {
  constexpr int PS = NB + 1, LF = 8;
  const int tid = threadIdx.x;
  float *T = sm.Tt;
  for (int e = tid; e < NB * NB; e += BT) T[(e / NB) * PS + e % NB] = 0.f;
  __syncthreads();
  if (tid < bw) {
    const int i = tid, a = (i / LF) * LF;
    for (int k = i; k < a + LF && k < bw; ++k) {
      if (k == i) {
        T[i * PS + k] = sm.tau[k];
      } else {
        float acc = 0.f;
        for (int l = i; l < k; ++l) acc = fmaf(T[i * PS + l], sm.Gm[l * PS + k], acc);
        T[i * PS + k] = -sm.tau[k] * acc;
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int h = LF; h < NB; h *= 2) {
    const int outs = (NB / (2 * h)) * h * h;
    // tmp = G12 T22 for every pair of sibling blocks
    for (int e = tid; e < outs; e += BT) {
      const int pr = e / (h * h), i = (e % (h * h)) / h, j = e % h;
      const int a = pr * 2 * h, b0 = a + h;
      float acc = 0.f;
      for (int l = 0; l <= j; ++l)
        if (b0 + l < bw && a + i < bw) acc = fmaf(sm.Gm[(a + i) * PS + b0 + l], T[(b0 + l) * PS + b0 + j], acc);
      sm.tmp[e] = acc;
    }
    __syncthreads();
    // T12 = -T11 tmp
    for (int e = tid; e < outs; e += BT) {
      const int pr = e / (h * h), i = (e % (h * h)) / h, j = e % h;
      const int a = pr * 2 * h, b0 = a + h;
      float acc = 0.f;
      for (int l = i; l < h; ++l) acc = fmaf(T[(a + i) * PS + a + l], sm.tmp[pr * h * h + l * h + j], acc);
      if (a + i < bw && b0 + j < bw) T[(a + i) * PS + b0 + j] = -acc;
    }
    __syncthreads();
  }
  for (int e = tid; e < bw * bw; e += BT) {
    const int i = e % bw, k = e / bw;
    Tp[i + k * NB] = T[i * PS + k];
  }
}

// Householder QR of the rows x cols matrix F (in place; ldf), compact WY with
// panels of NB columns.  Leaves R on and above F's diagonal (beta_j on the
// diagonal, before any sign change) and the Householder vectors below it
// (their unit leading entries implicit), and writes every panel's T
// (column-major, NB x NB) to Ts + panel * NB * NB.
//
// The panel lives in registers: thread t holds rows t, t + 256, ... (RPT of
// them) of all NB columns.  Column k takes one CTA-wide reduction of
//   S_c = sum_{r > k} x_r[k] x_r[c]   for every panel column c,
// which gives at once the norm (c = k), the reflector's action on the
// columns c > k, and the Gram entries g[l][k] = v_l . v_k (l < k) that the
// T factor needs; then every thread updates its own rows.
template <int NB, int RPT>
__device__ __noinline__ void cta_qr_factor(int rows_all, int cols, float *F, int ldf, float *Ts,
                                           float *Wg, float *Wg2, const Smem &sm) {
  constexpr int PS = NB + 1;
  constexpr int NW = BT / 32;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int j0 = 0; j0 < cols; j0 += NB) {
    const int bw = min(NB, cols - j0), rows = rows_all - j0;
    float x[RPT][NB];
#pragma unroll
    for (int s = 0; s < RPT; ++s) {
      const int r = tid + s * BT;
#pragma unroll
      for (int c = 0; c < NB; ++c)
        x[s][c] = (r < rows && c < bw) ? F[(j0 + r) + (long long)(j0 + c) * ldf] : 0.f;
    }
#pragma unroll
    for (int k = 0; k < NB; ++k) {
      if (k >= bw) break;
      if (tid == k) {
#pragma unroll
        for (int c = 0; c < NB; ++c) sm.rowk[c] = x[0][c];
      }
      // column sums in halves of 16 (register pressure): lanes L and L ^ 16
      // end with column h + (L & 15)
#pragma unroll
      for (int h = 0; h < NB; h += 16) {
        float pc[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) pc[c] = 0.f;
#pragma unroll
        for (int s = 0; s < RPT; ++s) {
          const int r = tid + s * BT;
          if (r > k && r < rows) {
            const float xk = x[s][k];
#pragma unroll
            for (int c = 0; c < 16; ++c) pc[c] = fmaf(xk, x[s][h + c], pc[c]);
          }
        }
        const float wsum = reduce_scatter<16>(pc, lane);
        if (lane < 16) sm.part[warp * NB + h + lane] = wsum;
      }
      __syncthreads();
      if (warp == 0) {
        float S = 0.f;
        if (lane < NB) {
#pragma unroll
          for (int w = 0; w < NW; ++w) S += sm.part[w * NB + lane];
        }
        const float sg = __shfl_sync(0xffffffffu, S, k);
        const float alpha = sm.rowk[k];
        float beta, tau, scale;
        if (sg == 0.f) {
          beta = alpha; tau = 0.f; scale = 0.f;  // already reduced: H_k = I
        } else {
          const float nrm = sqrtf(fmaf(alpha, alpha, sg));
          beta = alpha >= 0.f ? -nrm : nrm;
          tau = (beta - alpha) / beta;
          scale = 1.f / (alpha - beta);
        }
        if (lane < NB) {
          const float d = fmaf(scale, S, sm.rowk[lane]);  // v_k . (column lane), row k included
          if (lane < k) sm.Gm[lane * PS + k] = d;
          else if (lane > k) sm.fv[lane] = tau * d;
        }
        if (lane == 0) { sm.tau[k] = tau; sm.beta[k] = beta; sm.scale[k] = scale; }
      }
      __syncthreads();
      const float scale = sm.scale[k];
      float v[RPT];
#pragma unroll
      for (int s = 0; s < RPT; ++s) {
        const int r = tid + s * BT;
        v[s] = (r > k && r < rows) ? x[s][k] * scale : 0.f;
        if (r > k && r < rows) x[s][k] = v[s];
      }
#pragma unroll
      for (int c = k + 1; c < NB; ++c) {
        const float fc = sm.fv[c];
#pragma unroll
        for (int s = 0; s < RPT; ++s) x[s][c] = fmaf(-fc, v[s], x[s][c]);
        if (tid == k) x[0][c] -= fc;
      }
      if (tid == k) x[0][k] = sm.beta[k];
    }
    // ---- write back: R on and above the diagonal, V below it ----
#pragma unroll
    for (int s = 0; s < RPT; ++s) {
      const int r = tid + s * BT;
      if (r < rows) {
#pragma unroll
        for (int c = 0; c < NB; ++c) {
          if (c < bw) {
            F[(j0 + r) + (long long)(j0 + c) * ldf] = x[s][c];
          }
        }
      }
    }
    float *Tp = Ts + (size_t)(j0 / NB) * NB * NB;
    build_T<NB>(bw, sm, Tp);
    __syncthreads();
    // ---- trailing update C -= V T^T (V^T C) ----
    const int nc = cols - j0 - bw;
    if (nc > 0) {
      const float *Vp = F + j0 + (long long)j0 * ldf;
      float *Cp = F + j0 + (long long)(j0 + bw) * ldf;
      cta_gemm<true, NB, true>(bw, nc, rows, 1.f, Vp, ldf, Cp, ldf, 0.f, Wg, NB, sm.stage);
      cta_gemm<true, NB>(bw, nc, bw, 1.f, Tp, NB, Wg, NB, 0.f, Wg2, NB, sm.stage);
      cta_rank_update<NB, true>(rows, nc, bw, -1.f, Vp, ldf, Wg2, NB, Cp, ldf, sm.stage);
    }
  }
}

// Q (rows x cols, ldq) = H_1 ... H_cols [I; 0] from the panels cta_qr_factor
// left in F (below its diagonal) and Ts, then the sign fix diag(R) >= 0 read from F's diagonal;
// R (cols x cols, ldr) is written when non-null.
template <int NB>
__device__ __noinline__ void cta_qr_form(int rows_all, int cols, const float *F, int ldf,
                            const float *Ts, float *Wg, float *Wg2, float *Q, int ldq, float *R, int ldr,
                            const Smem &sm) {
  const int tid = threadIdx.x;
  for (long long e = tid; e < (long long)rows_all * cols; e += BT) {
    const int i = (int)(e % rows_all), j = (int)(e / rows_all);
    Q[i + (long long)j * ldq] = (i == j) ? 1.f : 0.f;
  }
  __syncthreads();
  const int npan = (cols + NB - 1) / NB;
  for (int p = npan - 1; p >= 0; --p) {
    const int j0 = p * NB, bw = min(NB, cols - j0), rows = rows_all - j0, nc = cols - j0;
    const float *Vp = F + j0 + (long long)j0 * ldf;
    const float *Tp = Ts + (size_t)p * NB * NB;
    float *Qp = Q + j0 + (long long)j0 * ldq;
    cta_gemm<true, NB, true>(bw, nc, rows, 1.f, Vp, ldf, Qp, ldq, 0.f, Wg, NB, sm.stage);
    cta_gemm<false, NB>(bw, nc, bw, 1.f, Tp, NB, Wg, NB, 0.f, Wg2, NB, sm.stage);
    cta_rank_update<NB, true>(rows, nc, bw, -1.f, Vp, ldf, Wg2, NB, Qp, ldq, sm.stage);
  }
  for (long long e = tid; e < (long long)rows_all * cols; e += BT) {
    const int i = (int)(e % rows_all), j = (int)(e / rows_all);
    if (F[j + (long long)j * ldf] < 0.f) Q[i + (long long)j * ldq] = -Q[i + (long long)j * ldq];
  }
  if (R) {
    for (int e = tid; e < cols * cols; e += BT) {
      const int i = e % cols, j = e / cols;
      float v = 0.f;
      if (i <= j) {
        v = F[i + (long long)j * ldf];
        if (F[i + (long long)i * ldf] < 0.f) v = -v;
      }
      R[i + (long long)j * ldr] = v;
    }
  }
  __syncthreads();
}

__device__ __noinline__ void cta_gaussian(uint64_t seed, int rows, int cols, float *G, int ldg) {
  const long long count = (long long)rows * cols, nblk = (count + 3) / 4;
  for (long long b = threadIdx.x; b < nblk; b += BT) {
    float z[4];
    gaussian_block_f32(seed, 0, (uint64_t)b, z);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const long long e = 4 * b + t;
      if (e < count) G[(e % rows) + (e / rows) * ldg] = z[t];
    }
  }
  __syncthreads();
}

__device__ void cta_copy(int rows, int cols, const float *X, int ldx, float *Y, int ldy) {
  for (long long e = threadIdx.x; e < (long long)rows * cols; e += BT) {
    const int i = (int)(e % rows), j = (int)(e / rows);
    Y[i + (long long)j * ldy] = X[i + (long long)j * ldx];
  }
  __syncthreads();
}

__global__ void batched_reset_kernel(BatchHeader *h) {
  h->next = 0u;
  h->status = PURL_OK;
}

template <int NB, int RPT, int MINB>
__global__ void __launch_bounds__(BT, MINB) urv_batched_kernel(Params p) {
  extern __shared__ float4 smem_raw[];
  float *sf = reinterpret_cast<float *>(smem_raw);
  Smem sm;
  sm.stage = sf;
  sm.Gm = sm.stage + stage_floats(NB, p.max_n);
  sm.Tt = sm.Gm + NB * (NB + 1);
  sm.tmp = sm.Tt + NB * (NB + 1);
  sm.part = sm.tmp + NB * NB / 2;
  sm.rowk = sm.part + (BT / 32) * NB;
  sm.fv = sm.rowk + NB;
  sm.tau = sm.fv + NB;
  sm.beta = sm.tau + NB;
  sm.scale = sm.beta + NB;
  sm.scal = reinterpret_cast<int *>(sm.scale + NB);
  float *slot = p.scratch + (size_t)blockIdx.x * p.slot_floats;
  float *Sm = slot + p.L.Sm, *Sn = slot + p.L.Sn;
  float *Wg = slot + p.L.Wg, *Wg2 = slot + p.L.Wg2, *Ts = slot + p.L.Ts;
  while (true) {
    if (threadIdx.x == 0) sm.scal[0] = (int)atomicAdd(&p.hdr->next, 1u);
    __syncthreads();
    const int idx = sm.scal[0];
    __syncthreads();
    if (idx >= p.count) break;
    const purl_batch_item it = p.items[idx];
    const int m = it.m, n = it.n;
    if (n < 1 || m < n || m > p.max_m || n > p.max_n || it.lda < m || it.ldu < m || it.ldr < n ||
        it.ldv < n || !it.A || !it.U || !it.R || !it.V) {
      if (threadIdx.x == 0) atomicCAS(&p.hdr->status, PURL_OK, PURL_ERR_UNSUPPORTED);
      continue;
    }
    // Y_0 = G in V's storage
    cta_gaussian(it.seed, n, n, it.V, it.ldv);
    const float *Y = it.V;
    int ldy = it.ldv;
    for (int i = 1; i <= p.q; ++i) {
      cta_gemm<false, 64>(m, n, n, 1.f, it.A, it.lda, Y, ldy, 0.f, Sm, m, sm.stage);  // A Y
      const float *Z = Sm;
      int ldz = m;
      if (p.reorth) {
        cta_qr_factor<NB, RPT>(m, n, Sm, m, Ts, Wg, Wg2, sm);
        cta_qr_form<NB>(m, n, Sm, m, Ts, Wg, Wg2, it.U, it.ldu, nullptr, 0, sm);
        Z = it.U;
        ldz = it.ldu;
      }
      cta_gemm<true, 64>(n, n, m, 1.f, it.A, it.lda, Z, ldz, 0.f, Sn, n, sm.stage);  // A^T Z
      Y = Sn;
      ldy = n;
      if (p.reorth && i < p.q) {
        cta_qr_factor<NB, RPT>(n, n, Sn, n, Ts, Wg, Wg2, sm);
        cta_qr_form<NB>(n, n, Sn, n, Ts, Wg, Wg2, it.V, it.ldv, nullptr, 0, sm);
        Y = it.V;
        ldy = it.ldv;
      }
    }
    if (Y != Sn) cta_copy(n, n, Y, ldy, Sn, n);
    // Eq. (5): Y_q = V Z'
    cta_qr_factor<NB, RPT>(n, n, Sn, n, Ts, Wg, Wg2, sm);
    cta_qr_form<NB>(n, n, Sn, n, Ts, Wg, Wg2, it.V, it.ldv, nullptr, 0, sm);
    // Eq. (6): A V = U R
    cta_gemm<false, 64>(m, n, n, 1.f, it.A, it.lda, it.V, it.ldv, 0.f, Sm, m, sm.stage);
    cta_qr_factor<NB, RPT>(m, n, Sm, m, Ts, Wg, Wg2, sm);
    cta_qr_form<NB>(m, n, Sm, m, Ts, Wg, Wg2, it.U, it.ldu, it.R, it.ldr, sm);
  }
}

__global__ void __launch_bounds__(256) gaussian_f32_kernel(uint64_t seed, uint64_t stream_id, int rows,
                                                           long long count, float *G, long long ldg) {
  const long long nblk = (count + 3) / 4;
  for (long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x; b < nblk;
       b += (long long)gridDim.x * blockDim.x) {
    float z[4];
    gaussian_block_f32(seed, stream_id, (uint64_t)b, z);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const long long e = 4 * b + t;
      if (e < count) G[(e % rows) + (e / rows) * ldg] = z[t];
    }
  }
}

using KernelFn = void (*)(Params);

KernelFn variant_kernel(int v) {
  switch (v) {
    case 0: return urv_batched_kernel<16, 2, 4>;
    case 1: return urv_batched_kernel<16, 2, 2>;
    case 2: return urv_batched_kernel<32, 2, 2>;
    case 3: return urv_batched_kernel<32, 2, 1>;
    case 4: return urv_batched_kernel<16, 4, 2>;
    default: return urv_batched_kernel<32, 4, 1>;
  }
}

// CTAs per SM that variant v reaches for (max_m, max_n) (0 if it cannot run).
// The kernel's dynamic shared-memory limit is a property of the function, not
// of the query: it is only ever raised (to the largest size any query needed),
// so a later query for smaller matrices cannot invalidate the launch of a
// larger batch whose occupancy was cached earlier.  Results are cached per
// (device, variant, max_m, max_n), so queries made during stream capture only
// read the cache.
std::mutex g_occ_mu;
std::map<std::tuple<int, int, int, int>, int> g_occ;
std::map<std::pair<int, int>, size_t> g_smem_attr;  // (device, variant) -> limit set

int variant_occupancy(int v, int max_m, int max_n) {
  const DeviceInfo *di = device_info();
  if (!di) return 0;
  std::lock_guard<std::mutex> lock(g_occ_mu);
  const auto key = std::make_tuple(di->device, v, max_m, max_n);
  auto it = g_occ.find(key);
  if (it != g_occ.end()) return it->second;
  int occ = 0;
  const size_t smem = smem_floats(kVariants[v].nb, max_n) * sizeof(float);
  KernelFn fn = variant_kernel(v);
  size_t &limit = g_smem_attr[std::make_pair(di->device, v)];
  bool ok = max_m <= kVariants[v].rpt * BT && smem <= (size_t)di->max_smem_optin;
  if (ok && smem > limit) {
    ok = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) == cudaSuccess;
    if (ok) limit = smem;
  }
  if (ok) {
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, fn, BT, smem) == cudaSuccess)
      occ = blocks < kVariants[v].minb ? blocks : kVariants[v].minb;
  }
  cudaGetLastError();
  g_occ[key] = occ;
  return occ;
}

std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int, int, int>, int> g_tuned;  // (device, count, max_m, max_n, q, reorth)

int default_variant(int max_m, int max_n) {
  for (int v = 0; v < kNumVariants; ++v)
    if (variant_occupancy(v, max_m, max_n) > 0) return v;
  return -1;
}

size_t workspace_for(int max_m, int max_n, int v, int *slots_out) {
  const DeviceInfo *di = device_info();
  if (!di) return 0;
  const int occ = variant_occupancy(v, max_m, max_n);
  if (occ <= 0) return 0;
  const int slots = di->num_sms * occ;
  if (slots_out) *slots_out = slots;
  const SlotLayout L = slot_layout(max_m, max_n, kVariants[v].nb);
  return 256 + (size_t)slots * L.total * sizeof(float);
}

int check_batch_args(int count, const purl_batch_item *items, int max_m, int max_n, int q) {
  if (count < 0) return -1;
  if (!items && count > 0) return -2;
  if (max_m < 1 || max_m > kMaxM) return -3;
  if (max_n < 1 || max_n > kMaxN || max_n > max_m) return -4;
  if (q < 0) return -5;
  return PURL_OK;
}

int launch_batched(int count, const purl_batch_item *items, int max_m, int max_n, int q, int reorth, int v,
                   void *workspace, size_t workspace_bytes, cudaStream_t s) {
  int slots = 0;
  const size_t need = workspace_for(max_m, max_n, v, &slots);
  if (need == 0) return PURL_ERR_UNSUPPORTED;
  if (!workspace || workspace_bytes < need || ((uintptr_t)workspace & 255) != 0) return PURL_ERR_NOMEM;
  Params p{};
  p.count = count;
  p.max_m = max_m;
  p.max_n = max_n;
  p.q = q;
  p.reorth = reorth ? 1 : 0;
  p.items = items;
  p.hdr = reinterpret_cast<BatchHeader *>(workspace);
  p.scratch = reinterpret_cast<float *>(static_cast<char *>(workspace) + 256);
  p.L = slot_layout(max_m, max_n, kVariants[v].nb);
  p.slot_floats = p.L.total;
  const int grid = count < slots ? count : slots;
  { LaunchScope ls(KC_OTHER, s, 0.0, 8.0, "batched_reset_kernel");
    batched_reset_kernel<<<1, 1, 0, s>>>(p.hdr); }
  PURL_CUDA_TRY(cudaGetLastError());
  if (grid == 0) return PURL_OK;
  const size_t smem = smem_floats(kVariants[v].nb, max_n) * sizeof(float);
  { LaunchScope ls(KC_OTHER, s, 0.0, 0.0, "urv_batched_kernel");
    variant_kernel(v)<<<grid, BT, smem, s>>>(p); }
  PURL_CUDA_TRY(cudaGetLastError());
  return PURL_OK;
}

}  // namespace

}  // namespace purl

using namespace purl;

extern "C" {

int purl_gaussian_f32(uint64_t seed, uint64_t stream_id, int rows, int cols, float *G, int ldg,
                      cudaStream_t stream) {
  if (rows < 0) return -3;
  if (cols < 0) return -4;
  if (!G && (long long)rows * cols > 0) return -5;
  if (ldg < (rows > 1 ? rows : 1)) return -6;
  const long long count = (long long)rows * cols;
  if (count == 0) return PURL_OK;
  const DeviceInfo *di = device_info();
  if (!di) return PURL_ERR_CUDA;
  const long long nblk = (count + 3) / 4, want = (nblk + 255) / 256;
  const int grid = (int)(want < (long long)di->num_sms * 8 ? want : (long long)di->num_sms * 8);
  { LaunchScope ls(KC_OTHER, stream, 0.0, 4.0 * count, "gaussian_f32_kernel");
    gaussian_f32_kernel<<<grid, 256, 0, stream>>>(seed, stream_id, rows, count, G, ldg); }
  return cudaGetLastError() == cudaSuccess ? PURL_OK : PURL_ERR_CUDA;
}

int purl_urv_batched_variants(void) { return kNumVariants; }

size_t purl_urv_batched_workspace_bytes(int max_m, int max_n, int variant) {
  if (check_batch_args(0, nullptr, max_m, max_n, 0) != PURL_OK) return 0;
  if (variant >= kNumVariants) return 0;
  if (variant >= 0) return workspace_for(max_m, max_n, variant, nullptr);
  size_t best = 0;
  for (int v = 0; v < kNumVariants; ++v) {
    const size_t b = workspace_for(max_m, max_n, v, nullptr);
    best = b > best ? b : best;
  }
  return best;
}

int purl_urv_factor_batched(int count, const purl_batch_item *items, int max_m, int max_n, int q, int reorth,
                            int variant, void *workspace, size_t workspace_bytes, cudaStream_t stream) {
  PURL_TRY(check_batch_args(count, items, max_m, max_n, q));
  if (variant >= kNumVariants) return -7;
  if (!device_info()) return PURL_ERR_CUDA;
  int v = variant;
  if (v < 0) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tuned.find(std::make_tuple(device_info()->device, count, max_m, max_n, q, reorth ? 1 : 0));
    v = it != g_tuned.end() ? it->second : default_variant(max_m, max_n);
  }
  if (v < 0) return PURL_ERR_UNSUPPORTED;
  return launch_batched(count, items, max_m, max_n, q, reorth, v, workspace, workspace_bytes, stream);
}

int purl_urv_batched_status(void *workspace, cudaStream_t stream) {
  if (!workspace) return -1;
  if (cudaStreamSynchronize(stream) != cudaSuccess) return PURL_ERR_CUDA;
  BatchHeader h{};
  if (cudaMemcpy(&h, workspace, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) return PURL_ERR_CUDA;
  return h.status;
}

int purl_urv_batched_autotune(int count, const purl_batch_item *items, int max_m, int max_n, int q, int reorth,
                              void *workspace, size_t workspace_bytes, cudaStream_t stream, int *variant_out,
                              float *ms_out) {
  PURL_TRY(check_batch_args(count, items, max_m, max_n, q));
  const DeviceInfo *di = device_info();
  if (!di) return PURL_ERR_CUDA;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return PURL_ERR_CUDA;
  int best = -1;
  float best_ms = 0.f;
  int st = PURL_OK;
  for (int v = 0; v < kNumVariants && st == PURL_OK; ++v) {
    const size_t need = workspace_for(max_m, max_n, v, nullptr);
    if (need == 0 || need > workspace_bytes) continue;
    st = launch_batched(count, items, max_m, max_n, q, reorth, v, workspace, workspace_bytes, stream);  // warm-up
    if (st != PURL_OK) break;
    if (cudaEventRecord(e0, stream) != cudaSuccess) { st = PURL_ERR_CUDA; break; }
    st = launch_batched(count, items, max_m, max_n, q, reorth, v, workspace, workspace_bytes, stream);
    if (st != PURL_OK) break;
    if (cudaEventRecord(e1, stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
      st = PURL_ERR_CUDA;
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (best < 0 || ms < best_ms) { best = v; best_ms = ms; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != PURL_OK) return st;
  if (best < 0) return PURL_ERR_NOMEM;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tuned[std::make_tuple(di->device, count, max_m, max_n, q, reorth ? 1 : 0)] = best;
  }
  if (variant_out) *variant_out = best;
  if (ms_out) *ms_out = best_ms;
  return PURL_OK;
}

}  // extern "C"
