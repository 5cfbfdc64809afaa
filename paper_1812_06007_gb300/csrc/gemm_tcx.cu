// gemm_tcx.cu -- BF16 tensor-core products with EXACT accumulation (sm_103a).
//
// The FP32 accumulator of tcgen05.mma does not round to nearest: measured on
// this GPU, a compensated 3-slice product over K = 512 is no more accurate
// than a 2-slice one (error ~ (K/16) 2^-23 of |C|).  This kernel removes that
// floor with the splitting of Ozaki et al. (error-free transformation of a
// matrix product into exact low-precision products): every operand row is
// scaled by a power of two and cut into slices of small integers
// (|alpha| <= 128, exact in BF16), so every product is an integer below 2^14
// and every partial sum of one slice-pair class over 256 of K is an integer
// of magnitude at most (S pairs) 256 2^14 <= 2^24 for S <= 4 -- exactly
// representable, so the accumulator never rounds.
//
// Per 256 of K ("chunk") the classes d = s + t (S of them) accumulate in
// their own TMEM columns; two chunk buffers alternate so the MMA warp fills
// one while the epilogue warps drain the other into per-thread double-FP32
// (hi, lo) sums by the error-free two-sum.  The only error left is the
// slicing itself: 2^(-8S) of each operand row's scale.
//
// Used by the mixed-precision QR (V^T C, the trailing update C - V W, the
// Gram matrix V^T V, Q formation) and by A V (Section 3, Eq. (6)).
//
// Wide configuration (S = 8, FP64 emulation): 8 digits of 8 bits carry every
// operand row to 2^-63 of its scale.  The 8 classes d = s + t < 8 of a
// 128-row N tile of 32 columns fill 2 x 8 x 32 = 512 TMEM columns; a class
// sums at most 8 pairs, so chunks are 128 of K (8 * 128 * 2^14 = 2^24).  All
// 8 slices of a 64-deep k-block of both operands would take 160 KB of shared
// memory, so a pipeline stage holds ONE A slice s with the B slices t < 8 - s
// it meets, and a k-block passes through 8 stages.  The epilogue drains each
// class as an exact integer into two 64-bit accumulators (classes 0-3 and
// 4-7, shifted to a common unit); the dropped pairs (s + t >= 8) weigh below
// 2^-59 of the row and column maxima, so the product is FP64-accurate.
#include <cuda.h>
#include <cuda_bf16.h>

#include "profile.cuh"
#include "qr.cuh"
#include "tc.cuh"
#include "tc_ptx.cuh"
#include "slice_int.cuh"

namespace purl {

int gemm_f64(bool ta, bool tb, int m, int n, int k, double alpha, const double *A, int lda, const double *B, int ldb,
             double beta, double *C, int ldc, cudaStream_t s);

namespace {

// warp 0 TMA, warp 1 MMA, then 16 epilogue warps: 4 per 32-lane quadrant of
// tensor memory, each draining a quarter of the tile's columns
constexpr int TCX_KBC = 4;        // k-blocks per exact chunk (4 x 64 = 256 of K)
constexpr int TCX_GROUP = 16;

// S slices per operand; ALL = every slice pair (s, t) instead of s + t < S
// (2S - 1 classes, used where the product of two sliced matrices must be
// exact, e.g. the Gram matrix of rounded Householder vectors); BN = N tile.
template <int S, bool ALL, int BN>
struct TcxCfg {
  static constexpr bool WIDE = S > 4;  // one A slice per stage, integer drains
  static constexpr int CLASSES = ALL ? 2 * S - 1 : S;
  static constexpr int KBC = WIDE ? 2 : TCX_KBC;  // k-blocks per exact chunk
  static constexpr int A_BYTES = TC_BM * TC_BK * 2;
  static constexpr int B_BYTES = BN * TC_BK * 2;
  static constexpr int STAGE_BYTES = WIDE ? A_BYTES + S * B_BYTES : S * (A_BYTES + B_BYTES);
  static constexpr int STAGES_RAW = (200 * 1024) / STAGE_BYTES;
  static constexpr int STAGES = STAGES_RAW > 8 ? 8 : STAGES_RAW;
  static constexpr int SMEM = STAGES * STAGE_BYTES + 1024;
  static constexpr int USED_COLS = 2 * CLASSES * BN;
  static constexpr int TMEM_COLS = USED_COLS <= 128 ? 128 : (USED_COLS <= 256 ? 256 : 512);
  static constexpr int EPI_WARPS = 16;  // 4 per TMEM lane quadrant: BN / 4 columns each
  static constexpr int THREADS = 64 + 32 * EPI_WARPS;
  static_assert(STAGES >= 2, "stages");
  static_assert(USED_COLS <= 512, "tensor memory");
  static_assert(BN % 32 == 0, "BN");
  static_assert(!WIDE || (!ALL && S <= 8), "wide: s + t < S classes of at most 8 pairs");
  static_assert(!WIDE || BN == 32, "wide: N tile of 32");
  static_assert(STAGE_BYTES % 1024 == 0, "stage alignment");
};

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// (hi, lo) += x, hi + lo exact up to the rounding of lo (error-free two-sum).
__device__ __forceinline__ void two_sum_acc(float &hi, float &lo, float x) {
  const float s = __fadd_rn(hi, x);
  const float bp = __fsub_rn(s, hi);
  const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(x, bp));
  hi = s;
  lo = __fadd_rn(lo, e);
}

template <int S, bool ALL, int BN>
__global__ void __launch_bounds__(TcxCfg<S, ALL, BN>::THREADS, 1)
    tcx_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, TcView va,
                    TcView vb, int M, int N, int K, int k_chunk, int splits, const int *__restrict__ scA,
                    const int *__restrict__ scB, TcEpilogue ep, DeviceControl *ctrl) {
  using Cfg = TcxCfg<S, ALL, BN>;
  constexpr int STAGES = Cfg::STAGES;
  constexpr int TCX_BN = BN;
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t full_bar[STAGES];
  __shared__ __align__(8) uint64_t empty_bar[STAGES];
  __shared__ __align__(8) uint64_t tfull_bar[2];
  __shared__ __align__(8) uint64_t tempty_bar[2];
  __shared__ __align__(8) uint64_t done_bar;
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tiles_m = (M + TC_BM - 1) / TC_BM, tiles_n = (N + TCX_BN - 1) / TCX_BN;
  const int tiles = tiles_m * tiles_n;
  const long long total = (long long)tiles * splits;
  const int per_group = TCX_GROUP * tiles_n;

  // Persistent: this block handles work items blockIdx.x, blockIdx.x + gridDim.x, ...
  // (work = split * tiles + tile).  Every role walks the same sequence.
  auto work_geometry = [&](long long work, int &m0, int &n0, int &kb0, int &nkb) {
    const int z = (int)(work / tiles), pid = (int)(work % tiles);
    const int first_m = (pid / per_group) * TCX_GROUP;
    const int gsize = min(tiles_m - first_m, TCX_GROUP);
    m0 = (first_m + (pid % per_group) % gsize) * TC_BM;
    n0 = ((pid % per_group) / gsize) * TCX_BN;
    kb0 = z * k_chunk;
    const int kend = min(K, kb0 + k_chunk);
    nkb = (kend - kb0 + TC_BK - 1) / TC_BK;
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull_bar[b], 1);
      mbar_init(&tempty_bar[b], Cfg::EPI_WARPS);
    }
    mbar_init(&done_bar, 1);
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                 "r"((uint32_t)Cfg::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;

  if (warp == 0) {
    if (lane == 0) {
      long long kt = 0;  // k-blocks issued so far (stage ring position)
      bool stop = false;
      for (long long work = blockIdx.x; work < total && !stop; work += gridDim.x) {
        int m0, n0, kb0, nkb;
        work_geometry(work, m0, n0, kb0, nkb);
        if constexpr (Cfg::WIDE) {
          // stage = (k-block kb, A slice s) with B slices t < S - s
          for (int kb = 0; kb < nkb && !stop; ++kb) {
            const int kx = kb0 + kb * TC_BK;
            for (int s = 0; s < S; ++s, ++kt) {
              const int st = (int)(kt % STAGES);
              const uint32_t ph = (uint32_t)(kt / STAGES) & 1u;
              if (!mbar_wait(&empty_bar[st], ph ^ 1u, ctrl, &s_abort)) { stop = true; break; }
              mbar_arrive_expect_tx(&full_bar[st], (uint32_t)(Cfg::A_BYTES + (S - s) * Cfg::B_BYTES));
              uint8_t *sa = smem + (size_t)st * Cfg::STAGE_BYTES;
              uint8_t *sb = sa + Cfg::A_BYTES;
              tma_load_3d(sa, &tmA, &full_bar[st], va.r0 + kx, va.c0 + m0, s);
              for (int t = 0; t < S - s; ++t)
                tma_load_3d(sb + t * Cfg::B_BYTES, &tmB, &full_bar[st], vb.r0 + kx, vb.c0 + n0, t);
            }
          }
        } else {
          for (int kb = 0; kb < nkb; ++kb, ++kt) {
            const int st = (int)(kt % STAGES);
            const uint32_t ph = (uint32_t)(kt / STAGES) & 1u;
            if (!mbar_wait(&empty_bar[st], ph ^ 1u, ctrl, &s_abort)) { stop = true; break; }
            mbar_arrive_expect_tx(&full_bar[st], (uint32_t)Cfg::STAGE_BYTES);
            uint8_t *sa = smem + (size_t)st * Cfg::STAGE_BYTES;
            uint8_t *sb = sa + S * Cfg::A_BYTES;
            const int kx = kb0 + kb * TC_BK;
#pragma unroll
            for (int s = 0; s < S; ++s) tma_load_3d(sa + s * Cfg::A_BYTES, &tmA, &full_bar[st], va.r0 + kx, va.c0 + m0, s);
#pragma unroll
            for (int s = 0; s < S; ++s) tma_load_3d(sb + s * Cfg::B_BYTES, &tmB, &full_bar[st], vb.r0 + kx, vb.c0 + n0, s);
          }
        }
      }
      // never leave the block with copies in flight: the last use of every stage
      // must have landed (bounded; normally already true)
      for (long long k = (kt > STAGES ? kt - STAGES : 0); k < kt; ++k)
        mbar_wait(&full_bar[k % STAGES], (uint32_t)(k / STAGES) & 1u, ctrl, &s_abort, false);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // The B slices of a stage lie back to back in shared memory (each a
      // 1024-byte-aligned block of 128-byte rows), and so do the classes in
      // tensor memory: all products of A slice s with B slices t = 0..T-1
      // are ONE MMA of N = T * BN columns writing classes s..s+T-1.
      long long kt = 0, ct = 0;  // k-block and chunk counters across work items
      bool stop = false;
      for (long long work = blockIdx.x; work < total && !stop; work += gridDim.x) {
        int m0, n0, kb0, nkb;
        work_geometry(work, m0, n0, kb0, nkb);
        if constexpr (Cfg::WIDE) {
          for (int kb = 0; kb < nkb && !stop; ++kb) {
            const int kin = kb % Cfg::KBC, b = (int)(ct & 1);
            if (kin == 0) {
              if (!mbar_wait(&tempty_bar[b], ((uint32_t)(ct >> 1) & 1u) ^ 1u, ctrl, &s_abort)) { stop = true; break; }
              tc_fence_after();
            }
            for (int s = 0; s < S; ++s, ++kt) {
              const int st = (int)(kt % STAGES);
              const uint32_t ph = (uint32_t)(kt / STAGES) & 1u;
              if (!mbar_wait(&full_bar[st], ph, ctrl, &s_abort)) { stop = true; break; }
              tc_fence_after();
              const uint32_t sa = smem_u32(smem + (size_t)st * Cfg::STAGE_BYTES);
              const uint32_t sb = sa + Cfg::A_BYTES;
              // B slices t < S - s: classes s..S-1
              const uint32_t dcol = tmem + (uint32_t)((b * Cfg::CLASSES + s) * TCX_BN);
              const uint32_t idesc = idesc_bf16(TC_BM, (S - s) * TCX_BN);
#pragma unroll
              for (int k = 0; k < TC_BK / 16; ++k) {
                const uint64_t ad = sw128_desc(sa + k * 32);
                const uint64_t bd = sw128_desc(sb + k * 32);
                // every class d is first reached at s = 0 (t = d): that product
                // opens the chunk's accumulator
                tc_mma(dcol, ad, bd, idesc, (kin == 0 && s == 0 && k == 0) ? 0u : 1u);
              }
              tc_commit(&empty_bar[st]);
            }
            if (!stop && (kin == Cfg::KBC - 1 || kb == nkb - 1)) {
              tc_commit(&tfull_bar[b]);
              ++ct;
            }
          }
          continue;
        }
        for (int kb = 0; kb < nkb; ++kb, ++kt) {
          const int kin = kb % TCX_KBC, b = (int)(ct & 1);
          if (kin == 0) {
            if (!mbar_wait(&tempty_bar[b], ((uint32_t)(ct >> 1) & 1u) ^ 1u, ctrl, &s_abort)) { stop = true; break; }
            tc_fence_after();
          }
          const int st = (int)(kt % STAGES);
          const uint32_t ph = (uint32_t)(kt / STAGES) & 1u;
          if (!mbar_wait(&full_bar[st], ph, ctrl, &s_abort)) { stop = true; break; }
          tc_fence_after();
          const uint32_t sa = smem_u32(smem + (size_t)st * Cfg::STAGE_BYTES);
          const uint32_t sb = sa + S * Cfg::A_BYTES;
#pragma unroll
          for (int s = 0; s < S; ++s) {
            // s + t < S: B slices 0..S-1-s, classes s..S-1, all first reached at
            // s = 0.  ALL: B slices 0..S-1, classes s..s+S-1; at s >= 1 the last
            // class s+S-1 is new (its first product overwrites), so that slice
            // is a second MMA.
            const int nt = ALL ? (s == 0 ? S : S - 1) : S - s;
            const uint32_t dcol = tmem + (uint32_t)((b * Cfg::CLASSES + s) * TCX_BN);
            const uint32_t idesc = idesc_bf16(TC_BM, nt * TCX_BN);
#pragma unroll
            for (int k = 0; k < TC_BK / 16; ++k) {
              const uint64_t ad = sw128_desc(sa + s * Cfg::A_BYTES + k * 32);
              const uint64_t bd = sw128_desc(sb + k * 32);
              // the first product of a class in a chunk overwrites its accumulator
              tc_mma(dcol, ad, bd, idesc, (kin == 0 && s == 0 && k == 0) ? 0u : 1u);
            }
            if (ALL && s >= 1) {
              const uint32_t dnew = tmem + (uint32_t)((b * Cfg::CLASSES + s + S - 1) * TCX_BN);
              constexpr uint32_t idesc1 = idesc_bf16(TC_BM, TCX_BN);
#pragma unroll
              for (int k = 0; k < TC_BK / 16; ++k) {
                const uint64_t ad = sw128_desc(sa + s * Cfg::A_BYTES + k * 32);
                const uint64_t bd = sw128_desc(sb + (S - 1) * Cfg::B_BYTES + k * 32);
                tc_mma(dnew, ad, bd, idesc1, (kin == 0 && k == 0) ? 0u : 1u);
              }
            }
          }
          tc_commit(&empty_bar[st]);
          if (kin == TCX_KBC - 1 || kb == nkb - 1) {
            tc_commit(&tfull_bar[b]);
            ++ct;
          }
        }
      }
      tc_commit(&done_bar);
    }
  } else {
    // ---------------- epilogue: drain chunks into double-FP32 sums, then write ----------------
    constexpr int HC = TCX_BN / (Cfg::EPI_WARPS / 4);  // columns per epilogue warp
    const int lane_base = 32 * (warp & 3);
    const int cbase = ((warp - 2) >> 2) * HC;  // which part of the columns
    long long ct = 0;
    bool ok = true;
    for (long long work = blockIdx.x; work < total && ok; work += gridDim.x) {
      int m0, n0, kb0, nkb;
      work_geometry(work, m0, n0, kb0, nkb);
      const int nch = (nkb + Cfg::KBC - 1) / Cfg::KBC;
      const bool reads_c = (ep.mode == 0 && ep.beta != 0.0);
      const int row = m0 + lane_base + lane;
      if (reads_c && row < M) {
        // pull this row's part of the C tile into L2 while the products run
        for (int j = 0; j < HC; ++j)
          if (n0 + cbase + j < N)
            asm volatile("prefetch.global.L2 [%0];" ::"l"(ep.C + row + (long long)(n0 + cbase + j) * ep.ldc));
      }
      // narrow: one double-FP32 sum of all classes; wide: exact integer sums
      // H (classes d < S - 4, unit 2^(32 - 8(S-1))) and L (classes d >= S - 4,
      // unit 2^(-8(S-1))), both relative to one class-0 product
      constexpr int NA = Cfg::WIDE ? 1 : HC, NW = Cfg::WIDE ? HC : 1;
      float hi[NA], lo[NA];
      long long accH[NW], accL[NW];
#pragma unroll
      for (int j = 0; j < NA; ++j) hi[j] = lo[j] = 0.0f;
#pragma unroll
      for (int j = 0; j < NW; ++j) accH[j] = accL[j] = 0;
      // the first batch of C is loaded before the wait for the tile's last
      // chunk, so its latency runs under that chunk's products
      constexpr int BATCH = HC < 8 ? HC : 8;  // independent loads of C kept in flight
      constexpr int PRE = 8;                      // of which loaded early
      double cpre[PRE];
#pragma unroll
      for (int jj = 0; jj < PRE; ++jj) cpre[jj] = 0.0;
      for (int c = 0; c < nch; ++c, ++ct) {
        const int b = (int)(ct & 1);
        if (c == nch - 1 && reads_c && row < M) {
#pragma unroll
          for (int jj = 0; jj < PRE; ++jj) {
            const int col = n0 + cbase + jj;
            cpre[jj] = (col < N) ? __ldcg(ep.C + row + (long long)col * ep.ldc) : 0.0;
          }
        }
        if (!mbar_wait(&tfull_bar[b], (uint32_t)(ct >> 1) & 1u, ctrl, &s_abort)) {
          ok = false;
          break;
        }
        tc_fence_after();
#pragma unroll
        for (int d = 0; d < Cfg::CLASSES; ++d) {
          const float w = __int_as_float((127 - 8 * d) << 23);  // 2^(-8d)
          const uint32_t taddr = tmem + ((uint32_t)lane_base << 16) + (uint32_t)((b * Cfg::CLASSES + d) * TCX_BN + cbase);
          if constexpr (Cfg::WIDE) {
            // class sums are exact integers below 2^24 in magnitude
            uint32_t v[HC];
            tmem_ld_cols<HC>(taddr, v);
            if (d < S - 4) {
              const int sh = 8 * (S - 5 - d);
#pragma unroll
              for (int j = 0; j < HC; ++j) accH[j] += (long long)__float2int_rz(__uint_as_float(v[j])) * (1LL << sh);
            } else {
              const int sh = 8 * (S - 1 - d);
#pragma unroll
              for (int j = 0; j < HC; ++j) accL[j] += (long long)__float2int_rz(__uint_as_float(v[j])) * (1LL << sh);
            }
            (void)w;
          } else if constexpr (HC >= 32) {
#pragma unroll
            for (int h = 0; h < HC / 32; ++h) {
              uint32_t v[32];
              tmem_ld32(taddr + (uint32_t)(h * 32), v);
#pragma unroll
              for (int j = 0; j < 32; ++j) two_sum_acc(hi[h * 32 + j], lo[h * 32 + j], __uint_as_float(v[j]) * w);
            }
          } else {
            uint32_t v[HC];
            tmem_ld_cols<HC>(taddr, v);
#pragma unroll
            for (int j = 0; j < HC; ++j) two_sum_acc(hi[j], lo[j], __uint_as_float(v[j]) * w);
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tempty_bar[b]);
      }
      if (ok && nkb > 0 && row < M) {
        const int ea = scA[va.c0 + row];
        // the common updates C = D and C = C - D take one or two FP64 adds;
        // hi and lo become exact doubles through integer bit assembly
        const bool plain = (ep.alpha == 1.0 && ep.beta == 0.0);
        const bool subtract = (ep.alpha == -1.0 && ep.beta == 1.0);
        const int z = (int)(work / tiles);
#pragma unroll
        for (int j0 = 0; j0 < HC; j0 += BATCH) {
          double cv[BATCH];
#pragma unroll
          for (int jj = 0; jj < BATCH; ++jj) {
            const int col = n0 + cbase + j0 + jj;
            cv[jj] = (j0 == 0 && jj < PRE) ? cpre[jj]
                                           : ((reads_c && col < N) ? __ldcg(ep.C + row + (long long)col * ep.ldc) : 0.0);
          }
#pragma unroll
          for (int jj = 0; jj < BATCH; ++jj) {
            const int j = j0 + jj;
            const int col = n0 + cbase + j;
            if (col < N) {
              const int k = ea + scB[vb.c0 + col] - 14;
              double dh, dl;
              if constexpr (Cfg::WIDE) {
                dh = int64_scaled_to_double(accH[j], k + 32 - 8 * (S - 1));
                dl = int64_scaled_to_double(accL[j], k - 8 * (S - 1));
              } else {
                dh = scaled_float_to_double(hi[j], k);
                dl = scaled_float_to_double(lo[j], k);
              }
              if (ep.mode == 0) {
                double *p = ep.C + row + (long long)col * ep.ldc;
                double x;
                if (subtract) x = (cv[jj] - dh) - dl;
                else if (plain) x = dh + dl;
                else {
                  const double val = dh + dl;
                  x = (ep.beta == 0.0) ? ep.alpha * val : fma(ep.alpha, val, ep.beta * cv[jj]);
                }
                *p = x;
                if (ep.out.base) {
                  __nv_bfloat16 *o = ep.out.base + row + (long long)col * ep.out.ld;
                  if (ep.out.scale) write_fixed_slices(x, ep.out.scale[col], o, ep.out.plane, ep.out.S);
                  else write_slices(x, o, ep.out.plane, ep.out.S);
                }
              } else {
                ep.Pd[(long long)z * M * N + row + (long long)col * M] = dh + dl;
              }
            }
          }
        }
      }
    }
  }
  __syncthreads();
  if (warp == 1) {
    if (lane == 0) mbar_wait(&done_bar, 0, ctrl, &s_abort, false);
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)Cfg::TMEM_COLS)
                 : "memory");
  }
}

// One block per column: exponent of the column maximum (or the given one),
// then the fixed-point slices of the column (integer arithmetic only).
// One block per column: exponent of the column maximum (or the given one),
// then the fixed-point slices of the column (integer arithmetic only).  When
// the column and the slice planes are aligned, a thread takes two rows at a
// time: one 16-byte load, one 4-byte store per slice for the pair.
template <int S>
__global__ void __launch_bounds__(256) split_exact_kernel(int R, int Cc, const double *__restrict__ X, long long ldx,
                                                          Slices dst, const int *__restrict__ scale_from) {
  __shared__ unsigned long long red[8];
  __shared__ int s_e;
  for (int c = blockIdx.x; c < Cc; c += gridDim.x) {
    const double *col = X + (long long)c * ldx;
    if (scale_from) {
      if (threadIdx.x == 0) s_e = scale_from[c];
    } else {
      unsigned long long mx = 0;
      for (int r = threadIdx.x; r < R; r += 256) mx = max(mx, abs_bits(col[r]));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
      __syncthreads();
      if (threadIdx.x == 0) {
        unsigned long long m = 0;
        for (int w = 0; w < 8; ++w) m = max(m, red[w]);
        s_e = exp_above_bits(m);
      }
    }
    __syncthreads();
    const int e = s_e;
    if (threadIdx.x == 0 && dst.scale) dst.scale[c] = e;
    unsigned short *out = reinterpret_cast<unsigned short *>(dst.base) + (long long)c * dst.ld;
    const bool pairs = ((reinterpret_cast<uintptr_t>(col) & 15) == 0) &&
                       ((reinterpret_cast<uintptr_t>(out) & 3) == 0) && ((dst.plane & 1) == 0);
    int r_done = 0;
    if (pairs) {
      const int R2 = R >> 1;
      const double2 *col2 = reinterpret_cast<const double2 *>(col);
      for (int r2 = threadIdx.x; r2 < R2; r2 += 256) {
        const double2 v = col2[r2];
        unsigned short d0[S], d1[S];
        fixed_digits<S>(v.x, e, d0);
        fixed_digits<S>(v.y, e, d1);
#pragma unroll
        for (int sl = 0; sl < S; ++sl)
          reinterpret_cast<unsigned *>(out + sl * dst.plane)[r2] = (unsigned)d0[sl] | ((unsigned)d1[sl] << 16);
      }
      r_done = R2 << 1;
    }
    for (int r = r_done + threadIdx.x; r < R; r += 256) {
      unsigned short d[S];
      fixed_digits<S>(col[r], e, d);
#pragma unroll
      for (int sl = 0; sl < S; ++sl) out[sl * dst.plane + r] = d[sl];
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256) col_norm_exp_kernel(int R, int Cc, const double *__restrict__ X, long long ldx,
                                                           int *e_out) {
  __shared__ double red[8];
  for (int c = blockIdx.x; c < Cc; c += gridDim.x) {
    const double *col = X + (long long)c * ldx;
    double s = 0.0;
    for (int r = threadIdx.x; r < R; r += 256) s = fma(col[r], col[r], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < 8; ++w) t += red[w];
      int e = 0;
      if (t > 0.0) frexp(sqrt(t) * (1.0 + 0x1.0p-20), &e);
      e_out[c] = e;
    }
    __syncthreads();
  }
}

template <int S, bool ALL, int BN>
int launch_tcx(const CUtensorMap &ma, const CUtensorMap &mb, TcView va, TcView vb, int M, int N, int K, int k_chunk,
               int splits, const int *scA, const int *scB, const TcEpilogue &ep, DeviceControl *ctrl,
               cudaStream_t s) {
  using Cfg = TcxCfg<S, ALL, BN>;
  static thread_local int attr_dev = -1;
  int dev = 0;
  cudaGetDevice(&dev);
  if (attr_dev != dev) {
    if (cudaFuncSetAttribute(tcx_gemm_kernel<S, ALL, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM) !=
        cudaSuccess)
      return PURL_ERR_CUDA;
    attr_dev = dev;
  }
  long long tiles = (long long)ceil_div(M, TC_BM) * ceil_div(N, BN);
  if (tiles * splits > 0x7fffffffLL) return PURL_ERR_UNSUPPORTED;
  const DeviceInfo *di = device_info();
  long long grid = tiles * splits;
  if (grid > di->num_sms) grid = di->num_sms;  // persistent: one block per SM walks the work list
  // issued tensor-core work: every slice pair is one BF16 product
  const int pairs = ALL ? S * S : S * (S + 1) / 2;
  double flops = 2.0 * M * (double)N * K * pairs;
  double bytes = (double)S * 2.0 * ((double)M * K + (double)N * K) +
                 (ep.mode == 0 ? 8.0 * M * N * (ep.beta != 0.0 ? 2 : 1) + (ep.out.base ? 2.0 * ep.out.S * M * N : 0)
                               : 8.0 * M * N * splits);
  LaunchScope ls(KC_GEMM_TC, s, flops, bytes, ep.tag ? ep.tag : "tcx_gemm_kernel");
  tcx_gemm_kernel<S, ALL, BN><<<(unsigned)grid, Cfg::THREADS, Cfg::SMEM, s>>>(ma, mb, va, vb, M, N, K, k_chunk,
                                                                             splits, scA, scB, ep, ctrl);
  return cudaGetLastError() == cudaSuccess ? PURL_OK : PURL_ERR_CUDA;
}

}  // namespace

int split_exact(int R, int Cc, const double *X, long long ldx, Slices dst, const int *scale_from, cudaStream_t s) {
  const DeviceInfo *di = device_info();
  if (!di) return PURL_ERR_CUDA;
  if (Cc <= 0) return PURL_OK;
  if (!scale_from && !dst.scale) return PURL_ERR_UNSUPPORTED;
  // a block reads its column twice (maximum, then digits): at most 4 columns
  // per SM in flight keep the second read in L2 for tall columns
  const int cap = R > 4096 ? di->num_sms * 4 : di->num_sms * 32;
  int grid = Cc < cap ? Cc : cap;
  LaunchScope ls(KC_SPLIT, s, 0.0, (8.0 + 2.0 * dst.S) * (double)R * Cc, "split_exact_kernel");
  switch (dst.S) {
    case 1: split_exact_kernel<1><<<grid, 256, 0, s>>>(R, Cc, X, ldx, dst, scale_from); break;
    case 2: split_exact_kernel<2><<<grid, 256, 0, s>>>(R, Cc, X, ldx, dst, scale_from); break;
    case 3: split_exact_kernel<3><<<grid, 256, 0, s>>>(R, Cc, X, ldx, dst, scale_from); break;
    case 4: split_exact_kernel<4><<<grid, 256, 0, s>>>(R, Cc, X, ldx, dst, scale_from); break;
    case 5: split_exact_kernel<5><<<grid, 256, 0, s>>>(R, Cc, X, ldx, dst, scale_from); break;
    case 6: split_exact_kernel<6><<<grid, 256, 0, s>>>(R, Cc, X, ldx, dst, scale_from); break;
    case 7: split_exact_kernel<7><<<grid, 256, 0, s>>>(R, Cc, X, ldx, dst, scale_from); break;
    case 8: split_exact_kernel<8><<<grid, 256, 0, s>>>(R, Cc, X, ldx, dst, scale_from); break;
    default: return PURL_ERR_UNSUPPORTED;
  }
  return cudaGetLastError() == cudaSuccess ? PURL_OK : PURL_ERR_CUDA;
}

int column_norm_exponents(int R, int Cc, const double *X, long long ldx, int *e, cudaStream_t s) {
  const DeviceInfo *di = device_info();
  if (!di) return PURL_ERR_CUDA;
  if (Cc <= 0) return PURL_OK;
  int grid = Cc < di->num_sms * 32 ? Cc : di->num_sms * 32;
  LaunchScope ls(KC_OTHER, s, 0.0, 8.0 * (double)R * Cc, "col_norm_exp_kernel");
  col_norm_exp_kernel<<<grid, 256, 0, s>>>(R, Cc, X, ldx, e);
  return cudaGetLastError() == cudaSuccess ? PURL_OK : PURL_ERR_CUDA;
}

int tcx_gemm_view_impl(const Slices &A, int a_r0, int a_c0, const Slices &B, int b_r0, int b_c0, int M, int N,
                       int K, int S, bool all_pairs, const TcEpilogue &ep, int splits, int k_chunk, cudaStream_t s) {
  const DeviceInfo *di = device_info();
  if (!di) return PURL_ERR_CUDA;
  if (M <= 0 || N <= 0) return PURL_OK;
  if (K <= 0 || k_chunk <= 0 || (k_chunk % (TC_BK * TCX_KBC)) != 0 || splits != ceil_div(K, k_chunk))
    return PURL_ERR_UNSUPPORTED;
  if (S < 1 || (S > 4 && (S != kTcxEmuSlices || all_pairs)) || A.S < S || B.S < S || !A.scale || !B.scale)
    return PURL_ERR_UNSUPPORTED;
  // wide sums: |H|, |L| < 2^48.1 per 128-deep chunk; K <= 2^20 keeps both
  // inside 64 bits
  if (S > 4 && K > (1 << 20)) return PURL_ERR_UNSUPPORTED;
  if ((a_r0 % 8) != 0 || (b_r0 % 8) != 0) return PURL_ERR_UNSUPPORTED;
  if (ep.mode == 2 && !ep.Pd) return PURL_ERR_UNSUPPORTED;
  if (ep.mode == 0 && !ep.C) return PURL_ERR_UNSUPPORTED;
  if (ep.mode != 0 && ep.mode != 2) return PURL_ERR_UNSUPPORTED;
  const int BN = (all_pairs || S > 4) ? 32 : 64;
  CUtensorMap ma, mb;
  PURL_TRY(make_map(&ma, A, a_r0 + K, a_c0 + M, TC_BM));
  PURL_TRY(make_map(&mb, B, b_r0 + K, b_c0 + N, BN));
  TcView va{a_r0, a_c0}, vb{b_r0, b_c0};
#define PURL_TCX(S_, ALL_, BN_) \
  return launch_tcx<S_, ALL_, BN_>(ma, mb, va, vb, M, N, K, k_chunk, splits, A.scale, B.scale, ep, di->ctrl, s)
  if (S == kTcxEmuSlices) PURL_TCX(kTcxEmuSlices, false, 32);
  if (!all_pairs) {
    if (S == 1) PURL_TCX(1, false, 64);
    if (S == 2) PURL_TCX(2, false, 64);
    if (S == 3) PURL_TCX(3, false, 64);
    PURL_TCX(4, false, 64);
  }
  if (S == 1) PURL_TCX(1, true, 32);
  if (S == 2) PURL_TCX(2, true, 32);
  if (S == 3) PURL_TCX(3, true, 32);
  PURL_TCX(4, true, 32);
#undef PURL_TCX
}

int tcx_gemm_view(const Slices &A, int a_r0, int a_c0, const Slices &B, int b_r0, int b_c0, int M, int N, int K, int S,
                  const TcEpilogue &ep, int splits, int k_chunk, cudaStream_t s) {
  return tcx_gemm_view_impl(A, a_r0, a_c0, B, b_r0, b_c0, M, N, K, S, false, ep, splits, k_chunk, s);
}

int tcx_gemm_all_pairs(const Slices &A, int a_r0, int a_c0, const Slices &B, int b_r0, int b_c0, int M, int N, int K,
                       int S, const TcEpilogue &ep, int splits, int k_chunk, cudaStream_t s) {
  return tcx_gemm_view_impl(A, a_r0, a_c0, B, b_r0, b_c0, M, N, K, S, true, ep, splits, k_chunk, s);
}

// Scratch layout of gemm_exact: slices of op(A) (K x M) and op(B) (K x N), their
// scales, and an FP64 staging buffer for the transposed operand.
static void gemm_exact_plan(Arena &ar, int m, int n, int k, int S, Slices *sa, Slices *sb, double **T) {
  const int kk = k > 0 ? k : 1, mm = m > 0 ? m : 1, nn = n > 0 ? n : 1;
  *sa = make_slices(ar.take<__nv_bfloat16>(slice_elems(kk, mm, S)), kk, mm, S);
  *sb = make_slices(ar.take<__nv_bfloat16>(slice_elems(kk, nn, S)), kk, nn, S);
  sa->scale = ar.take<int>(mm);
  sb->scale = ar.take<int>(nn);
  *T = ar.take<double>((size_t)kk * (size_t)(mm > nn ? mm : nn));
}

size_t gemm_exact_bytes(int m, int n, int k, int S) {
  Arena ar;
  Slices sa, sb;
  double *T;
  gemm_exact_plan(ar, m, n, k, S, &sa, &sb, &T);
  return ar.used;
}

int gemm_exact(bool ta, bool tb, int m, int n, int k, double alpha, const double *A, int lda, const double *B,
               int ldb, double beta, double *C, int ldc, int S, void *scratch, size_t scratch_bytes,
               cudaStream_t s) {
  if ((long long)m * n == 0) return PURL_OK;
  if (S < 1 || (S > 4 && S != kTcxEmuSlices)) return PURL_ERR_UNSUPPORTED;
  if (S > 4 && k > (1 << 20)) return PURL_ERR_UNSUPPORTED;
  if (k == 0) return gemm_f64(false, false, m, n, 0, 0.0, A, lda, B, ldb, beta, C, ldc, s);
  Arena ar;
  ar.base = static_cast<char *>(scratch);
  ar.size = scratch_bytes;
  Slices sa, sb;
  double *T;
  gemm_exact_plan(ar, m, n, k, S, &sa, &sb, &T);
  if (!ar.ok) return PURL_ERR_NOMEM;
  // operand rows along the columns of the sliced matrices: op(A)^T (K x M), op(B) (K x N)
  if (ta) {
    PURL_TRY(split_exact(k, m, A, lda, sa, nullptr, s));
  } else {
    PURL_TRY(transpose_f64(m, k, A, lda, T, k, s));
    PURL_TRY(split_exact(k, m, T, k, sa, nullptr, s));
  }
  if (tb) {
    PURL_TRY(transpose_f64(n, k, B, ldb, T, k, s));
    PURL_TRY(split_exact(k, n, T, k, sb, nullptr, s));
  } else {
    PURL_TRY(split_exact(k, n, B, ldb, sb, nullptr, s));
  }
  TcEpilogue ep;
  ep.mode = 0;
  ep.alpha = alpha;
  ep.beta = beta;
  ep.C = C;
  ep.ldc = ldc;
  return tcx_gemm_view(sa, 0, 0, sb, 0, 0, m, n, k, S, ep, 1, ceil_div(k, 256) * 256, s);
}

}  // namespace purl
