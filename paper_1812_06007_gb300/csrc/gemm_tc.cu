// gemm_tc.cu -- BF16 tensor-core product engine for sm_103a: TMA loads into
// 128-byte-swizzled shared memory, tcgen05.mma (kind::f16, BF16 x BF16 ->
// FP32) issued by one thread, the accumulator in tensor memory (TMEM), and an
// epilogue that reads TMEM with tcgen05.ld.
//
// This is the "efficient matrix-matrix multiplication routine" of Section 3
// for the mixed-precision path: the power-step products (one BF16 slice per
// operand) and, with 2 or 3 slices per operand, the compensated products of
// A V, of every QR trailing update and of Q formation.
//
// CTA = 6 warps: warp 0 issues TMA loads, warp 1 allocates TMEM and issues the
// MMAs, warps 2-5 run the epilogue (warp w reads TMEM lanes 32*(w%4)..+31).
// Tile 128 x BN x 64; a multi-stage shared-memory ring with full/empty
// mbarriers; every wait is bounded and records PURL_ERR_TIMEOUT on expiry.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <mutex>

#include "profile.cuh"
#include "tc.cuh"
#include "tc_ptx.cuh"
#include "slice_int.cuh"

namespace purl {

namespace {

constexpr int TC_THREADS = 192;
constexpr int TC_GROUP = 16;
constexpr int kSmemBudget = 200 * 1024;

template <int BN, int S>
struct TcCfg {
  static constexpr int A_BYTES = TC_BM * TC_BK * 2;
  static constexpr int B_BYTES = BN * TC_BK * 2;
  static constexpr int STAGE_BYTES = S * (A_BYTES + B_BYTES);
  static constexpr int STAGES_RAW = kSmemBudget / STAGE_BYTES;
  static constexpr int STAGES = STAGES_RAW > 8 ? 8 : STAGES_RAW;
  static constexpr int SMEM = STAGES * STAGE_BYTES + 1024;
  static constexpr int TMEM_COLS = BN < 32 ? 32 : BN;
  static_assert(STAGES >= 2, "tile too large for a 2-stage pipeline");
  static_assert(BN % 32 == 0 && BN >= 32 && BN <= 256, "BN");
};

template <int BN, int S>
__global__ void __launch_bounds__(TC_THREADS, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   TcView va, TcView vb, int M, int N, int K, int k_chunk, TcEpilogue ep,
                   DeviceControl *ctrl, uint32_t idesc) {
  using Cfg = TcCfg<BN, S>;
  constexpr int STAGES = Cfg::STAGES;
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t full_bar[STAGES];
  __shared__ __align__(8) uint64_t empty_bar[STAGES];
  __shared__ __align__(8) uint64_t acc_bar;
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // grouped raster: consecutive blocks walk TC_GROUP M-tiles before moving to
  // the next N-tile, so a wave shares A and B tiles in L2
  const int tiles_m = (M + TC_BM - 1) / TC_BM, tiles_n = (N + BN - 1) / BN;
  const int pid = blockIdx.x;
  const int per_group = TC_GROUP * tiles_n;
  const int first_m = (pid / per_group) * TC_GROUP;
  const int gsize = min(tiles_m - first_m, TC_GROUP);
  const int m0 = (first_m + (pid % per_group) % gsize) * TC_BM;
  const int n0 = ((pid % per_group) / gsize) * BN;
  const int kb0 = blockIdx.y * k_chunk;
  const int kend = min(K, kb0 + k_chunk);
  const int nkb = (kend - kb0 + TC_BK - 1) / TC_BK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    mbar_init(&acc_bar, 1);
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
      // ---------------- TMA producer ----------------
      int issued = 0;
      for (int kb = 0; kb < nkb; ++kb) {
        const int st = kb % STAGES;
        const uint32_t ph = (uint32_t)(kb / STAGES) & 1u;
        if (!mbar_wait(&empty_bar[st], ph ^ 1u, ctrl, &s_abort)) break;
        mbar_arrive_expect_tx(&full_bar[st], (uint32_t)Cfg::STAGE_BYTES);
        uint8_t *sa = smem + (size_t)st * Cfg::STAGE_BYTES;
        uint8_t *sb = sa + S * Cfg::A_BYTES;
        const int kx = kb0 + kb * TC_BK;
#pragma unroll
        for (int s = 0; s < S; ++s) tma_load_3d(sa + s * Cfg::A_BYTES, &tmA, &full_bar[st], va.r0 + kx, va.c0 + m0, s);
#pragma unroll
        for (int s = 0; s < S; ++s) tma_load_3d(sb + s * Cfg::B_BYTES, &tmB, &full_bar[st], vb.r0 + kx, vb.c0 + n0, s);
        issued = kb + 1;
      }
      // never leave the block with copies in flight: the last use of every stage
      // must have landed (bounded; normally already true)
      for (int kb = (issued > STAGES ? issued - STAGES : 0); kb < issued; ++kb)
        mbar_wait(&full_bar[kb % STAGES], (uint32_t)(kb / STAGES) & 1u, ctrl, &s_abort, false);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer ----------------
      for (int kb = 0; kb < nkb; ++kb) {
        const int st = kb % STAGES;
        const uint32_t ph = (uint32_t)(kb / STAGES) & 1u;
        if (!mbar_wait(&full_bar[st], ph, ctrl, &s_abort)) break;
        tc_fence_after();
        const uint32_t sa = smem_u32(smem + (size_t)st * Cfg::STAGE_BYTES);
        const uint32_t sb = sa + S * Cfg::A_BYTES;
        int prod = 0;
#pragma unroll
        for (int s = 0; s < S; ++s) {
#pragma unroll
          for (int t = 0; t < S - s; ++t) {
#pragma unroll
            for (int k = 0; k < TC_BK / 16; ++k) {
              const uint64_t ad = sw128_desc(sa + s * Cfg::A_BYTES + k * 32);
              const uint64_t bd = sw128_desc(sb + t * Cfg::B_BYTES + k * 32);
              tc_mma(tmem, ad, bd, idesc, (kb > 0 || prod > 0 || k > 0) ? 1u : 0u);
            }
            ++prod;
          }
        }
        tc_commit(&empty_bar[st]);
      }
      tc_commit(&acc_bar);
    }
  } else {
    // ---------------- epilogue (warps 2..5) ----------------
    const bool ok = mbar_wait(&acc_bar, 0, ctrl, &s_abort);
    tc_fence_after();
    if (ok && nkb > 0) {
      const int lane_base = 32 * (warp & 3);
      const int row = m0 + lane_base + lane;
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += 32) {
        uint32_t v[32];
        tmem_ld32(tmem + ((uint32_t)lane_base << 16) + (uint32_t)c0, v);
        if (row < M) {
          if (ep.mode == 0) {
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              const int col = n0 + c0 + j;
              if (col < N) {
                const double acc = scaled_float_to_double(__uint_as_float(v[j]), 0);
                double *p = ep.C + row + (long long)col * ep.ldc;
                const double x = (ep.beta == 0.0 && ep.alpha == 1.0)
                                     ? acc
                                     : ((ep.beta == 0.0) ? ep.alpha * acc : fma(ep.alpha, acc, ep.beta * *p));
                *p = x;
                if (ep.out.base)
                  write_slices(x, ep.out.base + row + (long long)col * ep.out.ld, ep.out.plane, ep.out.S);
              }
            }
          } else {
            float *P = ep.P + (long long)blockIdx.y * M * N;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              const int col = n0 + c0 + j;
              if (col < N) P[row + (long long)col * M] = __uint_as_float(v[j]);
            }
          }
        }
      }
    }
    tc_fence_before();
  }
  __syncthreads();
  if (warp == 1) {
    // every MMA of this block must be complete before TMEM is released
    if (lane == 0) mbar_wait(&acc_bar, 0, ctrl, &s_abort, false);
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"((uint32_t)Cfg::TMEM_COLS)
                 : "memory");
  }
}

// ------------------------------------------------------------- slicing ----
__global__ void split_kernel(int R, int Cc, const double *__restrict__ X, long long ldx, Slices dst) {
  long long total = (long long)R * Cc;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    int r = (int)(e % R), c = (int)(e / R);
    write_slices(X[r + c * ldx], dst.base + r + c * dst.ld, dst.plane, dst.S);
  }
}

// dst (Cc x R) = slices of X^T; 32 x 32 tiles through shared memory.
__global__ void split_t_kernel(int R, int Cc, const double *__restrict__ X, long long ldx, Slices dst) {
  __shared__ double tile[32][33];
  const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    int r = r0 + threadIdx.x, c = c0 + j;
    tile[j][threadIdx.x] = (r < R && c < Cc) ? X[r + (long long)c * ldx] : 0.0;
  }
  __syncthreads();
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    int c = c0 + threadIdx.x, r = r0 + j;  // dst(c, r) = X(r, c)
    if (r < R && c < Cc) write_slices(tile[threadIdx.x][j], dst.base + c + (long long)r * dst.ld, dst.plane, dst.S);
  }
}

// ------------------------------------------------- scaled plain slices ----
// Largest biased exponent field of the entries of X (atomicMax into *e).
__global__ void max_exp_kernel(int R, int Cc, const double *__restrict__ X, long long ldx, int *e) {
  long long total = (long long)R * Cc;
  int mx = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(i % R), c = (int)(i / R);
    const int ex = (int)((__double_as_longlong(X[r + c * ldx]) >> 52) & 0x7ff);
    mx = ex > mx ? ex : mx;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0 && mx > 0) atomicMax(e, mx);
}

// Power of two 2^s that puts the largest entry (below 2^(e - 1022)) just
// under 2^15 for FP16 or 2 for BF16; clamped so that the factor 2^s is a normal
// number (the scaling is exact unless an entry leaves the FP64 range).
__device__ __forceinline__ int slice_shift(int e, bool f16) {
  const int top = (f16 ? 15 : 1) - (e - 1022);
  return top < -1000 ? -1000 : (top > 1000 ? 1000 : top);
}

// 2^sh as a double (|sh| <= 1000: a normal number), built from its bits
__device__ __forceinline__ double pow2(int sh) { return __longlong_as_double((long long)(1023 + sh) << 52); }

__device__ __forceinline__ __nv_bfloat16 to_plain16(double x, bool f16) {
  if (f16) {
    const __half h = __double2half(x);
    return *reinterpret_cast<const __nv_bfloat16 *>(&h);
  }
  return __double2bfloat16(x);
}

__global__ void split_scaled_kernel(int R, int Cc, const double *__restrict__ X, long long ldx, Slices dst,
                                    const int *e) {
  const bool f16 = dst.f16 != 0;
  const double sc = pow2(slice_shift(*e, f16));
  long long total = (long long)R * Cc;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(i % R), c = (int)(i / R);
    dst.base[r + c * dst.ld] = to_plain16(X[r + c * ldx] * sc, f16);
  }
}

// dst (Cc x R) = 2^s X^T; 32 x 32 tiles through shared memory.
__global__ void split_scaled_t_kernel(int R, int Cc, const double *__restrict__ X, long long ldx, Slices dst,
                                      const int *e) {
  __shared__ double tile[32][33];
  const bool f16 = dst.f16 != 0;
  const double sc = pow2(slice_shift(*e, f16));
  const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    int r = r0 + threadIdx.x, c = c0 + j;
    tile[j][threadIdx.x] = (r < R && c < Cc) ? X[r + (long long)c * ldx] : 0.0;
  }
  __syncthreads();
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    int c = c0 + threadIdx.x, r = r0 + j;
    if (r < R && c < Cc) dst.base[c + (long long)r * dst.ld] = to_plain16(tile[threadIdx.x][j] * sc, f16);
  }
}

template <int BN, int S>
int launch_tc(const CUtensorMap &ma, const CUtensorMap &mb, TcView va, TcView vb, int M, int N, int K,
              int k_chunk, int splits, const TcEpilogue &ep, DeviceControl *ctrl, uint32_t idesc, cudaStream_t s) {
  using Cfg = TcCfg<BN, S>;
  static thread_local int attr_dev = -1;
  int dev = 0;
  cudaGetDevice(&dev);
  if (attr_dev != dev) {
    if (cudaFuncSetAttribute(tc_gemm_kernel<BN, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM) !=
        cudaSuccess)
      return PURL_ERR_CUDA;
    attr_dev = dev;
  }
  long long tiles = (long long)ceil_div(M, TC_BM) * ceil_div(N, BN);
  if (tiles > 0x7fffffffLL || splits > 65535) return PURL_ERR_UNSUPPORTED;
  dim3 grid((unsigned)tiles, splits);
  const int prods = S * (S + 1) / 2;
  double flops = 2.0 * M * (double)N * K * prods;  // issued tensor-core work: one product per slice pair
  double bytes = (double)S * 2.0 * ((double)M * K + (double)N * K) +
                 (ep.mode == 0 ? 8.0 * M * N * (ep.beta != 0.0 ? 2 : 1) + (ep.out.base ? 2.0 * ep.out.S * M * N : 0)
                               : 4.0 * M * N * splits);
  (void)prods;
  LaunchScope ls(KC_GEMM_TC, s, flops, bytes, ep.tag ? ep.tag : "tc_gemm_kernel");
  tc_gemm_kernel<BN, S><<<grid, TC_THREADS, Cfg::SMEM, s>>>(ma, mb, va, vb, M, N, K, k_chunk, ep, ctrl, idesc);
  return cudaGetLastError() == cudaSuccess ? PURL_OK : PURL_ERR_CUDA;
}

}  // namespace

// ------------------------------------------------------------ host side ---
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// Tensor map over the slices of an operand: x = row (K, contiguous) limited to
// k_end, y = column (M or N) limited to c_end, z = slice.
int make_map(CUtensorMap *map, const Slices &X, int k_end, int c_end, int box_rows) {
  auto enc = encode_fn();
  if (!enc) return PURL_ERR_UNSUPPORTED;
  if (((uintptr_t)X.base & 15) != 0 || (X.ld % 8) != 0 || (X.plane % 8) != 0) return PURL_ERR_UNSUPPORTED;
  cuuint64_t dims[3] = {(cuuint64_t)k_end, (cuuint64_t)c_end, (cuuint64_t)X.S};
  cuuint64_t strides[2] = {(cuuint64_t)X.ld * 2, (cuuint64_t)X.plane * 2};
  cuuint32_t box[3] = {(cuuint32_t)TC_BK, (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(map, X.f16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, X.base, dims,
                   strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? PURL_OK : PURL_ERR_UNSUPPORTED;
}


int split_slices(int R, int Cc, const double *X, long long ldx, Slices dst, cudaStream_t s) {
  const DeviceInfo *di = device_info();
  if (!di) return PURL_ERR_CUDA;
  long long total = (long long)R * Cc;
  if (total == 0) return PURL_OK;
  long long g = (total + 255) / 256;
  if (g > (long long)di->num_sms * 16) g = (long long)di->num_sms * 16;
  LaunchScope ls(KC_SPLIT, s, 0.0, (8.0 + 2.0 * dst.S) * total, "split_kernel");
  split_kernel<<<(int)g, 256, 0, s>>>(R, Cc, X, ldx, dst);
  return cudaGetLastError() == cudaSuccess ? PURL_OK : PURL_ERR_CUDA;
}

int split_slices_t(int R, int Cc, const double *X, long long ldx, Slices dst, cudaStream_t s) {
  if ((long long)R * Cc == 0) return PURL_OK;
  dim3 grid(ceil_div(R, 32), ceil_div(Cc, 32));
  if (grid.y > 65535) return PURL_ERR_UNSUPPORTED;
  LaunchScope ls(KC_SPLIT, s, 0.0, (8.0 + 2.0 * dst.S) * (double)R * Cc, "split_t_kernel");
  split_t_kernel<<<grid, dim3(32, 8), 0, s>>>(R, Cc, X, ldx, dst);
  return cudaGetLastError() == cudaSuccess ? PURL_OK : PURL_ERR_CUDA;
}

int split_scaled(int R, int Cc, const double *X, long long ldx, Slices dst, int *e_ws, bool transposed,
                 cudaStream_t s) {
  const DeviceInfo *di = device_info();
  if (!di) return PURL_ERR_CUDA;
  const long long total = (long long)R * Cc;
  if (total == 0) return PURL_OK;
  if (dst.S != 1) return PURL_ERR_UNSUPPORTED;
  PURL_TRY(zero_async(e_ws, sizeof(int), s));
  long long g = (total + 255) / 256;
  if (g > (long long)di->num_sms * 8) g = (long long)di->num_sms * 8;
  {
    LaunchScope ls(KC_SPLIT, s, 0.0, 8.0 * total, "max_exp_kernel");
    max_exp_kernel<<<(int)g, 256, 0, s>>>(R, Cc, X, ldx, e_ws);
  }
  PURL_CUDA_TRY(cudaGetLastError());
  if (transposed) {
    dim3 grid(ceil_div(R, 32), ceil_div(Cc, 32));
    if (grid.y > 65535) return PURL_ERR_UNSUPPORTED;
    LaunchScope ls(KC_SPLIT, s, 0.0, 10.0 * total, "split_scaled_t_kernel");
    split_scaled_t_kernel<<<grid, dim3(32, 8), 0, s>>>(R, Cc, X, ldx, dst, e_ws);
  } else {
    long long g2 = (total + 255) / 256;
    if (g2 > (long long)di->num_sms * 16) g2 = (long long)di->num_sms * 16;
    LaunchScope ls(KC_SPLIT, s, 0.0, 10.0 * total, "split_scaled_kernel");
    split_scaled_kernel<<<(int)g2, 256, 0, s>>>(R, Cc, X, ldx, dst, e_ws);
  }
  return cudaGetLastError() == cudaSuccess ? PURL_OK : PURL_ERR_CUDA;
}

void tc_choose_splits(int M, int N, int K, int num_sms, int max_splits, int *splits, int *k_chunk) {
  long long tiles = (long long)ceil_div(M, TC_BM) * ceil_div(N, 128);
  long long want = (2LL * num_sms + tiles - 1) / tiles;
  long long maxs = (K + 255) / 256;
  long long sp = want < maxs ? want : maxs;
  if (sp < 1) sp = 1;
  if (sp > max_splits) sp = max_splits;
  int chunk = ceil_div(ceil_div(K, (int)sp), TC_BK) * TC_BK;
  *k_chunk = chunk > 0 ? chunk : TC_BK;
  *splits = K > 0 ? ceil_div(K, *k_chunk) : 1;
}

// Views: A rows [a_r0, a_r0+K) x cols [a_c0, a_c0+M); same for B with N.
int tc_gemm_view(const Slices &A, int a_r0, int a_c0, const Slices &B, int b_r0, int b_c0, int M, int N, int K,
                 int S, const TcEpilogue &ep, int splits, int k_chunk, cudaStream_t s) {
  const DeviceInfo *di = device_info();
  if (!di) return PURL_ERR_CUDA;
  if (M <= 0 || N <= 0) return PURL_OK;
  if (K <= 0 || k_chunk <= 0 || (k_chunk % TC_BK) != 0 || splits != ceil_div(K, k_chunk)) return PURL_ERR_UNSUPPORTED;
  if (S < 1 || S > 3 || A.S < S || B.S < S) return PURL_ERR_UNSUPPORTED;
  // one operand type per MMA: never mix FP16 and BF16 (FP16 only as one plain slice)
  if (A.f16 != B.f16 || (A.f16 && S != 1)) return PURL_ERR_UNSUPPORTED;
  if ((a_r0 % 8) != 0 || (b_r0 % 8) != 0) return PURL_ERR_UNSUPPORTED;
  if (ep.mode == 1 && !ep.P) return PURL_ERR_UNSUPPORTED;
  if (ep.mode == 0 && !ep.C) return PURL_ERR_UNSUPPORTED;
  // N tile: the widest that fits the smem budget for S slices
  int BN = N > 128 ? 256 : (N > 64 ? 128 : (N > 32 ? 64 : 32));
  if (S == 3 && BN > 128) BN = 128;
  if (S == 2 && BN > 256) BN = 256;
  CUtensorMap ma, mb;
  PURL_TRY(make_map(&ma, A, a_r0 + K, a_c0 + M, TC_BM));
  PURL_TRY(make_map(&mb, B, b_r0 + K, b_c0 + N, BN));
  TcView va{a_r0, a_c0}, vb{b_r0, b_c0};
  const uint32_t idesc = A.f16 ? idesc_f16(TC_BM, BN) : idesc_bf16(TC_BM, BN);
#define PURL_TC_CASE(BN_, S_) \
  if (BN == BN_ && S == S_) return launch_tc<BN_, S_>(ma, mb, va, vb, M, N, K, k_chunk, splits, ep, di->ctrl, idesc, s);
  PURL_TC_CASE(32, 1) PURL_TC_CASE(64, 1) PURL_TC_CASE(128, 1) PURL_TC_CASE(256, 1)
  PURL_TC_CASE(32, 2) PURL_TC_CASE(64, 2) PURL_TC_CASE(128, 2) PURL_TC_CASE(256, 2)
  PURL_TC_CASE(32, 3) PURL_TC_CASE(64, 3) PURL_TC_CASE(128, 3)
#undef PURL_TC_CASE
  return PURL_ERR_UNSUPPORTED;
}

int tc_gemm(const Slices &A, const Slices &B, int M, int N, int K, int S, const TcEpilogue &ep, int splits,
            int k_chunk, cudaStream_t s) {
  return tc_gemm_view(A, 0, 0, B, 0, 0, M, N, K, S, ep, splits, k_chunk, s);
}

// ---------------------------------------------------------------------------
// Allocation-free variant of purl_gemm_tc.  Its operand slices (and the
// status word its bounded waits report to) live in one file-scope device
// array instead of memory from cudaMalloc/cudaMallocAsync, so it can be used
// by callers that must not allocate device memory.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)24 << 20;  // 24 MiB on every device that loads the library
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

struct NoAllocDevice {
  bool ready = false;
  unsigned char *scratch = nullptr;  // device address of g_noalloc_scratch on this device
};

__global__ void noalloc_scale_kernel(int m, int n, double beta, double *C, long long ldc) {
  long long total = (long long)m * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    int i = (int)(e % m), j = (int)(e / m);
    double *p = C + i + j * ldc;
    *p = (beta == 0.0) ? 0.0 : beta * *p;
  }
}

std::mutex g_noalloc_mu;
NoAllocDevice g_noalloc_devs[64];

// Once per device, with that device current: resolve the array's device
// address (the host-side symbol is not a device pointer) and clear the
// status word kept at its start.
int noalloc_setup(NoAllocDevice **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return PURL_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  NoAllocDevice &d = g_noalloc_devs[dev];
  if (!d.ready) {
    void *ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || ptr == nullptr) return PURL_ERR_CUDA;
    if (cudaMemset(ptr, 0, sizeof(DeviceControl)) != cudaSuccess) return PURL_ERR_CUDA;
    if (cudaDeviceSynchronize() != cudaSuccess) return PURL_ERR_CUDA;
    d.scratch = static_cast<unsigned char *>(ptr);
    d.ready = true;
  }
  *out = &d;
  return PURL_OK;
}

template <int BN, int S>
int noalloc_launch(const CUtensorMap &ma, const CUtensorMap &mb, int M, int N, int K, const TcEpilogue &ep,
                   DeviceControl *ctrl, cudaStream_t s) {
  using Cfg = TcCfg<BN, S>;
  if (cudaFuncSetAttribute(tc_gemm_kernel<BN, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM) !=
      cudaSuccess)
    return PURL_ERR_CUDA;
  long long tiles = (long long)ceil_div(M, TC_BM) * ceil_div(N, BN);
  if (tiles > 0x7fffffffLL) return PURL_ERR_UNSUPPORTED;
  TcView v0{0, 0};
  LaunchScope ls(KC_GEMM_TC, s, 2.0 * M * (double)N * K * (S * (S + 1) / 2),
                 (double)S * 2.0 * ((double)M * K + (double)N * K) + 8.0 * M * N * (ep.beta != 0.0 ? 2 : 1),
                 "tc noalloc");
  tc_gemm_kernel<BN, S><<<dim3((unsigned)tiles, 1), TC_THREADS, Cfg::SMEM, s>>>(ma, mb, v0, v0, M, N, K,
                                                                                 ceil_div(K, TC_BK) * TC_BK, ep, ctrl,
                                                                                 idesc_bf16(TC_BM, BN));
  return cudaGetLastError() == cudaSuccess ? PURL_OK : PURL_ERR_CUDA;
}

}  // namespace

}  // namespace purl

extern "C" int purl_gemm_tc_noalloc(char transa, char transb, int m, int n, int k, double alpha, const double *A,
                                    int lda, const double *B, int ldb, double beta, double *C, int ldc, int slices,
                                    cudaStream_t stream) {
  using namespace purl;
  const bool ta = (transa == 'T' || transa == 't'), tb = (transb == 'T' || transb == 't');
  if (!ta && transa != 'N' && transa != 'n') return -1;
  if (!tb && transb != 'N' && transb != 'n') return -2;
  if (m < 0) return -3;
  if (n < 0) return -4;
  if (k < 0) return -5;
  const int arows = ta ? k : m, brows = tb ? n : k;
  if (!A && (long long)m * k > 0) return -7;
  if (lda < (arows > 1 ? arows : 1)) return -8;
  if (!B && (long long)k * n > 0) return -9;
  if (ldb < (brows > 1 ? brows : 1)) return -10;
  if (!C && (long long)m * n > 0) return -12;
  if (ldc < (m > 1 ? m : 1)) return -13;
  if (slices < 1 || slices > 3) return -14;
  // the operand slices must fit in the static scratch (after the status word)
  const size_t ea = slice_elems(k > 0 ? k : 1, m > 0 ? m : 1, slices);
  const size_t eb = slice_elems(k > 0 ? k : 1, n > 0 ? n : 1, slices);
  const size_t off_a = 256, off_b = off_a + align_up(ea * sizeof(__nv_bfloat16), 256);
  if (off_b + align_up(eb * sizeof(__nv_bfloat16), 256) > kNoAllocScratchBytes) return PURL_ERR_NOMEM;
  if ((long long)m * n == 0) return PURL_OK;
  NoAllocDevice *nd = nullptr;
  PURL_TRY(noalloc_setup(&nd));
  int sms = 0, dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return PURL_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return PURL_ERR_CUDA;
  if (k == 0) {
    long long g = ((long long)m * n + 255) / 256;
    if (g > (long long)sms * 16) g = (long long)sms * 16;
    LaunchScope ls(KC_OTHER, stream, 0.0, 16.0 * m * n, "noalloc_scale_kernel");
    noalloc_scale_kernel<<<(int)g, 256, 0, stream>>>(m, n, beta, C, ldc);
    return cudaGetLastError() == cudaSuccess ? PURL_OK : PURL_ERR_CUDA;
  }
  DeviceControl *ctrl = reinterpret_cast<DeviceControl *>(nd->scratch);
  Slices sa = make_slices(reinterpret_cast<__nv_bfloat16 *>(nd->scratch + off_a), k, m, slices);
  Slices sb = make_slices(reinterpret_cast<__nv_bfloat16 *>(nd->scratch + off_b), k, n, slices);
  // operand A: rows K, cols M (K-major); operand B: rows K, cols N
  auto split = [&](bool transposed, int R, int Cc, const double *X, long long ldx, Slices dst) -> int {
    if (transposed) {
      dim3 grid(ceil_div(R, 32), ceil_div(Cc, 32));
      if (grid.y > 65535) return PURL_ERR_UNSUPPORTED;
      LaunchScope ls(KC_SPLIT, stream, 0.0, (8.0 + 2.0 * dst.S) * (double)R * Cc, "split_t_kernel");
      split_t_kernel<<<grid, dim3(32, 8), 0, stream>>>(R, Cc, X, ldx, dst);
    } else {
      long long g = ((long long)R * Cc + 255) / 256;
      if (g > (long long)sms * 16) g = (long long)sms * 16;
      LaunchScope ls(KC_SPLIT, stream, 0.0, (8.0 + 2.0 * dst.S) * (double)R * Cc, "split_kernel");
      split_kernel<<<(int)g, 256, 0, stream>>>(R, Cc, X, ldx, dst);
    }
    return cudaGetLastError() == cudaSuccess ? PURL_OK : PURL_ERR_CUDA;
  };
  if (ta) PURL_TRY(split(false, k, m, A, lda, sa));
  else PURL_TRY(split(true, m, k, A, lda, sa));
  if (tb) PURL_TRY(split(true, n, k, B, ldb, sb));
  else PURL_TRY(split(false, k, n, B, ldb, sb));
  int BN = n > 128 ? 256 : (n > 64 ? 128 : (n > 32 ? 64 : 32));
  if (slices == 3 && BN > 128) BN = 128;
  CUtensorMap ma, mb;
  PURL_TRY(make_map(&ma, sa, k, m, TC_BM));
  PURL_TRY(make_map(&mb, sb, k, n, BN));
  TcEpilogue ep;
  ep.mode = 0;
  ep.alpha = alpha;
  ep.beta = beta;
  ep.C = C;
  ep.ldc = ldc;
#define PURL_NA_CASE(BN_, S_) \
  if (BN == BN_ && slices == S_) return noalloc_launch<BN_, S_>(ma, mb, m, n, k, ep, ctrl, stream);
  PURL_NA_CASE(32, 1) PURL_NA_CASE(64, 1) PURL_NA_CASE(128, 1) PURL_NA_CASE(256, 1)
  PURL_NA_CASE(32, 2) PURL_NA_CASE(64, 2) PURL_NA_CASE(128, 2) PURL_NA_CASE(256, 2)
  PURL_NA_CASE(32, 3) PURL_NA_CASE(64, 3) PURL_NA_CASE(128, 3)
#undef PURL_NA_CASE
  return PURL_ERR_UNSUPPORTED;
}

namespace purl {

// Status word of the no-alloc entry point on the current device: read it and
// clear it (with the abort flag).  *status is PURL_OK when the entry point was
// never set up on this device.  Called by purl_device_status, so a bounded
// wait that ran out inside purl_gemm_tc_noalloc is reported like any other.
int noalloc_take_status(int *status) {
  *status = PURL_OK;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return PURL_ERR_CUDA;
  unsigned char *scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_devs[dev].ready) return PURL_OK;
    scratch = g_noalloc_devs[dev].scratch;
  }
  DeviceControl h{};
  if (cudaMemcpy(&h, scratch, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) return PURL_ERR_CUDA;
  if (h.status != PURL_OK || h.abort != 0) {
    const DeviceControl z{};
    if (cudaMemcpy(scratch, &z, sizeof(z), cudaMemcpyHostToDevice) != cudaSuccess) return PURL_ERR_CUDA;
  }
  *status = h.status;
  return PURL_OK;
}

// The no-alloc entry point's status word on the current device (set up like
// its first call), for the failure-detection probe.
int noalloc_control(DeviceControl **ctrl) {
  NoAllocDevice *nd = nullptr;
  PURL_TRY(noalloc_setup(&nd));
  *ctrl = reinterpret_cast<DeviceControl *>(nd->scratch);
  return PURL_OK;
}

}  // namespace purl
