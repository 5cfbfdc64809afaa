// finite.cu -- detection of non-finite input (the paper assumes finite data).
//
// A NaN or an infinity in A would pass silently through the tensor-core modes:
// their fixed-point slicing reads the exponent field of every entry as an
// integer, so a non-finite entry becomes a huge but finite row scale and the
// factorization comes back finite and wrong.  Every entry point that takes A
// therefore scans it once (8 bytes per entry read, nothing written), and when
// any entry has the all-ones exponent field it (i) records PURL_ERR_NONFINITE
// in the per-device status word and (ii) overwrites the outputs with NaN at
// the end of the call, so every mode behaves like FP64 arithmetic would.
#include "common.cuh"
#include "profile.cuh"

namespace purl {
namespace {

__device__ __forceinline__ bool not_finite(double x) {
  // exponent field 0x7ff: infinity or NaN (integer test, no FP64 compare)
  return ((__double_as_longlong(x) >> 52) & 0x7ff) == 0x7ff;
}

// One warp per column strip: rows walked with coalesced loads.
__global__ void finite_check_kernel(int m, int n, const double *__restrict__ A, long long lda, int *flag,
                                    DeviceControl *ctrl) {
  const int lane = threadIdx.x & 31;
  const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const long long rows32 = (m + 31) / 32;
  bool bad = false;
  for (long long w = warp; w < rows32 * n; w += nwarps) {
    const int j = (int)(w / rows32);
    const int i = (int)(w % rows32) * 32 + lane;
    if (i < m) bad |= not_finite(A[i + j * lda]);
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) {
    atomicExch(flag, 1);
    atomicCAS(&ctrl->status, PURL_OK, PURL_ERR_NONFINITE);
  }
}

__global__ void finite_poison_kernel(const int *flag, int m, int n, double *X, long long ldx) {
  if (*(volatile const int *)flag == 0) return;
  const double nan = __longlong_as_double(0x7ff8000000000000LL);
  const long long total = (long long)m * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x)
    X[(e % m) + (e / m) * ldx] = nan;
}

__global__ void zero_words_kernel(unsigned *p, long long words) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < words;
       i += (long long)gridDim.x * blockDim.x)
    p[i] = 0u;
}

}  // namespace

int zero_async(void *p, size_t bytes, cudaStream_t s) {
  const DeviceInfo *di = device_info();
  if (!di) return PURL_ERR_CUDA;
  const long long words = (long long)(bytes / 4);
  if (words == 0) return PURL_OK;
  long long blocks = (words + 255) / 256;
  if (blocks > (long long)di->num_sms * 4) blocks = (long long)di->num_sms * 4;
  LaunchScope ls(KC_OTHER, s, 0.0, (double)bytes, "zero_words_kernel");
  zero_words_kernel<<<(int)blocks, 256, 0, s>>>(static_cast<unsigned *>(p), words);
  return cudaGetLastError() == cudaSuccess ? PURL_OK : PURL_ERR_CUDA;
}

int finite_check(int m, int n, const double *A, long long lda, int *flag, cudaStream_t s) {
  const DeviceInfo *di = device_info();
  if (!di) return PURL_ERR_CUDA;
  PURL_TRY(zero_async(flag, sizeof(int), s));
  const long long total = (long long)m * n;
  if (total == 0) return PURL_OK;
  const long long warps = (long long)((m + 31) / 32) * n;
  long long blocks = (warps + 7) / 8;
  if (blocks > (long long)di->num_sms * 8) blocks = (long long)di->num_sms * 8;
  LaunchScope ls(KC_OTHER, s, 0.0, 8.0 * total, "finite_check_kernel");
  finite_check_kernel<<<(int)blocks, 256, 0, s>>>(m, n, A, lda, flag, di->ctrl);
  return cudaGetLastError() == cudaSuccess ? PURL_OK : PURL_ERR_CUDA;
}

int finite_poison(const int *flag, int m, int n, double *X, long long ldx, cudaStream_t s) {
  const DeviceInfo *di = device_info();
  if (!di) return PURL_ERR_CUDA;
  const long long total = (long long)m * n;
  if (total == 0 || X == nullptr) return PURL_OK;
  long long blocks = (total + 255) / 256;
  if (blocks > (long long)di->num_sms * 4) blocks = (long long)di->num_sms * 4;
  LaunchScope ls(KC_OTHER, s, 0.0, 4.0, "finite_poison_kernel");
  finite_poison_kernel<<<(int)blocks, 256, 0, s>>>(flag, m, n, X, ldx);
  return cudaGetLastError() == cudaSuccess ? PURL_OK : PURL_ERR_CUDA;
}

}  // namespace purl
