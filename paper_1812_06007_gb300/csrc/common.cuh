// common.cuh -- shared internals of libpurl (CUDA, sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include "purl.h"

namespace purl {

// ---------------------------------------------------------------- status --
#define PURL_CUDA_TRY(expr)                                   \
  do {                                                        \
    cudaError_t _e = (expr);                                  \
    if (_e != cudaSuccess) return PURL_ERR_CUDA;              \
  } while (0)

#define PURL_TRY(expr)                                        \
  do {                                                        \
    int _s = (expr);                                          \
    if (_s != PURL_OK) return _s;                             \
  } while (0)

// Per-device control block in device memory: the status word that bounded
// waits write when they give up, and an abort flag that makes the other
// blocks of the same launch stop waiting too.
struct DeviceControl {
  int status;
  int abort;
};

struct DeviceInfo {
  int device = -1;
  int num_sms = 0;
  int max_smem_optin = 0;
  DeviceControl *ctrl = nullptr;  // device pointer
};

// Lazily initialised per-device info (thread-safe).  Returns nullptr on a
// CUDA failure.
const DeviceInfo *device_info();

// The allocation-free product entry point keeps its own status word in its
// static device array: read and clear it (PURL_OK when never set up), and get
// its device address (setting the array up on first use).
int noalloc_take_status(int *status);
int noalloc_control(DeviceControl **ctrl);

// Zero `bytes` (a multiple of 4) of device memory with a kernel rather than
// cudaMemsetAsync, so that the many small clears of a factorization leave the
// copy engines to the caller's host transfers.
int zero_async(void *p, size_t bytes, cudaStream_t s);

// Non-finite input: finite_check zeroes *flag (device int), scans the m x n
// matrix and, if any entry is NaN or infinite, sets *flag and records
// PURL_ERR_NONFINITE in the device status word; finite_poison overwrites the
// m x n matrix X with NaN when *flag is set (one tiny launch otherwise).
int finite_check(int m, int n, const double *A, long long lda, int *flag, cudaStream_t s);
int finite_poison(const int *flag, int m, int n, double *X, long long ldx, cudaStream_t s);

// Spin budget of a device-side wait: number of polls before giving up
// (each poll is an L2 round trip of ~0.5-1 us, so this is several seconds).
constexpr long long kSpinLimit = 1LL << 23;

// ------------------------------------------------------ grid barrier ------
// Barrier among the `nblocks` co-resident blocks of a cooperative launch.
// `counter` starts at 0 for the launch; the i-th barrier (i = 0, 1, ...)
// completes when the counter reaches (i+1) * nblocks.  Arriving is a release
// reduction by thread 0 after a __syncthreads (publishing every write the
// block made before it), waiting an acquire poll by thread 0 followed by a
// __syncthreads (so every thread of the block sees what the others
// published).  Every wait is bounded: on expiry the block records
// PURL_ERR_TIMEOUT, raises the abort flag and returns false; callers then
// leave the kernel.
//
// In two halves, so that a block can do independent work between arriving and
// waiting.  grid_arrive: after a __syncthreads that orders the block's
// writes, thread 0 arrives.  grid_wait: thread 0 polls and the block learns
// the outcome; returns false when the wait gave up or another block aborted.
__device__ __forceinline__ void grid_arrive(unsigned *counter) {
  if (threadIdx.x == 0) asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(counter) : "memory");
}

__device__ __forceinline__ bool grid_wait(unsigned *counter, unsigned target, DeviceControl *ctrl,
                                          long long spin_limit = kSpinLimit) {
  __shared__ int s_ok2;
  if (threadIdx.x == 0) {
    int ok = 1;
    long long polls = 0;
    while (true) {
      unsigned v;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(counter) : "memory");
      if (v >= target) break;
      // the abort flag is a second L2 round trip: look at it every 64 polls
      if ((++polls & 63) == 0 && *(volatile int *)&ctrl->abort) { ok = 0; break; }
      if (polls > spin_limit) {
        atomicCAS(&ctrl->status, PURL_OK, PURL_ERR_TIMEOUT);
        atomicExch(&ctrl->abort, 1);
        ok = 0;
        break;
      }
    }
    s_ok2 = ok;
  }
  __syncthreads();
  return s_ok2 != 0;
}

__device__ __forceinline__ bool grid_barrier(unsigned *counter, unsigned target, DeviceControl *ctrl,
                                             long long spin_limit = kSpinLimit) {
  __syncthreads();
  grid_arrive(counter);
  return grid_wait(counter, target, ctrl, spin_limit);
}

// ---------------------------------------------------------- helpers -------
inline int ceil_div(int a, int b) { return (a + b - 1) / b; }
inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Bump allocator over a workspace.  With base == nullptr it only measures
// (take() returns nullptr and `used` grows), which is how workspace sizes are
// computed: the same plan function runs once to size and once to carve.
struct Arena {
  char *base = nullptr;
  size_t size = 0;
  size_t used = 0;
  bool ok = true;
  template <class T>
  T *take(size_t count) {
    size_t off = align_up(used, 256);
    used = off + align_up(count * sizeof(T), 256);
    if (base == nullptr) return nullptr;
    if (used > size) { ok = false; return nullptr; }
    return reinterpret_cast<T *>(base + off);
  }
};

}  // namespace purl
