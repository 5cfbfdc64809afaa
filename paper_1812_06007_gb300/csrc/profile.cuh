// profile.cuh -- launch accounting and opt-in CUDA-event timing per kernel class.
#pragma once

#include "common.cuh"

namespace purl {

enum KernelClass {
  KC_GEMM_F64 = 0,    // FP64 DFMA product engine
  KC_PANEL = 1,       // Householder panel (cooperative)
  KC_GEMM_TC = 2,     // BF16 tensor-core product (tcgen05)
  KC_SPLIT = 3,       // FP64 -> BF16 slicing
  KC_OTHER = 4,       // RNG, T factor, reductions, copies, sign fixes
  KC_COUNT = 5
};

// Counts every kernel launch; when timing is on, brackets the launch with two
// CUDA events on its stream and books `flops` / `bytes` to the class.
struct LaunchScope {
  LaunchScope(int cls, cudaStream_t s, double flops = 0.0, double bytes = 0.0, const char *name = nullptr);
  ~LaunchScope();
  int cls_;
  const char *name_;
  cudaStream_t s_;
  double flops_, bytes_;
  cudaEvent_t e0_ = nullptr, e1_ = nullptr;
};

}  // namespace purl
