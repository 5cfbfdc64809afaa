// diag.cu -- a probe of the library's failure detection (no counterpart in
// the paper).  Every device-side wait in the library is bounded: on expiry it
// records PURL_ERR_TIMEOUT in the per-device status word, raises the abort
// flag and returns, so a wait that can never complete (a block that never
// arrives, a copy that never lands) becomes an error the host can read
// instead of a hung GPU.  purl_wait_probe runs the library's grid barrier in
// a grid where one block is missing, with a short poll limit.
#include "common.cuh"
#include "profile.cuh"

namespace purl {
namespace {

__device__ unsigned g_probe_counter;

__global__ void wait_probe_kernel(unsigned target, long long polls, DeviceControl *ctrl) {
  grid_barrier(&g_probe_counter, target, ctrl, polls);
}

__global__ void probe_reset_kernel() { g_probe_counter = 0u; }

}  // namespace
}  // namespace purl

using namespace purl;

extern "C" {

static int wait_probe(int blocks, int missing, long long polls, DeviceControl *ctrl, cudaStream_t stream) {
  { LaunchScope ls(KC_OTHER, stream, 0.0, 0.0, "probe_reset_kernel");
    probe_reset_kernel<<<1, 1, 0, stream>>>(); }
  PURL_CUDA_TRY(cudaGetLastError());
  // the barrier completes at `blocks` arrivals; with `missing` one more is awaited
  void *args[] = {nullptr, nullptr, nullptr};
  unsigned target = (unsigned)(blocks + missing);
  args[0] = &target;
  args[1] = &polls;
  args[2] = &ctrl;
  LaunchScope ls(KC_OTHER, stream, 0.0, 0.0, "wait_probe_kernel");
  PURL_CUDA_TRY(cudaLaunchCooperativeKernel((const void *)wait_probe_kernel, dim3(blocks), dim3(32), args, 0, stream));
  return PURL_OK;
}

int purl_wait_probe(int blocks, int missing, long long polls, cudaStream_t stream) {
  if (blocks < 1 || blocks > 64) return -1;
  if (missing < 0 || missing > 1) return -2;
  if (polls < 1) return -3;
  const DeviceInfo *di = device_info();
  if (!di) return PURL_ERR_CUDA;
  return wait_probe(blocks, missing, polls, di->ctrl, stream);
}

int purl_wait_probe_noalloc(int blocks, int missing, long long polls, cudaStream_t stream) {
  if (blocks < 1 || blocks > 64) return -1;
  if (missing < 0 || missing > 1) return -2;
  if (polls < 1) return -3;
  DeviceControl *ctrl = nullptr;
  PURL_TRY(noalloc_control(&ctrl));
  return wait_probe(blocks, missing, polls, ctrl, stream);
}

}  // extern "C"
