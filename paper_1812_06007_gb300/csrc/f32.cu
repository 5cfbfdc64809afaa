// f32.cu -- FP32 storage for the factorization and its reverse mode.
//
// The entry points take and return FP32 matrices.  Inputs are widened to FP64
// in the workspace (exactly), the call runs in the requested mode -- by default
// PURL_MODE_FP32, whose products are 4-slice exact tensor-core products (FP32
// precision) -- and the FP64 results are rounded to FP32 once.
#include "common.cuh"
#include "profile.cuh"

namespace purl {
namespace {

__global__ void widen_kernel(int m, int n, const float *__restrict__ X, long long ldx, double *Y, long long ldy) {
  const long long total = (long long)m * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e % m), j = (int)(e / m);
    Y[i + j * ldy] = (double)X[i + j * ldx];
  }
}

__global__ void narrow_kernel(int m, int n, const double *__restrict__ X, long long ldx, float *Y, long long ldy) {
  const long long total = (long long)m * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e % m), j = (int)(e / m);
    Y[i + j * ldy] = __double2float_rn(X[i + j * ldx]);
  }
}

int grid_for_elems(long long total) {
  const DeviceInfo *di = device_info();
  long long g = (total + 255) / 256;
  const long long cap = (long long)di->num_sms * 16;
  return (int)(g > cap ? cap : (g < 1 ? 1 : g));
}

int widen(int m, int n, const float *X, int ldx, double *Y, int ldy, cudaStream_t s) {
  if ((long long)m * n == 0) return PURL_OK;
  LaunchScope ls(KC_OTHER, s, 0.0, 12.0 * m * (double)n, "widen_kernel");
  widen_kernel<<<grid_for_elems((long long)m * n), 256, 0, s>>>(m, n, X, ldx, Y, ldy);
  return cudaGetLastError() == cudaSuccess ? PURL_OK : PURL_ERR_CUDA;
}

int narrow(int m, int n, const double *X, int ldx, float *Y, int ldy, cudaStream_t s) {
  if ((long long)m * n == 0) return PURL_OK;
  LaunchScope ls(KC_OTHER, s, 0.0, 12.0 * m * (double)n, "narrow_kernel");
  narrow_kernel<<<grid_for_elems((long long)m * n), 256, 0, s>>>(m, n, X, ldx, Y, ldy);
  return cudaGetLastError() == cudaSuccess ? PURL_OK : PURL_ERR_CUDA;
}

// FP64 staging of the FP32 entry points: `count` matrices of rows x cols each,
// then the inner call's workspace.
struct F32Plan {
  double *buf[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  char *inner = nullptr;
  size_t inner_bytes = 0;
};

void f32_plan(Arena &ar, const int (*shape)[2], int count, size_t inner_bytes, F32Plan *p) {
  for (int i = 0; i < count; ++i)
    p->buf[i] = ar.take<double>((size_t)(shape[i][0] > 0 ? shape[i][0] : 1) * (shape[i][1] > 0 ? shape[i][1] : 1));
  p->inner_bytes = inner_bytes;
  p->inner = ar.take<char>(inner_bytes > 0 ? inner_bytes : 1);
}

// Stream-ordered scratch: the caller's workspace or one allocated on the stream.
struct F32Scratch {
  void *ptr = nullptr;
  bool owned = false;
  cudaStream_t s = 0;
  int acquire(void *ws, size_t ws_bytes, size_t need, cudaStream_t stream) {
    s = stream;
    if (ws) {
      if (ws_bytes < need || ((uintptr_t)ws & 255) != 0) return PURL_ERR_NOMEM;
      ptr = ws;
      return PURL_OK;
    }
    if (cudaMallocAsync(&ptr, need, stream) != cudaSuccess) return PURL_ERR_NOMEM;
    owned = true;
    return PURL_OK;
  }
  ~F32Scratch() {
    if (owned) cudaFreeAsync(ptr, s);
  }
};

}  // namespace
}  // namespace purl

using namespace purl;

extern "C" {

size_t purl_urv_f32_workspace_bytes(int m, int n, int mode) {
  const size_t inner = purl_urv_workspace_bytes(m, n, mode);
  if (inner == 0) return 0;
  const int shape[4][2] = {{m, n}, {m, n}, {n, n}, {n, n}};
  Arena ar;
  F32Plan p;
  f32_plan(ar, shape, 4, inner, &p);
  return ar.used;
}

int purl_urv_factor_f32(int m, int n, const float *A, int lda, int q, int reorth, uint64_t seed, float *U, int ldu,
                        float *R, int ldr, float *V, int ldv, int mode, void *workspace, size_t workspace_bytes,
                        cudaStream_t stream) {
  if (m < 0) return -1;
  if (n < 0) return -2;
  if (m < n) return PURL_ERR_SHAPE;
  if (!A && (long long)m * n > 0) return -3;
  if (lda < (m > 1 ? m : 1)) return -4;
  if (q < 0) return -5;
  if (!U && (long long)m * n > 0) return -8;
  if (ldu < (m > 1 ? m : 1)) return -9;
  if (!R && n > 0) return -10;
  if (ldr < (n > 1 ? n : 1)) return -11;
  if (!V && n > 0) return -12;
  if (ldv < (n > 1 ? n : 1)) return -13;
  const size_t need = purl_urv_f32_workspace_bytes(m, n, mode);
  if (need == 0) return -14;  // unsupported mode or size for the mode
  if (n == 0) return PURL_OK;
  if (!device_info()) return PURL_ERR_CUDA;
  F32Scratch scratch;
  PURL_TRY(scratch.acquire(workspace, workspace_bytes, need, stream));
  Arena ar;
  ar.base = static_cast<char *>(scratch.ptr);
  ar.size = workspace ? workspace_bytes : need;
  const int shape[4][2] = {{m, n}, {m, n}, {n, n}, {n, n}};
  F32Plan p;
  f32_plan(ar, shape, 4, purl_urv_workspace_bytes(m, n, mode), &p);
  if (!ar.ok) return PURL_ERR_NOMEM;
  double *A64 = p.buf[0], *U64 = p.buf[1], *R64 = p.buf[2], *V64 = p.buf[3];
  PURL_TRY(widen(m, n, A, lda, A64, m, stream));
  PURL_TRY(purl_urv_factor_ex(m, n, A64, m, q, reorth, seed, U64, m, R64, n, V64, n, mode, p.inner, p.inner_bytes,
                              stream));
  PURL_TRY(narrow(m, n, U64, m, U, ldu, stream));
  PURL_TRY(narrow(n, n, R64, n, R, ldr, stream));
  return narrow(n, n, V64, n, V, ldv, stream);
}

size_t purl_urv_backward_f32_workspace_bytes(int m, int n, int q, int mode) {
  const size_t inner = purl_urv_backward_ex_workspace_bytes(m, n, q, mode);
  if (inner == 0) return 0;
  const int shape[5][2] = {{m, n}, {m, n}, {n, n}, {n, n}, {m, n}};  // A, Ubar, Rbar, Vbar, Abar
  Arena ar;
  F32Plan p;
  f32_plan(ar, shape, 5, inner, &p);
  return ar.used;
}

int purl_urv_backward_f32(int m, int n, const float *A, int lda, int q, int reorth, uint64_t seed, const float *Ubar,
                          int ldub, const float *Rbar, int ldrb, const float *Vbar, int ldvb, float *Abar, int ldab,
                          int mode, void *workspace, size_t workspace_bytes, cudaStream_t stream) {
  if (m < 0) return -1;
  if (n < 0) return -2;
  if (m < n) return PURL_ERR_SHAPE;
  if (!A && (long long)m * n > 0) return -3;
  if (lda < (m > 1 ? m : 1)) return -4;
  if (q < 0) return -5;
  if (!Ubar && (long long)m * n > 0) return -8;
  if (ldub < (m > 1 ? m : 1)) return -9;
  if (!Rbar && n > 0) return -10;
  if (ldrb < (n > 1 ? n : 1)) return -11;
  if (!Vbar && n > 0) return -12;
  if (ldvb < (n > 1 ? n : 1)) return -13;
  if (!Abar && (long long)m * n > 0) return -14;
  if (ldab < (m > 1 ? m : 1)) return -15;
  const size_t need = purl_urv_backward_f32_workspace_bytes(m, n, q, mode);
  if (need == 0) return -16;  // unsupported mode or size for the mode
  if ((long long)m * n == 0) return PURL_OK;
  if (!device_info()) return PURL_ERR_CUDA;
  F32Scratch scratch;
  PURL_TRY(scratch.acquire(workspace, workspace_bytes, need, stream));
  Arena ar;
  ar.base = static_cast<char *>(scratch.ptr);
  ar.size = workspace ? workspace_bytes : need;
  const int shape[5][2] = {{m, n}, {m, n}, {n, n}, {n, n}, {m, n}};
  F32Plan p;
  f32_plan(ar, shape, 5, purl_urv_backward_ex_workspace_bytes(m, n, q, mode), &p);
  if (!ar.ok) return PURL_ERR_NOMEM;
  double *A64 = p.buf[0], *Ub = p.buf[1], *Rb = p.buf[2], *Vb = p.buf[3], *Ab = p.buf[4];
  PURL_TRY(widen(m, n, A, lda, A64, m, stream));
  PURL_TRY(widen(m, n, Ubar, ldub, Ub, m, stream));
  PURL_TRY(widen(n, n, Rbar, ldrb, Rb, n, stream));
  PURL_TRY(widen(n, n, Vbar, ldvb, Vb, n, stream));
  PURL_TRY(purl_urv_backward_ex(m, n, A64, m, q, reorth, seed, Ub, m, Rb, n, Vb, n, Ab, m, mode, p.inner,
                                p.inner_bytes, stream));
  return narrow(m, n, Ab, m, Abar, ldab, stream);
}

}  // extern "C"
