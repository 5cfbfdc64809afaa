// urv.cu -- the PowerURV driver (Section 3) and the C ABI of libpurl.
//
//   Y = G;  for i = 1..q:  Z = A Y      [Z <- Q(Z)  if reorth]
//                          Y = A^T Z    [Y <- Q(Y)  if reorth and i < q]
//   Eq. (5):  Y = V Z'  (Householder QR, diag(Z') >= 0)
//   Eq. (6):  A V = U R (Householder QR, diag(R) >= 0)
//
// The last power iterate needs no separate re-orthonormalisation: the QR of
// Eq. (5) is it.  q = 0 is DDH-URV (Section 2.2).  Everything is enqueued on
// the caller's stream; nothing synchronises.
#include <mutex>

#include "common.cuh"
#include "qr.cuh"
#include "qr_mixed.cuh"
#include "tc.cuh"

namespace purl {

int launch_gaussian(uint64_t seed, uint64_t stream_id, int rows, int cols, double *G, int ldg,
                    cudaStream_t stream, bool fp32_math = false);
int gemm_f64(bool ta, bool tb, int m, int n, int k, double alpha, const double *A, int lda,
             const double *B, int ldb, double beta, double *C, int ldc, cudaStream_t s);

// ------------------------------------------------------------ devices -----
const DeviceInfo *device_info() {
  static std::mutex mu;
  static DeviceInfo infos[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lock(mu);
  DeviceInfo &di = infos[dev];
  if (di.device == dev) return &di;
  int sms = 0, smem = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return nullptr;
  if (cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return nullptr;
  DeviceControl *ctrl = nullptr;
  if (cudaMalloc(&ctrl, sizeof(DeviceControl)) != cudaSuccess) return nullptr;
  if (cudaMemset(ctrl, 0, sizeof(DeviceControl)) != cudaSuccess) return nullptr;
  if (cudaDeviceSynchronize() != cudaSuccess) return nullptr;
  di.num_sms = sms;
  di.max_smem_optin = smem;
  di.ctrl = ctrl;
  di.device = dev;
  return &di;
}

// --------------------------------------------------------- workspace ------
// Slices per operand: the power-step products use one (plain BF16), the
// re-orthonormalisations of the power iteration use kReorthSlices and the two
// QRs that define V and U, R (Eqs. (5), (6)) and A V use kFinalSlices, all with
// exact accumulation.
constexpr int kReorthSlices = 2;
constexpr int kFinalSlices = 4;

struct UrvWork {
  int *finite = nullptr;                         // non-finite input flag
  double *buf[3] = {nullptr, nullptr, nullptr};  // each m x n
  QrWork qr;                                     // FP64 mode
  // mixed and FP64-emulation modes
  QrMixWork qm;
  Slices At1, An1, Ax, Ys, Zs, Vx;
  Slices Ae, Ze;  // FP64 emulation: A (m x n, scale per column), Z (m x n)
  int *pexp = nullptr;  // mixed modes: exponent scratch of the scaled power-step slices
};

// Slices per operand of the all-exact modes: every product, the power steps
// included, is an exact-accumulation product of S fixed-point slices.
// FP32 mode: 4 slices carry each operand row to 2^-32 of its scale.  Three
// (2^-24 of the row's largest entry) leave entries below that maximum with
// fewer than FP32's 24 bits, which measured ~1e-3 in ||I - Q^T Q||_F at
// n = 512, above FP32 Householder bounds (~4 n u = 1.2e-4).
constexpr int kFp32Slices = 4;
static int exact_slices(int mode) { return mode == PURL_MODE_FP32 ? kFp32Slices : kTcxEmuSlices; }

// FP64 emulation (S = kTcxEmuSlices, every operand row carried to 2^-63 of its
// scale) and FP32 (S = kFp32Slices): every product, including the power steps,
// with S exact slices.
static int urv_plan_emu(Arena &ar, int m, int n, int S, UrvWork *w) {
  PURL_TRY(qr_mixed_plan(ar, m, n, S, &w->qm));
  w->Ax = make_slices(ar.take<__nv_bfloat16>(slice_elems(n, m, S)), n, m, S);  // A^T: rows of A as operand rows
  w->Ax.scale = ar.take<int>(m > 0 ? m : 1);
  w->Ae = make_slices(ar.take<__nv_bfloat16>(slice_elems(m, n, S)), m, n, S);  // A: columns as operand rows
  w->Ae.scale = ar.take<int>(n > 0 ? n : 1);
  w->Ze = make_slices(ar.take<__nv_bfloat16>(slice_elems(m, n, S)), m, n, S);
  w->Ze.scale = ar.take<int>(n > 0 ? n : 1);
  w->Vx = make_slices(ar.take<__nv_bfloat16>(slice_elems(n, n, S)), n, n, S);  // Y, then V
  w->Vx.scale = ar.take<int>(n > 0 ? n : 1);
  return PURL_OK;
}

static int urv_plan(Arena &ar, int m, int n, int mode, UrvWork *w) {
  size_t mn = (size_t)(m > 0 ? m : 1) * (size_t)(n > 0 ? n : 1);
  w->finite = ar.take<int>(1);
  for (int i = 0; i < 3; ++i) w->buf[i] = ar.take<double>(mn);
  if (mode == PURL_MODE_FP64) return qr_plan(ar, m, n, mode, &w->qr);
  if (mode == PURL_MODE_FP64_EMU || mode == PURL_MODE_FP32) return urv_plan_emu(ar, m, n, exact_slices(mode), w);
  PURL_TRY(qr_mixed_plan(ar, m, n, kFinalSlices, &w->qm));
  const int f16 = mode == PURL_MODE_MIXED_FP16;
  w->pexp = ar.take<int>(1);
  w->At1 = make_slices(ar.take<__nv_bfloat16>(slice_elems(n, m, 1)), n, m, 1);
  w->An1 = make_slices(ar.take<__nv_bfloat16>(slice_elems(m, n, 1)), m, n, 1);
  w->Ax = make_slices(ar.take<__nv_bfloat16>(slice_elems(n, m, kFinalSlices)), n, m, kFinalSlices);
  w->Ax.scale = ar.take<int>(m > 0 ? m : 1);
  w->Ys = make_slices(ar.take<__nv_bfloat16>(slice_elems(n, n, 1)), n, n, 1);
  w->Zs = make_slices(ar.take<__nv_bfloat16>(slice_elems(m, n, 1)), m, n, 1);
  w->Vx = make_slices(ar.take<__nv_bfloat16>(slice_elems(n, n, kFinalSlices)), n, n, kFinalSlices);
  w->Vx.scale = ar.take<int>(n > 0 ? n : 1);
  w->At1.f16 = w->An1.f16 = w->Ys.f16 = w->Zs.f16 = f16;
  return PURL_OK;
}

static bool mode_ok(int mode) {
  return mode == PURL_MODE_FP64 || mode == PURL_MODE_FP32 || mode == PURL_MODE_MIXED_BF16 ||
         mode == PURL_MODE_MIXED_FP16 || mode == PURL_MODE_FP64_EMU;
}

// Slices of purl_qr's products in the tensor-core modes.
static int qr_slices(int mode) {
  return (mode == PURL_MODE_FP64_EMU || mode == PURL_MODE_FP32) ? exact_slices(mode) : kFinalSlices;
}

// The FP64-emulation products reduce over at most 2^20 rows (their 64-bit
// drains); a factorization with more rows is refused before any allocation.
constexpr int kEmuMaxRows = 1 << 20;
static bool emu_rows_ok(int mode, int rows) { return mode != PURL_MODE_FP64_EMU || rows <= kEmuMaxRows; }

// Stream-ordered scratch: the caller's workspace, or one allocated on the stream.
struct Scratch {
  void *ptr = nullptr;
  bool owned = false;
  cudaStream_t s = 0;
  int acquire(void *ws, size_t ws_bytes, size_t need, cudaStream_t stream) {
    s = stream;
    if (ws) {
      if (ws_bytes < need) return PURL_ERR_NOMEM;
      if (((uintptr_t)ws & 255) != 0) return PURL_ERR_NOMEM;
      ptr = ws;
      return PURL_OK;
    }
    if (need == 0) return PURL_OK;
    if (cudaMallocAsync(&ptr, need, stream) != cudaSuccess) return PURL_ERR_NOMEM;
    owned = true;
    return PURL_OK;
  }
  ~Scratch() {
    if (owned) cudaFreeAsync(ptr, s);
  }
};

static int urv_run_fp64(int m, int n, const double *A, int lda, int q, int reorth, uint64_t seed,
                        double *U, int ldu, double *R, int ldr, double *V, int ldv, UrvWork &w,
                        cudaStream_t s) {
  double *Y = w.buf[0], *Z = w.buf[1], *F = w.buf[2];
  PURL_TRY(launch_gaussian(seed, 0, n, n, Y, n, s));
  for (int i = 1; i <= q; ++i) {
    PURL_TRY(gemm_f64(false, false, m, n, n, 1.0, A, lda, Y, n, 0.0, F, m, s));  // F = A Y
    if (reorth) {
      PURL_TRY(qr_factor_f64(m, n, F, m, w.qr, s));
      PURL_TRY(qr_form_q_f64(m, n, F, m, w.qr, Z, m, s));
      PURL_TRY(qr_sign_fix(m, n, F, m, Z, m, nullptr, 0, s));
    } else {
      double *t = F; F = Z; Z = t;
    }
    PURL_TRY(gemm_f64(true, false, n, n, m, 1.0, A, lda, Z, m, 0.0, F, n, s));  // F = A^T Z
    if (reorth && i < q) {
      PURL_TRY(qr_factor_f64(n, n, F, n, w.qr, s));
      PURL_TRY(qr_form_q_f64(n, n, F, n, w.qr, Y, n, s));
      PURL_TRY(qr_sign_fix(n, n, F, n, Y, n, nullptr, 0, s));
    } else {
      double *t = F; F = Y; Y = t;
    }
  }
  // Eq. (5): (A^T A)^q G = V Z'
  PURL_TRY(qr_factor_f64(n, n, Y, n, w.qr, s));
  PURL_TRY(qr_form_q_f64(n, n, Y, n, w.qr, V, ldv, s));
  PURL_TRY(qr_sign_fix(n, n, Y, n, V, ldv, nullptr, 0, s));
  // Eq. (6): A V = U R
  PURL_TRY(gemm_f64(false, false, m, n, n, 1.0, A, lda, V, ldv, 0.0, F, m, s));
  PURL_TRY(qr_factor_f64(m, n, F, m, w.qr, s));
  PURL_TRY(qr_form_q_f64(m, n, F, m, w.qr, U, ldu, s));
  return qr_sign_fix(m, n, F, m, U, ldu, R, ldr, s);
}

// Mixed precision: power steps on the tensor cores with one plain BF16 or
// FP16 slice per operand and FP32 accumulation (they only shape the subspace),
// re-orthonormalisations with kReorthSlices exact slices, and the QRs of
// Eqs. (5)-(6) plus A V with kFinalSlices exact slices; Householder panels in
// FP64.  Every power-step operand is sliced as 2^s X with a power of two
// chosen from its largest entry (FP16's range is narrow, and the FP32 sums
// must not overflow); the scale is never undone, since each product is
// orthonormalised next (with reorth) or only its span enters the QR of
// Eq. (5) (without), and a positive scale changes neither.
static int urv_run_mixed(int m, int n, const double *A, int lda, int q, int reorth, uint64_t seed,
                         double *U, int ldu, double *R, int ldr, double *V, int ldv, UrvWork &w,
                         cudaStream_t s) {
  double *Y = w.buf[0], *Z = w.buf[1], *F = w.buf[2];
  TcEpilogue ep;
  ep.mode = 0;
  if (q > 0) {
    PURL_TRY(split_scaled(m, n, A, lda, w.At1, w.pexp, true, s));   // operand of A Y   (rows n = K, cols m = M)
    PURL_TRY(split_scaled(m, n, A, lda, w.An1, w.pexp, false, s));  // operand of A^T Z (rows m = K, cols n = M)
  }
  // G through the FP32 Box-Muller: its first use rounds it to BF16 / FP16
  // (with q = 0 it is orthonormalised by the mixed QR, whose panels are FP32)
  PURL_TRY(launch_gaussian(seed, 0, n, n, Y, n, s, true));
  for (int i = 1; i <= q; ++i) {
    PURL_TRY(split_scaled(n, n, Y, n, w.Ys, w.pexp, false, s));
    ep.C = F;
    ep.ldc = m;
    PURL_TRY(tc_gemm(w.At1, w.Ys, m, n, n, 1, ep, 1, ceil_div(n, 64) * 64, s));  // F = A Y
    if (reorth) {
      qr_mixed_use_slices(w.qm, kReorthSlices);
      PURL_TRY(qr_mixed_factor(m, n, F, m, w.qm, s));
      PURL_TRY(qr_mixed_form_q(m, n, F, m, w.qm, Z, m, s));
      PURL_TRY(qr_sign_fix(m, n, F, m, Z, m, nullptr, 0, s));
    } else {
      double *t = F; F = Z; Z = t;
    }
    PURL_TRY(split_scaled(m, n, Z, m, w.Zs, w.pexp, false, s));
    ep.C = F;
    ep.ldc = n;
    PURL_TRY(tc_gemm(w.An1, w.Zs, n, n, m, 1, ep, 1, ceil_div(m, 64) * 64, s));  // F = A^T Z
    if (reorth && i < q) {
      qr_mixed_use_slices(w.qm, kReorthSlices);
      PURL_TRY(qr_mixed_factor(n, n, F, n, w.qm, s));
      PURL_TRY(qr_mixed_form_q(n, n, F, n, w.qm, Y, n, s));
      PURL_TRY(qr_sign_fix(n, n, F, n, Y, n, nullptr, 0, s));
    } else {
      double *t = F; F = Y; Y = t;
    }
  }
  // Eq. (5): (A^T A)^q G = V Z'
  qr_mixed_use_slices(w.qm, kFinalSlices);
  PURL_TRY(qr_mixed_factor(n, n, Y, n, w.qm, s));
  PURL_TRY(qr_mixed_form_q(n, n, Y, n, w.qm, V, ldv, s));
  PURL_TRY(qr_sign_fix(n, n, Y, n, V, ldv, nullptr, 0, s));
  // A V with exact slices: A^T staged in Z (n x m), scale per row of A
  PURL_TRY(transpose_f64(m, n, A, lda, Z, n, s));
  PURL_TRY(split_exact(n, m, Z, n, w.Ax, nullptr, s));
  PURL_TRY(split_exact(n, n, V, ldv, w.Vx, nullptr, s));
  ep.C = F;
  ep.ldc = m;
  PURL_TRY(tcx_gemm_view(w.Ax, 0, 0, w.Vx, 0, 0, m, n, n, kFinalSlices, ep, 1, ceil_div(n, 256) * 256, s));
  // Eq. (6): A V = U R
  PURL_TRY(qr_mixed_factor(m, n, F, m, w.qm, s));
  PURL_TRY(qr_mixed_form_q(m, n, F, m, w.qm, U, ldu, s));
  return qr_sign_fix(m, n, F, m, U, ldu, R, ldr, s);
}

// FP64 emulated on the tensor cores: the FP64 path's algorithm with every
// product -- A Y, A^T Z, A V, and the trailing updates and Q formation of
// every QR -- as an exact-accumulation product of kTcxEmuSlices fixed-point
// BF16 slices, each operand row carried to 2^-63 of its scale.  Householder
// panels, their Gram matrices and the T factors stay in FP64.
static int urv_run_emu(int m, int n, const double *A, int lda, int q, int reorth, uint64_t seed,
                       double *U, int ldu, double *R, int ldr, double *V, int ldv, int S, UrvWork &w,
                       cudaStream_t s) {
  double *Y = w.buf[0], *Z = w.buf[1], *F = w.buf[2];
  qr_mixed_use_slices(w.qm, S);
  // A's slices, made once: A^T (rows of A as operand rows, staged in Z) for
  // A Y and A V, A itself (columns as operand rows) for A^T Z
  PURL_TRY(transpose_f64(m, n, A, lda, Z, n, s));
  PURL_TRY(split_exact(n, m, Z, n, w.Ax, nullptr, s));
  if (q > 0) PURL_TRY(split_exact(m, n, A, lda, w.Ae, nullptr, s));
  const int kn = ceil_div(n, 256) * 256, km = ceil_div(m, 256) * 256;
  TcEpilogue ep;
  ep.mode = 0;
  ep.tag = "tcx emu A Y";
  PURL_TRY(launch_gaussian(seed, 0, n, n, Y, n, s));
  for (int i = 1; i <= q; ++i) {
    PURL_TRY(split_exact(n, n, Y, n, w.Vx, nullptr, s));
    ep.C = F;
    ep.ldc = m;
    ep.tag = "tcx emu A Y";
    PURL_TRY(tcx_gemm_view(w.Ax, 0, 0, w.Vx, 0, 0, m, n, n, S, ep, 1, kn, s));  // F = A Y
    if (reorth) {
      PURL_TRY(qr_mixed_factor(m, n, F, m, w.qm, s));
      PURL_TRY(qr_mixed_form_q(m, n, F, m, w.qm, Z, m, s));
      PURL_TRY(qr_sign_fix(m, n, F, m, Z, m, nullptr, 0, s));
    } else {
      double *t = F; F = Z; Z = t;
    }
    PURL_TRY(split_exact(m, n, Z, m, w.Ze, nullptr, s));
    ep.C = F;
    ep.ldc = n;
    ep.tag = "tcx emu A^T Z";
    PURL_TRY(tcx_gemm_view(w.Ae, 0, 0, w.Ze, 0, 0, n, n, m, S, ep, 1, km, s));  // F = A^T Z
    if (reorth && i < q) {
      PURL_TRY(qr_mixed_factor(n, n, F, n, w.qm, s));
      PURL_TRY(qr_mixed_form_q(n, n, F, n, w.qm, Y, n, s));
      PURL_TRY(qr_sign_fix(n, n, F, n, Y, n, nullptr, 0, s));
    } else {
      double *t = F; F = Y; Y = t;
    }
  }
  // Eq. (5): (A^T A)^q G = V Z'
  PURL_TRY(qr_mixed_factor(n, n, Y, n, w.qm, s));
  PURL_TRY(qr_mixed_form_q(n, n, Y, n, w.qm, V, ldv, s));
  PURL_TRY(qr_sign_fix(n, n, Y, n, V, ldv, nullptr, 0, s));
  // A V, then Eq. (6): A V = U R
  PURL_TRY(split_exact(n, n, V, ldv, w.Vx, nullptr, s));
  ep.C = F;
  ep.ldc = m;
  ep.tag = "tcx emu A V";
  PURL_TRY(tcx_gemm_view(w.Ax, 0, 0, w.Vx, 0, 0, m, n, n, S, ep, 1, kn, s));
  PURL_TRY(qr_mixed_factor(m, n, F, m, w.qm, s));
  PURL_TRY(qr_mixed_form_q(m, n, F, m, w.qm, U, ldu, s));
  return qr_sign_fix(m, n, F, m, U, ldu, R, ldr, s);
}

static int urv_run(int m, int n, const double *A, int lda, int q, int reorth, uint64_t seed,
                   double *U, int ldu, double *R, int ldr, double *V, int ldv, int mode,
                   UrvWork &w, cudaStream_t s) {
  if (mode == PURL_MODE_MIXED_BF16 || mode == PURL_MODE_MIXED_FP16)
    return urv_run_mixed(m, n, A, lda, q, reorth, seed, U, ldu, R, ldr, V, ldv, w, s);
  if (mode == PURL_MODE_FP64_EMU || mode == PURL_MODE_FP32)
    return urv_run_emu(m, n, A, lda, q, reorth, seed, U, ldu, R, ldr, V, ldv, exact_slices(mode), w, s);
  return urv_run_fp64(m, n, A, lda, q, reorth, seed, U, ldu, R, ldr, V, ldv, w, s);
}

static int check_factor_args(int m, int n, const double *A, int lda, int q, double *U, int ldu,
                             double *R, int ldr, double *V, int ldv) {
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
  return PURL_OK;
}

}  // namespace purl

using namespace purl;

extern "C" {

const char *purl_status_str(int status) {
  switch (status) {
    case PURL_OK: return "ok";
    case PURL_ERR_SHAPE: return "m < n: factor the transpose instead";
    case PURL_ERR_NONFINITE: return "non-finite input";
    case PURL_ERR_TIMEOUT: return "a bounded device-side wait ran out";
    case PURL_ERR_CUDA: return "CUDA runtime error";
    case PURL_ERR_NOMEM: return "workspace allocation failed or too small";
    case PURL_ERR_UNSUPPORTED: return "unsupported on this device or build";
    default: return status < 0 ? "invalid argument (-i = i-th argument)" : "unknown status";
  }
}

const char *purl_version(void) { return "purl 0.1.0 sm_103a"; }

size_t purl_urv_workspace_bytes(int m, int n, int mode) {
  if (m < 0 || n < 0 || m < n || !mode_ok(mode) || !emu_rows_ok(mode, m)) return 0;
  Arena ar;
  UrvWork w;
  if (urv_plan(ar, m, n, mode, &w) != PURL_OK) return 0;
  return ar.used;
}

int purl_urv_factor_ex(int m, int n, const double *A, int lda, int q, int reorth, uint64_t seed,
                       double *U, int ldu, double *R, int ldr, double *V, int ldv, int mode,
                       void *workspace, size_t workspace_bytes, cudaStream_t stream) {
  int st = check_factor_args(m, n, A, lda, q, U, ldu, R, ldr, V, ldv);
  if (st != PURL_OK) return st;
  if (!mode_ok(mode)) return -14;
  if (!emu_rows_ok(mode, m)) return PURL_ERR_UNSUPPORTED;
  if (n == 0) return PURL_OK;
  if (!device_info()) return PURL_ERR_CUDA;
  size_t need = purl_urv_workspace_bytes(m, n, mode);
  Scratch scratch;
  PURL_TRY(scratch.acquire(workspace, workspace_bytes, need, stream));
  Arena ar;
  ar.base = static_cast<char *>(scratch.ptr);
  ar.size = workspace ? workspace_bytes : need;
  UrvWork w;
  PURL_TRY(urv_plan(ar, m, n, mode, &w));
  if (!ar.ok) return PURL_ERR_NOMEM;
  PURL_TRY(finite_check(m, n, A, lda, w.finite, stream));
  PURL_TRY(urv_run(m, n, A, lda, q, reorth, seed, U, ldu, R, ldr, V, ldv, mode, w, stream));
  PURL_TRY(finite_poison(w.finite, m, n, U, ldu, stream));
  PURL_TRY(finite_poison(w.finite, n, n, R, ldr, stream));
  return finite_poison(w.finite, n, n, V, ldv, stream);
}

int purl_urv_factor(int m, int n, const double *A, int lda, int q, int reorth, uint64_t seed,
                    double *U, int ldu, double *R, int ldr, double *V, int ldv,
                    cudaStream_t stream) {
  return purl_urv_factor_ex(m, n, A, lda, q, reorth, seed, U, ldu, R, ldr, V, ldv, PURL_MODE_FP64,
                            nullptr, 0, stream);
}

// ULV of a wide matrix through the URV of its transpose (Section 1): with
// A^T = U' R' V'^T (n x m, n >= m), A = V' R'^T U'^T, i.e. U = V' (m x m),
// L = R'^T (m x m, lower triangular, nonnegative diagonal), V = U' (n x m).
static int ulv_plan(Arena &ar, int m, int n, int mode, double **At, double **Rt, UrvWork *w) {
  *At = ar.take<double>((size_t)(n > 0 ? n : 1) * (size_t)(m > 0 ? m : 1));
  *Rt = ar.take<double>((size_t)(m > 0 ? m : 1) * (size_t)(m > 0 ? m : 1));
  return urv_plan(ar, n, m, mode, w);
}

size_t purl_ulv_workspace_bytes(int m, int n, int mode) {
  if (m < 0 || n < 0 || m > n || !mode_ok(mode) || !emu_rows_ok(mode, n)) return 0;
  Arena ar;
  double *At, *Rt;
  UrvWork w;
  if (ulv_plan(ar, m, n, mode, &At, &Rt, &w) != PURL_OK) return 0;
  return ar.used;
}

int purl_ulv_factor_ex(int m, int n, const double *A, int lda, int q, int reorth, uint64_t seed,
                       double *U, int ldu, double *L, int ldl, double *V, int ldv, int mode,
                       void *workspace, size_t workspace_bytes, cudaStream_t stream) {
  if (m < 0) return -1;
  if (n < 0) return -2;
  if (m > n) return PURL_ERR_SHAPE;
  if (!A && (long long)m * n > 0) return -3;
  if (lda < (m > 1 ? m : 1)) return -4;
  if (q < 0) return -5;
  if (!U && m > 0) return -8;
  if (ldu < (m > 1 ? m : 1)) return -9;
  if (!L && m > 0) return -10;
  if (ldl < (m > 1 ? m : 1)) return -11;
  if (!V && (long long)m * n > 0) return -12;
  if (ldv < (n > 1 ? n : 1)) return -13;
  if (!mode_ok(mode)) return -14;
  if (!emu_rows_ok(mode, n)) return PURL_ERR_UNSUPPORTED;
  if (m == 0) return PURL_OK;
  if (!device_info()) return PURL_ERR_CUDA;
  const size_t need = purl_ulv_workspace_bytes(m, n, mode);
  Scratch scratch;
  PURL_TRY(scratch.acquire(workspace, workspace_bytes, need, stream));
  Arena ar;
  ar.base = static_cast<char *>(scratch.ptr);
  ar.size = workspace ? workspace_bytes : need;
  double *At, *Rt;
  UrvWork w;
  PURL_TRY(ulv_plan(ar, m, n, mode, &At, &Rt, &w));
  if (!ar.ok) return PURL_ERR_NOMEM;
  PURL_TRY(finite_check(m, n, A, lda, w.finite, stream));
  PURL_TRY(transpose_f64(m, n, A, lda, At, n, stream));                                   // A^T, n x m
  PURL_TRY(urv_run(n, m, At, n, q, reorth, seed, V, ldv, Rt, m, U, ldu, mode, w, stream));  // A^T = V R' U^T
  PURL_TRY(transpose_f64(m, m, Rt, m, L, ldl, stream));                                   // L = R'^T
  PURL_TRY(finite_poison(w.finite, m, m, U, ldu, stream));
  PURL_TRY(finite_poison(w.finite, m, m, L, ldl, stream));
  return finite_poison(w.finite, n, m, V, ldv, stream);
}

int purl_gaussian(uint64_t seed, uint64_t stream_id, int rows, int cols, double *G, int ldg,
                  cudaStream_t stream) {
  if (rows < 0) return -3;
  if (cols < 0) return -4;
  if (!G && (long long)rows * cols > 0) return -5;
  if (ldg < (rows > 1 ? rows : 1)) return -6;
  return launch_gaussian(seed, stream_id, rows, cols, G, ldg, stream);
}

size_t purl_qr_workspace_bytes(int m, int n, int mode) {
  if (m < 0 || n < 0 || m < n || !mode_ok(mode) || !emu_rows_ok(mode, m)) return 0;
  Arena ar;
  int *flag = ar.take<int>(1);
  double *F = ar.take<double>((size_t)(m > 0 ? m : 1) * (size_t)(n > 0 ? n : 1));
  (void)F;
  (void)flag;
  if (mode == PURL_MODE_FP64) {
    QrWork w;
    if (qr_plan(ar, m, n, mode, &w) != PURL_OK) return 0;
  } else {
    QrMixWork w;
    if (qr_mixed_plan(ar, m, n, qr_slices(mode), &w) != PURL_OK) return 0;
  }
  return ar.used;
}

int purl_qr(int m, int n, const double *M, int ldm, double *Q, int ldq, double *R, int ldr,
            int mode, void *workspace, size_t workspace_bytes, cudaStream_t stream) {
  if (m < 0) return -1;
  if (n < 0) return -2;
  if (m < n) return PURL_ERR_SHAPE;
  if (!M && (long long)m * n > 0) return -3;
  if (ldm < (m > 1 ? m : 1)) return -4;
  if (Q && ldq < (m > 1 ? m : 1)) return -6;
  if (R && ldr < (n > 1 ? n : 1)) return -8;
  if (!mode_ok(mode)) return -9;
  if (!emu_rows_ok(mode, m)) return PURL_ERR_UNSUPPORTED;
  if (n == 0) return PURL_OK;
  if (!device_info()) return PURL_ERR_CUDA;
  size_t need = purl_qr_workspace_bytes(m, n, mode);
  Scratch scratch;
  PURL_TRY(scratch.acquire(workspace, workspace_bytes, need, stream));
  Arena ar;
  ar.base = static_cast<char *>(scratch.ptr);
  ar.size = workspace ? workspace_bytes : need;
  int *flag = ar.take<int>(1);
  double *F = ar.take<double>((size_t)m * n);
  if (mode == PURL_MODE_FP64) {
    QrWork w;
    PURL_TRY(qr_plan(ar, m, n, mode, &w));
    if (!ar.ok) return PURL_ERR_NOMEM;
    PURL_TRY(finite_check(m, n, M, ldm, flag, stream));
    PURL_TRY(copy_matrix(m, n, M, ldm, F, m, stream));
    PURL_TRY(qr_explicit(m, n, F, m, Q, ldq, R, ldr, mode, w, stream));
  } else {
    QrMixWork w;
    PURL_TRY(qr_mixed_plan(ar, m, n, qr_slices(mode), &w));
    if (!ar.ok) return PURL_ERR_NOMEM;
    PURL_TRY(finite_check(m, n, M, ldm, flag, stream));
    PURL_TRY(copy_matrix(m, n, M, ldm, F, m, stream));
    PURL_TRY(qr_mixed_factor(m, n, F, m, w, stream));
    if (Q) PURL_TRY(qr_mixed_form_q(m, n, F, m, w, Q, ldq, stream));
    PURL_TRY(qr_sign_fix(m, n, F, m, Q, ldq, R, ldr, stream));
  }
  PURL_TRY(finite_poison(flag, m, n, Q, ldq, stream));
  return finite_poison(flag, n, n, R, ldr, stream);
}

int purl_gemm_f64(char transa, char transb, int m, int n, int k, double alpha, const double *A,
                  int lda, const double *B, int ldb, double beta, double *C, int ldc,
                  cudaStream_t stream) {
  bool ta = (transa == 'T' || transa == 't'), tb = (transb == 'T' || transb == 't');
  if (!ta && transa != 'N' && transa != 'n') return -1;
  if (!tb && transb != 'N' && transb != 'n') return -2;
  if (m < 0) return -3;
  if (n < 0) return -4;
  if (k < 0) return -5;
  int arows = ta ? k : m, brows = tb ? n : k;
  if (!A && (long long)m * k > 0) return -7;
  if (lda < (arows > 1 ? arows : 1)) return -8;
  if (!B && (long long)k * n > 0) return -9;
  if (ldb < (brows > 1 ? brows : 1)) return -10;
  if (!C && (long long)m * n > 0) return -12;
  if (ldc < (m > 1 ? m : 1)) return -13;
  if (!device_info()) return PURL_ERR_CUDA;
  return gemm_f64(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, stream);
}

int purl_gemm_tc(char transa, char transb, int m, int n, int k, double alpha, const double *A,
                 int lda, const double *B, int ldb, double beta, double *C, int ldc, int slices,
                 int exact, cudaStream_t stream) {
  bool ta = (transa == 'T' || transa == 't'), tb = (transb == 'T' || transb == 't');
  if (!ta && transa != 'N' && transa != 'n') return -1;
  if (!tb && transb != 'N' && transb != 'n') return -2;
  if (m < 0) return -3;
  if (n < 0) return -4;
  if (k < 0) return -5;
  int arows = ta ? k : m, brows = tb ? n : k;
  if (!A && (long long)m * k > 0) return -7;
  if (lda < (arows > 1 ? arows : 1)) return -8;
  if (!B && (long long)k * n > 0) return -9;
  if (ldb < (brows > 1 ? brows : 1)) return -10;
  if (!C && (long long)m * n > 0) return -12;
  if (ldc < (m > 1 ? m : 1)) return -13;
  if (slices < 1 || (exact ? (slices > 4 && slices != kTcxEmuSlices) : slices > 3)) return -14;
  if (exact && slices > 4 && k > (1 << 20)) return PURL_ERR_UNSUPPORTED;
  if ((long long)m * n == 0) return PURL_OK;
  if (!device_info()) return PURL_ERR_CUDA;
  if (k == 0) return gemm_f64(false, false, m, n, 0, 0.0, A, lda, B, ldb, beta, C, ldc, stream);
  if (exact) {
    const size_t need = gemm_exact_bytes(m, n, k, slices);
    Scratch scratch;
    PURL_TRY(scratch.acquire(nullptr, 0, need, stream));
    return gemm_exact(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, slices, scratch.ptr, need, stream);
  }
  const size_t ea = slice_elems(k, m, slices), eb = slice_elems(k, n, slices);
  const size_t bytes = sizeof(__nv_bfloat16) * (ea + eb) + 1024;
  Scratch scratch;
  PURL_TRY(scratch.acquire(nullptr, 0, bytes, stream));
  Arena ar;
  ar.base = static_cast<char *>(scratch.ptr);
  ar.size = bytes;
  Slices sa = make_slices(ar.take<__nv_bfloat16>(ea), k, m, slices);
  Slices sb = make_slices(ar.take<__nv_bfloat16>(eb), k, n, slices);
  if (!ar.ok) return PURL_ERR_NOMEM;
  TcEpilogue ep;
  ep.mode = 0;
  ep.alpha = alpha;
  ep.beta = beta;
  ep.C = C;
  ep.ldc = ldc;
  // operand A: rows K, cols M (K-major); operand B: rows K, cols N
  if (ta) PURL_TRY(split_slices(k, m, A, lda, sa, stream));
  else PURL_TRY(split_slices_t(m, k, A, lda, sa, stream));
  if (tb) PURL_TRY(split_slices_t(n, k, B, ldb, sb, stream));
  else PURL_TRY(split_slices(k, n, B, ldb, sb, stream));
  return tc_gemm(sa, sb, m, n, k, slices, ep, 1, ceil_div(k, 64) * 64, stream);
}

int purl_urv_truncate(int m, int n, int k, const double *U, int ldu, const double *R, int ldr,
                      const double *V, int ldv, double *Ak, int ldak, cudaStream_t stream) {
  if (m < 0) return -1;
  if (n < 0) return -2;
  if (m < n) return PURL_ERR_SHAPE;
  if (k < 0 || k > n) return -3;
  if (!U && (long long)m * n > 0) return -4;
  if (ldu < (m > 1 ? m : 1)) return -5;
  if (!R && n > 0) return -6;
  if (ldr < (n > 1 ? n : 1)) return -7;
  if (!V && n > 0) return -8;
  if (ldv < (n > 1 ? n : 1)) return -9;
  if (!Ak && (long long)m * n > 0) return -10;
  if (ldak < (m > 1 ? m : 1)) return -11;
  if ((long long)m * n == 0) return PURL_OK;
  if (!device_info()) return PURL_ERR_CUDA;
  if (k == 0) return gemm_f64(false, false, m, n, 0, 0.0, U, ldu, R, ldr, 0.0, Ak, ldak, stream);
  Scratch scratch;
  PURL_TRY(scratch.acquire(nullptr, 0, sizeof(double) * (size_t)k * n, stream));
  double *W = static_cast<double *>(scratch.ptr);
  // W = R(1:k, :) V^T  (k x n), then A_k = U(:, 1:k) W
  PURL_TRY(gemm_f64(false, true, k, n, n, 1.0, R, ldr, V, ldv, 0.0, W, k, stream));
  return gemm_f64(false, false, m, n, k, 1.0, U, ldu, W, k, 0.0, Ak, ldak, stream);
}

int purl_urv_reconstruct(int m, int n, const double *U, int ldu, const double *R, int ldr,
                         const double *V, int ldv, double *Ak, int ldak, cudaStream_t stream) {
  return purl_urv_truncate(m, n, n, U, ldu, R, ldr, V, ldv, Ak, ldak, stream);
}

int purl_device_status(cudaStream_t stream) {
  const DeviceInfo *di = device_info();
  if (!di) return PURL_ERR_CUDA;
  if (cudaStreamSynchronize(stream) != cudaSuccess) return PURL_ERR_CUDA;
  DeviceControl h{};
  if (cudaMemcpy(&h, di->ctrl, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) return PURL_ERR_CUDA;
  DeviceControl z{};
  if (cudaMemcpy(di->ctrl, &z, sizeof(z), cudaMemcpyHostToDevice) != cudaSuccess) return PURL_ERR_CUDA;
  // the allocation-free entry point reports to a word of its own static array
  int na = PURL_OK;
  if (noalloc_take_status(&na) != PURL_OK) return PURL_ERR_CUDA;
  return h.status != PURL_OK ? h.status : na;
}

}  // extern "C"
