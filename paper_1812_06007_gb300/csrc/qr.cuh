// qr.cuh -- internal interface of the blocked Householder QR engine.
#pragma once

#include "common.cuh"
#include "tc.cuh"

namespace purl {

constexpr int QR_B = 32;            // panel width (columns per compact-WY block)
constexpr int QR_MAX_SPLITS = 64;   // split-K partial buffers for V^T C

struct QrWork {
  double *tau = nullptr;       // n reflector scalars
  double *T = nullptr;         // ceil(n/QR_B) blocks of QR_B x QR_B
  double *Vb = nullptr;        // explicit V of the current panel, m x QR_B
  double *Wp = nullptr;        // split-K partials of V^T C
  double *W2 = nullptr;        // op(T) V^T C, QR_B x n
  double *Gp = nullptr;        // split-K partials of V^T V
  double *part = nullptr;      // panel kernel: per-block partial sums (2 buffers)
  double *rowk = nullptr;      // panel kernel: pivot-row values (2 buffers)
  unsigned *counters = nullptr;  // one grid-barrier counter per panel
};

// Outputs of the tensor-core QR's fused panel tail (see panel_kernel): the
// Householder vectors rounded to the grid 2^(vexp - P), their slices vs
// (natural) and vts (transposed, one exponent per row), the Gram matrix
// partials gpart (blocks x bw(bw+1)/2) and their sum G (upper triangle column
// by column); panel_t then writes the T factor from G.
struct PanelTail {
  int vexp = 1, P = 31;
  unsigned epoch0 = 1;  // FP32 panel: epoch of column 0's tagged partial sums (see panel_kernel)
  Slices vs, vts;
  double *gpart = nullptr, *G = nullptr, *T = nullptr;
};

int qr_plan(Arena &ar, int m, int n, int mode, QrWork *w);
// One panel of the tensor-core QR with the fused tail (F, tau and the tail's
// outputs written; w.Vb is not).
int panel_factor_tail(int rows, int bw, double *Fp, int ldf, double *taup, unsigned *counter, QrWork &w,
                      const PanelTail &tail, cudaStream_t s);
// The panel's T from the Gram matrix its tail wrote (one block; tail.T).
int panel_t(int rows, int bw, const double *taup, const PanelTail &tail, cudaStream_t s);
int panel_factor(int rows, int bw, double *Fp, int ldf, double *taup, unsigned *counter, QrWork &w,
                 cudaStream_t s);
int larft_from_gram(int bw, int splits, const double *Gp, const double *taup, double *Tp, cudaStream_t s,
                    bool tau_from_gram = false);
int extract_v(int rows, int bw, const double *Fp, int ldf, double *Vb, cudaStream_t s);
int set_identity(int m, int n, double *Q, int ldq, cudaStream_t s);
int qr_factor_f64(int m, int n, double *F, int ldf, QrWork &w, cudaStream_t s);
int qr_form_q_f64(int m, int n, const double *F, int ldf, QrWork &w, double *Q, int ldq,
                  cudaStream_t s);
int qr_sign_fix(int m, int n, const double *F, int ldf, double *Q, int ldq, double *R, int ldr,
                cudaStream_t s);
int qr_explicit(int m, int n, double *F, int ldf, double *Q, int ldq, double *R, int ldr,
                int mode, QrWork &w, cudaStream_t s);
int transpose_f64(int R, int Cc, const double *X, int ldx, double *Y, int ldy, cudaStream_t s);
int copy_matrix(int m, int n, const double *X, int ldx, double *Y, int ldy, cudaStream_t s);

}  // namespace purl
