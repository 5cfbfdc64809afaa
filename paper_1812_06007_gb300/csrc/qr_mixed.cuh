// qr_mixed.cuh -- mixed-precision blocked Householder QR (internal).
#pragma once

#include "qr.cuh"
#include "tc.cuh"

namespace purl {

constexpr int QR_NB = 512;  // outer block: QR_NB / QR_B inner panels share one aggregated update

struct QrMixWork {
  QrWork base;       // tau, T, panel V (FP64), panel scratch, Gram partials
  int S = 3;         // slices per operand in every product
  int *col_exp = nullptr;  // per-column exponents of the active block's slices
  Slices Fs;         // slices of the matrix being factored, scale = col_exp
  Slices Qs;         // slices of the Q being formed, scale = col_exp
  Slices Vs;         // slices of the panel's V (rows x QR_B), own column scales
  Slices Vts;        // slices of V^T (QR_B x rows), scale per row of V
  double *Pd = nullptr;  // split-K FP64 partials of W^T = C^T V
  Slices W2s;        // slices of W2 = op(T) V^T C (QR_B x n), own column scales
  // outer (aggregated) blocks
  double *Tout = nullptr;  // ceil(n/QR_NB) blocks of QR_NB x QR_NB, upper triangular
  double *Vo = nullptr;    // explicit rounded V of the outer block (m x QR_NB, ld m)
  double *Vtl = nullptr;   // V~ = V op(T_out) (m x QR_NB, ld m)
  double *Go = nullptr;    // split-K partials of V^T V (QR_MAX_SPLITS x QR_NB x QR_NB)
  double *Tt = nullptr;    // scratch QR_NB x QR_NB (T_out^T, T-builder products)
  double *Gparts = nullptr;  // row-chunk partials of a panel's FP64 Gram matrix
  double *Pdo = nullptr;   // split-K partials of W^T (kOuterSplits x n x QR_NB)
  Slices Vos;        // slices of V (rows x QR_NB)
  Slices Vots;       // slices of V^T (QR_NB x rows), scale per row of V
  Slices Vtls;       // slices of V~ (rows x QR_NB)
  Slices Ts;         // slices of op(T_out) (QR_NB x QR_NB)
  Slices W2o;        // slices of W2 (QR_NB x n)
  unsigned *tcount = nullptr;  // grid-barrier counter of the T_out assembly
};

int qr_mixed_plan(Arena &ar, int m, int n, int S, QrMixWork *w);
// Work with S slices (<= the S the workspace was planned for) from now on.
inline void qr_mixed_use_slices(QrMixWork &w, int S) {
  w.S = S;
  w.Fs.S = S; w.Qs.S = S; w.Vs.S = S; w.Vts.S = S; w.W2s.S = S;
  w.Vos.S = S; w.Vots.S = S; w.Vtls.S = S; w.Ts.S = S; w.W2o.S = S;
}

// F (m x n, ld ldf) holds M on entry and the packed factor (R above the
// diagonal, Householder vectors below) on exit.
int qr_mixed_factor(int m, int n, double *F, int ldf, QrMixWork &w, cudaStream_t s);
// Q (m x n) from the packed factor; diag signs are NOT normalised here.
int qr_mixed_form_q(int m, int n, const double *F, int ldf, QrMixWork &w, double *Q, int ldq, cudaStream_t s);

}  // namespace purl
