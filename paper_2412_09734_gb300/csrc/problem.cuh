// Problem-level device data shared by the preprocessing and iteration code.
#pragma once

#include "common.cuh"

namespace mpax {

struct ProblemData {
  int m = 0, n = 0, nnz = 0;
  bool is_qp = false;
  cudaStream_t s = nullptr;  // library stream (non-blocking)

  // original data, FP64
  Csr A;                      // rp, col
  double* val = nullptr;      // A values
  double *c = nullptr, *lc = nullptr, *uc = nullptr, *l = nullptr, *u = nullptr;

  // QP: Q = diag(D) + F F^T, F is n x r
  int r = 0, f_nnz = 0;
  double* D = nullptr;
  Csr F;                      // n x r
  double* fval = nullptr;
  Csr Ft;                     // r x n (device transpose of F)
  int* permF = nullptr;

  // QP with a general sparse Q (mpax_qp_create): Q is n x n CSR, symmetric with
  // both triangles stored; D = 0 and F is an empty n x 1 matrix, so the
  // diagonal-plus-low-rank terms vanish and every Q product is a SpMV with Q.
  bool q_general = false;
  Csr Q;
  double* qval = nullptr;     // original values
  double* qval_s = nullptr;   // scaled: Dc_i Q_ij Dc_j

  // device transpose of A
  Csr At;
  int* permT = nullptr;
  bool transposed = false;

  // schedules
  Sched schedA, schedAt, schedF, schedFt, schedQ;
  bool scheduled = false;

  // scaling: A~ = diag(Dr) A diag(Dc)
  double *Dr = nullptr, *Dc = nullptr, *invDr = nullptr, *invDc = nullptr;
  double* val_s = nullptr;    // scaled A values, FP64 (A order)
  double* fval_s = nullptr;   // scaled F values (diag(Dc) F), FP64
  double* D_s = nullptr;      // scaled D (Dc^2 D)
  double* qdiag = nullptr;    // diag(Q) = D + row sums of F^2 (QP)
  double* rowred = nullptr;   // m work
  double* colred = nullptr;   // n work
  double* rowred2 = nullptr;  // m work (the next Ruiz round's norms)
  double* colred2 = nullptr;  // n work

  // scratch
  int* tmp_rows = nullptr;    // max(m, n, r) + 2 ints
  int* tmp_scan = nullptr;    // scan_tmp_ints(max(m, n, r) + 1)
  double* red = nullptr;      // reduction partials (kRedBlocks * 8)
  double* red_out = nullptr;  // 16 doubles
};

constexpr int kRedBlocks = 304;  // 2 x 152 SMs

// ---- preprocessing (prep.cu) ----
// Ruiz (ruiz_iters rounds) then optional Pock-Chambolle (alpha = 1) on A;
// fills Dr, Dc, invDr, invDc, val_s (and fval_s, D_s for QP).
cudaError_t compute_scaling(ProblemData& P, int ruiz_iters, bool pock_chambolle);
// out[0] = ||c~||, out[1] = ||b~||, out[2] = ||c||, out[3] = ||b|| into P.red_out (device).
cudaError_t bound_and_cost_norms(ProblemData& P);

template <typename T>
cudaError_t gather_cast(const double* src, const int* perm, T* dst, int n, cudaStream_t s);
template <typename T>
cudaError_t cast_vec(const double* src, T* dst, int n, cudaStream_t s);
// dst = src * d (elementwise, d may be nullptr = 1), or src / d when divide
template <typename T>
cudaError_t scale_cast(const double* src, const double* d, bool divide, T* dst, int n,
                       cudaStream_t s);

}  // namespace mpax
