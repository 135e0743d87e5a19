// Differentiation of the returned solution (FP64 on the device).
//
// LP: gradients of the optimal value at the returned point (x, y) by the
// envelope theorem: dv/dc = x, dv/dlc = y^+, dv/duc = -y^-, dv/dl = lam^+,
// dv/du = -lam^-, lam = c - A^T y.
//
// QP with Q = diag(D) + F F^T: implicit adjoint on the active set.  With F the
// free variables (strictly inside the box, or at a bound with a multiplier of
// at most delta') and R the active rows (equalities, and inequalities with
// y_i != 0), the solution satisfies
//     Q_FF x_F - A_RF^T y_R = -c_F - Q_FB x_B,    A_RF x_F = b_R - A_RB x_B,
// so for a loss gradient g = dL/dx the adjoint system
//     [[Q_FF, A_RF^T], [A_RF, 0]] [w; v] = [g_F; 0]
// gives dL/dc_F = -w, dL/db_R = v, dL/dD_j = -w_j x_j (j in F), zero elsewhere.
// The system is solved in the scaled variables w = D_c w~, v = D_r v~, where it
// reads [[Q~_FF, A~_RF^T], [A~_RF, 0]] [w~; v~] = [D_c g; 0], by MINRES
// (Paige-Saunders recurrences) with masked SpMVs of A~, A~^T and F~.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/mpax.h"
#include "problem.cuh"

namespace mpax {
ProblemData* problem_data(mpax_problem* p);
cudaStream_t problem_stream(mpax_problem* p);
}  // namespace mpax

namespace {

using namespace mpax;

int g1(long long k) { return (int)std::max(1LL, std::min(4096LL, (k + 255) / 256)); }
int wgrid(long long rows) { return (int)std::max(1LL, std::min(152LL * 8, (rows * 32 + 255) / 256)); }

// out_r = mask_r * (sum_p val[p] x[col[p]] + d_r x_r)   (d, mask nullable)
__global__ void k_rows(const int* __restrict__ rp, const int* __restrict__ col,
                       const double* __restrict__ val, const int* __restrict__ perm, int rows,
                       const double* __restrict__ x, const double* __restrict__ d,
                       const double* __restrict__ xd, const unsigned char* __restrict__ mask,
                       double* __restrict__ out, int accumulate) {
  const int lane = threadIdx.x & 31;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < rows; r += nw) {
    double s = 0.0;
    for (int p = rp[r] + lane; p < rp[r + 1]; p += 32)
      s += (perm ? val[perm[p]] : val[p]) * x[col[p]];
    s = warp_sum(s);
    if (lane == 0) {
      if (d) s += d[r] * xd[r];
      if (accumulate) s += out[r];
      out[r] = (mask && !mask[r]) ? 0.0 : s;
    }
  }
}

__global__ void k_dot_part(const double* __restrict__ a, const double* __restrict__ b, int n,
                           double* __restrict__ part) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    s += a[i] * b[i];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void k_sum_part(const double* __restrict__ part, int nb, double* __restrict__ out) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) s += part[i];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) *out = s;
}

// lam_j = (Ds x~ + F~ u)_j / Dc_j + c_j - (A^T y)_j with x~ = x / Dc, used for the
// active set; y in unscaled units; computed from the unscaled original data.
__global__ void k_active(const double* __restrict__ x, const double* __restrict__ lam,
                         const double* __restrict__ l, const double* __restrict__ u,
                         double tol_x, double tol_lam, int n, unsigned char* __restrict__ freem) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double lo = l[j], hi = u[j], xv = x[j];
  const bool nl = isfinite(lo) && (xv - lo <= tol_x * (1.0 + fabs(lo)));
  const bool nu = isfinite(hi) && (hi - xv <= tol_x * (1.0 + fabs(hi)));
  const bool weak = fabs(lam[j]) <= tol_lam;
  freem[j] = (!(nl || nu) || weak) ? 1 : 0;
}

__global__ void k_rows_active(const double* __restrict__ lc, const double* __restrict__ uc,
                              const double* __restrict__ y, int m,
                              unsigned char* __restrict__ rowm) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const bool eq = isfinite(lc[i]) && isfinite(uc[i]) && lc[i] == uc[i];
  rowm[i] = (eq || y[i] != 0.0) ? 1 : 0;
}

// elementwise helpers on the stacked vector of length N
__global__ void k_axpby(double* __restrict__ z, const double* __restrict__ a, double alpha,
                        const double* __restrict__ b, double beta, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    z[i] = alpha * a[i] + beta * (b ? b[i] : 0.0);
}

// w_new = (v - e w1 - dl w2) / g;  x += phi w_new;  (w1, w2, w) rotate on the host
__global__ void k_minres_w(const double* __restrict__ v, const double* __restrict__ w1,
                           const double* __restrict__ w2, double oldeps, double delta,
                           double denom, double* __restrict__ wout, double* __restrict__ x,
                           double phi, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double wn = (v[i] - oldeps * w1[i] - delta * w2[i]) * denom;
    wout[i] = wn;
    x[i] += phi * wn;
  }
}

// rhs_top = mask_F * Dc * g, rhs_bottom = 0
__global__ void k_rhs(const double* __restrict__ g, const double* __restrict__ Dc,
                      const unsigned char* __restrict__ freem, int n, int m,
                      double* __restrict__ b) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n + m; i += gridDim.x * blockDim.x)
    b[i] = (i < n) ? (freem[i] ? Dc[i] * g[i] : 0.0) : 0.0;
}

// dc = -Dc w~ (free), db = Dr v~ (active rows), dD = -(Dc w~) x (free)
__global__ void k_adj_out(const double* __restrict__ z, const double* __restrict__ Dc,
                          const double* __restrict__ Dr, const double* __restrict__ x,
                          const unsigned char* __restrict__ freem,
                          const unsigned char* __restrict__ rowm, int n, int m,
                          double* __restrict__ dc, double* __restrict__ db,
                          double* __restrict__ dD) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n + m; i += gridDim.x * blockDim.x) {
    if (i < n) {
      const double w = freem[i] ? Dc[i] * z[i] : 0.0;
      dc[i] = -w;
      if (dD) dD[i] = -w * x[i];
    } else {
      const int r = i - n;
      db[r] = rowm[r] ? Dr[r] * z[i] : 0.0;
    }
  }
}

// LP value gradients from x, y and lam = c - A^T y
__global__ void k_lp_grad(const double* __restrict__ x, const double* __restrict__ y,
                          const double* __restrict__ lam, int n, int m, double* dc, double* dlc,
                          double* duc, double* dl, double* du) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n + m; i += gridDim.x * blockDim.x) {
    if (i < n) {
      if (dc) dc[i] = x[i];
      if (dl) dl[i] = fmax(lam[i], 0.0);
      if (du) du[i] = -fmax(-lam[i], 0.0);
    } else {
      const int r = i - n;
      if (dlc) dlc[r] = fmax(y[r], 0.0);
      if (duc) duc[r] = -fmax(-y[r], 0.0);
    }
  }
}

// lam = c - A^T y + Q x (unscaled), from the unscaled data via A^T (perm) and F
__global__ void k_lam_finish(const double* __restrict__ aty, const double* __restrict__ c,
                             const double* __restrict__ qx, int n, double* __restrict__ lam) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  lam[j] = c[j] - aty[j] + (qx ? qx[j] : 0.0);
}

mpax_status afail(mpax_status s, const std::string& m) {
  set_last_error(m.c_str());
  return s;
}

struct DBuf {
  std::vector<void*> ptrs;
  ~DBuf() {
    for (void* p : ptrs) cudaFree(p);
  }
  template <typename T>
  T* get(size_t n, cudaError_t* e) {
    T* p = nullptr;
    if (*e == cudaSuccess) *e = cudaMalloc(&p, sizeof(T) * std::max<size_t>(n, 1));
    if (p) ptrs.push_back(p);
    return p;
  }
};

double dot(const double* a, const double* b, int n, double* part, double* out, cudaStream_t s) {
  k_dot_part<<<kRedBlocks, 256, 0, s>>>(a, b, n, part);
  k_sum_part<<<1, 256, 0, s>>>(part, kRedBlocks, out);
  double h = 0.0;
  cudaMemcpyAsync(&h, out, sizeof(double), cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  return h;
}

// Unscaled lam = Q x + c - A^T y on the device (x, y unscaled; n, m).
cudaError_t lambda_unscaled(ProblemData& P, const double* x, const double* y, double* lam,
                            double* tmpn, double* tmpr, cudaStream_t s) {
  // A^T y with the original values through the transpose permutation
  k_rows<<<wgrid(P.n), 256, 0, s>>>(P.At.rp, P.At.col, P.val, P.permT, P.n, y, nullptr,
                                     nullptr, nullptr, tmpn, 0);
  double* qx = nullptr;
  if (P.is_qp) {
    // u = F^T x (rows of F^T), then qx = F u + D x (rows of F)
    k_rows<<<wgrid(P.r), 256, 0, s>>>(P.Ft.rp, P.Ft.col, P.fval, P.permF, P.r, x, nullptr,
                                       nullptr, nullptr, tmpr, 0);
    k_rows<<<wgrid(P.n), 256, 0, s>>>(P.F.rp, P.F.col, P.fval, nullptr, P.n, tmpr, P.D, x,
                                       nullptr, lam, 0);
    if (P.q_general)  // + Q x for a general sparse Q (D = 0, F empty)
      k_rows<<<wgrid(P.n), 256, 0, s>>>(P.Q.rp, P.Q.col, P.qval, nullptr, P.n, x, nullptr,
                                         nullptr, nullptr, lam, 1);
    qx = lam;
  }
  k_lam_finish<<<g1(P.n), 256, 0, s>>>(tmpn, P.c, qx, P.n, lam);
  return cudaGetLastError();
}

}  // namespace

extern "C" {

mpax_status mpax_get_reduced_cost(mpax_problem* prob, double* lam, mpax_mem_kind kind) {
  if (!prob || !lam) return afail(MPAX_ERR_INVALID_ARGUMENT, "NULL argument");
  ProblemData& P = *problem_data(prob);
  const int n = P.n, m = P.m;
  cudaStream_t s = P.s;
  DBuf B;
  cudaError_t e = cudaSuccess;
  double* x = B.get<double>(n, &e);
  double* y = B.get<double>(m, &e);
  double* out = B.get<double>(n, &e);
  double* tmp = B.get<double>(n, &e);
  double* tmpr = B.get<double>(std::max(P.r, 1), &e);
  if (e) return afail(MPAX_ERR_OUT_OF_MEMORY, "reduced-cost buffers");
  mpax_status st = mpax_get_solution(prob, x, y, MPAX_MEM_DEVICE);
  if (st) return st;
  if ((e = lambda_unscaled(P, x, y, out, tmp, tmpr, s))) return afail(MPAX_ERR_CUDA, cudaGetErrorString(e));
  const cudaMemcpyKind k = kind == MPAX_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  if (n) e = cudaMemcpyAsync(lam, out, sizeof(double) * n, k, s);
  if (!e) e = cudaStreamSynchronize(s);
  if (e) return afail(MPAX_ERR_CUDA, cudaGetErrorString(e));
  return MPAX_OK;
}

mpax_status mpax_lp_value_grad(mpax_problem* prob, double* dc, double* dlc, double* duc,
                               double* dl, double* du, mpax_mem_kind kind) {
  if (!prob) return afail(MPAX_ERR_INVALID_ARGUMENT, "problem is NULL");
  ProblemData& P = *problem_data(prob);
  if (P.is_qp) return afail(MPAX_ERR_INVALID_ARGUMENT, "mpax_lp_value_grad needs an LP");
  const int n = P.n, m = P.m;
  DBuf B;
  cudaError_t e = cudaSuccess;
  double* x = B.get<double>(n, &e);
  double* y = B.get<double>(m, &e);
  double* lam = B.get<double>(n, &e);
  double* tmp = B.get<double>(n, &e);
  double* out = B.get<double>(3 * (size_t)n + 2 * (size_t)m, &e);
  if (e) return afail(MPAX_ERR_OUT_OF_MEMORY, "value gradient buffers");
  mpax_status st = mpax_get_solution(prob, x, y, MPAX_MEM_DEVICE);
  if (st) return st;
  cudaStream_t s = P.s;
  if ((e = lambda_unscaled(P, x, y, lam, tmp, nullptr, s))) return afail(MPAX_ERR_CUDA, cudaGetErrorString(e));
  double *odc = out, *odl = out + n, *odu = out + 2 * (size_t)n, *odlc = out + 3 * (size_t)n,
         *oduc = odlc + m;
  k_lp_grad<<<g1(n + m), 256, 0, s>>>(x, y, lam, n, m, odc, odlc, oduc, odl, odu);
  const cudaMemcpyKind k = kind == MPAX_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  double* dst[5] = {dc, dlc, duc, dl, du};
  double* src[5] = {odc, odlc, oduc, odl, odu};
  const int len[5] = {n, m, m, n, n};
  for (int q = 0; q < 5 && !e; ++q)
    if (dst[q] && len[q]) e = cudaMemcpyAsync(dst[q], src[q], sizeof(double) * len[q], k, s);
  if (!e) e = cudaStreamSynchronize(s);
  if (e) return afail(MPAX_ERR_CUDA, cudaGetErrorString(e));
  return MPAX_OK;
}

mpax_status mpax_qp_adjoint(mpax_problem* prob, const double* g, double* dc, double* db,
                            double* dD, double tol, int32_t max_iter, mpax_mem_kind kind,
                            double* info) {
  if (!prob || !g || !dc || !db) return afail(MPAX_ERR_INVALID_ARGUMENT, "NULL argument");
  ProblemData& P = *problem_data(prob);
  if (!P.is_qp) return afail(MPAX_ERR_INVALID_ARGUMENT, "mpax_qp_adjoint needs a QP");
  if (!(tol > 0) || max_iter < 1) return afail(MPAX_ERR_INVALID_ARGUMENT, "tol > 0, max_iter >= 1");
  const int n = P.n, m = P.m, N = n + m;
  cudaStream_t s = P.s;
  DBuf B;
  cudaError_t e = cudaSuccess;
  double* x = B.get<double>(n, &e);
  double* y = B.get<double>(m, &e);
  double* lam = B.get<double>(n, &e);
  double* tmpn = B.get<double>(n, &e);
  double* tmpr = B.get<double>(P.r, &e);
  double* gd = B.get<double>(n, &e);
  unsigned char* freem = B.get<unsigned char>(n, &e);
  unsigned char* rowm = B.get<unsigned char>(m, &e);
  double* vb[8];
  for (int q = 0; q < 8; ++q) vb[q] = B.get<double>(N, &e);
  double* Fts = B.get<double>(P.f_nnz, &e);  // scaled F^T values (transpose order)
  double* As_t = B.get<double>(P.nnz, &e);   // scaled A^T values
  double* part = B.get<double>(kRedBlocks, &e);
  double* one = B.get<double>(1, &e);
  if (e) return afail(MPAX_ERR_OUT_OF_MEMORY, "adjoint buffers");
  mpax_status st = mpax_get_solution(prob, x, y, MPAX_MEM_DEVICE);
  if (st) return st;
  const cudaMemcpyKind kin = kind == MPAX_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  if ((e = cudaMemcpyAsync(gd, g, sizeof(double) * n, kin, s))) return afail(MPAX_ERR_CUDA, cudaGetErrorString(e));
  // active sets from the returned point
  if ((e = lambda_unscaled(P, x, y, lam, tmpn, tmpr, s))) return afail(MPAX_ERR_CUDA, cudaGetErrorString(e));
  double cinf = 0.0;
  {
    std::vector<double> hc(n);
    cudaMemcpyAsync(hc.data(), P.c, sizeof(double) * n, cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    for (double v : hc) cinf = std::max(cinf, std::fabs(v));
  }
  k_active<<<g1(n), 256, 0, s>>>(x, lam, P.l, P.u, 1e-7, 1e-7 * (1.0 + cinf), n, freem);
  k_rows_active<<<g1(m), 256, 0, s>>>(P.lc, P.uc, y, m, rowm);
  // scaled transposed values (FP64) for the masked products
  gather_cast<double>(P.val_s, P.permT, As_t, P.nnz, s);
  gather_cast<double>(P.fval_s, P.permF, Fts, P.f_nnz, s);
  // MINRES on K z = b, z = [w~; v~]
  double *xz = vb[0], *r1 = vb[1], *r2 = vb[2], *yv = vb[3], *v = vb[4], *w = vb[5], *w1 = vb[6],
         *w2 = vb[7];
  auto matvec = [&](const double* in, double* out) {
    // top: mask_F (Ds in_top + F~ (F~^T in_top) + A~^T in_bot)
    k_rows<<<wgrid(P.r), 256, 0, s>>>(P.Ft.rp, P.Ft.col, Fts, nullptr, P.r, in, nullptr,
                                       nullptr, nullptr, tmpr, 0);
    k_rows<<<wgrid(n), 256, 0, s>>>(P.F.rp, P.F.col, P.fval_s, nullptr, n, tmpr, P.D_s, in,
                                     nullptr, out, 0);
    if (P.q_general)
      k_rows<<<wgrid(n), 256, 0, s>>>(P.Q.rp, P.Q.col, P.qval_s, nullptr, n, in, nullptr,
                                       nullptr, nullptr, out, 1);
    k_rows<<<wgrid(n), 256, 0, s>>>(P.At.rp, P.At.col, As_t, nullptr, n, in + n, nullptr,
                                     nullptr, freem, out, 1);
    // bottom: mask_R A~ in_top
    k_rows<<<wgrid(m), 256, 0, s>>>(P.A.rp, P.A.col, P.val_s, nullptr, m, in, nullptr, nullptr,
                                     rowm, out + n, 0);
  };
  k_rhs<<<g1(N), 256, 0, s>>>(gd, P.Dc, freem, n, m, r1);
  cudaMemsetAsync(xz, 0, sizeof(double) * N, s);
  cudaMemsetAsync(w, 0, sizeof(double) * N, s);
  cudaMemsetAsync(w2, 0, sizeof(double) * N, s);
  cudaMemcpyAsync(r2, r1, sizeof(double) * N, cudaMemcpyDeviceToDevice, s);
  cudaMemcpyAsync(yv, r1, sizeof(double) * N, cudaMemcpyDeviceToDevice, s);
  double beta1 = std::sqrt(dot(r1, r1, N, part, one, s));
  int itn = 0;
  double phibar = beta1;
  if (beta1 > 0.0) {
    double oldb = 0.0, beta = beta1, dbar = 0.0, epsln = 0.0, cs = -1.0, sn = 0.0;
    for (itn = 1; itn <= max_iter; ++itn) {
      k_axpby<<<g1(N), 256, 0, s>>>(v, yv, 1.0 / beta, nullptr, 0.0, N);
      matvec(v, yv);
      if (itn >= 2) k_axpby<<<g1(N), 256, 0, s>>>(yv, yv, 1.0, r1, -beta / oldb, N);
      const double alfa = dot(v, yv, N, part, one, s);
      k_axpby<<<g1(N), 256, 0, s>>>(yv, yv, 1.0, r2, -alfa / beta, N);
      std::swap(r1, r2);  // r1 <- r2
      cudaMemcpyAsync(r2, yv, sizeof(double) * N, cudaMemcpyDeviceToDevice, s);
      oldb = beta;
      beta = std::sqrt(dot(r2, yv, N, part, one, s));
      const double oldeps = epsln;
      const double delta = cs * dbar + sn * alfa;
      const double gbar = sn * dbar - cs * alfa;
      epsln = sn * beta;
      dbar = -cs * beta;
      double gamma = std::sqrt(gbar * gbar + beta * beta);
      gamma = std::max(gamma, 1e-300);
      cs = gbar / gamma;
      sn = beta / gamma;
      const double phi = cs * phibar;
      phibar = sn * phibar;
      // w1 <- w2, w2 <- w, w <- (v - oldeps w1 - delta w2) / gamma, x += phi w
      double* t = w1;
      w1 = w2;
      w2 = w;
      w = t;
      k_minres_w<<<g1(N), 256, 0, s>>>(v, w1, w2, oldeps, delta, 1.0 / gamma, w, xz, phi, N);
      if (phibar <= tol * beta1 || beta == 0.0) break;
    }
  }
  if ((e = cudaGetLastError())) return afail(MPAX_ERR_CUDA, cudaGetErrorString(e));
  double* odc = tmpn;
  double* odb = lam;  // reuse (m <= n not assumed: allocate when needed)
  DBuf B2;
  if (m > n) odb = B2.get<double>(m, &e);
  double* odD = dD ? gd : nullptr;
  k_adj_out<<<g1(N), 256, 0, s>>>(xz, P.Dc, P.Dr, x, freem, rowm, n, m, odc, odb, odD);
  const cudaMemcpyKind k = kind == MPAX_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  e = cudaMemcpyAsync(dc, odc, sizeof(double) * n, k, s);
  if (!e && m) e = cudaMemcpyAsync(db, odb, sizeof(double) * m, k, s);
  if (!e && dD) e = cudaMemcpyAsync(dD, odD, sizeof(double) * n, k, s);
  if (!e) e = cudaStreamSynchronize(s);
  if (e) return afail(MPAX_ERR_CUDA, cudaGetErrorString(e));
  if (info) {
    info[0] = (double)itn;
    info[1] = beta1 > 0 ? phibar / beta1 : 0.0;
  }
  return MPAX_OK;
}

}  // extern "C"
