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
#include "epilogues.cuh"
#include "kernels.cuh"
#include "problem.cuh"
#include "spmv_launch.cuh"

namespace mpax {
ProblemData* problem_data(mpax_problem* p);
cudaStream_t problem_stream(mpax_problem* p);
}  // namespace mpax

namespace {

using namespace mpax;

int g1(long long k) { return (int)std::max(1LL, std::min(4096LL, (k + 255) / 256)); }
// MINRES: steps per captured graph (the period of the buffer rotations) and
// graphs launched between two reads of the state by the host
constexpr int kMinresGraphSteps = 3;
constexpr int kMinresGraphsPerCheck = 8;
int wgrid(long long rows) { return (int)std::max(1LL, std::min(152LL * 8, (rows * 32 + 255) / 256)); }

// out_r = mask_r * (sum_p val[p] x[col[p]] + d_r x_r)   (d, mask nullable)
// (skip nullable: a device flag that, when set, turns the launch into a no-op)
__global__ void k_rows(const int* __restrict__ rp, const int* __restrict__ col,
                       const double* __restrict__ val, const int* __restrict__ perm, int rows,
                       const double* __restrict__ x, const double* __restrict__ d,
                       const double* __restrict__ xd, const unsigned char* __restrict__ mask,
                       double* __restrict__ out, int accumulate, const int* skip = nullptr) {
  if (skip && *skip) return;
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

// ---- MINRES with its scalars resident on the device --------------------------
// One MINRES step (Paige-Saunders, no preconditioner) on the masked KKT matrix
//   K = [[mask_F (D~ + F~ F~^T + Q~) mask_F, mask_F A~^T mask_R], [mask_R A~ mask_F, 0]]
// runs on the solver's row schedules of A, A^T, F, F^T and Q (the fused SpMV
// kernels of kernels.cuh, FP64), none of the launches returning a scalar to the
// host:
//   u = F~^T v_top            (schedule of F^T; low-rank Q only)
//   aux = F~ u, or Q~ v_top   (schedule of F, or of Q for a general Q)
//   y_top = mask_F (A~^T v_bot + aux + D~ v_top)   (schedule of A^T)
//   y_bot = mask_R A~ v_top                          (schedule of A, forked branch)
//     both fused with the first Lanczos update y -= (beta / beta_old) r1 (from the
//     second step on) and per-item partials of v.y
//   k_mr_alpha  alpha = v.y from the partials of both products, in a fixed order
//   k_mr_b      y -= (alpha / beta) r2; the last block to finish sums the
//               partials of y.y, takes beta' = sqrt(y.y) and the Givens
//               recurrences, and sets `done` when phibar <= tol beta1, beta' = 0
//               or the step limit is reached
//   k_mr_c      w' = (v - eps_old w1 - delta w2) / gamma;  x += phi w';  v = y / beta'
// after which r1 <- r2, r2 <- y, w1 <- w2, w2 <- w' rotate buffers on the host.
// The steps are captured as one CUDA graph and the host reads the state only
// every few dozen steps; a step launched after convergence finds `done` set and
// does nothing.  "Last block" is an arrival counter (atomicAdd after a fence, no
// waiting); every sum runs in a fixed order, so results do not depend on the
// number of steps between host checks.
struct MinresState {
  double beta1, tol;
  double beta, oldb, dbar, epsln, cs, sn, phibar, alfa;
  double oldeps, delta, inv_gamma, phi;  // the w update of the latest step
  int itn, max_iter, done, w_applied;    // w_applied == itn: no w update pending
};

// Arrival at the end of a kernel: true in the whole of the block that arrives last.
// The counter is reset for the next launch by that block.
__device__ __forceinline__ bool arrive_last(unsigned* cnt, bool* flag) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    *flag = atomicAdd(cnt, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (*flag) __threadfence();
  return *flag;
}

// Fixed-order sum of count partials written by other blocks or launches (read
// through L2); the total in thread 0.
__device__ __forceinline__ double sum_parts(const double* part, int count, double* sh) {
  double s = 0.0;
  for (int i = threadIdx.x; i < count; i += blockDim.x) s += __ldcg(part + i);
  return block_sum(s, sh);
}

// Row epilogues of the MINRES products (the interface of epilogues.cuh).
// out_r = s: u = F~^T v_top and aux = F~ u (or Q~ v_top).
struct EpiMrStore {
  static constexpr int NQ = 1;  // no partials: check stays 0
  struct Pre {};
  const MinresState* st;
  double* out;
  int check = 0;
  __device__ __forceinline__ bool skip() const { return st->done != 0; }
  __device__ __forceinline__ void load() {}
  __device__ __forceinline__ void pre(int, Pre&) const {}
  __device__ __forceinline__ void row(int r, double s, const Pre&, double*) { out[r] = s; }
};

// One block row of y = K v (top: rows of A^T, bottom: rows of A), then
// y -= (beta / beta_old) r1 and the partial [0] v.y.
struct EpiMrRow {
  static constexpr int NQ = 1;
  struct Pre {
    double v, r1, aux, d;
    unsigned char keep;
  };
  MinresState* st;
  const double* v;   // the stacked vector, offset to this block's rows
  double* y;         // likewise
  const double* r1;  // likewise
  const double* aux;  // nullable (top only): F~ u or Q~ v_top
  const double* ds;   // nullable (top only): D~
  const unsigned char* mask;
  int check = 1;
  bool sub;
  double c;
  __device__ __forceinline__ bool skip() const { return st->done != 0; }
  __device__ __forceinline__ void load() {
    sub = st->itn >= 1;
    c = sub ? -st->beta / st->oldb : 0.0;
  }
  __device__ __forceinline__ void pre(int r, Pre& p) const {
    p.v = v[r];
    p.r1 = sub ? r1[r] : 0.0;
    p.aux = aux ? aux[r] : 0.0;
    p.d = ds ? ds[r] : 0.0;
    p.keep = mask[r];
  }
  __device__ __forceinline__ void row(int r, double s, const Pre& p, double* acc) {
    double yi = p.keep ? s + p.aux + p.d * p.v : 0.0;
    if (sub) yi += c * p.r1;
    y[r] = yi;
    acc[0] += p.v * yi;
  }
};

// alpha = v.y from the per-item partials of the top product, then the bottom's:
// block b sums a contiguous share of that sequence, the last block to finish
// sums the blocks' totals in block order.
constexpr int kAlphaBlocks = 32;
__global__ void k_mr_alpha(MinresState* __restrict__ st, const double* __restrict__ pt, int nt,
                           const double* __restrict__ pb, int nb, double* __restrict__ apart,
                           unsigned* __restrict__ cnt) {
  __shared__ double sh[32];
  __shared__ bool last;
  if (blockIdx.x == 0 && threadIdx.x == 0) st->w_applied = st->itn;  // no w update pending
  if (st->done) return;
  const long long total = (long long)nt + nb;
  const int lo = (int)(total * blockIdx.x / gridDim.x);
  const int hi = (int)(total * (blockIdx.x + 1) / gridDim.x);
  double t = 0.0;
  for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) t += __ldcg(i < nt ? pt + i : pb + (i - nt));
  t = block_sum(t, sh);
  if (threadIdx.x == 0) apart[blockIdx.x] = t;
  if (!arrive_last(cnt, &last)) return;
  const double a = sum_parts(apart, gridDim.x, sh);
  if (threadIdx.x == 0) {
    st->alfa = a;
    *cnt = 0;
  }
}

__global__ void k_mr_b(MinresState* __restrict__ st, double* __restrict__ y,
                       const double* __restrict__ r2, int n, double* __restrict__ part,
                       unsigned* __restrict__ cnt) {
  __shared__ double sh[32];
  __shared__ bool last;
  if (st->done) return;
  const double c = -st->alfa / st->beta;
  double s = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double yi = y[i] + c * r2[i];
    y[i] = yi;
    s += yi * yi;
  }
  s = block_sum(s, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
  if (!arrive_last(cnt, &last)) return;
  const double bsq = sum_parts(part, gridDim.x, sh);
  if (threadIdx.x != 0) return;
  *cnt = 0;
  const double alfa = st->alfa;
  const double beta = sqrt(bsq);
  const double cs = st->cs, sn = st->sn, dbar = st->dbar;
  st->oldeps = st->epsln;
  st->delta = cs * dbar + sn * alfa;
  const double gbar = sn * dbar - cs * alfa;
  st->epsln = sn * beta;
  st->dbar = -cs * beta;
  const double gamma = fmax(sqrt(gbar * gbar + beta * beta), 1e-300);
  st->cs = gbar / gamma;
  st->sn = beta / gamma;
  st->inv_gamma = 1.0 / gamma;
  st->phi = st->cs * st->phibar;
  st->phibar = st->sn * st->phibar;
  st->oldb = st->beta;
  st->beta = beta;
  st->itn += 1;
  if (st->phibar <= st->tol * st->beta1 || beta == 0.0 || st->itn >= st->max_iter) st->done = 1;
}

__global__ void k_mr_c(const MinresState* __restrict__ st, double* __restrict__ v,
                       const double* __restrict__ w1, const double* __restrict__ w2,
                       double* __restrict__ w, double* __restrict__ x,
                       const double* __restrict__ y, int n) {
  if (st->w_applied == st->itn) return;  // no step ran since the last update
  const double oldeps = st->oldeps, delta = st->delta, ig = st->inv_gamma, phi = st->phi;
  const bool next = !st->done;
  const double ib = next ? 1.0 / st->beta : 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double wn = (v[i] - oldeps * w1[i] - delta * w2[i]) * ig;
    w[i] = wn;
    x[i] += phi * wn;
    if (next) v[i] = ib * y[i];
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
  double* part_b = B.get<double>(kRedBlocks, &e);
  double* u = B.get<double>(std::max(P.r, 1), &e);
  unsigned* cnt = B.get<unsigned>(2, &e);
  double* one = B.get<double>(1, &e);
  MinresState* mst = B.get<MinresState>(1, &e);
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
  k_rhs<<<g1(N), 256, 0, s>>>(gd, P.Dc, freem, n, m, r1);
  cudaMemsetAsync(xz, 0, sizeof(double) * N, s);
  cudaMemsetAsync(w, 0, sizeof(double) * N, s);
  cudaMemsetAsync(w2, 0, sizeof(double) * N, s);
  cudaMemcpyAsync(r2, r1, sizeof(double) * N, cudaMemcpyDeviceToDevice, s);
  cudaMemsetAsync(cnt, 0, sizeof(unsigned) * 2, s);
  const double beta1 = std::sqrt(dot(r1, r1, N, part, one, s));
  MinresState hs{};
  hs.beta1 = beta1;
  hs.tol = tol;
  hs.beta = beta1;
  hs.cs = -1.0;
  hs.phibar = beta1;
  hs.max_iter = max_iter;
  hs.done = beta1 > 0.0 ? 0 : 1;
  if ((e = cudaMemcpyAsync(mst, &hs, sizeof(hs), cudaMemcpyHostToDevice, s)))
    return afail(MPAX_ERR_CUDA, cudaGetErrorString(e));
  if (beta1 > 0.0) {
    k_axpby<<<g1(N), 256, 0, s>>>(v, r2, 1.0 / beta1, nullptr, 0.0, N);
    cudaStream_t s2 = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    e = cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking);
    if (!e) e = cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming);
    if (!e) e = cudaEventCreateWithFlags(&ev_join, cudaEventDisableTiming);
    struct Release {
      cudaStream_t& s2;
      cudaEvent_t &a, &b;
      ~Release() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
        if (s2) cudaStreamDestroy(s2);
      }
    } release{s2, ev_fork, ev_join};
    if (e) return afail(MPAX_ERR_CUDA, cudaGetErrorString(e));
    const bool lowrank = !P.q_general && P.r > 0 && P.f_nnz > 0;
    // the products run in FP64 with the wide register budget whatever kernel the
    // solver's precision was tuned to
    auto wide = [](const Sched& sc) {
      Sched w = sc;
      w.kind = kSpmvItemWide;
      return w;
    };
    const Sched sA = wide(P.schedA), sAt = wide(P.schedAt), sF = wide(P.schedF),
                sFt = wide(P.schedFt), sQ = wide(P.schedQ);
    auto step = [&]() {
      const double* aux = nullptr;
      if (lowrank) {
        launch_spmv<double>(sFt, P.Ft, Fts, InPlain<double>{v}, EpiMrStore{mst, u}, 0, s);
        launch_spmv<double>(sF, P.F, P.fval_s, InPlain<double>{u}, EpiMrStore{mst, tmpn}, 0, s);
        aux = tmpn;
      } else if (P.q_general) {
        launch_spmv<double>(sQ, P.Q, P.qval_s, InPlain<double>{v}, EpiMrStore{mst, tmpn}, 0, s);
        aux = tmpn;
      }
      // the bottom block on a forked branch: it reads only v
      cudaEventRecord(ev_fork, s);
      cudaStreamWaitEvent(s2, ev_fork, 0);
      EpiMrRow eb{mst, v + n, yv + n, r1 + n, nullptr, nullptr, rowm};
      launch_spmv<double>(sA, P.A, P.val_s, InPlain<double>{v}, eb, 0, s2);
      cudaEventRecord(ev_join, s2);
      EpiMrRow et{mst, v, yv, r1, aux, P.D_s, freem};
      launch_spmv<double>(sAt, P.At, As_t, InPlain<double>{v + n}, et, 0, s);
      cudaStreamWaitEvent(s, ev_join, 0);
      k_mr_alpha<<<kAlphaBlocks, 256, 0, s>>>(mst, sAt.part, sAt.n_items, sA.part, sA.n_items,
                                              part, cnt);
      k_mr_b<<<kRedBlocks, 256, 0, s>>>(mst, yv, r2, N, part_b, cnt + 1);
      double* t = w1;  // w1 <- w2, w2 <- w, w <- (the free buffer)
      w1 = w2;
      w2 = w;
      w = t;
      k_mr_c<<<g1(N), 256, 0, s>>>(mst, v, w1, w2, w, xz, yv, N);
      t = r1;  // r1 <- r2, r2 <- y, y <- (the free buffer)
      r1 = r2;
      r2 = yv;
      yv = t;
    };
    // Both rotations have period 3: a graph of three steps leaves every pointer
    // where it found it, so one captured graph serves every launch.
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    if ((e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal)))
      return afail(MPAX_ERR_CUDA, cudaGetErrorString(e));
    for (int k = 0; k < kMinresGraphSteps; ++k) step();
    e = cudaStreamEndCapture(s, &g);
    if (!e) e = cudaGraphInstantiate(&ge, g, 0);
    if (g) cudaGraphDestroy(g);
    for (long long launched = 0; !e && launched < max_iter;) {
      for (int k = 0; k < kMinresGraphsPerCheck && !e && launched < max_iter; ++k) {
        e = cudaGraphLaunch(ge, s);
        launched += kMinresGraphSteps;
      }
      if (!e) e = cudaMemcpyAsync(&hs, mst, sizeof(hs), cudaMemcpyDeviceToHost, s);
      if (!e) e = cudaStreamSynchronize(s);
      if (!e && hs.done) break;
    }
    if (ge) cudaGraphExecDestroy(ge);
    if (e) return afail(MPAX_ERR_CUDA, cudaGetErrorString(e));
  }
  const int itn = hs.itn;
  const double phibar = hs.phibar;
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
