// Restarted PDHG iteration on the device: r^2HPDHG (Algorithm 1) for LP and
// rAPDHG (Algorithm 2) for QP, in FP64 or mixed precision.
//
// A check block of `check_every` iterations is a fixed launch sequence
//   [F~^T x_md (QP)], primal fused SpMV^T, dual fused SpMV     (per iteration)
//   [F~^T xavg (QP)], KKT SpMV, KKT SpMV^T, finalize, restart (per check)
// captured once as a CUDA graph and replayed.  The finalize kernel (one CTA)
// reduces the FP64 partials in a fixed order, evaluates the relative KKT test,
// the restart rule and the primal-weight update, and refreshes the device
// state; a host thread only reads a mapped status word one block behind.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <map>
#include <mutex>
#include <vector>

#include <type_traits>

#include "engine.cuh"
#include "epilogues.cuh"
#include "kernels.cuh"
#include "spmv_launch.cuh"
#include "unrolled.cuh"

namespace mpax {

namespace {

int grid1(long long k) { return (int)std::max(1LL, std::min(4096LL, (k + 255) / 256)); }

// ---------------------------------------------------------------------------
// small kernels
// ---------------------------------------------------------------------------

template <typename T>
__global__ void k_fill(T* v, int n, T val) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    v[i] = val;
}

template <typename T>
__global__ void k_copy(T* __restrict__ d, const T* __restrict__ s, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    d[i] = s[i];
}

// dst = src / D (src nullable: zeros), cast to T
template <typename T>
__global__ void k_div_in(const double* __restrict__ src, const double* __restrict__ D,
                         T* __restrict__ dst, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    dst[i] = src ? (T)(src[i] / D[i]) : (T)0;
}

template <typename T>
__global__ void k_to_double(const T* __restrict__ v, const double* __restrict__ D,
                            double* __restrict__ out, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    out[i] = D ? D[i] * (double)v[i] : (double)v[i];
}

template <typename T>
__global__ void k_from_double(const double* __restrict__ v, T* __restrict__ out, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    out[i] = (T)v[i];
}

// x^{n,k} rebuilt from (w, anchor) with coefficient slot idx (see EpiPrimalLP)
template <typename T>
__global__ void k_materialize_lp(T* __restrict__ out, const T* __restrict__ w,
                                 const T* __restrict__ xa, const DevState* st, int idx, int n) {
  const T b = (T)st->coef_b[idx];
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
    out[j] = (b == (T)1) ? xa[j] : w[j] + b * (xa[j] - w[j]);
}

// Halpern (LP) or averaging (QP) coefficients for a block starting at k_base.
__device__ void fill_table(DevState* st, int len) {
  const long long kb = st->k_base;
  for (int i = threadIdx.x; i <= len + 1 && i < kMaxCheckEvery + 2; i += blockDim.x) {
    if (st->is_qp) {
      const double k = (double)(kb + i);
      st->coef_a[i] = 2.0 / (k + 2.0);
      st->coef_b[i] = 0.0;
    } else {
      const double kp = (double)(kb - 1 + i);
      st->coef_a[i] = (kp + 1.0) / (kp + 2.0);
      st->coef_b[i] = 1.0 / (kp + 2.0);
    }
  }
}

// Unrolled differentiation, backward: open the previous tape record
// (tape_cursor - 1): its step sizes and averaging table, iteration on.
__global__ void k_tape_open(DevState* st, char* const* tab) {
  __shared__ int len;
  if (threadIdx.x == 0) {
    const long long slot = --st->tape_cursor;
    const TapeHead* h = reinterpret_cast<const TapeHead*>(tab[slot]);
    st->tau = h->tau;
    st->sigma = h->sigma;
    st->inv_sigma = 1.0 / h->sigma;
    st->k_base = h->k_base;
    st->done = 0;
    len = h->len;
  }
  __syncthreads();
  fill_table(st, len);
}

__global__ void k_set_cursor(DevState* st, long long v) { st->tape_cursor = v; }

__global__ void k_set_table(DevState* st, long long k_base, int len) {
  if (threadIdx.x == 0) st->k_base = k_base;
  __syncthreads();
  fill_table(st, len);
}

__global__ void k_set_steps(DevState* st, double tau, double sigma, double gamma) {
  st->tau = tau;
  st->sigma = sigma;
  st->inv_sigma = 1.0 / sigma;
  st->gamma = gamma;
  st->done = 0;
}

__device__ void set_step_sizes(DevState* st) {
  if (st->is_qp) {
    const double sigma = st->eta * st->omega;
    const double denom = st->norm_Q + sigma * st->norm_A * st->norm_A;
    st->sigma = sigma;
    st->tau = denom > 0.0 ? st->step_safety / denom : 1.0;
  } else {
    st->tau = st->eta / st->omega;
    st->sigma = st->eta * st->omega;
  }
  st->inv_sigma = 1.0 / st->sigma;
}

struct InitParams {
  double eps_abs, eps_rel, r_suff, r_nec, r_art, pw_smooth, step_safety, gamma;
  double eps_pi, eps_di;
  long long iter_limit;
  int check_every, is_qp, stall_limit, feas_mode;
};

// red: [0] ||c~||, [1] ||b~||, [2] ||c||, [3] ||b||  (norm_A, norm_Q already in st)
__global__ void k_init_state(DevState* st, InitParams p, const double* red) {
  if (threadIdx.x == 0) {
    st->eps_abs = p.eps_abs;
    st->eps_rel = p.eps_rel;
    st->r_suff = p.r_suff;
    st->r_nec = p.r_nec;
    st->r_art = p.r_art;
    st->pw_smooth = p.pw_smooth;
    st->step_safety = p.step_safety;
    st->gamma = p.gamma;
    st->iter_limit = p.iter_limit;
    st->check_every = p.check_every;
    st->is_qp = p.is_qp;
    const double nc = red[0], nb = red[1];
    // a polishing run has a zero objective (mode 1) or zero bounds (mode 2): the
    // initial primal weight is then 1, as the zero norm gives
    st->omega = (nc > 1e-10 && nb > 1e-10 && p.feas_mode == 0) ? nc / nb : 1.0;
    st->feas_mode = p.feas_mode;
    st->c_norm = red[2];
    st->b_norm = red[3];
    st->eta = st->norm_A > 0.0 ? p.step_safety / st->norm_A : 1.0;
    set_step_sizes(st);
    st->total = 0;
    st->k_base = 0;
    st->restarts = 0;
    st->checks = 0;
    st->done = 0;
    st->restart_flag = 0;
    st->termination = 0;
    st->have_anchor = 0;
    st->r_anchor = 0.0;
    st->r_prev = 0.0;
    st->rel_kkt = INFINITY;
    st->best_rel = INFINITY;
    st->stall_count = 0;
    st->stall_limit = p.stall_limit;
    st->eps_pi = p.eps_pi;
    st->eps_di = p.eps_di;
  }
  __syncthreads();
  fill_table(st, p.check_every);
}

// Candidate rays of an LP check (scaled space): rx = x^ - x_anchor, and
// ry = y^ - y_anchor projected onto the recession cone of Y (ry_i >= 0 where
// uc_i = +inf, ry_i <= 0 where lc_i = -inf).
template <typename T>
__global__ void k_ray_prep(const T* __restrict__ xhat, const T* __restrict__ xa, int n,
                           const T* __restrict__ yhat, const T* __restrict__ ya,
                           const double* __restrict__ lc, const double* __restrict__ uc, int m,
                           const int* skip, T* __restrict__ rx, T* __restrict__ ry) {
  if (skip && *skip) return;
  const int stride = gridDim.x * blockDim.x;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) rx[j] = xhat[j] - xa[j];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
    T d = yhat[i] - ya[i];
    if (!isfinite(uc[i]) && d < (T)0) d = (T)0;
    if (!isfinite(lc[i]) && d > (T)0) d = (T)0;
    ry[i] = d;
  }
}

__global__ void k_power_start(DevState* st) {
  st->pw_scale = 1.0;
  st->pw_nu = 0.0;
  st->pw_d = 0.0;
  st->pw_done = 0;
  st->pw_iters = 0;
}

// One power-iteration round done: sum of squares of g in part[0..n).
// mode 0 (A~^T A~): nu = sqrt(||g||); mode 1 (Q~): nu = ||g||.  v_next = g/||g||
// through pw_scale.  Writes the estimate to norm_A or norm_Q.
// Every finite bound of the pair (lo, hi) set to zero (the dual polishing problem).
template <typename T>
__global__ void k_zero_finite(T* __restrict__ lo, T* __restrict__ hi, int k) {
  const int stride = gridDim.x * blockDim.x;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += stride) {
    if (isfinite(lo[i])) lo[i] = (T)0;
    if (isfinite(hi[i])) hi[i] = (T)0;
  }
}

// ||A~||_2 := 1, the bound of the Pock-Chambolle round (power_max_iter = 0).
__global__ void k_power_bound(DevState* st, int mode) {
  st->pw_nu = 1.0;
  st->pw_done = 1;
  st->pw_iters = 0;
  if (mode == 0) st->norm_A = 1.0;
}

// The normalised start vector of the power iterations (power_start_raw).
template <typename T>
__global__ void k_power_vec(T* __restrict__ v, int n, double inv_norm) {
  const int stride = gridDim.x * blockDim.x;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride)
    v[j] = (T)(power_start_raw(j) * inv_norm);
}

// ||raw start vector||_2 for n entries (host, once per size).
double power_start_norm(int n) {
  thread_local int cached_n = -1;
  thread_local double cached = 1.0;
  if (n != cached_n) {
    double s = 0.0;
    for (int j = 0; j < n; ++j) {
      const double r = power_start_raw(j);
      s += r * r;
    }
    cached = s > 0.0 ? std::sqrt(s) : 1.0;
    cached_n = n;
  }
  return cached;
}

__global__ void k_power_finalize(const double* __restrict__ part, int n, DevState* st, int t,
                                 double tol, int mode, double cap, int max_iter) {
  __shared__ double sh[32];
  if (st->pw_done) return;
  double v = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) v += part[i];
  v = block_sum(v, sh);
  if (threadIdx.x == 0) {
    const double nrm = sqrt(v);
    if (nrm == 0.0) {
      st->pw_nu = 0.0;
      st->pw_done = 1;
    } else {
      const double nu = (mode == 0) ? sqrt(nrm) : nrm;
      const double prev = st->pw_nu;
      st->pw_scale = 1.0 / nrm;
      st->pw_nu = nu;
      double est = nu;
      if (t > 1 && power_stop(nu, prev, &st->pw_d, tol, cap, &est)) {
        st->pw_nu = est;
        st->pw_done = 1;
      } else if (t >= max_iter && isfinite(cap)) {
        st->pw_nu = cap;  // out of rounds: the certified bound
      }
    }
    st->pw_iters = t;
    if (mode == 0) st->norm_A = st->pw_nu;
    else st->norm_Q = st->pw_nu;
  }
}

__device__ double sum_slot(const double* part, int q, int n, double* sh) {
  double v = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) v += part[(size_t)q * n + i];
  return block_sum(v, sh);
}

// First level of the check reductions: block b sums the fixed chunk b of every
// partial-sum slot (A^T slots 0..qt-1, then A slots 0..qa-1) into out[q][b].
constexpr int kChunks = 128;
// Check quantities reduced per check: 10 partial slots of the A^T schedule
// (0-1 restart metric, 2-5 KKT columns, 6-9 ray columns) then 6 of the A
// schedule (0-1 restart metric, 2-3 KKT rows, 4-5 ray rows).
constexpr int kCheckQt = 10, kCheckQa = 6, kCheckQ = kCheckQt + kCheckQa;
__global__ void k_part_reduce(const double* __restrict__ partAt, int nAt, int qt,
                              const double* __restrict__ partA, int nA, int qa,
                              const int* skip, double* __restrict__ out) {
  __shared__ double sh[32];
  if (skip && *skip) return;
  for (int q = 0; q < qt + qa; ++q) {
    const double* p = q < qt ? partAt + (size_t)q * nAt : partA + (size_t)(q - qt) * nA;
    const int n = q < qt ? nAt : nA;
    const int chunk = (n + kChunks - 1) / kChunks;
    const int lo = blockIdx.x * chunk, hi = min(n, lo + chunk);
    double v = 0;
    for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) v += p[i];
    v = block_sum(v, sh);
    if (threadIdx.x == 0) out[q * kChunks + blockIdx.x] = v;
  }
}

// Check of Algorithm 1 / 2 after a block of `len` iterations.
//   partAt slots: 0 sum(x^-x)^2, 1 sum(x^-x_anchor)^2 (QP: averages), 2..5 KKT column terms
//   partA  slots: 0 sum(y^-y)^2, 1 sum(y^-y_anchor)^2, 2..3 KKT row terms
__global__ void k_finalize_check(const double* __restrict__ partAt, int nAt,
                                 const double* __restrict__ partA, int nA, DevState* st,
                                 HostStatus* hs, int len, int next_len) {
  __shared__ double sh[32];
  __shared__ double vals[kCheckQ];
  if (st->done) return;
  // partAt / partA hold the kChunks first-level sums of every slot (k_part_reduce)
  for (int q = 0; q < kCheckQ; ++q) {
    const double v = sum_slot(partAt, q, kChunks, sh);
    if (threadIdx.x == 0) vals[q] = v;
  }
  (void)partA;
  (void)nA;
  (void)nAt;
  __syncthreads();
  if (threadIdx.x == 0) {
    const double P0 = vals[0], P1 = vals[1], C0 = vals[2], C1 = vals[3], C2 = vals[4],
                 C3 = vals[5], D0 = vals[10], D1 = vals[11], K0 = vals[12], K1 = vals[13];
    const double RC0 = vals[6], RC1 = vals[7], RC2 = vals[8], RC3 = vals[9], RR0 = vals[14],
                 RR1 = vals[15];
    st->total += len;
    st->checks += 1;
    const double nrp = sqrt(K0), nrd = sqrt(C0);
    const double pobj = C1 + 0.5 * C3;
    const double dobj = K1 + C2 - 0.5 * C3;
    const double gap = fabs(pobj - dobj);
    const double bn = st->b_norm, cn = st->c_norm;
    const double rel = fmax(fmax(nrp / (1.0 + bn), nrd / (1.0 + cn)),
                            gap / (1.0 + fabs(pobj) + fabs(dobj)));
    st->primal_res = nrp;
    st->dual_res = nrd;
    st->pobj = pobj;
    st->dobj = dobj;
    st->gap = gap;
    st->rel_kkt = rel;
    const double ea = st->eps_abs, er = st->eps_rel;
    const bool conv = st->feas_mode == 1   ? nrp <= ea + er * bn
                      : st->feas_mode == 2 ? nrd <= ea + er * cn
                                           : nrp <= ea + er * bn && nrd <= ea + er * cn &&
                                                 gap <= ea + er * (fabs(pobj) + fabs(dobj));
    int term = 0;
    if (!isfinite(rel) || !isfinite(P0) || !isfinite(D0) || !isfinite(P1) || !isfinite(D1))
      term = MPAX_TERM_NUMERICAL_ERROR;
    else if (conv) term = MPAX_TERM_OPTIMAL;
    else if (st->total >= st->iter_limit) term = MPAX_TERM_ITERATION_LIMIT;
    if (!term && !st->is_qp) {
      // infeasibility certificates from the cycle's move (the oracle's reading):
      // a Farkas ray with positive objective and reduced costs in their cone, or
      // a recession ray of the primal with negative cost
      const double obj = RR1 + RC1;
      if (st->eps_pi > 0.0 && obj > 0.0 && sqrt(RC0) <= st->eps_pi * obj)
        term = MPAX_TERM_PRIMAL_INFEASIBLE;
      else if (st->eps_di > 0.0 && RC2 < 0.0 && sqrt(RR0 + RC3) <= st->eps_di * (-RC2))
        term = MPAX_TERM_DUAL_INFEASIBLE;
    }
    if (!term && st->stall_limit > 0) {
      // the precision floor: no 10% improvement of the KKT error over a window of
      // max(stall_limit, checks / 4) checks.  The window grows with the solve, so a
      // slow but steady decrease (a few per cent per check) is not taken for a
      // floor, while a plateau costs at most a quarter more iterations.
      const long long window =
          st->stall_limit > st->checks / 4 ? (long long)st->stall_limit : st->checks / 4;
      if (rel < 0.9 * st->best_rel) {
        st->best_rel = rel;
        st->stall_count = 0;
      } else if (++st->stall_count >= window) {
        term = kTermStalled;
      }
    }
    st->restart_flag = 0;
    if (term) {
      st->termination = term;
      st->done = 1;
    } else {
      const double r = st->is_qp ? rel : sqrt(st->omega * P0 + D0 / st->omega);
      const long long kc = st->k_base + len;
      const bool restart = !st->have_anchor || r <= st->r_suff * st->r_anchor ||
                           (r <= st->r_nec * st->r_anchor && r > st->r_prev) ||
                           (double)kc >= st->r_art * (double)st->total;
      st->last_restart_metric = r;
      if (restart) {
        const double dx = sqrt(P1), dy = sqrt(D1);
        if (dx > 1e-10 && dy > 1e-10) {
          const double th = st->pw_smooth;
          st->omega = exp(th * log(dy / dx) + (1.0 - th) * log(st->omega));
        }
        set_step_sizes(st);
        if (st->rs_count < kRestartLog) {
          st->rs_iter[st->rs_count] = st->total;
          st->rs_omega[st->rs_count] = st->omega;
        }
        st->rs_count += 1;
        st->k_base = 0;
        st->have_anchor = 1;
        st->r_anchor = r;
        st->r_prev = r;
        st->restarts += 1;
        st->restart_flag = 1;
      } else {
        st->r_prev = r;
        st->k_base = kc;
      }
    }
    hs->total = st->total;
    hs->restarts = st->restarts;
    hs->checks = st->checks;
    hs->rel_kkt = rel;
    hs->pobj = pobj;
    hs->dobj = dobj;
    hs->primal_res = nrp;
    hs->dual_res = nrd;
    hs->gap = gap;
    hs->omega = st->omega;
    hs->termination = st->termination;
    __threadfence_system();
    hs->done = st->done;
    __threadfence_system();
  }
  __syncthreads();
  if (!st->done) fill_table(st, next_len);
}

// Restart of Algorithm 1: anchor and iterate <- (x^, y^).
template <typename T>
__global__ void k_restart_lp(const DevState* st, int n, int m, const T* __restrict__ xhat,
                             T* __restrict__ xa, T* __restrict__ xbar, T* __restrict__ wbuf,
                             const T* __restrict__ yhat, T* __restrict__ ya, T* __restrict__ y) {
  if (st->done || !st->restart_flag) return;
  const int stride = gridDim.x * blockDim.x;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
    const T v = xhat[j];
    xa[j] = v;
    xbar[j] = v;
    wbuf[j] = v;
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
    const T v = yhat[i];
    ya[i] = v;
    y[i] = v;
  }
}

// Restart of Algorithm 2: x, anchor <- xavg; y, anchor <- yavg.
template <typename T>
__global__ void k_restart_qp(const DevState* st, int n, int m, const T* __restrict__ xavg,
                             T* __restrict__ x, T* __restrict__ xanc,
                             const T* __restrict__ yavg, T* __restrict__ y,
                             T* __restrict__ yanc) {
  if (st->done || !st->restart_flag) return;
  const int stride = gridDim.x * blockDim.x;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
    const T v = xavg[j];
    x[j] = v;
    xanc[j] = v;
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
    const T v = yavg[i];
    y[i] = v;
    yanc[i] = v;
  }
}

__global__ void k_kkt_finalize(const double* __restrict__ partAt, int nAt,
                               const double* __restrict__ partA, int nA, const DevState* st,
                               double* out) {
  __shared__ double sh[32];
  __shared__ double vals[6];
  // partAt holds the chunk sums of the A^T slots 0..kCheckQt-1 then the A slots
  // (KKT columns in A^T slots 2..5, KKT rows in A slots 2..3)
  for (int q = 0; q < 4; ++q) {
    const double v = sum_slot(partAt, 2 + q, nAt, sh);
    if (threadIdx.x == 0) vals[q] = v;
  }
  for (int q = 0; q < 2; ++q) {
    const double v = sum_slot(partAt, kCheckQt + 2 + q, nAt, sh);
    if (threadIdx.x == 0) vals[4 + q] = v;
  }
  (void)partA;
  (void)nA;
  __syncthreads();
  if (threadIdx.x == 0) {
    const double nrp = sqrt(vals[4]), nrd = sqrt(vals[0]);
    const double pobj = vals[1] + 0.5 * vals[3];
    const double dobj = vals[5] + vals[2] - 0.5 * vals[3];
    const double gap = fabs(pobj - dobj);
    out[0] = nrp;
    out[1] = nrd;
    out[2] = pobj;
    out[3] = dobj;
    out[4] = gap;
    out[5] = fmax(fmax(nrp / (1.0 + st->b_norm), nrd / (1.0 + st->c_norm)),
                  gap / (1.0 + fabs(pobj) + fabs(dobj)));
  }
}

// ---- autotuner helpers ------------------------------------------------------
// Signature of a schedule's matrix: sizes, precision and the log2 histogram of
// row lengths (bin b counts rows of length in [2^(b-1), 2^b), bin 0 empty rows).
constexpr int kTuneBins = 32;
constexpr int kTuneReps = 10;
struct TuneKey {
  long long v[5 + kTuneBins];
  bool operator<(const TuneKey& o) const {
    return std::lexicographical_compare(v, v + 5 + kTuneBins, o.v, o.v + 5 + kTuneBins);
  }
};

__global__ void k_row_hist(const int* __restrict__ rp, int rows, int* __restrict__ hist) {
  __shared__ int h[kTuneBins];
  if (threadIdx.x < kTuneBins) h[threadIdx.x] = 0;
  __syncthreads();
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < rows; i += gridDim.x * blockDim.x) {
    const int len = rp[i + 1] - rp[i];
    atomicAdd(&h[len == 0 ? 0 : 32 - __clz(len)], 1);  // integer counts: order-free
  }
  __syncthreads();
  if (threadIdx.x < kTuneBins && h[threadIdx.x]) atomicAdd(hist + threadIdx.x, h[threadIdx.x]);
}

cudaError_t tune_key(const Csr& K, int n_items, size_t tsize, int* scratch, cudaStream_t s,
                     TuneKey* key) {
  int h[kTuneBins];
  cudaError_t e = cudaMemsetAsync(scratch, 0, sizeof(h), s);
  if (e) return e;
  if (K.rows > 0) k_row_hist<<<grid1(K.rows), 256, 0, s>>>(K.rp, K.rows, scratch);
  if ((e = cudaMemcpyAsync(h, scratch, sizeof(h), cudaMemcpyDeviceToHost, s))) return e;
  if ((e = cudaStreamSynchronize(s))) return e;
  key->v[0] = K.rows;
  key->v[1] = K.cols;
  key->v[2] = K.nnz;
  key->v[3] = n_items;
  key->v[4] = (long long)tsize;
  for (int b = 0; b < kTuneBins; ++b) key->v[5 + b] = h[b];
  return cudaSuccess;
}

std::mutex& tune_mutex() {
  static std::mutex m;
  return m;
}
std::map<TuneKey, int>& tune_cache() {
  static std::map<TuneKey, int> c;
  return c;
}
bool tune_lookup(const TuneKey& k, int* kind) {
  std::lock_guard<std::mutex> g(tune_mutex());
  auto it = tune_cache().find(k);
  if (it == tune_cache().end()) return false;
  *kind = it->second;
  return true;
}
void tune_store(const TuneKey& k, int kind) {
  std::lock_guard<std::mutex> g(tune_mutex());
  tune_cache()[k] = kind;
}

// Average microseconds of `reps` launches of f (after one untimed launch),
// CUDA events on the stream the launches use.
template <class F>
cudaError_t time_launches(cudaStream_t s, int reps, double* us, F f) {
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e) return e;
  if ((e = cudaEventCreate(&e1))) {
    cudaEventDestroy(e0);
    return e;
  }
  f();
  cudaEventRecord(e0, s);
  for (int r = 0; r < reps; ++r) f();
  cudaEventRecord(e1, s);
  e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (!e) e = cudaEventElapsedTime(&ms, e0, e1);
  if (!e) e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *us = 1000.0 * ms / reps;
  return e;
}

template <typename T>
T* dalloc(size_t n, cudaError_t* e) {
  T* p = nullptr;
  if (*e == cudaSuccess) *e = cudaMalloc(&p, sizeof(T) * std::max<size_t>(n, 1));
  return p;
}

}  // namespace

// ---------------------------------------------------------------------------
// Engine
// ---------------------------------------------------------------------------

template <typename T>
class Engine final : public EngineBase {
 public:
  Engine(ProblemData* P, cudaError_t* e) : P_(P) {
    const int m = P->m, n = P->n;
    valA_ = dalloc<T>((size_t)P->nnz + kPad, e);
    valAt_ = dalloc<T>((size_t)P->nnz + kPad, e);
    c_ = dalloc<T>(n, e);
    l_ = dalloc<T>(n, e);
    u_ = dalloc<T>(n, e);
    lc_ = dalloc<T>(m, e);
    uc_ = dalloc<T>(m, e);
    xbar_ = dalloc<T>(n, e);
    wbuf_ = dalloc<T>(n, e);
    xa_ = dalloc<T>(n, e);
    xhat_ = dalloc<T>(n, e);
    xprev_ = dalloc<T>(n, e);
    rayx_ = dalloc<T>(n, e);
    rayy_ = dalloc<T>(m, e);
    pv_ = dalloc<T>(n, e);
    pg_ = dalloc<T>(n, e);
    y_ = dalloc<T>(m, e);
    ya_ = dalloc<T>(m, e);
    yhat_ = dalloc<T>(m, e);
    yprev_ = dalloc<T>(m, e);
    pw_ = dalloc<T>(m, e);
    if (P->is_qp) {
      x_ = dalloc<T>(n, e);
      xavg_ = dalloc<T>(n, e);
      xref_ = dalloc<T>(n, e);
      xanc_ = dalloc<T>(n, e);
      yavg_ = dalloc<T>(m, e);
      yanc_ = dalloc<T>(m, e);
      Ds_ = dalloc<T>(n, e);
      fval_ = dalloc<T>((size_t)P->f_nnz + kPad, e);
      ftval_ = dalloc<T>((size_t)P->f_nnz + kPad, e);
      uvec_ = dalloc<T>(P->r, e);
      uvec2_ = dalloc<T>(P->r, e);
      if (P->q_general) {
        qv_ = dalloc<T>((size_t)P->Q.nnz + kPad, e);
        qvec_ = dalloc<T>(n, e);
        qvec2_ = dalloc<T>(n, e);
      }
    }
    st_ = dalloc<DevState>(1, e);
    if (*e == cudaSuccess) *e = cudaHostAlloc(&hs_, sizeof(HostStatus), cudaHostAllocMapped);
    if (*e == cudaSuccess) *e = cudaHostGetDevicePointer((void**)&hs_dev_, hs_, 0);
    if (*e == cudaSuccess) *e = cudaMemsetAsync(st_, 0, sizeof(DevState), P->s);
  }

  ~Engine() override {
    for (auto& kv : graphs_) cudaGraphExecDestroy(kv.second);
    for (auto& ev : prof_ev_) cudaEventDestroy(ev);
    void* bufs[] = {valA_, valAt_, c_,    l_,    u_,    lc_,   uc_,    xbar_, wbuf_,
                    xa_,   xhat_,  xprev_, pv_,  pg_,   y_,    ya_,    yhat_, yprev_,
                    pw_,   x_,     xavg_, xref_, xanc_, yavg_, yanc_,  Ds_,   fval_,
                    ftval_, uvec_, uvec2_, rayx_, rayy_, qv_, qvec_, qvec2_, st_};
    for (void* b : bufs)
      if (b) cudaFree(b);
    if (hs_) cudaFreeHost(hs_);
    tape_free();
    if (tape_tab_) cudaFree(tape_tab_);
    if (tape_tab_h_) cudaFreeHost(tape_tab_h_);
  }

  cudaError_t set_feasibility(int mode) override {
    ProblemData& P = *P_;
    cudaStream_t s = P.s;
    feas_mode_ = mode;
    if (mode == 1 && P.n) return cudaMemsetAsync(c_, 0, sizeof(T) * P.n, s);
    if (mode == 2) {
      if (P.n) k_zero_finite<T><<<grid1(P.n), 256, 0, s>>>(l_, u_, P.n);
      if (P.m) k_zero_finite<T><<<grid1(P.m), 256, 0, s>>>(lc_, uc_, P.m);
      return cudaGetLastError();
    }
    return cudaSuccess;
  }

  cudaError_t load_values() override {
    ProblemData& P = *P_;
    cudaStream_t s = P.s;
    cudaError_t e;
    feas_mode_ = 0;
    if ((e = cast_vec<T>(P.val_s, valA_, P.nnz, s))) return e;
    if ((e = gather_cast<T>(P.val_s, P.permT, valAt_, P.nnz, s))) return e;
    if ((e = scale_cast<T>(P.c, P.Dc, false, c_, P.n, s))) return e;
    if ((e = scale_cast<T>(P.l, P.Dc, true, l_, P.n, s))) return e;
    if ((e = scale_cast<T>(P.u, P.Dc, true, u_, P.n, s))) return e;
    if ((e = scale_cast<T>(P.lc, P.Dr, false, lc_, P.m, s))) return e;
    if ((e = scale_cast<T>(P.uc, P.Dr, false, uc_, P.m, s))) return e;
    if (P.is_qp) {
      if ((e = cast_vec<T>(P.D_s, Ds_, P.n, s))) return e;
      if ((e = cast_vec<T>(P.fval_s, fval_, P.f_nnz, s))) return e;
      if ((e = gather_cast<T>(P.fval_s, P.permF, ftval_, P.f_nnz, s))) return e;
      if (P.q_general && (e = cast_vec<T>(P.qval_s, qv_, P.Q.nnz, s))) return e;
    }
    return cudaGetLastError();
  }

  // ---- norms by power iteration -------------------------------------------
  cudaError_t power(int mode, const mpax_options& o, long long* launches) {
    ProblemData& P = *P_;
    cudaStream_t s = P.s;
    const int n = P.n;
    k_power_start<<<1, 1, 0, s>>>(st_);
    *launches += 1;
    if (o.power_max_iter == 0) {  // the certified bound of the Pock-Chambolle round
      k_power_bound<<<1, 1, 0, s>>>(st_, mode);
      *launches += 1;
      return cudaGetLastError();
    }
    k_power_vec<T><<<grid1(n), 256, 0, s>>>(pv_, n, 1.0 / power_start_norm(n));
    *launches += 1;
    T* v = pv_;
    T* g = pg_;
    const int* skip = &st_->pw_done;
    for (int t = 1; t <= o.power_max_iter; ++t) {
      EpiStore<T> e1{skip, nullptr, &st_->pw_scale, nullptr, nullptr, nullptr, 0};
      EpiStore<T> e2{skip, g, nullptr, nullptr, nullptr, nullptr, 1};
      if (mode == 0) {
        e1.out = pw_;
        launch_spmv<T>(P.schedA, P.A, valA_, InPlain<T>{v}, e1, 0, s);
        launch_spmv<T>(P.schedAt, P.At, valAt_, InPlain<T>{pw_}, e2, 0, s);
        k_part_reduce<<<kChunks, 256, 0, s>>>(P.schedAt.part, P.schedAt.n_items, 1, nullptr, 0,
                                              0, skip, P.red);
        k_power_finalize<<<1, 256, 0, s>>>(P.red, kChunks, st_, t, o.power_tol, 0,
                                           o.pock_chambolle ? 1.0 : INFINITY, o.power_max_iter);
      } else if (P.q_general) {
        // g = Q~ (v pw_scale), sum of squares for the norm
        EpiStore<T> eq{skip, g, &st_->pw_scale, nullptr, nullptr, nullptr, 1};
        launch_spmv<T>(P.schedQ, P.Q, qv_, InPlain<T>{v}, eq, 0, s);
        k_part_reduce<<<kChunks, 256, 0, s>>>(P.schedQ.part, P.schedQ.n_items, 1, nullptr, 0,
                                              0, skip, P.red);
        k_power_finalize<<<1, 256, 0, s>>>(P.red, kChunks, st_, t, o.power_tol, 1, INFINITY,
                                           o.power_max_iter);
      } else {
        e1.out = uvec_;
        launch_spmv<T>(P.schedFt, P.Ft, ftval_, InPlain<T>{v}, e1, 0, s);
        e2.diag = Ds_;
        e2.din = v;
        e2.d_scale = &st_->pw_scale;
        launch_spmv<T>(P.schedF, P.F, fval_, InPlain<T>{uvec_}, e2, 0, s);
        k_part_reduce<<<kChunks, 256, 0, s>>>(P.schedF.part, P.schedF.n_items, 1, nullptr, 0,
                                              0, skip, P.red);
        k_power_finalize<<<1, 256, 0, s>>>(P.red, kChunks, st_, t, o.power_tol, 1, INFINITY,
                                           o.power_max_iter);
      }
      *launches += 4;
      std::swap(v, g);
      if (t % 8 == 0) {
        int done = 0;
        cudaError_t e = cudaMemcpyAsync(&done, &st_->pw_done, sizeof(int),
                                        cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e) return e;
        if (done) break;
      }
    }
    return cudaGetLastError();
  }

  // ---- autotuner: which kernel runs the A and A^T schedules -------------------
  cudaError_t tune(const mpax_options& o, long long* launches) override {
    ProblemData& P = *P_;
    cudaStream_t s = P.s;
    Sched* sc[2] = {&P.schedA, &P.schedAt};
    const Csr* K[2] = {&P.A, &P.At};
    for (double& u : tune_us_) u = 0.0;
    for (int q = 0; q < 2; ++q) {
      int kind = kSpmvItem;
      if (o.spmv_kernel >= 0) {
        kind = o.spmv_kernel;
      } else if (sc[q]->n_items > 0) {
        TuneKey key;
        cudaError_t e = tune_key(*K[q], sc[q]->n_items, sizeof(T), P.tmp_rows, s, &key);
        if (e) return e;
        key.v[4] += P.is_qp ? 100 : 0;  // the iteration's epilogues differ
        if (!tune_lookup(key, &kind)) {
          // a previous solve may have left `done` set, which makes every epilogue
          // skip its work; init_state clears the state again after tuning
          if ((e = cudaMemsetAsync(st_, 0, sizeof(DevState), s))) return e;
          double best = INFINITY;
          for (int k = 0; k < kSpmvKinds; ++k) {
            sc[q]->kind = k;
            double us = 0.0;
            e = time_launches(s, kTuneReps, &us, [&]() { tune_launch(q); });
            if (e) return e;
            *launches += kTuneReps + 1;
            if (k == kSpmvPipe) {
              // a bounded wait that gave up disqualifies the kernel (its error
              // word is cleared so that the chosen kernel starts clean)
              int herr = 0;
              int* w = sc[q]->cnt + sc[q]->n_items;
              if ((e = cudaMemcpyAsync(&herr, w, sizeof(int), cudaMemcpyDeviceToHost, s))) return e;
              if ((e = cudaStreamSynchronize(s))) return e;
              if (herr) {
                if ((e = cudaMemsetAsync(w, 0, sizeof(int), s))) return e;
                us = INFINITY;
              }
            }
            tune_us_[kSpmvKinds * q + k] = us;
            // another kind must beat the default shape by 3%: kinds within the
            // timing noise would otherwise flip between processes
            const double score = (k == kSpmvItem) ? us : us * 1.03;
            if (score < best) {
              best = score;
              kind = k;
            }
          }
          tune_store(key, kind);
        }
      }
      if (sc[q]->kind != kind) ++sched_generation;  // graphs captured the old kernel
      sc[q]->kind = kind;
      tune_kind_[q] = kind;
    }
    return cudaGetLastError();
  }

  // The error words of the pipelined SpMV (a bounded wait that gave up):
  // cudaErrorTimeout when one is set.
  cudaError_t pipe_errors() {
    ProblemData& P = *P_;
    const Sched* sc[2] = {&P.schedA, &P.schedAt};
    for (const Sched* q : sc) {
      if (!q->cnt || q->kind != kSpmvPipe) continue;
      int h = 0;
      cudaError_t e = cudaMemcpy(&h, q->cnt + q->n_items, sizeof(int), cudaMemcpyDeviceToHost);
      if (e) return e;
      if (h) return cudaErrorTimeout;
    }
    return cudaSuccess;
  }

  // One launch of the iteration's half-step on schedule q (0: A, the dual step;
  // 1: A^T, the primal step) with its own epilogue, on the engine's iterate
  // buffers: tuning runs before the iterate is initialised, so what these
  // launches write is overwritten before the solve reads it.
  void tune_launch(int q) {
    ProblemData& P = *P_;
    cudaStream_t s = P.s;
    if (!P.is_qp) {
      if (q == 0) {
        EpiDualLP<T> ed{st_, y_, ya_, lc_, uc_, yhat_, yprev_, 0, 0, 0};
        launch_spmv<T>(P.schedA, P.A, valA_, InPlain<T>{xbar_}, ed, 0, s);
      } else {
        EpiPrimalLP<T> ep{st_, xbar_, xbar_, xa_, c_, l_, u_, nullptr, xhat_, xprev_, 0, 0, 0};
        launch_spmv<T>(P.schedAt, P.At, valAt_, InPlain<T>{y_}, ep, 0, s);
      }
    } else if (q == 0) {
      EpiDualQP<T> ed{st_, y_, yavg_, yanc_, lc_, uc_, 0, 0};
      launch_spmv<T>(P.schedA, P.A, valA_, InPlain<T>{xref_}, ed, 0, s);
    } else {
      EpiPrimalQP<T> ep{st_, x_,  xavg_,   xref_,    xanc_, c_,    l_,     u_, Ds_, P.F.rp,
                        P.F.col, fval_, uvec_, xprev_, 0,   0,   0,  nullptr, nullptr,
                        P.q_general ? qvec_ : nullptr};
      launch_spmv<T>(P.schedAt, P.At, valAt_, InPlain<T>{y_}, ep, 0, s);
    }
  }

  void tune_info(int* kind, double* us) const override {
    for (int q = 0; q < 2; ++q) kind[q] = tune_kind_[q];
    for (int i = 0; i < 2 * kSpmvKinds; ++i) us[i] = tune_us_[i];
  }

  cudaError_t init_state(const mpax_options& o, long long* launches) override {
    ProblemData& P = *P_;
    cudaError_t e;
    if ((e = cudaMemsetAsync(st_, 0, sizeof(DevState), P.s))) return e;
    if (P.m > 0 && P.nnz > 0) {
      if ((e = power(0, o, launches))) return e;
    }
    if (P.is_qp) {
      if ((e = power(1, o, launches))) return e;
    }
    InitParams ip;
    ip.eps_abs = o.eps_abs;
    ip.eps_rel = o.eps_rel;
    ip.r_suff = o.restart_sufficient;
    ip.r_nec = o.restart_necessary;
    ip.r_art = o.restart_artificial;
    ip.pw_smooth = o.primal_weight_smoothing;
    ip.step_safety = o.step_safety;
    ip.gamma = o.reflection_gamma;
    ip.iter_limit = o.iteration_limit;
    ip.check_every = o.check_every;
    ip.is_qp = P.is_qp ? 1 : 0;
    ip.stall_limit = (o.precision == MPAX_PREC_MIXED && o.fp64_continuation) ? o.stall_checks : 0;
    ip.eps_pi = o.eps_primal_infeasible;
    ip.eps_di = o.eps_dual_infeasible;
    ip.feas_mode = feas_mode_;
    k_init_state<<<1, 256, 0, P.s>>>(st_, ip, P.red_out);
    *launches += 1;
    gamma_one_ = (o.reflection_gamma == 1.0);
    return cudaGetLastError();
  }

  cudaError_t init_iterate(const double* x0, const double* y0) override {
    ProblemData& P = *P_;
    cudaStream_t s = P.s;
    const int n = P.n, m = P.m;
    if (n) k_div_in<T><<<grid1(n), 256, 0, s>>>(x0, P.Dc, xhat_, n);
    if (m) k_div_in<T><<<grid1(m), 256, 0, s>>>(y0, P.Dr, yhat_, m);
    T* xs[] = {xa_, xbar_, wbuf_, xprev_, x_, xavg_, xref_, xanc_};
    T* ys[] = {ya_, y_, yprev_, yavg_, yanc_};
    for (T* d : xs)
      if (d && n) k_copy<T><<<grid1(n), 256, 0, s>>>(d, xhat_, n);
    for (T* d : ys)
      if (d && m) k_copy<T><<<grid1(m), 256, 0, s>>>(d, yhat_, m);
    use_xsrc_ = false;
    return cudaGetLastError();
  }

  // ---- one block -------------------------------------------------------------
  void launch_block(int len, bool plain, bool record_all, bool prof) {
    ProblemData& P = *P_;
    cudaStream_t s = P.s;
    const bool qp = P.is_qp;
    if (tape_on_ && !plain) {
      k_tape_save<T><<<grid1(std::max(P.n, P.m)), 256, 0, s>>>(
          st_, tape_tab_, kTapeSlots, P.n, P.m, x_, xavg_, y_, yavg_, len);
      launches_ += 1;
    }
    // QP: u = F~^T x_md (or Q~ x_md) of step it + 1 depends only on the point the
    // primal half-step of step it wrote, so it rides in the dual half-step's launch
    // (two independent schedules, one spmv_fused_pair); the first step of a block
    // follows a check and a possible restart and launches it on its own.
    bool aux_ready = false;
    for (int it = 0; it < len; ++it) {
      const bool last = (it == len - 1) && !plain;
      const int rec = (record_all || last) ? 1 : 0;
      const int chk = last ? 1 : 0;
      if (!qp) {
        EpiPrimalLP<T> ep{st_, xbar_, gamma_one_ ? xbar_ : wbuf_, xa_, c_, l_, u_,
                          (it == 0 && use_xsrc_) ? xprev_ : nullptr, xhat_, xprev_, it, rec,
                          chk};
        prof_begin(prof, 0);
        launch_spmv<T>(P.schedAt, P.At, valAt_, InPlain<T>{y_}, ep, 0, s);
        prof_end(prof, 0);
        EpiDualLP<T> ed{st_, y_, ya_, lc_, uc_, yhat_, yprev_, it, rec, chk};
        prof_begin(prof, 1);
        launch_spmv<T>(P.schedA, P.A, valA_, InPlain<T>{xbar_}, ed, 0, s);
        prof_end(prof, 1);
        launches_ += 2;
      } else {
        if (P.f_nnz > 0 && !aux_ready) {
          EpiStore<T> eu{&st_->done, uvec_, nullptr, nullptr, nullptr, nullptr, 0};
          prof_begin(prof, 4);
          launch_spmv<T>(P.schedFt, P.Ft, ftval_, InMomentum<T>{x_, xavg_, st_, it}, eu, 0, s);
          prof_end(prof, 4);
          launches_ += 1;
        }
        if (P.q_general && !aux_ready) {
          EpiStore<T> eq{&st_->done, qvec_, nullptr, nullptr, nullptr, nullptr, 0};
          prof_begin(prof, 4);
          launch_spmv<T>(P.schedQ, P.Q, qv_, InMomentum<T>{x_, xavg_, st_, it}, eq, 0, s);
          prof_end(prof, 4);
          launches_ += 1;
        }
        aux_ready = false;
        EpiPrimalQP<T> ep{st_, x_,  xavg_,    xref_,    xanc_,  c_,     l_,    u_,
                          Ds_, P.F.rp, P.F.col, fval_, uvec_, xprev_, it,    rec, chk,
                          nullptr, nullptr, P.q_general ? qvec_ : nullptr};
        prof_begin(prof, 0);
        launch_spmv<T>(P.schedAt, P.At, valAt_, InPlain<T>{y_}, ep, 0, s);
        prof_end(prof, 0);
        EpiDualQP<T> ed{st_, y_, yavg_, yanc_, lc_, uc_, it, chk};
        // the pair launch when the next step's product exists and is not timed apart
        const bool pair = !prof && it + 1 < len && (P.f_nnz > 0) != P.q_general;
        if (pair) {
          const InMomentum<T> nx{x_, xavg_, st_, it + 1};
          if (P.f_nnz > 0) {
            EpiStore<T> eu{&st_->done, uvec_, nullptr, nullptr, nullptr, nullptr, 0};
            aux_ready = launch_spmv_pair<T>(P.schedA, P.A, valA_, InPlain<T>{xref_}, ed,
                                            P.schedFt, P.Ft, ftval_, nx, eu, s);
          } else {
            EpiStore<T> eq{&st_->done, qvec_, nullptr, nullptr, nullptr, nullptr, 0};
            aux_ready = launch_spmv_pair<T>(P.schedA, P.A, valA_, InPlain<T>{xref_}, ed,
                                            P.schedQ, P.Q, qv_, nx, eq, s);
          }
        }
        if (!aux_ready) {
          prof_begin(prof, 1);
          launch_spmv<T>(P.schedA, P.A, valA_, InPlain<T>{xref_}, ed, 0, s);
          prof_end(prof, 1);
        }
        launches_ += 2;
      }
    }
    use_xsrc_ = false;
    if (plain) return;
    kkt_launch(&st_->done, prof);
    if (!qp) ray_launch(&st_->done);
    k_part_reduce<<<kChunks, 256, 0, s>>>(P.schedAt.part, P.schedAt.n_items, kCheckQt,
                                          P.schedA.part, P.schedA.n_items, kCheckQa,
                                          &st_->done, P.red);
    k_finalize_check<<<1, 512, 0, s>>>(P.red, kChunks, nullptr, 0, st_, hs_dev_, len, block_);
    launches_ += 1;
    if (!qp) {
      k_restart_lp<T><<<grid1(std::max(P.n, P.m)), 256, 0, s>>>(
          st_, P.n, P.m, xhat_, xa_, xbar_, gamma_one_ ? xbar_ : wbuf_, yhat_, ya_, y_);
    } else {
      k_restart_qp<T><<<grid1(std::max(P.n, P.m)), 256, 0, s>>>(st_, P.n, P.m, xavg_, x_,
                                                                 xanc_, yavg_, y_, yanc_);
    }
    launches_ += 2;
  }

  // KKT SpMVs at (x^, y^) (LP) or (xavg, yavg) (QP), partial slots 2..
  // Infeasibility rays of an LP check: the anchor moves (k_ray_prep), then A~ rx
  // and A~^T ry with the ray epilogues into partial slots 4-5 (A) and 6-9 (A^T).
  void ray_launch(const int* skip) {
    ProblemData& P = *P_;
    cudaStream_t s = P.s;
    k_ray_prep<T><<<grid1(std::max(P.n, P.m)), 256, 0, s>>>(xhat_, xa_, P.n, yhat_, ya_, P.lc,
                                                             P.uc, P.m, skip, rayx_, rayy_);
    EpiRayRow<T> er{skip, P.invDr, P.Dr, P.lc, P.uc, rayy_, 1};
    launch_spmv<T>(P.schedA, P.A, valA_, InPlain<T>{rayx_}, er, 4, s);
    EpiRayCol<T> ec{skip, P.invDc, P.Dc, P.c, P.l, P.u, rayx_, 1};
    launch_spmv<T>(P.schedAt, P.At, valAt_, InPlain<T>{rayy_}, ec, 6, s);
    launches_ += 3;
  }

  void kkt_launch(const int* skip, bool prof) {
    ProblemData& P = *P_;
    cudaStream_t s = P.s;
    const bool qp = P.is_qp;
    const T* xv = qp ? xavg_ : xhat_;
    const T* yv = qp ? yavg_ : yhat_;
    if (qp && P.f_nnz > 0) {
      EpiStore<T> eu{skip, uvec2_, nullptr, nullptr, nullptr, nullptr, 0};
      launch_spmv<T>(P.schedFt, P.Ft, ftval_, InPlain<T>{xv}, eu, 0, s);
      launches_ += 1;
    }
    EpiKktRow<T> er{skip, P.invDr, P.Dr, P.lc, P.uc, yv, 1};
    prof_begin(prof, 2);
    launch_spmv<T>(P.schedA, P.A, valA_, InPlain<T>{xv}, er, 2, s);
    prof_end(prof, 2);
    if (qp && P.q_general) {
      EpiStore<T> eq{skip, qvec2_, nullptr, nullptr, nullptr, nullptr, 0};
      launch_spmv<T>(P.schedQ, P.Q, qv_, InPlain<T>{xv}, eq, 0, s);
      launches_ += 1;
    }
    EpiKktCol<T> ec{skip, P.invDc, P.Dc, P.c, P.l, P.u, xv, qp ? 1 : 0, P.D_s,
                    P.F.rp, P.F.col, P.fval_s, uvec2_, 1,
                    (qp && P.q_general) ? qvec2_ : nullptr};
    prof_begin(prof, 3);
    launch_spmv<T>(P.schedAt, P.At, valAt_, InPlain<T>{yv}, ec, 2, s);
    prof_end(prof, 3);
    launches_ += 2;
  }

  // ---- profiling with CUDA events (no graphs) ---------------------------------
  void prof_begin(bool prof, int cls) {
    if (!prof) return;
    if (prof_used_ + 2 > prof_ev_.size()) {
      for (int i = 0; i < 64; ++i) {
        cudaEvent_t ev;
        cudaEventCreate(&ev);
        prof_ev_.push_back(ev);
      }
    }
    cudaEventRecord(prof_ev_[prof_used_], P_->s);
    prof_cls_.push_back(cls);
  }
  void prof_end(bool prof, int) {
    if (!prof) return;
    cudaEventRecord(prof_ev_[prof_used_ + 1], P_->s);
    prof_used_ += 2;
  }
  void prof_collect(RunInfo* info) {
    for (size_t i = 0; i < prof_cls_.size(); ++i) {
      float ms = 0;
      cudaEventElapsedTime(&ms, prof_ev_[2 * i], prof_ev_[2 * i + 1]);
      info->profile_ms[prof_cls_[i]] += ms;
      info->profile_launches[prof_cls_[i]] += 1;
    }
    prof_cls_.clear();
    prof_used_ = 0;
  }

  int tune_kind_[2] = {0, 0};
  double tune_us_[2 * kSpmvKinds] = {};

  cudaError_t block_graph(int len, cudaGraphExec_t* out) {
    if (graph_gen_ != sched_generation) {
      for (auto& kv : graphs_) cudaGraphExecDestroy(kv.second);
      graphs_.clear();
      graph_launches_.clear();
      graph_gen_ = sched_generation;
    }
    const long long key = (long long)len + 4096LL * block_ + (gamma_one_ ? (1LL << 40) : 0) +
                          (tape_on_ ? (1LL << 41) : 0);
    auto itg = graphs_.find(key);
    if (itg != graphs_.end()) {
      *out = itg->second;
      return cudaSuccess;
    }
    cudaStream_t s = P_->s;
    cudaGraph_t g;
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e) return e;
    const long long before = launches_;
    launch_block(len, false, false, false);
    graph_launches_[key] = launches_ - before;
    launches_ = before;
    e = cudaStreamEndCapture(s, &g);
    if (e) return e;
    cudaGraphExec_t ge;
    e = cudaGraphInstantiate(&ge, g, 0);
    cudaGraphDestroy(g);
    if (e) return e;
    graphs_[key] = ge;
    graph_key_ = key;
    *out = ge;
    return cudaSuccess;
  }

  cudaError_t run(const mpax_options& o, RunInfo* info) override {
    ProblemData& P = *P_;
    cudaStream_t s = P.s;
    cudaError_t e;
    block_ = o.check_every;
    hs_->done = 0;
    hs_->total = 0;
    hs_->checks = 0;
    launches_ = 0;
    const bool prof = o.profile_kernels != 0;
    const bool graphs = o.use_graphs != 0 && !prof;
    const long long limit = o.iteration_limit;
    tape_on_ = o.record_tape != 0 && P.is_qp;
    tape_valid_ = false;
    tape_slots_ = 0;
    if (tape_on_) {
      if ((e = tape_init())) return e;
    } else {
      tape_free();
    }
    const auto t0 = std::chrono::steady_clock::now();
    cudaEvent_t ev[2];
    cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming);
    cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming);
    long long launched = 0;
    long long last_print = -1;
    bool stop = false;
    for (long long b = 0; !stop; ++b) {
      const int len = (int)std::min<long long>(block_, limit - launched);
      if (tape_on_ && (e = tape_ensure(b))) break;
      if (graphs) {
        cudaGraphExec_t ge;
        if ((e = block_graph(len, &ge))) break;
        if ((e = cudaGraphLaunch(ge, s))) break;
        launches_ += graph_launches_[graph_key_];
      } else {
        launch_block(len, false, false, prof);
      }
      if ((e = cudaEventRecord(ev[b & 1], s))) break;
      launched += len;
      if (prof) {
        if ((e = cudaEventSynchronize(ev[b & 1]))) break;
        prof_collect(info);
        stop = hs_->done != 0;
      } else if (b >= 1) {
        if ((e = cudaEventSynchronize(ev[(b - 1) & 1]))) break;
        stop = hs_->done != 0;
      }
      if (o.verbose && hs_->checks != last_print &&
          hs_->checks % std::max(1, o.display_frequency) == 0) {
        last_print = hs_->checks;
        std::printf("mpax  iter %10lld  rel_kkt %.3e  pobj %+.8e  dobj %+.8e  omega %.3e\n",
                    (long long)hs_->total, (double)hs_->rel_kkt, (double)hs_->pobj,
                    (double)hs_->dobj, (double)hs_->omega);
        std::fflush(stdout);
      }
      if (!stop && launched >= limit) {
        if ((e = cudaEventSynchronize(ev[b & 1]))) break;
        stop = true;
      }
      if (!stop && o.time_limit < INFINITY) {
        const double el =
            std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (el >= o.time_limit) {
          info->time_limit_hit = true;
          stop = true;
        }
      }
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    if (e) return e;
    if ((e = cudaStreamSynchronize(s))) return e;
    if ((e = pipe_errors())) return e;
    DevState h;
    if ((e = read_state(&h))) return e;
    if (tape_on_) {
      tape_on_ = false;
      if (h.tape_err) return cudaErrorMemoryAllocation;
      tape_slots_ = h.checks;
      tape_valid_ = true;
    }
    info->termination = h.termination;
    if (!h.done && info->time_limit_hit) info->termination = MPAX_TERM_TIME_LIMIT;
    info->iterations = h.total;
    info->restarts = h.restarts;
    info->checks = h.checks;
    info->launches = launches_;
    return cudaSuccess;
  }

  // ---- tape of a QP solve and the unrolled reverse sweep -----------------------
  cudaError_t tape_init() {
    ProblemData& P = *P_;
    cudaError_t e;
    const size_t bytes = sizeof(TapeHead) + sizeof(T) * (2 * (size_t)P.n + 2 * (size_t)P.m);
    const size_t rec = (bytes + 255) / 256 * 256;
    if (rec != tape_rec_bytes_) tape_free();
    tape_rec_bytes_ = rec;
    if (!tape_tab_) {
      if ((e = cudaMalloc(&tape_tab_, sizeof(char*) * kTapeSlots))) return e;
      if ((e = cudaMemsetAsync(tape_tab_, 0, sizeof(char*) * kTapeSlots, P.s))) return e;
      if ((e = cudaHostAlloc(&tape_tab_h_, sizeof(char*) * kTapeSlots, cudaHostAllocDefault)))
        return e;
    }
    return cudaSuccess;
  }

  // Records for blocks 0..slot exist (chunks of kTapeChunk records).
  cudaError_t tape_ensure(long long slot) {
    const long long have = (long long)tape_chunks_.size() * kTapeChunk;
    if (slot < have) return cudaSuccess;
    if (slot >= kTapeSlots) return cudaErrorMemoryAllocation;
    char* chunk = nullptr;
    cudaError_t e = cudaMalloc(&chunk, tape_rec_bytes_ * kTapeChunk);
    if (e) return e;
    tape_chunks_.push_back(chunk);
    for (int k = 0; k < kTapeChunk; ++k) tape_tab_h_[have + k] = chunk + k * tape_rec_bytes_;
    return cudaMemcpyAsync(tape_tab_ + have, tape_tab_h_ + have, sizeof(char*) * kTapeChunk,
                           cudaMemcpyHostToDevice, P_->s);
  }

  void tape_free() {
    if (tape_chunks_.empty()) return;
    cudaStreamSynchronize(P_->s);
    for (char* c : tape_chunks_) cudaFree(c);
    tape_chunks_.clear();
    if (tape_tab_) cudaMemsetAsync(tape_tab_, 0, sizeof(char*) * kTapeSlots, P_->s);
    tape_valid_ = false;
    tape_slots_ = 0;
  }

  // One block of the taped path again from its restored start state, with the
  // forward kernels recording x_md and the clamp codes of every step.
  void replay_block(int len, T* xmd, unsigned char* cx, unsigned char* cy) {
    ProblemData& P = *P_;
    cudaStream_t s = P.s;
    const size_t n = P.n, m = P.m;
    bool aux_ready = false;  // the step's momentum product came with the last dual launch
    for (int it = 0; it < len; ++it) {
      if (P.f_nnz > 0 && !aux_ready) {
        EpiStore<T> eu{&st_->done, uvec_, nullptr, nullptr, nullptr, nullptr, 0};
        launch_spmv<T>(P.schedFt, P.Ft, ftval_, InMomentum<T>{x_, xavg_, st_, it}, eu, 0, s);
        launches_ += 1;
      }
      if (P.q_general && !aux_ready) {
        EpiStore<T> eq{&st_->done, qvec_, nullptr, nullptr, nullptr, nullptr, 0};
        launch_spmv<T>(P.schedQ, P.Q, qv_, InMomentum<T>{x_, xavg_, st_, it}, eq, 0, s);
        launches_ += 1;
      }
      aux_ready = false;
      EpiPrimalQP<T, true> ep{st_, x_,    xavg_,  xref_,  xanc_, c_,     l_,  u_,
                              Ds_, P.F.rp, P.F.col, fval_, uvec_, xprev_, it, 0,
                              0,   xmd + it * n, cx + it * n, P.q_general ? qvec_ : nullptr};
      launch_spmv<T>(P.schedAt, P.At, valAt_, InPlain<T>{y_}, ep, 0, s);
      EpiDualQP<T, true> ed{st_, y_, yavg_, yanc_, lc_, uc_, it, 0, cy + it * m};
      if (it + 1 < len && (P.f_nnz > 0) != P.q_general) {  // as in launch_block
        const InMomentum<T> nx{x_, xavg_, st_, it + 1};
        EpiStore<T> ea{&st_->done, P.f_nnz > 0 ? uvec_ : qvec_, nullptr, nullptr, nullptr,
                       nullptr, 0};
        aux_ready = P.f_nnz > 0
                        ? launch_spmv_pair<T>(P.schedA, P.A, valA_, InPlain<T>{xref_}, ed,
                                              P.schedFt, P.Ft, ftval_, nx, ea, s)
                        : launch_spmv_pair<T>(P.schedA, P.A, valA_, InPlain<T>{xref_}, ed,
                                              P.schedQ, P.Q, qv_, nx, ea, s);
      }
      if (!aux_ready) launch_spmv<T>(P.schedA, P.A, valA_, InPlain<T>{xref_}, ed, 0, s);
      launches_ += 2;
    }
  }

  cudaError_t unrolled_backward(const double* gx, const double* gy, double* gc, double* glc,
                                double* guc, double* gl, double* gu, double* gD, bool use_graphs,
                                long long* launches) override {
    if constexpr (!std::is_same<T, double>::value) {
      return cudaErrorNotSupported;
    } else {
      ProblemData& P = *P_;
      cudaStream_t s = P.s;
      const int n = P.n, m = P.m;
      if (!tape_valid_ || tape_slots_ <= 0) return cudaErrorNotReady;
      cudaError_t e;
      std::vector<TapeHead> H((size_t)tape_slots_);
      for (long long b = 0; b < tape_slots_; ++b)
        if ((e = cudaMemcpyAsync(&H[b], tape_tab_h_[b], sizeof(TapeHead), cudaMemcpyDeviceToHost,
                                 s)))
          return e;
      if ((e = cudaStreamSynchronize(s))) return e;
      int lmax = 1;
      for (const TapeHead& h : H) lmax = std::max(lmax, h.len);
      // scratch: adjoints, the replayed block's x_md and codes, the saved state
      e = cudaSuccess;
      double* ax = dalloc<double>(n, &e);
      double* axa = dalloc<double>(n, &e);
      double* uu = dalloc<double>(n, &e);
      double* ay = dalloc<double>(m, &e);
      double* aya = dalloc<double>(m, &e);
      double* ws = dalloc<double>(m, &e);
      double* tq = dalloc<double>(std::max(P.r, 1), &e);
      double* qu = P.q_general ? dalloc<double>(n, &e) : nullptr;
      T* xmd = dalloc<T>((size_t)lmax * n, &e);
      unsigned char* cx = dalloc<unsigned char>((size_t)lmax * n, &e);
      unsigned char* cy = dalloc<unsigned char>((size_t)lmax * m, &e);
      T* sv = dalloc<T>(2 * (size_t)n + 2 * (size_t)m, &e);
      DevState* sts = dalloc<DevState>(1, &e);
      void* bufs[] = {ax, axa, uu, ay, aya, ws, tq, qu, xmd, cx, cy, sv, sts};
      auto release = [&]() {
        cudaStreamSynchronize(s);
        for (void* b : bufs)
          if (b) cudaFree(b);
      };
      if (e) {
        release();
        return e;
      }
      const long long l0 = launches_;
      // the returned point and the state survive the sweep
      cudaMemcpyAsync(sts, st_, sizeof(DevState), cudaMemcpyDeviceToDevice, s);
      const size_t nn = n, mm = m;
      cudaMemcpyAsync(sv, x_, sizeof(T) * nn, cudaMemcpyDeviceToDevice, s);
      cudaMemcpyAsync(sv + nn, xavg_, sizeof(T) * nn, cudaMemcpyDeviceToDevice, s);
      cudaMemcpyAsync(sv + 2 * nn, y_, sizeof(T) * mm, cudaMemcpyDeviceToDevice, s);
      cudaMemcpyAsync(sv + 2 * nn + mm, yavg_, sizeof(T) * mm, cudaMemcpyDeviceToDevice, s);
      for (double* g : {gc, gl, gu, gD}) cudaMemsetAsync(g, 0, sizeof(double) * nn, s);
      for (double* g : {glc, guc})
        if (m) cudaMemsetAsync(g, 0, sizeof(double) * mm, s);
      const int gN = grid1(std::max(n, m));
      k_rev_seed<<<gN, 256, 0, s>>>(gx, gy, P.Dc, P.Dr, n, m, ax, axa, ay, aya);
      k_set_cursor<<<1, 1, 0, s>>>(st_, tape_slots_);
      launches_ += 2;
      // One block backwards: every launch reads its block's scalars from the
      // device state, so the sequence is captured once per block length as a
      // CUDA graph and replayed for every block.
      // The reverse epilogues carry more state than the forward ones: in FP64 the
      // default register budget (the forward kind the tuner may keep) spills them,
      // so the reverse products run with the wide budget instead.
      Sched sAtRev = P.schedAt, sARev = P.schedA;
      if (sizeof(T) == 8 && sAtRev.kind == kSpmvItem) sAtRev.kind = kSpmvItemWide;
      if (sizeof(T) == 8 && sARev.kind == kSpmvItem) sARev.kind = kSpmvItemWide;
      auto rev_block = [&](int L) {
        k_tape_open<<<1, 256, 0, s>>>(st_, tape_tab_);
        k_tape_restore<T><<<gN, 256, 0, s>>>(st_, tape_tab_, n, m, x_, xavg_, y_, yavg_, ax,
                                             axa, ay, aya);
        launches_ += 2;
        replay_block(L, xmd, cx, cy);
        if (m) {
          k_rev_r1<<<grid1(m), 256, 0, s>>>(st_, L - 1, m, cy + (size_t)(L - 1) * mm, ay, aya,
                                            ws, glc, guc);
          launches_ += 1;
        }
        for (int it = L - 1; it >= 0; --it) {
          EpiRevPrimal<T> ep{st_, ax, axa, uu, gc, gl, gu, gD, cx + (size_t)it * nn, Ds_,
                             P.F.rp, P.F.col, fval_, tq,
                             it < L - 1 ? xmd + (size_t)(it + 1) * nn : nullptr, it, 0, qu};
          launch_spmv<T>(sAtRev, P.At, valAt_, InPlain<T>{ws}, ep, 0, s);
          // F~^T uu (or Q~ uu) and the reverse dual step both read only uu: one launch
          EpiRevDual<T> ed{st_, ay, aya, ws, glc, guc,
                           it > 0 ? cy + (size_t)(it - 1) * mm : nullptr, it, 0};
          bool paired = false;
          if (P.f_nnz > 0) {
            EpiStore<T> eu{nullptr, tq, nullptr, nullptr, nullptr, nullptr, 0};
            paired = launch_spmv_pair<T>(sARev, P.A, valA_, InPlain<T>{uu}, ed, P.schedFt, P.Ft,
                                         ftval_, InPlain<T>{uu}, eu, s);
            if (!paired) {
              launch_spmv<T>(P.schedFt, P.Ft, ftval_, InPlain<T>{uu}, eu, 0, s);
              launches_ += 1;
            }
          } else if (P.q_general) {
            EpiStore<T> eq{nullptr, qu, nullptr, nullptr, nullptr, nullptr, 0};
            paired = launch_spmv_pair<T>(sARev, P.A, valA_, InPlain<T>{uu}, ed, P.schedQ, P.Q,
                                         qv_, InPlain<T>{uu}, eq, s);
            if (!paired) {
              launch_spmv<T>(P.schedQ, P.Q, qv_, InPlain<T>{uu}, eq, 0, s);
              launches_ += 1;
            }
          }
          if (!paired) launch_spmv<T>(sARev, P.A, valA_, InPlain<T>{uu}, ed, 0, s);
          launches_ += 2;
        }
        k_rev_r4<T><<<grid1(n), 256, 0, s>>>(st_, 0, n, Ds_, P.F.rp, P.F.col, fval_, tq, uu, xmd,
                                             qu, ax, axa, gD);
        launches_ += 1;
      };
      std::map<int, std::pair<cudaGraphExec_t, long long>> rg;
      for (long long b = tape_slots_ - 1; b >= 0 && !e; --b) {
        const int L = H[b].len;
        if (!use_graphs) {
          rev_block(L);
          continue;
        }
        auto it = rg.find(L);
        if (it == rg.end()) {
          cudaGraph_t g;
          if ((e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal))) break;
          const long long before = launches_;
          rev_block(L);
          const long long nl = launches_ - before;
          launches_ = before;
          if ((e = cudaStreamEndCapture(s, &g))) break;
          cudaGraphExec_t ge;
          e = cudaGraphInstantiate(&ge, g, 0);
          cudaGraphDestroy(g);
          if (e) break;
          it = rg.emplace(L, std::make_pair(ge, nl)).first;
        }
        if ((e = cudaGraphLaunch(it->second.first, s))) break;
        launches_ += it->second.second;
      }
      for (auto& kv : rg) cudaGraphExecDestroy(kv.second.first);
      if (e) {
        release();
        return e;
      }
      k_rev_unscale<<<gN, 256, 0, s>>>(P.Dc, P.Dr, n, m, gc, gl, gu, gD, glc, guc);
      cudaMemcpyAsync(x_, sv, sizeof(T) * nn, cudaMemcpyDeviceToDevice, s);
      cudaMemcpyAsync(xavg_, sv + nn, sizeof(T) * nn, cudaMemcpyDeviceToDevice, s);
      cudaMemcpyAsync(y_, sv + 2 * nn, sizeof(T) * mm, cudaMemcpyDeviceToDevice, s);
      cudaMemcpyAsync(yavg_, sv + 2 * nn + mm, sizeof(T) * mm, cudaMemcpyDeviceToDevice, s);
      cudaMemcpyAsync(st_, sts, sizeof(DevState), cudaMemcpyDeviceToDevice, s);
      launches_ += 1;
      *launches += launches_ - l0;
      e = cudaGetLastError();
      release();
      return e;
    }
  }

  // ---- lower-level access -----------------------------------------------------
  cudaError_t set_iterate(const double* x, const double* y, const double* xa, const double* ya,
                          long long k, double tau, double sigma, double gamma) override {
    ProblemData& P = *P_;
    cudaStream_t s = P.s;
    const int n = P.n, m = P.m;
    gamma_one_ = (gamma == 1.0);
    if (!P.is_qp) {
      if (n) {
        k_from_double<T><<<grid1(n), 256, 0, s>>>(x, xprev_, n);
        k_from_double<T><<<grid1(n), 256, 0, s>>>(x, xbar_, n);
        k_from_double<T><<<grid1(n), 256, 0, s>>>(x, wbuf_, n);
        k_from_double<T><<<grid1(n), 256, 0, s>>>(xa, xa_, n);
      }
      if (m) {
        k_from_double<T><<<grid1(m), 256, 0, s>>>(y, y_, m);
        k_from_double<T><<<grid1(m), 256, 0, s>>>(ya, ya_, m);
      }
      use_xsrc_ = true;
    } else {
      if (n) {
        k_from_double<T><<<grid1(n), 256, 0, s>>>(x, x_, n);
        k_from_double<T><<<grid1(n), 256, 0, s>>>(xa, xavg_, n);
        k_from_double<T><<<grid1(n), 256, 0, s>>>(xa, xanc_, n);
      }
      if (m) {
        k_from_double<T><<<grid1(m), 256, 0, s>>>(y, y_, m);
        k_from_double<T><<<grid1(m), 256, 0, s>>>(ya, yavg_, m);
        k_from_double<T><<<grid1(m), 256, 0, s>>>(ya, yanc_, m);
      }
    }
    st_is_qp_kernel();
    k_set_steps<<<1, 1, 0, s>>>(st_, tau, sigma, gamma);
    k_cur_ = k;
    return cudaGetLastError();
  }

  void st_is_qp_kernel() {
    // is_qp flag for the coefficient tables when set_iterate runs before a solve
    InitParams ip{};
    (void)ip;
    const int v = P_->is_qp ? 1 : 0;
    cudaMemcpyAsync(&st_->is_qp, &v, sizeof(int), cudaMemcpyHostToDevice, P_->s);
    cudaStreamSynchronize(P_->s);
  }

  cudaError_t iterate(long long iters) override {
    cudaStream_t s = P_->s;
    while (iters > 0) {
      const int len = (int)std::min<long long>(iters, kMaxCheckEvery);
      k_set_table<<<1, 256, 0, s>>>(st_, k_cur_, len);
      launch_block(len, true, true, false);
      k_cur_ += len;
      iters -= len;
    }
    return cudaGetLastError();
  }

  cudaError_t get_iterate(double* x, double* y, double* xh, double* yh) override {
    ProblemData& P = *P_;
    cudaStream_t s = P.s;
    const int n = P.n, m = P.m;
    if (!P.is_qp) {
      k_set_table<<<1, 256, 0, s>>>(st_, k_cur_, 1);
      if (n) {
        k_materialize_lp<T><<<grid1(n), 256, 0, s>>>(pv_, gamma_one_ ? xbar_ : wbuf_, xa_, st_,
                                                     0, n);
        if (x) k_to_double<T><<<grid1(n), 256, 0, s>>>(pv_, nullptr, x, n);
        if (xh) k_to_double<T><<<grid1(n), 256, 0, s>>>(xhat_, nullptr, xh, n);
      }
      if (m) {
        if (y) k_to_double<T><<<grid1(m), 256, 0, s>>>(y_, nullptr, y, m);
        if (yh) k_to_double<T><<<grid1(m), 256, 0, s>>>(yhat_, nullptr, yh, m);
      }
    } else {
      if (n && x) k_to_double<T><<<grid1(n), 256, 0, s>>>(x_, nullptr, x, n);
      if (n && xh) k_to_double<T><<<grid1(n), 256, 0, s>>>(xavg_, nullptr, xh, n);
      if (m && y) k_to_double<T><<<grid1(m), 256, 0, s>>>(y_, nullptr, y, m);
      if (m && yh) k_to_double<T><<<grid1(m), 256, 0, s>>>(yavg_, nullptr, yh, m);
    }
    return cudaGetLastError();
  }

  cudaError_t get_solution(double* x, double* y) override {
    ProblemData& P = *P_;
    cudaStream_t s = P.s;
    const T* xv = P.is_qp ? xavg_ : xhat_;
    const T* yv = P.is_qp ? yavg_ : yhat_;
    if (x && P.n) k_to_double<T><<<grid1(P.n), 256, 0, s>>>(xv, P.Dc, x, P.n);
    if (y && P.m) k_to_double<T><<<grid1(P.m), 256, 0, s>>>(yv, P.Dr, y, P.m);
    return cudaGetLastError();
  }

  cudaError_t kkt_at(const double* x, const double* y, double* out6) override {
    ProblemData& P = *P_;
    cudaStream_t s = P.s;
    T* xv = P.is_qp ? xavg_ : xhat_;
    T* yv = P.is_qp ? yavg_ : yhat_;
    if (P.n) k_div_in<T><<<grid1(P.n), 256, 0, s>>>(x, P.Dc, xv, P.n);
    if (P.m) k_div_in<T><<<grid1(P.m), 256, 0, s>>>(y, P.Dr, yv, P.m);
    // zero the partial slots so empty schedules contribute nothing
    if (P.schedA.part) cudaMemsetAsync(P.schedA.part, 0, sizeof(double) * kPartQ * std::max(P.schedA.n_items, 1), s);
    if (P.schedAt.part) cudaMemsetAsync(P.schedAt.part, 0, sizeof(double) * kPartQ * std::max(P.schedAt.n_items, 1), s);
    kkt_launch(nullptr, false);
    k_part_reduce<<<kChunks, 256, 0, s>>>(P.schedAt.part, P.schedAt.n_items, kCheckQt,
                                          P.schedA.part, P.schedA.n_items, 4, nullptr, P.red);
    k_kkt_finalize<<<1, 256, 0, s>>>(P.red, kChunks, nullptr, 0, st_, out6);
    return cudaGetLastError();
  }

  cudaError_t read_state(DevState* h) override {
    cudaError_t e = cudaMemcpyAsync(h, st_, sizeof(DevState), cudaMemcpyDeviceToHost, P_->s);
    if (e) return e;
    return cudaStreamSynchronize(P_->s);
  }

 private:
  ProblemData* P_;
  T *valA_ = nullptr, *valAt_ = nullptr;
  T *c_ = nullptr, *l_ = nullptr, *u_ = nullptr, *lc_ = nullptr, *uc_ = nullptr;
  T *xbar_ = nullptr, *wbuf_ = nullptr, *xa_ = nullptr, *xhat_ = nullptr, *xprev_ = nullptr;
  T *rayx_ = nullptr, *rayy_ = nullptr;  // infeasibility rays of an LP check
  int feas_mode_ = 0;                     // polishing mode of the loaded data
  T *pv_ = nullptr, *pg_ = nullptr, *pw_ = nullptr;
  T *y_ = nullptr, *ya_ = nullptr, *yhat_ = nullptr, *yprev_ = nullptr;
  T *x_ = nullptr, *xavg_ = nullptr, *xref_ = nullptr, *xanc_ = nullptr;
  T *yavg_ = nullptr, *yanc_ = nullptr;
  T *Ds_ = nullptr, *fval_ = nullptr, *ftval_ = nullptr, *uvec_ = nullptr, *uvec2_ = nullptr;
  T *qv_ = nullptr, *qvec_ = nullptr, *qvec2_ = nullptr;  // general sparse Q
  DevState* st_ = nullptr;
  HostStatus* hs_ = nullptr;
  HostStatus* hs_dev_ = nullptr;
  bool gamma_one_ = true;
  bool use_xsrc_ = false;
  long long k_cur_ = 0;
  int block_ = 64;
  long long launches_ = 0;
  std::map<long long, cudaGraphExec_t> graphs_;
  std::map<long long, long long> graph_launches_;
  unsigned long long graph_gen_ = 0;
  long long graph_key_ = 0;
  std::vector<cudaEvent_t> prof_ev_;
  std::vector<int> prof_cls_;
  size_t prof_used_ = 0;
  // tape of a QP solve: one record per check block (TapeHead + x, xavg, y, yavg)
  static constexpr long long kTapeSlots = 1LL << 20;
  static constexpr int kTapeChunk = 16;
  bool tape_on_ = false, tape_valid_ = false;
  long long tape_slots_ = 0;
  size_t tape_rec_bytes_ = 0;
  char** tape_tab_ = nullptr;    // device: record of block b
  char** tape_tab_h_ = nullptr;  // pinned host mirror
  std::vector<char*> tape_chunks_;
};

EngineBase* make_engine(ProblemData* P, int precision, cudaError_t* err) {
  *err = cudaSuccess;
  EngineBase* e;
  if (precision == MPAX_PREC_FP64) e = new Engine<double>(P, err);
  else e = new Engine<float>(P, err);
  if (*err != cudaSuccess) {
    delete e;
    return nullptr;
  }
  return e;
}

}  // namespace mpax
