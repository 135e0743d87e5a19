// Ragged batch of independent LPs solved by r^2HPDHG (Algorithm 1) in ONE
// persistent kernel launch.
//
// The paper batches same-shape instances by vectorising the solver (Sec. 3.2).
// Here instances may differ in size: they are packed back to back as one
// block-diagonal problem, so the device transpose and the Ruiz/Pock-Chambolle
// scaling (row- and column-local operations) of the single-problem path apply
// unchanged.  The iteration itself runs in one launch: each CTA takes the next
// unsolved instance from an atomic work counter and runs the whole restarted
// loop for it -- power iteration, initial primal weight, half-steps, relative
// KKT checks, restarts, primal-weight updates, termination -- with the two
// gathered vectors of the instance (y for the SpMV^T, the reflected primal point
// for the SpMV) held in shared memory, or, for an instance too large for that,
// in global memory (the same code through generic pointers).  All reductions are fixed-order CTA
// trees in FP64; no instance waits on another, so no grid-wide synchronisation
// exists and a finished CTA simply takes the next instance.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/mpax.h"
#include "problem.cuh"

namespace mpax {

// Threads of the CTA that solves one instance, and CTAs per SM at 64 registers a
// thread.  Measured on 4,096 instances of the bench recipe: FP32 1024 threads 0.323 s
// per batch (instance p50 6.5 ms), 512 threads 0.334 s (11.8 ms), 256 threads
// 0.435 s; FP64 512 threads 0.461 s, 1024 threads 0.488 s, 256 threads 0.80 s.
template <typename T>
constexpr int kBatchThreads = sizeof(T) == 4 ? 1024 : 512;
template <typename T>
constexpr int kBatchMinB = 1024 / kBatchThreads<T>;
constexpr double kBatchMaxSeconds = 600.0;
// Lanes cooperating on one row of an instance (a power of two <= 32).  Rows of
// the batch recipe hold ~1-40 nonzeros: measured on 4096 instances, 2 lanes per
// row (0.325 s per batch mixed, 0.450 s FP64) beat 8 (0.490 / 0.956 s) and 1
// (0.521 / 0.597 s) -- with 8 lanes a row's shuffle reduction and its one-lane
// epilogue cost more than its two or three loads per lane.
#ifndef MPAX_BATCH_LPR
#define MPAX_BATCH_LPR 2
#endif
constexpr int kLPR = MPAX_BATCH_LPR;
// Rows each lane group carries per step of a half-step (their memory round
// trips overlap).  With 2-lane groups a step already covers 256 rows, and 1 row
// per group measured best (0.325 against 0.329 s per 4096-instance batch).
#ifndef MPAX_BATCH_ROWS
#define MPAX_BATCH_ROWS 1
#endif
constexpr int kBR = MPAX_BATCH_ROWS;
// Values and columns each lane loads per row before using any (see rows_dot).
// Measured on 1024 instances of the bench recipe: 1 (0.369 s per batch, mixed)
// beats 2 (0.370 s) and 4 (0.405 s): at 64 registers deeper batches spill.
#ifndef MPAX_BATCH_UNROLL
#define MPAX_BATCH_UNROLL 1
#endif
constexpr int kBU = MPAX_BATCH_UNROLL;
// 1: stage each instance's row pointers in shared memory when two CTAs per SM
//    still fit (<= 100 KB of shared memory per CTA).
#ifndef MPAX_BATCH_SMEM_RP
#define MPAX_BATCH_SMEM_RP 1
#endif

template <typename T>
struct BatchArgs {
  int B;
  const long long* m_off;
  const long long* n_off;
  const int* rp;      // A (block diagonal, global columns)
  const int* col;
  const T* val;
  const int* rpt;     // A^T (columns are global rows of A)
  const int* colt;
  const T* valt;
  const T *c, *l, *u, *lc, *uc;                 // scaled data
  const double *c0, *l0, *u0, *lc0, *uc0, *Dr, *Dc;  // originals and scaling
  T *w, *xa, *xhat, *ya, *yhat, *gbuf;          // iterate storage
  double *xout, *yout;
  int* status;
  long long* iters;
  long long* restarts;
  double *relkkt, *pobj, *secs;
  int* next;
  // Shared-memory pool of a CTA: smem_vec elements for the instance's two
  // gathered vectors (y, m_b entries, then the primal vector, n_b entries) and
  // then rp_cap ints for its row pointers.  An instance with m_b + n_b >
  // smem_vec keeps both vectors in global memory instead (gys, gxs: its slices
  // of two m- and n-vectors); one with m_b + n_b + 2 > rp_cap reads its row
  // pointers in place.
  int smem_vec;
  int rp_cap;
  T* gys;
  T* gxs;
  double eps_abs, eps_rel, r_suff, r_nec, r_art, pw_smooth, step_safety, power_tol;
  long long iter_limit;
  long long time_limit_ns;  // from the start of the launch, on the device clock
  int check_every, power_max_iter;
  const int* todo;  // instances of this launch (nullptr: all B, in order)
  int n_todo;       // work items of this launch
  int warm;         // 1: start from the returned points (xout, yout) instead of zero
  double power_cap; // certified bound on ||A~_b||_2 (1 after Pock-Chambolle, else inf)
  int stall_limit;  // > 0: end an instance whose KKT error stops improving (FP32 floor)
  long long stage_cap;  // bytes of the shared pool an instance may stage whole (0: none)
};

__device__ __forceinline__ double bsum(double v, double* sh) {
  v = block_sum(v, sh);
  __shared__ double bc;
  if (threadIdx.x == 0) bc = v;
  __syncthreads();
  const double r = bc;
  __syncthreads();
  return r;
}

template <typename T>
__device__ __forceinline__ T group_sum(T v) {
#pragma unroll
  for (int o = kLPR / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, kLPR);
  return v;
}

__device__ __forceinline__ double bound_val(double lo, double hi) {
  const bool fl = isfinite(lo), fu = isfinite(hi);
  if (fl && fu) return (fabs(lo) >= fabs(hi)) ? lo : hi;
  if (fl) return lo;
  if (fu) return hi;
  return 0.0;
}

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Dot products of kBR rows (one per slot r, lane offset already in pp[r]) with
// the shared-memory vector vec (columns offset by off): each pass issues up to
// kBU values and columns per row and lane before any of them is used, so a row
// of up to kBU * kLPR nonzeros costs one memory round trip.
template <typename T>
__device__ __forceinline__ void rows_dot(const int* pp, const int* pe, const T* __restrict__ val,
                                         const int* __restrict__ col, const T* vec, int off,
                                         T* sr) {
  for (int base = 0;; base += kBU * kLPR) {
    T v[kBR][kBU];
    int c[kBR][kBU];
    bool any = false;
#pragma unroll
    for (int r = 0; r < kBR; ++r)
#pragma unroll
      for (int u = 0; u < kBU; ++u) {
        const int p = pp[r] + base + u * kLPR;
        if (p < pe[r]) {
          v[r][u] = val[p];
          c[r][u] = col[p];
          any = true;
        }
      }
    if (!any) break;
#pragma unroll
    for (int r = 0; r < kBR; ++r)
#pragma unroll
      for (int u = 0; u < kBU; ++u) {
        const int p = pp[r] + base + u * kLPR;
        if (p < pe[r]) sr[r] += v[r][u] * vec[c[r][u] - off];
      }
  }
}

// Shared-memory pool of an instance run with kStage (T elements, then ints):
// ys[mb] xs[nb] val[z] valt[z] c l u w xa xhat gbuf [nb each] lc uc ya yhat [mb each]
// | rp[mb+1] rpt[nb+1] col[z] colt[z], z the instance's nonzeros.
__host__ __device__ __forceinline__ long long stage_bytes(long long mb, long long nb, long long z,
                                                          int tsize) {
  return tsize * (5 * mb + 8 * nb + 2 * z) + 4 * (mb + nb + 2 + 2 * z);
}

// The arrays of one instance as the loop reads them.  Row pointers index val()
// and col() (global offsets in place, local ones when staged); columns hold
// global indices (less n0 for A, m0 for A^T); vectors are indexed locally.  In
// place, every array is the kernel parameter's pointer plus the instance offset
// (no register holds it); staged, it is the pool position that mb, nb and z fix.
template <typename T, bool kStage>
struct Inst {
  const BatchArgs<T>& a;
  int m0, n0, mb, nb, z;
  const int *rp, *rpt;
  T* sp;  // staged: the pool after ys and xs
#define MPAX_INST_ARR(Type, name, staged, inplace) \
  __device__ __forceinline__ Type* name() const {    \
    if constexpr (kStage) return staged;             \
    else return inplace;                             \
  }
  MPAX_INST_ARR(const T, val, sp, a.val)
  MPAX_INST_ARR(const T, valt, sp + z, a.valt)
  MPAX_INST_ARR(const T, c, sp + 2 * z, a.c + n0)
  MPAX_INST_ARR(const T, l, sp + 2 * z + nb, a.l + n0)
  MPAX_INST_ARR(const T, u, sp + 2 * z + 2 * nb, a.u + n0)
  MPAX_INST_ARR(T, w, sp + 2 * z + 3 * nb, a.w + n0)
  MPAX_INST_ARR(T, xa, sp + 2 * z + 4 * nb, a.xa + n0)
  MPAX_INST_ARR(T, xhat, sp + 2 * z + 5 * nb, a.xhat + n0)
  MPAX_INST_ARR(T, gbuf, sp + 2 * z + 6 * nb, a.gbuf + n0)
  MPAX_INST_ARR(const T, lc, sp + 2 * z + 7 * nb, a.lc + m0)
  MPAX_INST_ARR(const T, uc, sp + 2 * z + 7 * nb + mb, a.uc + m0)
  MPAX_INST_ARR(T, ya, sp + 2 * z + 7 * nb + 2 * mb, a.ya + m0)
  MPAX_INST_ARR(T, yhat, sp + 2 * z + 7 * nb + 3 * mb, a.yhat + m0)
  MPAX_INST_ARR(int, srp, reinterpret_cast<int*>(sp + 2 * z + 7 * nb + 4 * mb), nullptr)
  MPAX_INST_ARR(const int, col, srp() + (mb + 1) + (nb + 1), a.col)
  MPAX_INST_ARR(const int, colt, srp() + (mb + 1) + (nb + 1) + z, a.colt)
#undef MPAX_INST_ARR
};

// kStage: the whole instance -- both matrices, the scaled data and every
// iterate vector -- is copied into the shared pool first, so the loop touches
// global memory only at checks (the unscaled data) and at the end.  Otherwise
// the two gathered vectors sit at ys, xs (shared or global) and the rest is
// read in place, with the row pointers staged at srp when they fit.
template <typename T, bool kStage>
__device__ __forceinline__ void solve_instance(const BatchArgs<T>& a, int b, T* ys, T* xs,
                                               int* srp, double* sh,
                                               unsigned long long t_launch) {
  const unsigned long long t_start = gtimer();
  __shared__ int s_late;
  const int m0 = (int)a.m_off[b], mb = (int)(a.m_off[b + 1] - a.m_off[b]);
  const int n0 = (int)a.n_off[b], nb = (int)(a.n_off[b + 1] - a.n_off[b]);
  const int grp = threadIdx.x / kLPR, gl = threadIdx.x % kLPR;
  const int G = blockDim.x / kLPR;
  const int z0 = a.rp[m0];
  Inst<T, kStage> v{a, m0, n0, mb, nb, a.rp[m0 + mb] - z0, a.rp + m0, a.rpt + n0, xs + nb};
  if constexpr (kStage) {
    // ys (the pool's start) and xs = ys + mb come first; copy the rest in
    const int zt0 = a.rpt[n0];
    int* srp_a = v.srp();
    int* srp_t = srp_a + (mb + 1);
    T* sval = const_cast<T*>(v.val());
    T* svalt = const_cast<T*>(v.valt());
    int* scol = const_cast<int*>(v.col());
    int* scolt = const_cast<int*>(v.colt());
    for (int i = threadIdx.x; i <= mb; i += blockDim.x) srp_a[i] = a.rp[m0 + i] - z0;
    for (int j = threadIdx.x; j <= nb; j += blockDim.x) srp_t[j] = a.rpt[n0 + j] - zt0;
    for (int p = threadIdx.x; p < v.z; p += blockDim.x) {
      sval[p] = a.val[z0 + p];
      scol[p] = a.col[z0 + p];
      svalt[p] = a.valt[zt0 + p];
      scolt[p] = a.colt[zt0 + p];
    }
    T* sc = const_cast<T*>(v.c());
    T* sl = const_cast<T*>(v.l());
    T* su = const_cast<T*>(v.u());
    for (int j = threadIdx.x; j < nb; j += blockDim.x) {
      sc[j] = a.c[n0 + j];
      sl[j] = a.l[n0 + j];
      su[j] = a.u[n0 + j];
    }
    T* slc = const_cast<T*>(v.lc());
    T* suc = const_cast<T*>(v.uc());
    for (int i = threadIdx.x; i < mb; i += blockDim.x) {
      slc[i] = a.lc[m0 + i];
      suc[i] = a.uc[m0 + i];
    }
    __syncthreads();
    v.rp = srp_a;
    v.rpt = srp_t;
  } else if (srp) {
    // Row pointers of A_b and A_b^T: staged in shared memory when they fit (one
    // global round trip less in every step of a half-step), else read in place.
    int* sa = srp;
    int* st = srp + (mb + 1);
    for (int i = threadIdx.x; i <= mb; i += blockDim.x) sa[i] = a.rp[m0 + i];
    for (int j = threadIdx.x; j <= nb; j += blockDim.x) st[j] = a.rpt[n0 + j];
    __syncthreads();
    v.rp = sa;
    v.rpt = st;
  }
  const int* rpl = v.rp;
  const int* rptl = v.rpt;

  // ---- power iteration for ||A~_b||_2 from the common start vector ----------
  double ss0 = 0.0;
  for (int j = threadIdx.x; j < nb; j += blockDim.x) {
    const double r = power_start_raw(j);
    ss0 += r * r;
  }
  const double inv0 = 1.0 / sqrt(fmax(bsum(ss0, sh), 1e-300));
  for (int j = threadIdx.x; j < nb; j += blockDim.x) xs[j] = (T)(power_start_raw(j) * inv0);
  __syncthreads();
  double nA = 0.0, nu_prev = 0.0, d_prev = 0.0;
  const bool has_rows = mb > 0 && rpl[mb] > rpl[0];
  if (has_rows && a.power_max_iter == 0) nA = a.power_cap;  // the certified bound
  for (int t = 1; has_rows && t <= a.power_max_iter; ++t) {
    for (int i0 = 0; i0 < mb; i0 += G) {
      const int i = i0 + grp;
      const bool in_i = i < mb;
      T s = 0;
      for (int p = in_i ? rpl[i] + gl : 0; in_i && p < rpl[i + 1]; p += kLPR)
        s += v.val()[p] * xs[v.col()[p] - n0];
      s = group_sum(s);
      if (gl == 0 && in_i) ys[i] = s;
    }
    __syncthreads();
    double acc = 0.0;
    for (int j0 = 0; j0 < nb; j0 += G) {
      const int j = j0 + grp;
      const bool in_j = j < nb;
      T s = 0;
      for (int p = in_j ? rptl[j] + gl : 0; in_j && p < rptl[j + 1]; p += kLPR)
        s += v.valt()[p] * ys[v.colt()[p] - m0];
      s = group_sum(s);
      if (gl == 0 && in_j) {
        v.gbuf()[j] = s;
        acc += (double)s * (double)s;
      }
    }
    const double nrm = sqrt(bsum(acc, sh));
    if (nrm == 0.0) {
      nA = 0.0;
      break;
    }
    const double nu = sqrt(nrm);
    for (int j = threadIdx.x; j < nb; j += blockDim.x) xs[j] = (T)((double)v.gbuf()[j] / nrm);
    __syncthreads();
    nA = nu;
    double est = nu;
    if (t > 1 && power_stop(nu, nu_prev, &d_prev, a.power_tol, a.power_cap, &est)) {
      nA = est;
      break;
    }
    if (t == a.power_max_iter && isfinite(a.power_cap)) nA = a.power_cap;
    nu_prev = nu;
  }

  // ---- initial primal weight, norms of the unscaled data ------------------
  double s_cs = 0, s_bs = 0, s_c = 0, s_b = 0;
  for (int j = threadIdx.x; j < nb; j += blockDim.x) {
    const double cs = (double)v.c()[j];
    s_cs += cs * cs;
    s_c += a.c0[n0 + j] * a.c0[n0 + j];
  }
  for (int i = threadIdx.x; i < mb; i += blockDim.x) {
    const double bs = bound_val((double)v.lc()[i], (double)v.uc()[i]);
    const double bo = bound_val(a.lc0[m0 + i], a.uc0[m0 + i]);
    s_bs += bs * bs;
    s_b += bo * bo;
  }
  const double ncs = sqrt(bsum(s_cs, sh)), nbs = sqrt(bsum(s_bs, sh));
  const double c_norm = sqrt(bsum(s_c, sh)), b_norm = sqrt(bsum(s_b, sh));
  double omega = (ncs > 1e-10 && nbs > 1e-10) ? ncs / nbs : 1.0;
  const double eta = nA > 0.0 ? a.step_safety / nA : 1.0;
  double tau = eta / omega, sigma = eta * omega;

  // ---- start at zero, or (warm) at the returned point of an earlier launch,
  // taken back into the scaled space: anchor, reflected point, duals ---------
  for (int j = threadIdx.x; j < nb; j += blockDim.x) {
    const T x = a.warm ? (T)(a.xout[n0 + j] / a.Dc[n0 + j]) : (T)0;
    v.xa()[j] = x;
    v.w()[j] = x;
    v.xhat()[j] = x;
  }
  for (int i = threadIdx.x; i < mb; i += blockDim.x) {
    const T y = a.warm ? (T)(a.yout[m0 + i] / a.Dr[m0 + i]) : (T)0;
    ys[i] = y;
    v.ya()[i] = y;
    v.yhat()[i] = y;
  }
  __syncthreads();

  long long total = 0, k = 0, restarts = 0;
  double r_anchor = 0.0, r_prev = 0.0, rel = INFINITY, pobj = 0.0;
  bool have_anchor = false;
  int term = 0;
  long long checks = 0, stall_count = 0;
  double best_rel = INFINITY;
  while (true) {
    const int len = (int)min((long long)a.check_every, a.iter_limit - total);
    double P0 = 0, P1 = 0, D0 = 0, D1 = 0;
    const T tt = (T)tau, ss = (T)sigma, iss = (T)(1.0 / sigma);
    for (int it = 0; it < len; ++it) {
      const bool chk = (it == len - 1);
      const T rb = (T)(1.0 / (double)(k + 1));  // rebuild weight of x^{n,k}
      const T hb = (T)(1.0 / (double)(k + 2));  // Halpern weight of the anchor
      // primal half-step over the rows of A^T (eq. 3, first line).  Each kLPR-lane
      // group takes kBR rows per step (j, j + G, ...) and issues the row pointers,
      // the epilogue operands and both rows' products before reducing, so every
      // dependent round trip to memory is shared by kBR rows.
      for (int j0 = 0; j0 < nb; j0 += kBR * G) {
        int jr[kBR], pp[kBR], pe[kBR];
        T sr[kBR], x0r[kBR], wr[kBR], cr[kBR], lr[kBR], ur[kBR];
#pragma unroll
        for (int r = 0; r < kBR; ++r) {
          jr[r] = j0 + r * G + grp;
          const bool in = jr[r] < nb;
          pp[r] = in ? rptl[jr[r]] + gl : 0;
          pe[r] = in ? rptl[jr[r] + 1] : 0;
          sr[r] = 0;
          if (gl == 0 && in) {
            const int j = jr[r];
            x0r[r] = v.xa()[j];
            wr[r] = v.w()[j];
            cr[r] = v.c()[j];
            lr[r] = v.l()[j];
            ur[r] = v.u()[j];
          }
        }
        rows_dot<T>(pp, pe, v.valt(), v.colt(), ys, m0, sr);
#pragma unroll
        for (int r = 0; r < kBR; ++r) sr[r] = group_sum(sr[r]);
        if (gl == 0) {
#pragma unroll
          for (int r = 0; r < kBR; ++r) {
            if (jr[r] >= nb) continue;
            const int j = jr[r];
            const T x0 = x0r[r], wv = wr[r];
            const T x = (k == 0) ? x0 : wv + rb * (x0 - wv);
            const T xh = clampv<T>(x - tt * (cr[r] - sr[r]), lr[r], ur[r]);
            const T wn = (T)2 * xh - x;
            v.w()[j] = wn;
            xs[j] = wn;
            if (chk) {
              v.xhat()[j] = xh;
              const double d0 = (double)xh - (double)x, d1 = (double)xh - (double)x0;
              P0 += d0 * d0;
              P1 += d1 * d1;
            }
          }
        }
      }
      __syncthreads();
      // dual half-step over the rows of A (eq. 3, second line) and Halpern (eq. 4),
      // kBR rows per group and step as above
      for (int i0 = 0; i0 < mb; i0 += kBR * G) {
        int ir[kBR], pp[kBR], pe[kBR];
        T sr[kBR], yar[kBR], lcr[kBR], ucr[kBR];
#pragma unroll
        for (int r = 0; r < kBR; ++r) {
          ir[r] = i0 + r * G + grp;
          const bool in = ir[r] < mb;
          pp[r] = in ? rpl[ir[r]] + gl : 0;
          pe[r] = in ? rpl[ir[r] + 1] : 0;
          sr[r] = 0;
          if (gl == 0 && in) {
            const int i = ir[r];
            yar[r] = v.ya()[i];
            lcr[r] = v.lc()[i];
            ucr[r] = v.uc()[i];
          }
        }
        rows_dot<T>(pp, pe, v.val(), v.col(), xs, n0, sr);
#pragma unroll
        for (int r = 0; r < kBR; ++r) sr[r] = group_sum(sr[r]);
        if (gl == 0) {
#pragma unroll
          for (int r = 0; r < kBR; ++r) {
            if (ir[r] >= mb) continue;
            const int i = ir[r];
            const T y0 = ys[i], y0a = yar[r];
            const T t = y0 * iss - sr[r];
            const T yh = ss * (t - clampv<T>(t, -ucr[r], -lcr[r]));
            const T z = (T)2 * yh - y0;
            ys[i] = z + hb * (y0a - z);
            if (chk) {
              v.yhat()[i] = yh;
              const double d0 = (double)yh - (double)y0, d1 = (double)yh - (double)y0a;
              D0 += d0 * d0;
              D1 += d1 * d1;
            }
          }
        }
      }
      __syncthreads();
      ++k;
      ++total;
    }
    // ---- check: relative KKT error of (x^, y^) on the unscaled problem ----
    for (int j = threadIdx.x; j < nb; j += blockDim.x) xs[j] = v.xhat()[j];
    __syncthreads();
    double K0 = 0, K1 = 0, C0 = 0, C1 = 0, C2 = 0;
    for (int i0 = 0; i0 < mb; i0 += G) {
      const int i = i0 + grp;
      const bool in_i = i < mb;
      T s = 0;
      for (int p = in_i ? rpl[i] + gl : 0; in_i && p < rpl[i + 1]; p += kLPR)
        s += v.val()[p] * xs[v.col()[p] - n0];
      s = group_sum(s);
      if (gl == 0 && in_i) {
        const int g = m0 + i;
        const double ax = (double)s / a.Dr[g];
        const double lo = a.lc0[g], hi = a.uc0[g];
        const double r = ax - fmin(fmax(ax, lo), hi);
        K0 += r * r;
        const double y = a.Dr[g] * (double)v.yhat()[i];
        if (y > 0.0 && isfinite(lo)) K1 += lo * y;
        if (y < 0.0 && isfinite(hi)) K1 += hi * y;
      }
    }
    for (int j0 = 0; j0 < nb; j0 += G) {
      const int j = j0 + grp;
      const bool in_j = j < nb;
      T s = 0;
      for (int p = in_j ? rptl[j] + gl : 0; in_j && p < rptl[j + 1]; p += kLPR)
        s += v.valt()[p] * v.yhat()[v.colt()[p] - m0];
      s = group_sum(s);
      if (gl == 0 && in_j) {
        const int g = n0 + j;
        const double aty = (double)s / a.Dc[g];
        const double x = a.Dc[g] * (double)xs[j];
        const double lam = a.c0[g] - aty;
        const double lo = a.l0[g], hi = a.u0[g];
        const bool lf = isfinite(lo), uf = isfinite(hi);
        const double lh = (lf && uf) ? lam : lf ? fmax(lam, 0.0) : uf ? fmin(lam, 0.0) : 0.0;
        const double rd = lam - lh;
        C0 += rd * rd;
        C1 += a.c0[g] * x;
        C2 += (lf ? lo * fmax(lh, 0.0) : 0.0) + (uf ? hi * fmin(lh, 0.0) : 0.0);
      }
    }
    P0 = bsum(P0, sh);
    P1 = bsum(P1, sh);
    D0 = bsum(D0, sh);
    D1 = bsum(D1, sh);
    K0 = bsum(K0, sh);
    K1 = bsum(K1, sh);
    C0 = bsum(C0, sh);
    C1 = bsum(C1, sh);
    C2 = bsum(C2, sh);
    const double nrp = sqrt(K0), nrd = sqrt(C0);
    pobj = C1;
    const double dobj = K1 + C2;
    const double gap = fabs(pobj - dobj);
    rel = fmax(fmax(nrp / (1.0 + b_norm), nrd / (1.0 + c_norm)),
               gap / (1.0 + fabs(pobj) + fabs(dobj)));
    const bool conv = nrp <= a.eps_abs + a.eps_rel * b_norm &&
                      nrd <= a.eps_abs + a.eps_rel * c_norm &&
                      gap <= a.eps_abs + a.eps_rel * (fabs(pobj) + fabs(dobj));
    if (!isfinite(rel) || !isfinite(P0) || !isfinite(D0)) term = MPAX_TERM_NUMERICAL_ERROR;
    else if (conv) term = MPAX_TERM_OPTIMAL;
    else if (total >= a.iter_limit) term = MPAX_TERM_ITERATION_LIMIT;
    // one thread reads the clock so that the decision is uniform over the block
    if (threadIdx.x == 0) s_late = (long long)(gtimer() - t_launch) >= a.time_limit_ns;
    __syncthreads();
    if (!term && s_late) term = MPAX_TERM_TIME_LIMIT;
    __syncthreads();
    // the FP32 floor: no 10% improvement of the KKT error over stall_limit
    // checks.  Unlike the single-problem rule the window does not grow: a batch
    // instance is small and latency-bound, FP64 costs it about twice per
    // iteration, and an FP32 run that keeps finding slightly lower minima while
    // it drifts would otherwise run on.  Every quantity here is uniform over the
    // block.
    ++checks;
    if (!term && a.stall_limit > 0) {
      const long long window = a.stall_limit;
      if (rel < 0.9 * best_rel) {
        best_rel = rel;
        stall_count = 0;
      } else if (++stall_count >= window) {
        term = kTermStalled;
      }
    }
    if (term) break;
    // restart rule and primal weight (the same rule as the single-problem path)
    const double r = sqrt(omega * P0 + D0 / omega);
    const bool restart = !have_anchor || r <= a.r_suff * r_anchor ||
                         (r <= a.r_nec * r_anchor && r > r_prev) ||
                         (double)k >= a.r_art * (double)total;
    if (restart) {
      const double dx = sqrt(P1), dy = sqrt(D1);
      if (dx > 1e-10 && dy > 1e-10)
        omega = exp(a.pw_smooth * log(dy / dx) + (1.0 - a.pw_smooth) * log(omega));
      tau = eta / omega;
      sigma = eta * omega;
      have_anchor = true;
      r_anchor = r;
      r_prev = r;
      k = 0;
      ++restarts;
      for (int j = threadIdx.x; j < nb; j += blockDim.x) {
        const T x = v.xhat()[j];
        v.xa()[j] = x;
        v.w()[j] = x;
      }
      for (int i = threadIdx.x; i < mb; i += blockDim.x) {
        const T y = v.yhat()[i];
        v.ya()[i] = y;
        ys[i] = y;
      }
    } else {
      r_prev = r;
    }
    __syncthreads();
  }
  // ---- returned point (x^, y^), unscaled; per-instance statistics ---------
  for (int j = threadIdx.x; j < nb; j += blockDim.x)
    a.xout[n0 + j] = a.Dc[n0 + j] * (double)v.xhat()[j];
  for (int i = threadIdx.x; i < mb; i += blockDim.x)
    a.yout[m0 + i] = a.Dr[m0 + i] * (double)v.yhat()[i];
  if (threadIdx.x == 0) {
    // a warm launch continues an instance: its counts and time add to the earlier ones
    a.status[b] = term;
    a.iters[b] = (a.warm ? a.iters[b] : 0) + total;
    a.restarts[b] = (a.warm ? a.restarts[b] : 0) + restarts;
    a.relkkt[b] = rel;
    a.pobj[b] = pobj;
    a.secs[b] = (a.warm ? a.secs[b] : 0.0) + (double)(gtimer() - t_start) * 1e-9;
  }
  __syncthreads();
}

// kStaging: the launch may stage whole instances (a separate instantiation, so
// that the many-instance kernel carries only the two in-place call sites).
template <typename T, bool kStaging>
__global__ void __launch_bounds__(kBatchThreads<T>, kBatchMinB<T>) batch_lp_kernel(BatchArgs<T> a) {
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ double sh[32];
  __shared__ int s_inst;
  T* pool = reinterpret_cast<T*>(sm);
  int* rpool = reinterpret_cast<int*>(pool + a.smem_vec);
  const unsigned long long t_launch = gtimer();  // used by thread 0 only
  while (true) {
    if (threadIdx.x == 0) s_inst = atomicAdd(a.next, 1);
    __syncthreads();
    const int w = s_inst;
    __syncthreads();
    if (w >= a.n_todo) return;
    const int b = a.todo ? a.todo[w] : w;
    const int mb = (int)(a.m_off[b + 1] - a.m_off[b]), nb = (int)(a.n_off[b + 1] - a.n_off[b]);
    const int z = a.rp[a.m_off[b + 1]] - a.rp[a.m_off[b]];
    int* srp = (mb + nb + 2 <= a.rp_cap) ? rpool : nullptr;
    // three call sites: the whole instance in shared memory; its two gathered
    // vectors in shared memory (shared loads for the gathers); everything global
    if (kStaging && stage_bytes(mb, nb, z, (int)sizeof(T)) <= a.stage_cap)
      solve_instance<T, true>(a, b, pool, pool + mb, nullptr, sh, t_launch);
    else if (mb + nb <= a.smem_vec)
      solve_instance<T, false>(a, b, pool, pool + mb, srp, sh, t_launch);
    else
      solve_instance<T, false>(a, b, a.gys + a.m_off[b], a.gxs + a.n_off[b], srp, sh, t_launch);
  }
}

// z[b] = rp[m_off[b]], b = 0..B
__global__ void k_first_nnz(const long long* __restrict__ rp, const long long* __restrict__ m_off,
                            int B, long long* __restrict__ z) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b <= B) z[b] = rp[m_off[b]];
}

// row -> instance via binary search in m_off; global column = n_off[b] + local
__global__ void k_globalize_cols(const long long* __restrict__ m_off,
                                 const long long* __restrict__ n_off, int B,
                                 const long long* __restrict__ rp, int rows,
                                 int* __restrict__ col, int* flags) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows) return;
  int lo = 0, hi = B;  // find b with m_off[b] <= i < m_off[b+1]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (m_off[mid] <= i) lo = mid;
    else hi = mid;
  }
  const long long nb = n_off[lo + 1] - n_off[lo];
  for (long long p = rp[i]; p < rp[i + 1]; ++p) {
    const int c = col[p];
    if (c < 0 || c >= nb) atomicOr(flags, 1);
    col[p] = (int)(n_off[lo] + c);
  }
}

// ---- B copies of one LP's constraints (the replicated batch) -----------------
__global__ void k_rep_rowptr(const long long* __restrict__ rp, int m, long long nnz, int B,
                             long long* __restrict__ out) {
  const long long total = (long long)B * m;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const long long b = t / m, i = t - b * m;
    out[t + 1] = rp[i + 1] + b * nnz;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) out[0] = 0;
}

template <typename V>
__global__ void k_tile(const V* __restrict__ src, long long len, int B, V* __restrict__ dst) {
  const long long total = len * B;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x)
    dst[t] = src[t % len];
}

// ---- SPO+ (Sec. 3.4): the surrogate loss of predicted costs ------------------
// c' = 2 c_hat - c_true, the costs of the solve that gives x~.
__global__ void k_spo_costs(const double* __restrict__ c_hat, const double* __restrict__ c_true,
                            long long len, double* __restrict__ out) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < len;
       t += (long long)gridDim.x * blockDim.x)
    out[t] = 2.0 * c_hat[t] - c_true[t];
}

// One block per instance b (coordinates [off[b], off[b+1]), or b*n.. with off
// null): loss_b = -c'^T x~ + 2 c_hat^T x* - z*_b and grad = 2 (x* - x~), where
// x~ minimises c'^T x (Elmachtoub and Grigas 2022).  Fixed-order FP64 sums.
__global__ void k_spo_loss(const long long* __restrict__ off, int n, const double* __restrict__ cp,
                           const double* __restrict__ c_hat, const double* __restrict__ x_true,
                           const double* __restrict__ z_true, const double* __restrict__ x_tl,
                           double* __restrict__ loss, double* __restrict__ grad) {
  __shared__ double sh[32];
  const int b = blockIdx.x;
  const long long j0 = off ? off[b] : (long long)b * n, j1 = off ? off[b + 1] : j0 + n;
  double v = 0.0, t = 0.0;
  for (long long j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
    const double xt = x_tl[j], xs = x_true[j];
    v += cp[j] * xt;
    t += c_hat[j] * xs;
    grad[j] = 2.0 * (xs - xt);
  }
  v = block_sum(v, sh);
  __syncthreads();
  t = block_sum(t, sh);
  if (threadIdx.x == 0) loss[b] = -v + 2.0 * t - z_true[b];
}

}  // namespace mpax

// ============================================================================

using namespace mpax;

struct mpax_batch {
  mpax_problem* prob = nullptr;  // the block-diagonal problem
  int B = 0;
  long long* m_off = nullptr;  // device
  long long* n_off = nullptr;
  std::vector<long long> h_moff, h_noff;
  std::vector<long long> h_zoff;  // row_ptr at each instance's first row
  int max_m = 0, max_n = 0;
  int* next = nullptr;
  int* status = nullptr;
  long long* iters = nullptr;
  long long* restarts = nullptr;
  double *relkkt = nullptr, *pobj = nullptr, *secs = nullptr, *xout = nullptr, *yout = nullptr;
  void* work = nullptr;  // iterate storage and scaled data (precision dependent)
  size_t work_bytes = 0;
  bool solved = false;
  double solve_seconds = 0.0;
  long long launches = 0;
  int* todo = nullptr;     // device list of instances continued in FP64
  int fp64_instances = 0;  // instances of the last solve continued in FP64
  double* spo = nullptr;   // SPO+ staging of host arguments: 3 sum(n) + B doubles
};

namespace mpax {
// defined in api.cu
ProblemData* problem_data(mpax_problem* p);
cudaStream_t problem_stream(mpax_problem* p);
void problem_order_after_user(mpax_problem* p);
void problem_order_user_after(mpax_problem* p);
}  // namespace mpax

namespace {

mpax_status bfail(mpax_status s, const std::string& m) {
  set_last_error(m.c_str());
  return s;
}

// Bytes of shared memory an instance's two vectors may take (larger instances
// keep them in global memory).
constexpr long long kBatchVecBytes = 200 * 1024;
// Shared-memory bytes an instance may stage whole (matrices, data and iterates)
// when the launch has at most one instance per SM.  With more instances nothing
// is staged whole: a pool of that size shrinks the L1 share of every CTA, and
// on 4096 instances of the ragged recipe (about 15% small enough at 100 KB)
// the batch took 0.57 s against 0.35 s without.
constexpr long long kStageFew = 200 * 1024;

// The arguments and shared-memory size of one batch launch in precision T.
template <typename T>
struct BatchLaunch {
  BatchArgs<T> a;
  size_t smem = 0;
};

// Scaled data and iterate storage of the launch in T (in *work, grown to fit),
// its arguments and its shared-memory pool; allow_stage: whole instances may be
// staged.
template <typename T>
mpax_status batch_prepare(mpax_batch* bt, const mpax_options* o, long long* launches,
                          const int* todo, const int* todo_host, int n_todo, int warm,
                          int stall_limit, bool allow_stage, void** work, size_t* work_bytes,
                          BatchLaunch<T>* L) {
  ProblemData& P = *problem_data(bt->prob);
  cudaStream_t s = P.s;
  const int m = P.m, n = P.n, nnz = P.nnz;
  // scaled data and iterate storage in the iteration precision
  const size_t need =
      sizeof(T) * ((size_t)2 * (nnz + kPad) + 10 * (size_t)n + 8 * (size_t)m + 96);
  if (*work_bytes < need) {
    if (*work) cudaFree(*work);
    *work = nullptr;
    *work_bytes = 0;
    if (cudaMalloc(work, need) != cudaSuccess) return bfail(MPAX_ERR_OUT_OF_MEMORY, "batch work");
    *work_bytes = need;
  }
  T* p = reinterpret_cast<T*>(*work);
  auto take = [&](size_t k) {
    T* r = p;
    p += (k + 15) / 16 * 16;
    return r;
  };
  T* valA = take(nnz + kPad);
  T* valAt = take(nnz + kPad);
  T *c = take(n), *l = take(n), *u = take(n), *lc = take(m), *uc = take(m);
  T *w = take(n), *xa = take(n), *xhat = take(n), *gbuf = take(n);
  T *ya = take(m), *yhat = take(m);
  T *gys = take(m), *gxs = take(n);
  cudaError_t e;
  if ((e = cast_vec<T>(P.val_s, valA, nnz, s))) return bfail(MPAX_ERR_CUDA, cudaGetErrorString(e));
  if ((e = gather_cast<T>(P.val_s, P.permT, valAt, nnz, s)))
    return bfail(MPAX_ERR_CUDA, cudaGetErrorString(e));
  scale_cast<T>(P.c, P.Dc, false, c, n, s);
  scale_cast<T>(P.l, P.Dc, true, l, n, s);
  scale_cast<T>(P.u, P.Dc, true, u, n, s);
  scale_cast<T>(P.lc, P.Dr, false, lc, m, s);
  scale_cast<T>(P.uc, P.Dr, false, uc, m, s);
  *launches += 7;
  BatchArgs<T>& a = L->a;
  a.B = bt->B;
  a.m_off = bt->m_off;
  a.n_off = bt->n_off;
  a.rp = P.A.rp;
  a.col = P.A.col;
  a.val = valA;
  a.rpt = P.At.rp;
  a.colt = P.At.col;
  a.valt = valAt;
  a.c = c;
  a.l = l;
  a.u = u;
  a.lc = lc;
  a.uc = uc;
  a.c0 = P.c;
  a.l0 = P.l;
  a.u0 = P.u;
  a.lc0 = P.lc;
  a.uc0 = P.uc;
  a.Dr = P.Dr;
  a.Dc = P.Dc;
  a.w = w;
  a.xa = xa;
  a.xhat = xhat;
  a.ya = ya;
  a.yhat = yhat;
  a.gbuf = gbuf;
  a.xout = bt->xout;
  a.yout = bt->yout;
  a.status = bt->status;
  a.iters = bt->iters;
  a.restarts = bt->restarts;
  a.relkkt = bt->relkkt;
  a.pobj = bt->pobj;
  a.secs = bt->secs;
  a.next = bt->next;
  a.gys = gys;
  a.gxs = gxs;
  a.eps_abs = o->eps_abs;
  a.eps_rel = o->eps_rel;
  a.r_suff = o->restart_sufficient;
  a.r_nec = o->restart_necessary;
  a.r_art = o->restart_artificial;
  a.pw_smooth = o->primal_weight_smoothing;
  a.step_safety = o->step_safety;
  a.power_tol = o->power_tol;
  a.iter_limit = o->iteration_limit;
  // the whole batch is one launch: it always ends, at the latest kBatchMaxSeconds
  // after it starts, even with no iteration or time limit given
  a.time_limit_ns = (long long)(std::min(o->time_limit, kBatchMaxSeconds) * 1e9);
  a.check_every = o->check_every;
  a.power_max_iter = o->power_max_iter;
  a.power_cap = o->pock_chambolle ? 1.0 : INFINITY;
  // the shared pool fits the largest instance of this launch that fits in
  // kBatchVecBytes; larger instances run from global memory
  const long long vec_cap = kBatchVecBytes / (long long)sizeof(T);
  long long vmax = 0, rmax = 0;
  for (int w = 0; w < n_todo; ++w) {
    const int b = todo_host ? todo_host[w] : w;
    const long long v = (bt->h_moff[b + 1] - bt->h_moff[b]) + (bt->h_noff[b + 1] - bt->h_noff[b]);
    if (v <= vec_cap) vmax = std::max(vmax, v);
    rmax = std::max(rmax, v + 2);
  }
  a.smem_vec = (int)((vmax + 3) / 4 * 4);
  size_t smem = sizeof(T) * (size_t)a.smem_vec;
  // row pointers staged when two CTAs per SM still fit
  a.rp_cap = (MPAX_BATCH_SMEM_RP && smem + sizeof(int) * (size_t)rmax <= 100 * 1024)
                 ? (int)rmax : 0;
  smem += sizeof(int) * (size_t)a.rp_cap;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // whole-instance staging when every instance of the launch has an SM of its own
  const long long cap = (allow_stage && o->batch_stage && n_todo <= sms) ? kStageFew : 0;
  long long smax = 0;
  for (int w = 0; w < n_todo; ++w) {
    const int b = todo_host ? todo_host[w] : w;
    const long long need = stage_bytes(bt->h_moff[b + 1] - bt->h_moff[b],
                                       bt->h_noff[b + 1] - bt->h_noff[b],
                                       bt->h_zoff[b + 1] - bt->h_zoff[b], (int)sizeof(T));
    if (need <= cap) smax = std::max(smax, need);
  }
  a.stage_cap = smax;
  L->smem = std::max(smem, (size_t)((smax + 15) / 16 * 16));
  a.todo = todo;
  a.n_todo = n_todo;
  a.warm = warm;
  a.stall_limit = stall_limit;
  if ((e = cudaGetLastError())) return bfail(MPAX_ERR_CUDA, cudaGetErrorString(e));
  return MPAX_OK;
}

// Resident CTAs of `kernel` on the whole GPU (at least one per SM).
template <class K>
int batch_grid(K kernel, int threads, size_t smem, int n_todo) {
  int occ = 0, dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, threads, smem);
  return std::min(n_todo, std::max(1, occ) * sms);
}

template <typename T>
mpax_status run_batch(mpax_batch* bt, const mpax_options* o, long long* launches,
                      const int* todo, const int* todo_host, int n_todo, int warm,
                      int stall_limit) {
  BatchLaunch<T> L;
  mpax_status st = batch_prepare<T>(bt, o, launches, todo, todo_host, n_todo, warm, stall_limit,
                                    true, &bt->work, &bt->work_bytes, &L);
  if (st) return st;
  cudaStream_t s = problem_data(bt->prob)->s;
  auto kernel = L.a.stage_cap > 0 ? batch_lp_kernel<T, true> : batch_lp_kernel<T, false>;
  const int grid = batch_grid(kernel, kBatchThreads<T>, L.smem, n_todo);
  cudaMemsetAsync(bt->next, 0, sizeof(int), s);
  kernel<<<grid, kBatchThreads<T>, L.smem, s>>>(L.a);
  *launches += 1;
  cudaError_t e = cudaGetLastError();
  if (e) return bfail(MPAX_ERR_CUDA, cudaGetErrorString(e));
  return MPAX_OK;
}

}  // namespace

extern "C" {

mpax_status mpax_lp_batch_create(int32_t B, const int64_t* m_off, const int64_t* n_off,
                                 const int64_t* row_ptr, const int32_t* col_idx,
                                 const double* val, const double* c, const double* lc,
                                 const double* uc, const double* l, const double* u,
                                 mpax_mem_kind kind, void* cuda_stream, mpax_batch** out) {
  if (!out) return bfail(MPAX_ERR_INVALID_ARGUMENT, "out must not be NULL");
  *out = nullptr;
  if (B < 1) return bfail(MPAX_ERR_INVALID_ARGUMENT, "B must be >= 1");
  if (!m_off || !n_off || !row_ptr) return bfail(MPAX_ERR_INVALID_ARGUMENT, "NULL offsets");
  std::vector<long long> hm(B + 1), hn(B + 1);
  const cudaMemcpyKind k = kind == MPAX_MEM_HOST ? cudaMemcpyHostToHost : cudaMemcpyDeviceToHost;
  if (cudaMemcpy(hm.data(), m_off, sizeof(long long) * (B + 1), k) != cudaSuccess ||
      cudaMemcpy(hn.data(), n_off, sizeof(long long) * (B + 1), k) != cudaSuccess)
    return bfail(MPAX_ERR_CUDA, "copy of the offsets failed");
  if (hm[0] != 0 || hn[0] != 0) return bfail(MPAX_ERR_INVALID_ARGUMENT, "offsets must start at 0");
  int max_m = 0, max_n = 0;
  for (int b = 0; b < B; ++b) {
    if (hm[b + 1] < hm[b] || hn[b + 1] < hn[b])
      return bfail(MPAX_ERR_INVALID_ARGUMENT, "offsets must be non-decreasing");
    max_m = std::max<long long>(max_m, hm[b + 1] - hm[b]);
    max_n = std::max<long long>(max_n, hn[b + 1] - hn[b]);
  }
  if (hm[B] >= (1LL << 31) || hn[B] >= (1LL << 31))
    return bfail(MPAX_ERR_UNSUPPORTED, "total rows and columns must be < 2^31");
  const int m = (int)hm[B], n = (int)hn[B];
  long long nnz = 0;
  if (cudaMemcpy(&nnz, row_ptr + m, sizeof(long long), k) != cudaSuccess)
    return bfail(MPAX_ERR_CUDA, "copy of row_ptr failed");
  // device copies of the structure with columns made global
  long long *d_moff = nullptr, *d_noff = nullptr, *d_rp = nullptr;
  int *d_col = nullptr, *flags = nullptr;
  cudaError_t e = cudaMalloc(&d_moff, sizeof(long long) * (B + 1));
  if (!e) e = cudaMalloc(&d_noff, sizeof(long long) * (B + 1));
  if (!e) e = cudaMalloc(&d_rp, sizeof(long long) * (m + 1));
  if (!e) e = cudaMalloc(&d_col, sizeof(int) * std::max<long long>(nnz, 1));
  if (!e) e = cudaMalloc(&flags, sizeof(int));
  if (!e) e = cudaMemcpy(d_moff, hm.data(), sizeof(long long) * (B + 1), cudaMemcpyHostToDevice);
  if (!e) e = cudaMemcpy(d_noff, hn.data(), sizeof(long long) * (B + 1), cudaMemcpyHostToDevice);
  const cudaMemcpyKind kin = kind == MPAX_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  if (!e) e = cudaMemcpy(d_rp, row_ptr, sizeof(long long) * (m + 1), kin);
  if (!e && nnz > 0) e = cudaMemcpy(d_col, col_idx, sizeof(int) * nnz, kin);
  // row_ptr at each instance's first row (sizes the whole-instance staging)
  std::vector<long long> hz(B + 1);
  long long* d_z = nullptr;
  if (!e) e = cudaMalloc(&d_z, sizeof(long long) * (B + 1));
  if (!e) k_first_nnz<<<(B + 256) / 256, 256>>>(d_rp, d_moff, B, d_z);
  if (!e) e = cudaMemcpy(hz.data(), d_z, sizeof(long long) * (B + 1), cudaMemcpyDeviceToHost);
  if (d_z) cudaFree(d_z);
  if (!e) e = cudaMemset(flags, 0, sizeof(int));
  if (!e && m > 0) k_globalize_cols<<<(m + 255) / 256, 256>>>(d_moff, d_noff, B, d_rp, m, d_col, flags);
  int hf = 0;
  if (!e) e = cudaMemcpy(&hf, flags, sizeof(int), cudaMemcpyDeviceToHost);
  mpax_problem* prob = nullptr;
  mpax_status st = MPAX_OK;
  if (!e && hf) st = bfail(MPAX_ERR_INVALID_ARGUMENT, "a column index is outside its instance");
  if (!e && !hf) {
    // values and vectors go through the single-problem create (copy + validation);
    // host inputs are staged on the device first so that every pointer is device memory
    const double* dv[6] = {val, c, lc, uc, l, u};
    const long long cnt[6] = {nnz, n, m, m, n, n};
    double* tmp[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    if (kind == MPAX_MEM_HOST) {
      for (int q = 0; q < 6 && !e; ++q) {
        e = cudaMalloc(&tmp[q], sizeof(double) * std::max<long long>(cnt[q], 1));
        if (!e && cnt[q] > 0) e = cudaMemcpy(tmp[q], dv[q], sizeof(double) * cnt[q], cudaMemcpyHostToDevice);
        dv[q] = tmp[q];
      }
    }
    if (!e)
      st = mpax_lp_create(m, n, nnz, (const int64_t*)d_rp, d_col, dv[0], dv[1], dv[2], dv[3],
                          dv[4], dv[5], MPAX_MEM_DEVICE, cuda_stream, &prob);
    for (double* t : tmp)
      if (t) cudaFree(t);
  }
  cudaFree(d_rp);
  cudaFree(d_col);
  cudaFree(flags);
  if (e) {
    cudaFree(d_moff);
    cudaFree(d_noff);
    return bfail(MPAX_ERR_CUDA, cudaGetErrorString(e));
  }
  if (st) {
    cudaFree(d_moff);
    cudaFree(d_noff);
    return st;
  }
  mpax_batch* bt = new mpax_batch();
  e = cudaMalloc(&bt->next, sizeof(int));
  if (!e) e = cudaMalloc(&bt->status, sizeof(int) * B);
  if (!e) e = cudaMalloc(&bt->iters, sizeof(long long) * B);
  if (!e) e = cudaMalloc(&bt->restarts, sizeof(long long) * B);
  if (!e) e = cudaMalloc(&bt->relkkt, sizeof(double) * B);
  if (!e) e = cudaMalloc(&bt->pobj, sizeof(double) * B);
  if (!e) e = cudaMalloc(&bt->secs, sizeof(double) * B);
  if (!e) e = cudaMalloc(&bt->xout, sizeof(double) * std::max(n, 1));
  if (!e) e = cudaMalloc(&bt->yout, sizeof(double) * std::max(m, 1));
  bt->prob = prob;
  bt->B = B;
  bt->m_off = d_moff;
  bt->n_off = d_noff;
  bt->h_moff = hm;
  bt->h_noff = hn;
  bt->h_zoff = hz;
  bt->max_m = max_m;
  bt->max_n = max_n;
  if (e) {
    mpax_batch_destroy(bt);
    return bfail(MPAX_ERR_OUT_OF_MEMORY, "batch output arrays");
  }
  *out = bt;
  return MPAX_OK;
}

mpax_status mpax_batch_solve(mpax_batch* bt, const mpax_options* o) {
  if (!bt || !o) return bfail(MPAX_ERR_INVALID_ARGUMENT, "NULL argument");
  if (o->reflection_gamma != 1.0)
    return bfail(MPAX_ERR_UNSUPPORTED, "the batch path implements reflection_gamma = 1");
  if (o->check_every < 1 || o->iteration_limit < 1 || o->ruiz_iters < 0 ||
      !(o->step_safety > 0 && o->step_safety < 1) || o->power_max_iter < 0 ||
      (o->power_max_iter == 0 && !o->pock_chambolle) ||
      !(o->time_limit >= 0) || (o->batch_stage != 0 && o->batch_stage != 1))
    return bfail(MPAX_ERR_INVALID_ARGUMENT, "invalid options");
  if (o->precision != MPAX_PREC_FP64 && o->precision != MPAX_PREC_MIXED)
    return bfail(MPAX_ERR_INVALID_ARGUMENT, "bad precision");
  const auto t0 = std::chrono::steady_clock::now();
  ProblemData& P = *problem_data(bt->prob);
  cudaStream_t s = P.s;
  problem_order_after_user(bt->prob);
  long long launches = 0;
  cudaError_t e = transpose_csr(P.A, P.At, P.permT, P.tmp_rows, P.tmp_scan, s);
  if (!e) e = compute_scaling(P, o->ruiz_iters, o->pock_chambolle != 0);
  launches += 6 + 5 * o->ruiz_iters + 8;
  if (e) return bfail(MPAX_ERR_CUDA, cudaGetErrorString(e));
  const bool cont = o->precision == MPAX_PREC_MIXED && o->fp64_continuation;
  mpax_status st =
      o->precision == MPAX_PREC_FP64
          ? run_batch<double>(bt, o, &launches, nullptr, nullptr, bt->B, 0, 0)
          : run_batch<float>(bt, o, &launches, nullptr, nullptr, bt->B, 0,
                             cont ? o->stall_checks : 0);
  if (st) return st;
  if (cont) {
    // FP64 continuation of the instances that stalled in FP32, warm-started
    // from their returned points, in one more persistent launch
    std::vector<int> hs(bt->B), todo;
    e = cudaMemcpyAsync(hs.data(), bt->status, sizeof(int) * bt->B, cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaStreamSynchronize(s);
    if (e) return bfail(MPAX_ERR_CUDA, cudaGetErrorString(e));
    for (int b = 0; b < bt->B; ++b)
      if (hs[b] == kTermStalled) todo.push_back(b);
    bt->fp64_instances = (int)todo.size();
    if (!todo.empty()) {
      if (!bt->todo && (e = cudaMalloc(&bt->todo, sizeof(int) * bt->B)))
        return bfail(MPAX_ERR_OUT_OF_MEMORY, "batch continuation list");
      e = cudaMemcpyAsync(bt->todo, todo.data(), sizeof(int) * todo.size(),
                          cudaMemcpyHostToDevice, s);
      if (e) return bfail(MPAX_ERR_CUDA, cudaGetErrorString(e));
      st = run_batch<double>(bt, o, &launches, bt->todo, todo.data(), (int)todo.size(), 1, 0);
      if (st) return st;
    }
  }
  e = cudaStreamSynchronize(s);
  if (e) return bfail(MPAX_ERR_CUDA, cudaGetErrorString(e));
  problem_order_user_after(bt->prob);
  bt->solved = true;
  bt->launches = launches;
  bt->solve_seconds =
      std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return MPAX_OK;
}

mpax_status mpax_batch_get_solution(const mpax_batch* bt, double* x, double* y,
                                    mpax_mem_kind kind) {
  if (!bt) return bfail(MPAX_ERR_INVALID_ARGUMENT, "NULL batch");
  if (!bt->solved) return bfail(MPAX_ERR_NOT_SOLVED, "call mpax_batch_solve first");
  const cudaMemcpyKind k = kind == MPAX_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  const long long n = bt->h_noff[bt->B], m = bt->h_moff[bt->B];
  cudaError_t e = cudaSuccess;
  if (x && n) e = cudaMemcpy(x, bt->xout, sizeof(double) * n, k);
  if (!e && y && m) e = cudaMemcpy(y, bt->yout, sizeof(double) * m, k);
  if (e) return bfail(MPAX_ERR_CUDA, cudaGetErrorString(e));
  return MPAX_OK;
}

mpax_status mpax_batch_get_stats(const mpax_batch* bt, mpax_batch_stats* stats, int32_t* status,
                                 int64_t* iterations, double* rel_kkt, double* primal_obj,
                                 double* seconds) {
  if (!bt || !stats) return bfail(MPAX_ERR_INVALID_ARGUMENT, "NULL argument");
  if (!bt->solved) return bfail(MPAX_ERR_NOT_SOLVED, "call mpax_batch_solve first");
  const int B = bt->B;
  std::vector<int> hs(B);
  std::vector<long long> hi(B), hr(B);
  std::vector<double> hk(B), hp(B), ht(B);
  cudaError_t e = cudaMemcpy(hs.data(), bt->status, sizeof(int) * B, cudaMemcpyDeviceToHost);
  if (!e) e = cudaMemcpy(hi.data(), bt->iters, sizeof(long long) * B, cudaMemcpyDeviceToHost);
  if (!e) e = cudaMemcpy(hr.data(), bt->restarts, sizeof(long long) * B, cudaMemcpyDeviceToHost);
  if (!e) e = cudaMemcpy(hk.data(), bt->relkkt, sizeof(double) * B, cudaMemcpyDeviceToHost);
  if (!e) e = cudaMemcpy(hp.data(), bt->pobj, sizeof(double) * B, cudaMemcpyDeviceToHost);
  if (!e) e = cudaMemcpy(ht.data(), bt->secs, sizeof(double) * B, cudaMemcpyDeviceToHost);
  if (e) return bfail(MPAX_ERR_CUDA, cudaGetErrorString(e));
  std::memset(stats, 0, sizeof(*stats));
  stats->B = B;
  std::vector<double> sorted = ht;
  std::sort(sorted.begin(), sorted.end());
  for (int b = 0; b < B; ++b) {
    stats->n_optimal += hs[b] == MPAX_TERM_OPTIMAL;
    stats->iterations_total += hi[b];
    stats->iterations_max = std::max<long long>(stats->iterations_max, hi[b]);
    stats->restarts_total += hr[b];
    stats->rel_kkt_max = std::max(stats->rel_kkt_max, hk[b]);
  }
  auto pct = [&](double q) {
    const size_t i = std::min<size_t>(sorted.size() - 1, (size_t)std::ceil(q * sorted.size()) - 1);
    return sorted[i];
  };
  stats->instance_seconds_p50 = pct(0.50);
  stats->instance_seconds_p99 = pct(0.99);
  stats->instance_seconds_max = sorted.back();
  stats->solve_seconds = bt->solve_seconds;
  stats->kernel_launches = bt->launches;
  stats->fp64_instances = bt->fp64_instances;
  for (int b = 0; b < B; ++b) {
    if (status) status[b] = hs[b];
    if (iterations) iterations[b] = hi[b];
    if (rel_kkt) rel_kkt[b] = hk[b];
    if (primal_obj) primal_obj[b] = hp[b];
    if (seconds) seconds[b] = ht[b];
  }
  return MPAX_OK;
}

mpax_status mpax_lp_batch_create_replicated(int32_t B, int32_t m, int32_t n, int64_t nnz,
                                            const int64_t* row_ptr, const int32_t* col_idx,
                                            const double* val, const double* lc,
                                            const double* uc, const double* l, const double* u,
                                            mpax_mem_kind kind, void* cuda_stream,
                                            mpax_batch** out) {
  if (!out) return bfail(MPAX_ERR_INVALID_ARGUMENT, "out must not be NULL");
  *out = nullptr;
  if (B < 1 || m < 0 || n < 0 || nnz < 0)
    return bfail(MPAX_ERR_INVALID_ARGUMENT, "B >= 1 and non-negative sizes required");
  if (!row_ptr || (nnz > 0 && (!col_idx || !val)) || (m > 0 && (!lc || !uc)) ||
      (n > 0 && (!l || !u)))
    return bfail(MPAX_ERR_INVALID_ARGUMENT, "a required array pointer is NULL");
  if ((long long)B * m >= (1LL << 31) || (long long)B * n >= (1LL << 31) ||
      (long long)B * nnz >= (1LL << 31))
    return bfail(MPAX_ERR_UNSUPPORTED, "B copies must hold < 2^31 rows, columns and nonzeros");
  const cudaMemcpyKind k = kind == MPAX_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  // one copy of the set on the device, then B copies of it (columns stay local)
  const long long Bm = (long long)B * m, Bn = (long long)B * n, Bz = (long long)B * nnz;
  long long *rp1 = nullptr, *rpB = nullptr, *moff = nullptr, *noff = nullptr;
  int *col1 = nullptr, *colB = nullptr;
  double* v1 = nullptr;  // nnz + 2m + 2n
  double* vB = nullptr;  // B (nnz + 3n + 2m): values, c (zero), lc, uc, l, u
  cudaError_t e = cudaMalloc(&rp1, sizeof(long long) * (m + 1));
  if (!e) e = cudaMalloc(&rpB, sizeof(long long) * (Bm + 1));
  if (!e) e = cudaMalloc(&moff, sizeof(long long) * (B + 1));
  if (!e) e = cudaMalloc(&noff, sizeof(long long) * (B + 1));
  if (!e) e = cudaMalloc(&col1, sizeof(int) * std::max<long long>(nnz, 1));
  if (!e) e = cudaMalloc(&colB, sizeof(int) * std::max<long long>(Bz, 1));
  if (!e) e = cudaMalloc(&v1, sizeof(double) * std::max<long long>(nnz + 2LL * m + 2LL * n, 1));
  if (!e) e = cudaMalloc(&vB, sizeof(double) * std::max<long long>(Bz + 3 * Bn + 2 * Bm, 1));
  double* valB = vB;
  double* cB = vB + Bz;
  double* lcB = cB + Bn;
  double* ucB = lcB + Bm;
  double* lB = ucB + Bm;
  double* uB = lB + Bn;
  if (!e) e = cudaMemcpyAsync(rp1, row_ptr, sizeof(long long) * (m + 1), k, s);
  if (!e && nnz) e = cudaMemcpyAsync(col1, col_idx, sizeof(int) * nnz, k, s);
  if (!e && nnz) e = cudaMemcpyAsync(v1, val, sizeof(double) * nnz, k, s);
  if (!e && m) e = cudaMemcpyAsync(v1 + nnz, lc, sizeof(double) * m, k, s);
  if (!e && m) e = cudaMemcpyAsync(v1 + nnz + m, uc, sizeof(double) * m, k, s);
  if (!e && n) e = cudaMemcpyAsync(v1 + nnz + 2LL * m, l, sizeof(double) * n, k, s);
  if (!e && n) e = cudaMemcpyAsync(v1 + nnz + 2LL * m + n, u, sizeof(double) * n, k, s);
  std::vector<long long> hm(B + 1), hn(B + 1);
  for (int b = 0; b <= B; ++b) {
    hm[b] = (long long)b * m;
    hn[b] = (long long)b * n;
  }
  if (!e) e = cudaMemcpyAsync(moff, hm.data(), sizeof(long long) * (B + 1), cudaMemcpyHostToDevice, s);
  if (!e) e = cudaMemcpyAsync(noff, hn.data(), sizeof(long long) * (B + 1), cudaMemcpyHostToDevice, s);
  if (!e) {
    const int g = 1024;
    k_rep_rowptr<<<g, 256, 0, s>>>(rp1, m, nnz, B, rpB);
    if (nnz) k_tile<int><<<g, 256, 0, s>>>(col1, nnz, B, colB);
    if (nnz) k_tile<double><<<g, 256, 0, s>>>(v1, nnz, B, valB);
    if (m) k_tile<double><<<g, 256, 0, s>>>(v1 + nnz, m, B, lcB);
    if (m) k_tile<double><<<g, 256, 0, s>>>(v1 + nnz + m, m, B, ucB);
    if (n) k_tile<double><<<g, 256, 0, s>>>(v1 + nnz + 2LL * m, n, B, lB);
    if (n) k_tile<double><<<g, 256, 0, s>>>(v1 + nnz + 2LL * m + n, n, B, uB);
    if (Bn) e = cudaMemsetAsync(cB, 0, sizeof(double) * Bn, s);
    if (!e) e = cudaGetLastError();
    if (!e) e = cudaStreamSynchronize(s);
  }
  mpax_status st = MPAX_ERR_CUDA;
  if (!e)
    st = mpax_lp_batch_create(B, (const int64_t*)moff, (const int64_t*)noff,
                              (const int64_t*)rpB, colB, valB, cB, lcB, ucB, lB, uB,
                              MPAX_MEM_DEVICE, cuda_stream, out);
  cudaStreamSynchronize(s);
  for (void* p : {(void*)rp1, (void*)rpB, (void*)moff, (void*)noff, (void*)col1, (void*)colB,
                  (void*)v1, (void*)vB})
    if (p) cudaFree(p);
  if (e) return bfail(e == cudaErrorMemoryAllocation ? MPAX_ERR_OUT_OF_MEMORY : MPAX_ERR_CUDA,
                      cudaGetErrorString(e));
  return st;
}

mpax_status mpax_batch_set_costs(mpax_batch* bt, const double* c, mpax_mem_kind kind) {
  if (!bt || !c) return bfail(MPAX_ERR_INVALID_ARGUMENT, "NULL argument");
  ProblemData& P = *problem_data(bt->prob);
  const long long n = bt->h_noff[bt->B];
  problem_order_after_user(bt->prob);
  const cudaMemcpyKind k = kind == MPAX_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  cudaError_t e = n ? cudaMemcpyAsync(P.c, c, sizeof(double) * n, k, P.s) : cudaSuccess;
  if (!e) e = cudaStreamSynchronize(P.s);
  if (e) return bfail(MPAX_ERR_CUDA, cudaGetErrorString(e));
  problem_order_user_after(bt->prob);
  bt->solved = false;
  return MPAX_OK;
}

mpax_status mpax_batch_get_objective(const mpax_batch* bt, double* v, mpax_mem_kind kind) {
  if (!bt || !v) return bfail(MPAX_ERR_INVALID_ARGUMENT, "NULL argument");
  if (!bt->solved) return bfail(MPAX_ERR_NOT_SOLVED, "call mpax_batch_solve first");
  const cudaMemcpyKind k = kind == MPAX_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  const cudaError_t e = cudaMemcpy(v, bt->pobj, sizeof(double) * bt->B, k);
  if (e) return bfail(MPAX_ERR_CUDA, cudaGetErrorString(e));
  return MPAX_OK;
}

mpax_status mpax_batch_spo_plus(mpax_batch* bt, const mpax_options* o, const double* c_hat,
                                const double* c_true, const double* x_true,
                                const double* z_true, double* loss, double* grad,
                                mpax_mem_kind kind) {
  if (!bt || !o || !c_hat || !c_true || !x_true || !z_true || !loss || !grad)
    return bfail(MPAX_ERR_INVALID_ARGUMENT, "NULL argument");
  ProblemData& P = *problem_data(bt->prob);
  cudaStream_t s = P.s;
  const int B = bt->B;
  const long long n = bt->h_noff[B];
  problem_order_after_user(bt->prob);
  cudaError_t e = cudaSuccess;
  if (kind == MPAX_MEM_HOST) {
    // stage the host arguments: c_hat, c_true, x_true (sum n each), z_true (B)
    if (!bt->spo) e = cudaMalloc(&bt->spo, sizeof(double) * (3 * std::max<long long>(n, 1) + B));
    double* d = bt->spo;
    if (!e && n) e = cudaMemcpyAsync(d, c_hat, sizeof(double) * n, cudaMemcpyHostToDevice, s);
    if (!e && n) e = cudaMemcpyAsync(d + n, c_true, sizeof(double) * n, cudaMemcpyHostToDevice, s);
    if (!e && n)
      e = cudaMemcpyAsync(d + 2 * n, x_true, sizeof(double) * n, cudaMemcpyHostToDevice, s);
    if (!e) e = cudaMemcpyAsync(d + 3 * n, z_true, sizeof(double) * B, cudaMemcpyHostToDevice, s);
    c_hat = d;
    c_true = d + n;
    x_true = d + 2 * n;
    z_true = d + 3 * n;
  }
  if (!e && n) {
    k_spo_costs<<<(int)std::min<long long>(4096, (n + 255) / 256), 256, 0, s>>>(c_hat, c_true,
                                                                              n, P.c);
    e = cudaGetLastError();
  }
  if (!e) e = cudaStreamSynchronize(s);
  if (e) return bfail(MPAX_ERR_CUDA, cudaGetErrorString(e));
  problem_order_user_after(bt->prob);
  bt->solved = false;
  mpax_status st = mpax_batch_solve(bt, o);
  if (st) return st;
  problem_order_after_user(bt->prob);
  double* dl = loss;
  double* dg = grad;
  if (kind == MPAX_MEM_HOST) {
    // results go through the work area of the staged inputs (c_true is no longer needed)
    dg = bt->spo + n;
    dl = bt->spo + 3 * n;  // z_true is read before loss is written, block by block
  }
  k_spo_loss<<<B, 256, 0, s>>>(bt->n_off, 0, P.c, c_hat, x_true, z_true, bt->xout, dl, dg);
  e = cudaGetLastError();
  if (!e && kind == MPAX_MEM_HOST) {
    if (n) e = cudaMemcpyAsync(grad, dg, sizeof(double) * n, cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaMemcpyAsync(loss, dl, sizeof(double) * B, cudaMemcpyDeviceToHost, s);
  }
  if (!e) e = cudaStreamSynchronize(s);
  if (e) return bfail(MPAX_ERR_CUDA, cudaGetErrorString(e));
  problem_order_user_after(bt->prob);
  return MPAX_OK;
}

void mpax_batch_destroy(mpax_batch* bt) {
  if (!bt) return;
  if (bt->prob) mpax_destroy(bt->prob);
  void* bufs[] = {bt->m_off, bt->n_off, bt->next, bt->status, bt->iters, bt->restarts,
                  bt->relkkt, bt->pobj, bt->secs, bt->xout, bt->yout, bt->work, bt->todo,
                  bt->spo};
  for (void* b : bufs)
    if (b) cudaFree(b);
  delete bt;
}

}  // extern "C"
