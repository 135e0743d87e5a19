// Row epilogues of the fused SpMV kernels: the elementwise half of each PDHG
// half-step, fused with the SpMV that produces its row sums.
//
// Interface: load() reads the DevState scalars once per warp; pre(r, p) issues
// the loads of row r's operands (called before the SpMV loads so that they are
// in flight together); row(r, s, p, acc) receives s = (K v)_r, computes, stores
// and, when `check` is set, accumulates NQ FP64 partial sums.
//
// Weighted sums of two points are written as anchor-relative affine updates,
// v + b (anchor - v), so the two weights sum to one exactly in any precision;
// with separately rounded FP32 weights (k+1)/(k+2) and 1/(k+2) the iterate
// would drift by ~1e-7 relatively per iteration over long restart cycles.
#pragma once

#include "common.cuh"

namespace mpax {

// ---- r^2HPDHG (Algorithm 1) -------------------------------------------------
//
// Storage of the Halpern iterate: the current primal iterate of the cycle,
//   x^{n,k} = w^k + (1/(k+1)) (x^{n,0} - w^k),
// is rebuilt from the stored reflected point w^k = (1+gamma) x^ - gamma x of the
// previous step and the anchor x^{n,0} (eq. 4 rewritten), so a primal
// half-step reads (w, anchor, c, l, u) and writes only w (plus xbar = 2x^ - x,
// the vector the dual SpMV gathers, which is w itself when gamma = 1).

// Primal half-step over the rows of A^T (one row per variable j):
//   x^ = proj_[l,u](x - tau (c - A^T y))            (eq. 3, first line)
//   xbar = 2 x^ - x, w = (1+gamma) x^ - gamma x      (eq. 4)
// check partials: [0] sum (x^ - x)^2, [1] sum (x^ - x^{n,0})^2
template <typename T>
struct EpiPrimalLP {
  static constexpr int NQ = 2;
  struct Pre {
    T w, x0, c, l, u, xs;
  };
  const DevState* st;
  T* xbar;
  T* wbuf;  // == xbar when gamma == 1
  const T* xa;
  const T* c;
  const T* l;
  const T* u;
  const T* xsrc;  // non-null: take x from here instead of rebuilding it
  T* xhat;
  T* xprev;
  int it, record, check;
  T tau, rb, g;
  __device__ __forceinline__ bool skip() const { return st->done != 0; }
  __device__ __forceinline__ void load() {
    tau = (T)st->tau;
    rb = (T)st->coef_b[it];
    g = (T)st->gamma;
  }
  __device__ __forceinline__ void pre(int j, Pre& p) const {
    p.w = wbuf[j];
    p.x0 = xa[j];
    p.c = c[j];
    p.l = l[j];
    p.u = u[j];
    p.xs = xsrc ? xsrc[j] : (T)0;
  }
  __device__ __forceinline__ void row(int j, T t, const Pre& p, double* acc) {
    T x;
    if (xsrc) x = p.xs;
    else x = (rb == (T)1) ? p.x0 : p.w + rb * (p.x0 - p.w);
    const T xh = clampv<T>(x - tau * (p.c - t), p.l, p.u);
    xbar[j] = (T)2 * xh - x;
    if (wbuf != xbar) wbuf[j] = ((T)1 + g) * xh - g * x;
    if (record) {
      xhat[j] = xh;
      xprev[j] = x;
    }
    if (check) {
      const double d0 = (double)xh - (double)x, d1 = (double)xh - (double)p.x0;
      acc[0] += d0 * d0;
      acc[1] += d1 * d1;
    }
  }
};

// Dual half-step over the rows of A (one row per constraint i), s = (A xbar)_i:
//   v = y/sigma - s;  y^ = sigma (v - proj_[-uc,-lc](v))   (eq. 3, second line;
//   y - sigma s = sigma v)
//   y+ = z + b (y^{n,0} - z),  z = (1+gamma) y^ - gamma y, b = 1/(k+2)   (eq. 4)
// check partials: [0] sum (y^ - y)^2, [1] sum (y^ - y^{n,0})^2
template <typename T>
struct EpiDualLP {
  static constexpr int NQ = 2;
  struct Pre {
    T y, ya, lc, uc;
  };
  const DevState* st;
  T* y;
  const T* ya;
  const T* lc;
  const T* uc;
  T* yhat;
  T* yprev;
  int it, record, check;
  T sigma, inv_sigma, hb, g;
  __device__ __forceinline__ bool skip() const { return st->done != 0; }
  __device__ __forceinline__ void load() {
    sigma = (T)st->sigma;
    inv_sigma = (T)st->inv_sigma;
    hb = (T)st->coef_b[it + 1];
    g = (T)st->gamma;
  }
  __device__ __forceinline__ void pre(int i, Pre& p) const {
    p.y = y[i];
    p.ya = ya[i];
    p.lc = lc[i];
    p.uc = uc[i];
  }
  __device__ __forceinline__ void row(int i, T s, const Pre& p, double* acc) {
    const T v = p.y * inv_sigma - s;
    const T yh = sigma * (v - clampv<T>(v, -p.uc, -p.lc));
    const T z = ((T)1 + g) * yh - g * p.y;
    y[i] = z + hb * (p.ya - z);
    if (record) {
      yhat[i] = yh;
      yprev[i] = p.y;
    }
    if (check) {
      const double d0 = (double)yh - (double)p.y, d1 = (double)yh - (double)p.ya;
      acc[0] += d0 * d0;
      acc[1] += d1 * d1;
    }
  }
};

// ---- rAPDHG (Algorithm 2) ---------------------------------------------------
// beta_k = theta_k = coef_a[it] = 2/(k+2).  Q~ = diag(Ds) + F~ F~^T with
// u = F~^T x_md computed by the SpMV launched just before.

// Primal step over the rows of A^T, t = (A^T y)_j:
//   x_md = xavg + beta (x - xavg);  q = Ds x_md + (F~ u)_j
//   x+ = proj_[l,u](x - tau (q + c - t))            (eq. 6)
//   xref = 2 x+ - x;  xavg+ = xavg + theta (x+ - xavg)
// check partials: [1] sum (xavg+ - x_anchor)^2
// TAPE (replay of a block for the reverse sweep): also writes x_md and the
// clamp code of the projection (0 inside, 1 at l, 2 at u).
template <typename T, bool TAPE = false>
struct EpiPrimalQP {
  static constexpr int NQ = 2;
  struct Pre {
    T x, xa, xn, c, l, u, d;
    int f0, f1;
  };
  const DevState* st;
  T* x;
  T* xavg;
  T* xref;
  const T* xanc;
  const T* c;
  const T* l;
  const T* u;
  const T* Ds;
  const int* frp;
  const int* fcol;
  const T* fval;
  const T* uvec;
  T* xprev;
  int it, record, check;
  T* tape_xmd;
  unsigned char* tape_code;
  const T* qadd;  // general sparse Q: (Q~ x_md)_j from the SpMV launched before
  T tau, beta;
  __device__ __forceinline__ bool skip() const { return st->done != 0; }
  __device__ __forceinline__ void load() {
    tau = (T)st->tau;
    beta = (T)st->coef_a[it];
  }
  __device__ __forceinline__ void pre(int j, Pre& p) const {
    p.x = x[j];
    p.xa = xavg[j];
    p.xn = check ? xanc[j] : (T)0;
    p.c = c[j];
    p.l = l[j];
    p.u = u[j];
    p.d = Ds[j];
    p.f0 = frp[j];
    p.f1 = frp[j + 1];
  }
  __device__ __forceinline__ void row(int j, T t, const Pre& p, double* acc) {
    const T xmd = p.xa + beta * (p.x - p.xa);
    T q = p.d * xmd;
    for (int k = p.f0; k < p.f1; ++k) q += fval[k] * uvec[fcol[k]];
    if (qadd) q += qadd[j];
    const T vx = p.x - tau * (q + p.c - t);
    const T xn = clampv<T>(vx, p.l, p.u);
    if constexpr (TAPE) {
      tape_xmd[j] = xmd;
      tape_code[j] = clamp_code<T>(vx, p.l, p.u);
    }
    xref[j] = (T)2 * xn - p.x;
    x[j] = xn;
    const T xan = p.xa + beta * (xn - p.xa);
    xavg[j] = xan;
    if (record) xprev[j] = p.x;
    if (check) {
      const double d1 = (double)xan - (double)p.xn;
      acc[1] += d1 * d1;
    }
  }
};

// Dual step over the rows of A, s = (A xref)_i (eq. 5 second line), then the
// weighted average.  check partials: [1] sum (yavg+ - y_anchor)^2
// TAPE: also writes the clamp code of proj_[-uc,-lc] (0 inside, 1 at -uc, 2 at -lc).
template <typename T, bool TAPE = false>
struct EpiDualQP {
  static constexpr int NQ = 2;
  struct Pre {
    T y, ya, yn, lc, uc;
  };
  const DevState* st;
  T* y;
  T* yavg;
  const T* yanc;
  const T* lc;
  const T* uc;
  int it, check;
  unsigned char* tape_code;
  T sigma, inv_sigma, theta;
  __device__ __forceinline__ bool skip() const { return st->done != 0; }
  __device__ __forceinline__ void load() {
    sigma = (T)st->sigma;
    inv_sigma = (T)st->inv_sigma;
    theta = (T)st->coef_a[it];
  }
  __device__ __forceinline__ void pre(int i, Pre& p) const {
    p.y = y[i];
    p.ya = yavg[i];
    p.yn = check ? yanc[i] : (T)0;
    p.lc = lc[i];
    p.uc = uc[i];
  }
  __device__ __forceinline__ void row(int i, T s, const Pre& p, double* acc) {
    const T v = p.y * inv_sigma - s;
    const T yn = sigma * (v - clampv<T>(v, -p.uc, -p.lc));
    if constexpr (TAPE) tape_code[i] = clamp_code<T>(v, -p.uc, -p.lc);
    y[i] = yn;
    const T yan = p.ya + theta * (yn - p.ya);
    yavg[i] = yan;
    if (check) {
      const double d1 = (double)yan - (double)p.yn;
      acc[1] += d1 * d1;
    }
  }
};

// ---- relative KKT error (unscaled problem), FP64 ---------------------------

// Rows of A, s = (A~ x~)_i:  (A x)_i = s / Dr_i.
// partials: [0] sum r_p^2, [1] sum (lc y^+ - uc y^-) (finite bounds only)
template <typename T>
struct EpiKktRow {
  static constexpr int NQ = 2;
  struct Pre {
    double idr, dr, lc, uc;
    T yv;
  };
  const int* skipf;
  const double* invDr;
  const double* Dr;
  const double* lc;
  const double* uc;
  const T* yv;
  int check;
  __device__ __forceinline__ bool skip() const { return skipf && *skipf != 0; }
  __device__ __forceinline__ void load() {}
  __device__ __forceinline__ void pre(int i, Pre& p) const {
    p.idr = invDr[i];
    p.dr = Dr[i];
    p.lc = lc[i];
    p.uc = uc[i];
    p.yv = yv[i];
  }
  __device__ __forceinline__ void row(int i, T s, const Pre& p, double* acc) {
    const double ax = (double)s * p.idr;
    const double rp = ax - fmin(fmax(ax, p.lc), p.uc);
    acc[0] += rp * rp;
    const double y = p.dr * (double)p.yv;
    double term = 0.0;
    if (y > 0.0 && isfinite(p.lc)) term = p.lc * y;
    if (y < 0.0 && isfinite(p.uc)) term = p.uc * y;
    acc[1] += term;
  }
};

// Rows of A^T, t = (A~^T y~)_j:  (A^T y)_j = t / Dc_j,  x_j = Dc_j x~_j,
// lam = Q x + c - A^T y, (Q x)_j = (Ds x~ + F~ u)_j / Dc_j.
// partials: [0] sum r_d^2, [1] sum c x, [2] sum (l lh^+ - u lh^-), [3] sum x Q x
template <typename T>
struct EpiKktCol {
  static constexpr int NQ = 4;
  struct Pre {
    double idc, dc, c, l, u;
    T xv;
  };
  const int* skipf;
  const double* invDc;
  const double* Dc;
  const double* c;
  const double* l;
  const double* u;
  const T* xv;
  int is_qp;
  const double* Ds;
  const int* frp;
  const int* fcol;
  const double* fval;
  const T* uvec;
  int check;
  const T* qadd;  // general sparse Q: (Q~ x~)_j
  __device__ __forceinline__ bool skip() const { return skipf && *skipf != 0; }
  __device__ __forceinline__ void load() {}
  __device__ __forceinline__ void pre(int j, Pre& p) const {
    p.idc = invDc[j];
    p.dc = Dc[j];
    p.c = c[j];
    p.l = l[j];
    p.u = u[j];
    p.xv = xv[j];
  }
  __device__ __forceinline__ void row(int j, T t, const Pre& p, double* acc) {
    const double aty = (double)t * p.idc;
    const double xs = (double)p.xv;
    const double x = p.dc * xs;
    double qx = 0.0;
    if (is_qp) {
      double q = Ds[j] * xs;
      for (int k = frp[j]; k < frp[j + 1]; ++k) q += fval[k] * (double)uvec[fcol[k]];
      if (qadd) q += (double)qadd[j];
      qx = q * p.idc;
    }
    const double lam = qx + p.c - aty;
    const bool lf = isfinite(p.l), uf = isfinite(p.u);
    double lh;
    if (lf && uf) lh = lam;
    else if (lf) lh = fmax(lam, 0.0);
    else if (uf) lh = fmin(lam, 0.0);
    else lh = 0.0;
    const double rd = lam - lh;
    acc[0] += rd * rd;
    acc[1] += p.c * x;
    acc[2] += (lf ? p.l * fmax(lh, 0.0) : 0.0) + (uf ? p.u * fmin(lh, 0.0) : 0.0);
    acc[3] += x * qx;
  }
};

// ---- infeasibility rays (LP) ----------------------------------------------------
// The candidate rays of a check are the moves since the cycle's anchor, in the
// scaled space: rx~ = x^ - x_anchor, and ry~ = y^ - y_anchor projected onto the
// recession cone of Y (k_ray_prep).  Unscaled: dx = Dc rx~, dy = Dr ry~.
//
// Rows of A, s = (A~ rx~)_i:  (A dx)_i = s / Dr_i.
// partials: [0] ||A dx - proj_R(A dx)||^2 (R: recession cone of [lc_i, uc_i]),
//           [1] sum lc_i dy_i^+ - uc_i dy_i^- (finite terms): the Farkas ray's row
//               objective
template <typename T>
struct EpiRayRow {
  static constexpr int NQ = 2;
  struct Pre {
    double idr, dr, lc, uc;
    T ry;
  };
  const int* skipf;
  const double* invDr;
  const double* Dr;
  const double* lc;
  const double* uc;
  const T* ry;
  int check;
  __device__ __forceinline__ bool skip() const { return skipf && *skipf != 0; }
  __device__ __forceinline__ void load() {}
  __device__ __forceinline__ void pre(int i, Pre& p) const {
    p.idr = invDr[i];
    p.dr = Dr[i];
    p.lc = lc[i];
    p.uc = uc[i];
    p.ry = ry[i];
  }
  __device__ __forceinline__ void row(int i, T s, const Pre& p, double* acc) {
    const double ax = (double)s * p.idr;
    const bool lf = isfinite(p.lc), uf = isfinite(p.uc);
    const double pr = (lf && uf) ? 0.0 : lf ? fmax(ax, 0.0) : uf ? fmin(ax, 0.0) : ax;
    acc[0] += (ax - pr) * (ax - pr);
    const double y = p.dr * (double)p.ry;
    double term = 0.0;
    if (y > 0.0 && lf) term = p.lc * y;
    if (y < 0.0 && uf) term = p.uc * y;
    acc[1] += term;
  }
};

// Rows of A^T, t = (A~^T ry~)_j:  lam_j = -(A^T dy)_j = -t / Dc_j.
// partials: [0] ||lam - proj_Lambda(lam)||^2, [1] sum l_j lh_j^+ - u_j lh_j^- (the
//           Farkas ray's column objective, lh = proj_Lambda(lam)), [2] c^T dx,
//           [3] ||dx - proj_X(dx)||^2 (X: recession cone of [l_j, u_j])
template <typename T>
struct EpiRayCol {
  static constexpr int NQ = 4;
  struct Pre {
    double idc, dc, c, l, u;
    T rx;
  };
  const int* skipf;
  const double* invDc;
  const double* Dc;
  const double* c;
  const double* l;
  const double* u;
  const T* rx;
  int check;
  __device__ __forceinline__ bool skip() const { return skipf && *skipf != 0; }
  __device__ __forceinline__ void load() {}
  __device__ __forceinline__ void pre(int j, Pre& p) const {
    p.idc = invDc[j];
    p.dc = Dc[j];
    p.c = c[j];
    p.l = l[j];
    p.u = u[j];
    p.rx = rx[j];
  }
  __device__ __forceinline__ void row(int j, T t, const Pre& p, double* acc) {
    const double lam = -(double)t * p.idc;
    const bool lf = isfinite(p.l), uf = isfinite(p.u);
    const double lh = (lf && uf) ? lam : lf ? fmax(lam, 0.0) : uf ? fmin(lam, 0.0) : 0.0;
    acc[0] += (lam - lh) * (lam - lh);
    acc[1] += (lf ? p.l * fmax(lh, 0.0) : 0.0) + (uf ? p.u * fmin(lh, 0.0) : 0.0);
    const double dx = p.dc * (double)p.rx;
    acc[2] += p.c * dx;
    const double px = (lf && uf) ? 0.0 : lf ? fmax(dx, 0.0) : uf ? fmin(dx, 0.0) : dx;
    acc[3] += (dx - px) * (dx - px);
  }
};

// ---- plain products (power iteration, Q~ v) ----------------------------------
// out_r = s * s_scale + diag_r * din_r * d_scale; partial [0] sum out^2
template <typename T>
struct EpiStore {
  static constexpr int NQ = 1;
  struct Pre {
    T d, di;
  };
  const int* skipf;
  T* out;
  const double* s_scale;  // nullable: 1
  const T* diag;          // nullable
  const T* din;
  const double* d_scale;  // nullable: 1
  int check;
  T ss, ds;
  __device__ __forceinline__ bool skip() const { return skipf && *skipf != 0; }
  __device__ __forceinline__ void load() {
    ss = s_scale ? (T)*s_scale : (T)1;
    ds = d_scale ? (T)*d_scale : (T)1;
  }
  __device__ __forceinline__ void pre(int r, Pre& p) const {
    p.d = diag ? diag[r] : (T)0;
    p.di = diag ? din[r] : (T)0;
  }
  __device__ __forceinline__ void row(int r, T s, const Pre& p, double* acc) {
    T v = s * ss;
    if (diag) v += p.d * (p.di * ds);
    out[r] = v;
    if (check) acc[0] += (double)v * (double)v;
  }
};

}  // namespace mpax
