// Row epilogues of the fused SpMV kernels: the elementwise half of each PDHG
// half-step, fused with the SpMV that produces its row sums.
//
// Each epilogue is called once per row with s = (K v)_row, accumulates up to
// NQ FP64 partial sums when `check` is set, and reads its scalars from the
// device-resident DevState in load().
#pragma once

#include "common.cuh"

namespace mpax {

// ---- r^2HPDHG (Algorithm 1) -------------------------------------------------
//
// Storage of the Halpern iterate: the current primal iterate of the cycle,
//   x^{n,k} = a_k w^k + b_k x^{n,0},  a_k = k/(k+1), b_k = 1/(k+1),
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
  T tau, ra, rb, g;
  __device__ __forceinline__ bool skip() const { return st->done != 0; }
  __device__ __forceinline__ void load() {
    tau = (T)st->tau;
    ra = (T)st->coef_a[it];
    rb = (T)st->coef_b[it];
    g = (T)st->gamma;
  }
  __device__ __forceinline__ void row(int j, T t, double* acc) {
    const T x0 = xa[j];
    T x;
    if (xsrc) {
      x = xsrc[j];
    } else {
      x = (ra == (T)0) ? x0 : ra * wbuf[j] + rb * x0;
    }
    const T xh = clampv<T>(x - tau * (c[j] - t), l[j], u[j]);
    xbar[j] = (T)2 * xh - x;
    if (wbuf != xbar) wbuf[j] = ((T)1 + g) * xh - g * x;
    if (record) {
      xhat[j] = xh;
      xprev[j] = x;
    }
    if (check) {
      const double d0 = (double)xh - (double)x, d1 = (double)xh - (double)x0;
      acc[0] += d0 * d0;
      acc[1] += d1 * d1;
    }
  }
};

// Dual half-step over the rows of A (one row per constraint i), s = (A xbar)_i:
//   v = y/sigma - s;  y^ = sigma (v - proj_[-uc,-lc](v))   (eq. 3, second line;
//   y - sigma s = sigma v)
//   y+ = a ((1+gamma) y^ - gamma y) + b y^{n,0}            (eq. 4)
// check partials: [0] sum (y^ - y)^2, [1] sum (y^ - y^{n,0})^2
template <typename T>
struct EpiDualLP {
  static constexpr int NQ = 2;
  const DevState* st;
  T* y;
  const T* ya;
  const T* lc;
  const T* uc;
  T* yhat;
  T* yprev;
  int it, record, check;
  T sigma, inv_sigma, ha, hb, g;
  __device__ __forceinline__ bool skip() const { return st->done != 0; }
  __device__ __forceinline__ void load() {
    sigma = (T)st->sigma;
    inv_sigma = (T)st->inv_sigma;
    ha = (T)st->coef_a[it + 1];
    hb = (T)st->coef_b[it + 1];
    g = (T)st->gamma;
  }
  __device__ __forceinline__ void row(int i, T s, double* acc) {
    const T y0 = y[i];
    const T y0a = ya[i];
    const T v = y0 * inv_sigma - s;
    const T yh = sigma * (v - clampv<T>(v, -uc[i], -lc[i]));
    y[i] = ha * (((T)1 + g) * yh - g * y0) + hb * y0a;
    if (record) {
      yhat[i] = yh;
      yprev[i] = y0;
    }
    if (check) {
      const double d0 = (double)yh - (double)y0, d1 = (double)yh - (double)y0a;
      acc[0] += d0 * d0;
      acc[1] += d1 * d1;
    }
  }
};

// ---- rAPDHG (Algorithm 2) ---------------------------------------------------
// beta_k = theta_k = coef_a[it] = 2/(k+2).  Q~ = diag(Ds) + F~ F~^T with
// u = F~^T x_md computed by the SpMV launched just before.

// Primal step over the rows of A^T, t = (A^T y)_j:
//   x_md = (1-beta) xavg + beta x;  q = Ds x_md + (F~ u)_j
//   x+ = proj_[l,u](x - tau (q + c - t))            (eq. 6)
//   xref = 2 x+ - x;  xavg+ = (1-theta) xavg + theta x+
// check partials: [1] sum (xavg+ - x_anchor)^2
template <typename T>
struct EpiPrimalQP {
  static constexpr int NQ = 2;
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
  T tau, beta;
  __device__ __forceinline__ bool skip() const { return st->done != 0; }
  __device__ __forceinline__ void load() {
    tau = (T)st->tau;
    beta = (T)st->coef_a[it];
  }
  __device__ __forceinline__ void row(int j, T t, double* acc) {
    const T x0 = x[j];
    const T xa = xavg[j];
    const T xmd = ((T)1 - beta) * xa + beta * x0;
    T q = Ds[j] * xmd;
    for (int p = frp[j]; p < frp[j + 1]; ++p) q += fval[p] * uvec[fcol[p]];
    const T xn = clampv<T>(x0 - tau * (q + c[j] - t), l[j], u[j]);
    xref[j] = (T)2 * xn - x0;
    x[j] = xn;
    const T xan = ((T)1 - beta) * xa + beta * xn;
    xavg[j] = xan;
    if (record) xprev[j] = x0;
    if (check) {
      const double d1 = (double)xan - (double)xanc[j];
      acc[1] += d1 * d1;
    }
  }
};

// Dual step over the rows of A, s = (A xref)_i (eq. 5 second line), then the
// weighted average.  check partials: [1] sum (yavg+ - y_anchor)^2
template <typename T>
struct EpiDualQP {
  static constexpr int NQ = 2;
  const DevState* st;
  T* y;
  T* yavg;
  const T* yanc;
  const T* lc;
  const T* uc;
  int it, check;
  T sigma, inv_sigma, theta;
  __device__ __forceinline__ bool skip() const { return st->done != 0; }
  __device__ __forceinline__ void load() {
    sigma = (T)st->sigma;
    inv_sigma = (T)st->inv_sigma;
    theta = (T)st->coef_a[it];
  }
  __device__ __forceinline__ void row(int i, T s, double* acc) {
    const T y0 = y[i];
    const T v = y0 * inv_sigma - s;
    const T yn = sigma * (v - clampv<T>(v, -uc[i], -lc[i]));
    y[i] = yn;
    const T yan = ((T)1 - theta) * yavg[i] + theta * yn;
    yavg[i] = yan;
    if (check) {
      const double d1 = (double)yan - (double)yanc[i];
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
  const int* skipf;
  const double* invDr;
  const double* Dr;
  const double* lc;
  const double* uc;
  const T* yv;
  int check;
  __device__ __forceinline__ bool skip() const { return skipf && *skipf != 0; }
  __device__ __forceinline__ void load() {}
  __device__ __forceinline__ void row(int i, T s, double* acc) {
    const double ax = (double)s * invDr[i];
    const double lo = lc[i], hi = uc[i];
    const double rp = ax - fmin(fmax(ax, lo), hi);
    acc[0] += rp * rp;
    const double y = Dr[i] * (double)yv[i];
    double term = 0.0;
    if (y > 0.0 && isfinite(lo)) term = lo * y;
    if (y < 0.0 && isfinite(hi)) term = hi * y;
    acc[1] += term;
  }
};

// Rows of A^T, t = (A~^T y~)_j:  (A^T y)_j = t / Dc_j,  x_j = Dc_j x~_j,
// lam = Q x + c - A^T y, (Q x)_j = (Ds x~ + F~ u)_j / Dc_j.
// partials: [0] sum r_d^2, [1] sum c x, [2] sum (l lh^+ - u lh^-), [3] sum x Q x
template <typename T>
struct EpiKktCol {
  static constexpr int NQ = 4;
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
  __device__ __forceinline__ bool skip() const { return skipf && *skipf != 0; }
  __device__ __forceinline__ void load() {}
  __device__ __forceinline__ void row(int j, T t, double* acc) {
    const double aty = (double)t * invDc[j];
    const double xs = (double)xv[j];
    const double x = Dc[j] * xs;
    double qx = 0.0;
    if (is_qp) {
      double q = Ds[j] * xs;
      for (int p = frp[j]; p < frp[j + 1]; ++p) q += fval[p] * (double)uvec[fcol[p]];
      qx = q * invDc[j];
    }
    const double lam = qx + c[j] - aty;
    const double lo = l[j], hi = u[j];
    const bool lf = isfinite(lo), uf = isfinite(hi);
    double lh;
    if (lf && uf) lh = lam;
    else if (lf) lh = fmax(lam, 0.0);
    else if (uf) lh = fmin(lam, 0.0);
    else lh = 0.0;
    const double rd = lam - lh;
    acc[0] += rd * rd;
    acc[1] += c[j] * x;
    acc[2] += (lf ? lo * fmax(lh, 0.0) : 0.0) + (uf ? hi * fmin(lh, 0.0) : 0.0);
    acc[3] += x * qx;
  }
};

// ---- plain products (power iteration, Q~ v) ----------------------------------
// out_r = s * s_scale + diag_r * din_r * d_scale; partial [0] sum out^2
template <typename T>
struct EpiStore {
  static constexpr int NQ = 1;
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
  __device__ __forceinline__ void row(int r, T s, double* acc) {
    T v = s * ss;
    if (diag) v += diag[r] * (din[r] * ds);
    out[r] = v;
    if (check) acc[0] += (double)v * (double)v;
  }
};

}  // namespace mpax
