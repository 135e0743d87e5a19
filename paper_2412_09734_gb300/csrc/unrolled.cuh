// Differentiation of a QP solve by unrolling rAPDHG (Algorithm 2; Sec. 3.4
// obtains QP gradients by differentiating through the solver's iterations).
//
// Along the path a solve took -- its restarts, step sizes and stopping point
// held fixed -- the returned point (D_c xavg, D_r yavg) is a piecewise-affine
// function of the data (c, lc, uc, l, u, D).  The Jacobian of one step depends
// only on which coordinates the two projections clamped and on the momentum
// point x_md, so the reverse sweep needs no stored iterate per step:
//
//   Tape (forward).  One record per check block: step sizes, the block's first
//   inner counter and length, whether the check after it restarted, and the
//   state (x, xavg, y, yavg) the block started from (TapeHead + 2n + 2m values).
//   Records live in chunks allocated as the solve advances; a device table maps
//   the block index to its record.
//
//   Backward, block by block from the last: restore the block's start state,
//   replay the block with the forward kernels (which then also write x_md and
//   the clamp codes of each step), and run its steps backwards.
//
// One step backwards, b = 2/(k+2), adjoints (ax, ay, axa, aya) of
// (x+, y+, xavg+, yavg+), scaled data:
//   R1 (rows of A)    ty = ay + b aya;  w = ty where vy was clamped, else 0;
//                     guc += sigma w (clamped at -uc), glc += sigma w (at -lc);
//                     ws = -sigma w;  ay <- w;  aya <- (1 - b) aya
//   R2 (rows of A^T)  t = (A^T ws)_j;  tx = ax + b axa + 2 t;  u = tx inside
//                     the box, else 0, and gl / gu += tx at l / u;
//                     gc += -tau u;  ax <- u - t
//   R3                tq = F^T u  (general sparse Q: qu = Q~ u)
//   R4 (rows of F)    gq = -tau u;  gxmd = D gq - tau (F tq + qu)_j;  gD += gq x_md;
//                     ax += b gxmd;  axa <- (1 - b)(axa + gxmd)
//   R5 (rows of A)    ay += tau (A u)_i
// Inside a block, R4 of step t runs in the epilogue of R2 of step t-1 and R1
// of step t-1 in the epilogue of R5 of step t: three launches per step
// backwards (A^T SpMV, F^T SpMV, A SpMV), as forwards.
#pragma once

#include "common.cuh"

namespace mpax {

struct TapeHead {
  double tau, sigma;
  long long k_base;
  int len, restart_after;
  double pad[4];
};
static_assert(sizeof(TapeHead) == 64, "tape record head is 64 bytes");

// Forward: record of the block about to run, at slot = checks done so far.
// The previous record learns whether the check before this block restarted.
template <typename T>
__global__ void k_tape_save(DevState* st, char* const* tab, long long cap, int n, int m,
                            const T* __restrict__ x, const T* __restrict__ xavg,
                            const T* __restrict__ y, const T* __restrict__ yavg, int len) {
  if (st->done) return;
  const long long slot = st->checks;
  char* rec = slot < cap ? tab[slot] : nullptr;
  if (rec == nullptr) {
    if (blockIdx.x == 0 && threadIdx.x == 0) st->tape_err = 1;
    return;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    TapeHead* h = reinterpret_cast<TapeHead*>(rec);
    h->tau = st->tau;
    h->sigma = st->sigma;
    h->k_base = st->k_base;
    h->len = len;
    h->restart_after = 0;
    if (slot > 0) reinterpret_cast<TapeHead*>(tab[slot - 1])->restart_after = st->restart_flag;
  }
  T* v = reinterpret_cast<T*>(rec + sizeof(TapeHead));
  const size_t nn = (size_t)n, mm = (size_t)m;
  const int stride = gridDim.x * blockDim.x;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
    v[j] = x[j];
    v[nn + j] = xavg[j];
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
    v[2 * nn + i] = y[i];
    v[2 * nn + mm + i] = yavg[i];
  }
}

// Backward: restore the open record's start state; where the check after the
// block restarted (x, y <- xavg, yavg), fold the adjoints of x, y into those of
// the averages.
template <typename T>
__global__ void k_tape_restore(const DevState* st, char* const* tab, int n, int m,
                               T* __restrict__ x, T* __restrict__ xavg, T* __restrict__ y,
                               T* __restrict__ yavg, double* __restrict__ ax,
                               double* __restrict__ axa, double* __restrict__ ay,
                               double* __restrict__ aya) {
  const char* rec = tab[st->tape_cursor];
  const int fold = reinterpret_cast<const TapeHead*>(rec)->restart_after;
  const T* v = reinterpret_cast<const T*>(rec + sizeof(TapeHead));
  const size_t nn = (size_t)n, mm = (size_t)m;
  const int stride = gridDim.x * blockDim.x;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
    x[j] = v[j];
    xavg[j] = v[nn + j];
    if (fold) {
      axa[j] += ax[j];
      ax[j] = 0.0;
    }
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
    y[i] = v[2 * nn + i];
    yavg[i] = v[2 * nn + mm + i];
    if (fold) {
      aya[i] += ay[i];
      ay[i] = 0.0;
    }
  }
}

// R1 of step `it` on its own (the last step of a block).
__global__ void k_rev_r1(const DevState* st, int it, int m, const unsigned char* __restrict__ cy,
                         double* __restrict__ ay, double* __restrict__ aya,
                         double* __restrict__ ws, double* __restrict__ glc,
                         double* __restrict__ guc) {
  const double b = st->coef_a[it], sigma = st->sigma;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    const double a = aya[i];
    const unsigned char c = cy[i];
    const double w = c == 0 ? 0.0 : ay[i] + b * a;
    if (c == 1) guc[i] += sigma * w;
    else if (c == 2) glc[i] += sigma * w;
    ws[i] = -sigma * w;
    ay[i] = w;
    aya[i] = (1.0 - b) * a;
  }
}

// R4 of step `it` on its own (the first step of a block).
template <typename T>
__global__ void k_rev_r4(const DevState* st, int it, int n, const T* __restrict__ Ds,
                         const int* __restrict__ frp, const int* __restrict__ fcol,
                         const T* __restrict__ fval, const double* __restrict__ tq,
                         const double* __restrict__ u, const T* __restrict__ xmd,
                         const double* __restrict__ qu, double* __restrict__ ax,
                         double* __restrict__ axa, double* __restrict__ gD) {
  const double b = st->coef_a[it], tau = st->tau;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    double fq = qu ? qu[j] : 0.0;
    for (int k = frp[j]; k < frp[j + 1]; ++k) fq += (double)fval[k] * tq[fcol[k]];
    const double gq = -tau * u[j];
    const double gxmd = (double)Ds[j] * gq - tau * fq;
    gD[j] += gq * (double)xmd[j];
    ax[j] += b * gxmd;
    axa[j] = (1.0 - b) * (axa[j] + gxmd);
  }
}

// R2 of step `it` over the rows of A^T (t = (A^T ws)_j), preceded per row by
// R4 of step it + 1 when xmd_next is set.
template <typename T>
struct EpiRevPrimal {
  static constexpr int NQ = 1;
  struct Pre {
    double ax, axa, u1, x1, d;
    int f0, f1;
    unsigned char c;
  };
  const DevState* st;
  double* ax;
  double* axa;
  double* u;
  double* gc;
  double* gl;
  double* gu;
  double* gD;
  const unsigned char* cx;  // codes of step it
  const T* Ds;
  const int* frp;
  const int* fcol;
  const T* fval;
  const double* tq;     // F^T u of step it + 1
  const T* xmd_next;    // x_md of step it + 1; nullptr: no R4 here
  int it, check;
  const double* qu;     // general sparse Q: Q~ u of step it + 1 (else nullptr)
  double tau, b, b1;
  __device__ __forceinline__ bool skip() const { return false; }
  __device__ __forceinline__ void load() {
    tau = st->tau;
    b = st->coef_a[it];
    b1 = xmd_next ? st->coef_a[it + 1] : 0.0;
  }
  __device__ __forceinline__ void pre(int j, Pre& p) const {
    p.ax = ax[j];
    p.axa = axa[j];
    p.c = cx[j];
    if (xmd_next) {
      p.u1 = u[j];
      p.x1 = (double)xmd_next[j];
      p.d = (double)Ds[j];
      p.f0 = frp[j];
      p.f1 = frp[j + 1];
    }
  }
  __device__ __forceinline__ void row(int j, T t, const Pre& p, double*) {
    double axj = p.ax, axaj = p.axa;
    if (xmd_next) {
      double fq = 0.0;
      for (int k = p.f0; k < p.f1; ++k) fq += (double)fval[k] * tq[fcol[k]];
      if (qu) fq += qu[j];
      const double gq = -tau * p.u1;
      const double gxmd = p.d * gq - tau * fq;
      gD[j] += gq * p.x1;
      axj += b1 * gxmd;
      axaj = (1.0 - b1) * (axaj + gxmd);
    }
    const double tt = (double)t;
    const double tx = axj + b * axaj + 2.0 * tt;
    double uu = 0.0;
    if (p.c == 0) uu = tx;
    else if (p.c == 1) gl[j] += tx;
    else gu[j] += tx;
    gc[j] += -tau * uu;
    u[j] = uu;
    ax[j] = uu - tt;
    axa[j] = axaj;
  }
};

// R5 of step `it` over the rows of A (s = (A u)_i), followed per row by R1 of
// step it - 1 when cy_prev is set.
template <typename T>
struct EpiRevDual {
  static constexpr int NQ = 1;
  struct Pre {
    double ay, aya;
    unsigned char c;
  };
  const DevState* st;
  double* ay;
  double* aya;
  double* ws;
  double* glc;
  double* guc;
  const unsigned char* cy_prev;  // codes of step it - 1; nullptr: no R1 here
  int it, check;
  double tau, sigma, b0;
  __device__ __forceinline__ bool skip() const { return false; }
  __device__ __forceinline__ void load() {
    tau = st->tau;
    sigma = st->sigma;
    b0 = cy_prev ? st->coef_a[it - 1] : 0.0;
  }
  __device__ __forceinline__ void pre(int i, Pre& p) const {
    p.ay = ay[i];
    p.aya = cy_prev ? aya[i] : 0.0;
    p.c = cy_prev ? cy_prev[i] : 0;
  }
  __device__ __forceinline__ void row(int i, T s, const Pre& p, double*) {
    double ayi = p.ay + tau * (double)s;
    if (cy_prev) {
      const double w = p.c == 0 ? 0.0 : ayi + b0 * p.aya;
      if (p.c == 1) guc[i] += sigma * w;
      else if (p.c == 2) glc[i] += sigma * w;
      ws[i] = -sigma * w;
      ayi = w;
      aya[i] = (1.0 - b0) * p.aya;
    }
    ay[i] = ayi;
  }
};

// Seeds of the reverse sweep: the loss gradients on the returned averages,
// in scaled variables (x = D_c xavg, y = D_r yavg); gy nullable.
__global__ void k_rev_seed(const double* __restrict__ gx, const double* __restrict__ gy,
                           const double* __restrict__ Dc, const double* __restrict__ Dr, int n,
                           int m, double* __restrict__ ax, double* __restrict__ axa,
                           double* __restrict__ ay, double* __restrict__ aya) {
  const int stride = gridDim.x * blockDim.x;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
    axa[j] = Dc[j] * gx[j];
    ax[j] = 0.0;
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
    aya[i] = gy ? Dr[i] * gy[i] : 0.0;
    ay[i] = 0.0;
  }
}

// Scaled gradients to the data's: c~ = Dc c, l~ = l / Dc, u~ = u / Dc,
// lc~ = Dr lc, uc~ = Dr uc, D~ = Dc^2 D (in place).
__global__ void k_rev_unscale(const double* __restrict__ Dc, const double* __restrict__ Dr,
                              int n, int m, double* __restrict__ gc, double* __restrict__ gl,
                              double* __restrict__ gu, double* __restrict__ gD,
                              double* __restrict__ glc, double* __restrict__ guc) {
  const int stride = gridDim.x * blockDim.x;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
    const double d = Dc[j];
    gc[j] *= d;
    gl[j] /= d;
    gu[j] /= d;
    gD[j] *= d * d;
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
    glc[i] *= Dr[i];
    guc[i] *= Dr[i];
  }
}

}  // namespace mpax
