// Batch of LPs sharing one dense constraint matrix: B instances
//     min c_k^T x  s.t.  lc <= A x <= uc,  l <= x <= u,   k = 0..B-1,
// solved together by r^2HPDHG (Algorithm 1) with per-instance step sizes,
// primal weights, restarts and termination.  Stacking the instances' iterates
// as the columns of X (n x B) and Y (m x B) turns the two matrix-vector products
// of every iteration into dense GEMMs, A X and A^T Y (the paper batches
// same-shape instances by vectorisation, Sec. 3.2; with a shared A the batched
// product is a dense contraction), which run on the tensor cores.
//
// Precision: the scaled matrix and the iterates are split into BF16 pairs
// v = v_hi + v_lo (v_hi = bf16(v), v_lo = bf16(v - v_hi)); each product is the
// sum of three BF16 GEMMs with FP32 accumulation, A_hi X_lo + A_lo X_hi +
// A_hi X_hi: each operand keeps about 16 significant bits and the dropped
// A_lo X_lo term is of order 2^-16 relative, so a product is accurate to about
// 2^-16 relative per term (an FP32 product: 2^-24).  The split of
// the iterates is written by the fused update kernels, so a GEMM reads BF16
// operands only.  The GEMMs are plain library GEMMs (cuBLAS); the PDHG update,
// projection, Halpern step, splitting and the FP64 check reductions are this
// file's kernels.  A plain FP32 product path (SGEMM on the FP32 pipes) is kept
// for comparison.
//
// Layout: A is row-major m x n, i.e. column-major n x m; X, Y and every
// per-instance vector are column-major (column k = instance k).
#include <cuda_bf16.h>

#include <algorithm>
#include <chrono>
#include <climits>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/mpax.h"
#include "umma_host.h"
#include "common.cuh"

namespace mpax {

namespace {

int g1(long long k) { return (int)std::max(1LL, std::min(8192LL, (k + 255) / 256)); }
// Grid of the per-instance elementwise kernels: x over `len` coordinates (256
// threads, up to 4 coordinates each), y over the B instances (65,535 at most; the
// kernels loop over the rest).
dim3 grid2d(long long len, int B) {
  const long long bx = std::max(1LL, std::min(1024LL, (len + 1023) / 1024));
  return dim3((unsigned)bx, (unsigned)std::max(1, std::min(B, 65535)));
}

mpax_status sfail(mpax_status s, const std::string& m) {
  set_last_error(m.c_str());
  return s;
}

// ---- per-instance state --------------------------------------------------------
struct Inst {
  double tau, sigma, omega, r_anchor, r_prev, rel, pobj, dobj, c_norm, best_rel;
  long long k, total, restarts, done_at, checks, stall_count;
  int done, status, restart, have_anchor, stalled;
};

// ---- dense scaling (row-major m x n): row/column infinity- and 1-norms ----------
__global__ void k_row_red(const float* __restrict__ A, int m, int n, int sum,
                          double* __restrict__ out) {
  __shared__ double sh[32];
  for (int i = blockIdx.x; i < m; i += gridDim.x) {
    double acc = 0.0;
    const float* r = A + (size_t)i * n;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      const double v = fabs((double)r[j]);
      acc = sum ? acc + v : fmax(acc, v);
    }
    if (sum) {
      acc = block_sum(acc, sh);
    } else {
      // fixed-order max tree
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc = fmax(acc, __shfl_xor_sync(0xffffffffu, acc, o));
      __syncthreads();
      if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
      __syncthreads();
      if (threadIdx.x < 32) {
        acc = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc = fmax(acc, __shfl_xor_sync(0xffffffffu, acc, o));
      }
    }
    if (threadIdx.x == 0) out[i] = acc;
    __syncthreads();
  }
}

// column reduction: thread per column, sequential over rows (coalesced in j)
__global__ void k_col_red(const float* __restrict__ A, int m, int n, int sum,
                          double* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double acc = 0.0;
  for (int i = 0; i < m; ++i) {
    const double v = fabs((double)A[(size_t)i * n + j]);
    acc = sum ? acc + v : fmax(acc, v);
  }
  out[j] = acc;
}

__global__ void k_factor(double* __restrict__ norm, int k, double* __restrict__ D) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= k) return;
  const double v = norm[i];
  const double d = v > 0.0 ? 1.0 / sqrt(v) : 1.0;
  norm[i] = d;
  D[i] *= d;
}

// dst_ij = (src_ij * dr_i) * dc_j
__global__ void k_scale_dense(const float* __restrict__ src, float* __restrict__ dst, int m,
                              int n, const double* __restrict__ dr,
                              const double* __restrict__ dc) {
  const size_t total = (size_t)m * n;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / n), j = (int)(e % n);
    dst[e] = (float)(((double)src[e] * dr[i]) * dc[j]);
  }
}

__global__ void k_split(const float* __restrict__ a, __nv_bfloat16* __restrict__ hi,
                        __nv_bfloat16* __restrict__ lo, size_t total) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const float v = a[e];
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    hi[e] = h;
    lo[e] = __float2bfloat16_rn(v - __bfloat162float(h));
  }
}

__device__ __forceinline__ void split_store(float v, __nv_bfloat16* hi, __nv_bfloat16* lo,
                                            size_t e) {
  const __nv_bfloat16 h = __float2bfloat16_rn(v);
  hi[e] = h;
  lo[e] = __float2bfloat16_rn(v - __bfloat162float(h));
}

// ---- fused updates ----------------------------------------------------------------
struct Vecs {
  int m, n, B;
  const float *ct, *l, *u, *lc, *uc;  // scaled: ct n x B, l/u n, lc/uc m
  float *w, *xa, *xhat, *T;             // n x B
  float *y, *ya, *yhat, *S;             // m x B
  __nv_bfloat16 *xh_hi, *xh_lo, *y_hi, *y_lo;  // BF16 splits: B rows of ldx / ldy
  double* part;                          // per-column partials [q][k]
  Inst* inst;
  long long ldx, ldy;                    // row strides of the splits (n, m rounded to 8)
};

// primal: T = A~^T Y; x = w + (anchor - w)/(k+1); x^ = proj(x - tau (c~ - T));
// w <- 2 x^ - x (also split to BF16 for the next product)
// tpart (B = 1 only): T is the sum of the GEMV's tchunks partials, in order.
// Grid: x over the coordinates of an instance, y over instances (grid2d).
__global__ void k_primal(Vecs v, int check, const float* __restrict__ tpart, int tchunks) {
  for (int k = blockIdx.y; k < v.B; k += gridDim.y)
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < v.n; j += gridDim.x * blockDim.x) {
    const size_t e = (size_t)k * v.n + j;
    const Inst& I = v.inst[k];
    if (I.done) continue;
    float t;
    if (tpart) {
      t = 0.0f;
      for (int c = 0; c < tchunks; ++c) t += tpart[(size_t)c * v.n + j];
    } else {
      t = v.T[e];
    }
    const float rb = (float)(1.0 / (double)(I.k + 1));
    const float x0 = v.xa[e], wv = v.w[e];
    const float x = (I.k == 0) ? x0 : wv + rb * (x0 - wv);
    const float xh = fminf(fmaxf(x - (float)I.tau * (v.ct[e] - t), v.l[j]), v.u[j]);
    const float wn = 2.0f * xh - x;
    v.w[e] = wn;
    split_store(wn, v.xh_hi, v.xh_lo, (size_t)k * v.ldx + j);
    if (check) v.xhat[e] = xh;
  }
}

// dual: S = A~ xbar; y^ = sigma (v - proj_[-uc,-lc](v)), v = y/sigma - S;
// y <- z + (anchor - z)/(k+2), z = 2 y^ - y (also split)
// spart (B = 1 only): S is the sum of the GEMV's schunks partials, in order.
__global__ void k_dual(Vecs v, int check, const float* __restrict__ spart, int schunks) {
  for (int k = blockIdx.y; k < v.B; k += gridDim.y)
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < v.m; i += gridDim.x * blockDim.x) {
    const size_t e = (size_t)k * v.m + i;
    const Inst& I = v.inst[k];
    if (I.done) continue;
    float sv;
    if (spart) {
      sv = 0.0f;
      for (int c = 0; c < schunks; ++c) sv += spart[(size_t)c * v.m + i];
    } else {
      sv = v.S[e];
    }
    const float sg = (float)I.sigma, isg = (float)(1.0 / I.sigma);
    const float hb = (float)(1.0 / (double)(I.k + 2));
    const float y0 = v.y[e];
    const float vv = y0 * isg - sv;
    const float yh = sg * (vv - fminf(fmaxf(vv, -v.uc[i]), -v.lc[i]));
    const float z = 2.0f * yh - y0;
    const float yn = z + hb * (v.ya[e] - z);
    v.y[e] = yn;
    split_store(yn, v.y_hi, v.y_lo, (size_t)k * v.ldy + i);
    if (check) v.yhat[e] = yh;
  }
}

__global__ void k_advance(Inst* inst, int B) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < B && !inst[k].done) {
    inst[k].k += 1;
    inst[k].total += 1;
  }
}

// Per-column check reductions (one block per instance, fixed order).
// The products S = A~ x^ and T = A~^T y^ were formed into S and T by the caller.
// part[q * B + k]: 0 sum (x^-x)^2 .. computed here from w/xa? -- see k_check_prep.
struct KktArgs {
  int m, n, B;
  const float *xhat, *yhat, *S, *T, *xprev_w, *xa, *yprev, *ya;
  const double *Dr, *Dc, *c0, *lc0, *uc0, *l0, *u0;  // c0: n x B unscaled costs
  double* part;
};

__global__ void k_kkt_cols(KktArgs a, const Inst* inst) {
  __shared__ double sh[32];
  const int k = blockIdx.x;
  if (inst[k].done) return;
  const size_t on = (size_t)k * a.n, om = (size_t)k * a.m;
  double rd2 = 0, cx = 0, bt = 0;
  for (int j = threadIdx.x; j < a.n; j += blockDim.x) {
    const double aty = (double)a.T[on + j] / a.Dc[j];
    const double x = a.Dc[j] * (double)a.xhat[on + j];
    const double c = a.c0[on + j];
    const double lam = c - aty;
    const double lo = a.l0[j], hi = a.u0[j];
    const bool lf = isfinite(lo), uf = isfinite(hi);
    const double lh = (lf && uf) ? lam : lf ? fmax(lam, 0.0) : uf ? fmin(lam, 0.0) : 0.0;
    rd2 += (lam - lh) * (lam - lh);
    cx += c * x;
    bt += (lf ? lo * fmax(lh, 0.0) : 0.0) + (uf ? hi * fmin(lh, 0.0) : 0.0);
  }
  double rp2 = 0, yt = 0;
  for (int i = threadIdx.x; i < a.m; i += blockDim.x) {
    const double ax = (double)a.S[om + i] / a.Dr[i];
    const double lo = a.lc0[i], hi = a.uc0[i];
    const double r = ax - fmin(fmax(ax, lo), hi);
    rp2 += r * r;
    const double y = a.Dr[i] * (double)a.yhat[om + i];
    if (y > 0.0 && isfinite(lo)) yt += lo * y;
    if (y < 0.0 && isfinite(hi)) yt += hi * y;
  }
  const double v[5] = {rd2, cx, bt, rp2, yt};
  for (int q = 0; q < 5; ++q) {
    const double s = block_sum(v[q], sh);
    if (threadIdx.x == 0) a.part[(size_t)q * a.B + k] = s;
  }
}

// restart metric pieces: x = w_prev rebuilt is not stored; use the stored x^ and the
// iterate before the check step (xprev) to form |x^ - x|^2 and |x^ - anchor|^2
__global__ void k_fixed_point_cols(const float* __restrict__ xhat, const float* __restrict__ xprev,
                                   const float* __restrict__ xa, const float* __restrict__ yhat,
                                   const float* __restrict__ yprev, const float* __restrict__ ya,
                                   int m, int n, int B, const Inst* inst, double* part) {
  __shared__ double sh[32];
  const int k = blockIdx.x;
  if (inst[k].done) return;
  const size_t on = (size_t)k * n, om = (size_t)k * m;
  double p0 = 0, p1 = 0, d0 = 0, d1 = 0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const double a = (double)xhat[on + j] - (double)xprev[on + j];
    const double b = (double)xhat[on + j] - (double)xa[on + j];
    p0 += a * a;
    p1 += b * b;
  }
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const double a = (double)yhat[om + i] - (double)yprev[om + i];
    const double b = (double)yhat[om + i] - (double)ya[om + i];
    d0 += a * a;
    d1 += b * b;
  }
  const double v[4] = {p0, p1, d0, d1};
  for (int q = 0; q < 4; ++q) {
    const double s = block_sum(v[q], sh);
    if (threadIdx.x == 0) part[(size_t)(5 + q) * B + k] = s;
  }
}

struct CheckParams {
  double eps_abs, eps_rel, r_suff, r_nec, r_art, pw_smooth, eta, b_norm;
  long long iter_limit, now_ns, time_limit_ns;
  int B, check_no, stall_limit;
};

__global__ void k_check_finalize(Inst* inst, const double* part, CheckParams p) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= p.B) return;
  Inst& I = inst[k];
  I.restart = 0;
  if (I.done) return;
  const double rd2 = part[0 * p.B + k], cx = part[1 * p.B + k], bt = part[2 * p.B + k],
               rp2 = part[3 * p.B + k], yt = part[4 * p.B + k];
  const double P0 = part[5 * p.B + k], P1 = part[6 * p.B + k], D0 = part[7 * p.B + k],
               D1 = part[8 * p.B + k];
  const double nrp = sqrt(rp2), nrd = sqrt(rd2), pobj = cx, dobj = yt + bt;
  const double gap = fabs(pobj - dobj);
  const double rel = fmax(fmax(nrp / (1.0 + p.b_norm), nrd / (1.0 + I.c_norm)),
                          gap / (1.0 + fabs(pobj) + fabs(dobj)));
  I.rel = rel;
  I.pobj = pobj;
  I.dobj = dobj;
  const bool conv = nrp <= p.eps_abs + p.eps_rel * p.b_norm &&
                    nrd <= p.eps_abs + p.eps_rel * I.c_norm &&
                    gap <= p.eps_abs + p.eps_rel * (fabs(pobj) + fabs(dobj));
  int term = 0;
  if (!isfinite(rel)) term = MPAX_TERM_NUMERICAL_ERROR;
  else if (conv) term = MPAX_TERM_OPTIMAL;
  else if (I.total >= p.iter_limit) term = MPAX_TERM_ITERATION_LIMIT;
  else if (p.now_ns >= p.time_limit_ns) term = MPAX_TERM_TIME_LIMIT;
  if (term) {
    I.done = 1;
    I.status = term;
    I.done_at = p.now_ns;
    return;
  }
  // the BF16x3 floor (the single-problem rule): no 10% improvement of the KKT
  // error over max(stall_limit, checks / 4) checks marks the instance stalled;
  // the host then continues the batch with FP32 products
  I.checks += 1;
  if (p.stall_limit > 0 && !I.stalled) {
    const long long window = p.stall_limit > I.checks / 4 ? (long long)p.stall_limit : I.checks / 4;
    if (rel < 0.9 * I.best_rel) {
      I.best_rel = rel;
      I.stall_count = 0;
    } else if (++I.stall_count >= window) {
      I.stalled = 1;
    }
  }
  const double r = sqrt(I.omega * P0 + D0 / I.omega);
  const bool restart = !I.have_anchor || r <= p.r_suff * I.r_anchor ||
                       (r <= p.r_nec * I.r_anchor && r > I.r_prev) ||
                       (double)I.k >= p.r_art * (double)I.total;
  if (restart) {
    const double dx = sqrt(P1), dy = sqrt(D1);
    if (dx > 1e-10 && dy > 1e-10)
      I.omega = exp(p.pw_smooth * log(dy / dx) + (1.0 - p.pw_smooth) * log(I.omega));
    I.tau = p.eta / I.omega;
    I.sigma = p.eta * I.omega;
    I.have_anchor = 1;
    I.r_anchor = r;
    I.r_prev = r;
    I.k = 0;
    I.restarts += 1;
    I.restart = 1;
  } else {
    I.r_prev = r;
  }
}

__global__ void k_restart_apply(Vecs v) {
  const int tot = v.n + v.m;
  for (int k = blockIdx.y; k < v.B; k += gridDim.y) {
    if (!v.inst[k].restart) continue;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < tot; t += gridDim.x * blockDim.x) {
      if (t < v.n) {
        const size_t e = (size_t)k * v.n + t;
        const float xh = v.xhat[e];
        v.xa[e] = xh;
        v.w[e] = xh;
        split_store(xh, v.xh_hi, v.xh_lo, (size_t)k * v.ldx + t);
      } else {
        const size_t f = (size_t)k * v.m + (t - v.n);
        const float yh = v.yhat[f];
        v.ya[f] = yh;
        v.y[f] = yh;
        split_store(yh, v.y_hi, v.y_lo, (size_t)k * v.ldy + (t - v.n));
      }
    }
  }
}

// x (before the check step) rebuilt for the fixed-point residual: x = w + (xa - w)/(k+1)
__global__ void k_rebuild_x(const float* __restrict__ w, const float* __restrict__ xa,
                            float* __restrict__ out, int n, int B, const Inst* inst) {
  for (int k = blockIdx.y; k < B; k += gridDim.y)
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    const size_t e = (size_t)k * n + j;
    const Inst& I = inst[k];
    const float rb = (float)(1.0 / (double)(I.k + 1));
    out[e] = (I.k == 0) ? xa[e] : w[e] + rb * (xa[e] - w[e]);
  }
}

__global__ void k_copy_f(const float* __restrict__ s, float* __restrict__ d, size_t total) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x)
    d[e] = s[e];
}

__global__ void k_init_inst(Inst* inst, int B, const double* cnorm_s, const double* cnorm,
                            double bnorm_s, double eta) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= B) return;
  Inst I;
  memset(&I, 0, sizeof(I));
  const double nc = cnorm_s[k];
  I.omega = (nc > 1e-10 && bnorm_s > 1e-10) ? nc / bnorm_s : 1.0;
  I.tau = eta / I.omega;
  I.sigma = eta * I.omega;
  I.c_norm = cnorm[k];
  I.rel = INFINITY;
  I.best_rel = INFINITY;
  inst[k] = I;
}

// ||column k||_2 of an n x B column-major double matrix, optionally scaled by D
__global__ void k_colnorm(const double* __restrict__ Cm, const double* __restrict__ D, int n,
                          double* __restrict__ out) {
  __shared__ double sh[32];
  const int k = blockIdx.x;
  double s = 0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const double v = Cm[(size_t)k * n + j] * (D ? D[j] : 1.0);
    s += v * v;
  }
  s = block_sum(s, sh);
  if (threadIdx.x == 0) out[k] = sqrt(s);
}

__global__ void k_scale_costs(const double* __restrict__ C0, const double* __restrict__ Dc, int n,
                              size_t total, float* __restrict__ ct) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x)
    ct[e] = (float)(C0[e] * Dc[e % n]);
}

__global__ void k_scale_vec(const double* __restrict__ v, const double* __restrict__ D, int div,
                            int n, float* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (float)(div ? v[i] / D[i] : v[i] * D[i]);
}

__global__ void k_unscale_out(const float* __restrict__ v, const double* __restrict__ D, int n,
                              size_t total, double* __restrict__ out) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x)
    out[e] = D[e % n] * (double)v[e];
}

__global__ void k_bound_norm(const double* lc, const double* uc, const double* Dr, int m,
                             double* out) {
  __shared__ double sh[32];
  double s = 0, ss = 0;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const double lo = lc[i], hi = uc[i];
    auto bnd = [](double a, double b) {
      const bool fa = isfinite(a), fb = isfinite(b);
      if (fa && fb) return fabs(a) >= fabs(b) ? a : b;
      if (fa) return a;
      if (fb) return b;
      return 0.0;
    };
    const double b = bnd(lo, hi), bs = bnd(lo * Dr[i], hi * Dr[i]);
    s += b * b;
    ss += bs * bs;
  }
  s = block_sum(s, sh);
  __syncthreads();
  ss = block_sum(ss, sh);
  if (threadIdx.x == 0) {
    out[0] = sqrt(s);
    out[1] = sqrt(ss);
  }
}

__global__ void k_vec_norm_part(const float* __restrict__ v, size_t n, double* __restrict__ out) {
  __shared__ double sh[32];
  double s = 0;
  for (size_t i = threadIdx.x; i < n; i += blockDim.x) s += (double)v[i] * (double)v[i];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) *out = sqrt(s);
}

__global__ void k_scale_f(float* __restrict__ v, size_t n, const double* __restrict__ nrm) {
  const double inv = *nrm > 0 ? 1.0 / *nrm : 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    v[i] = (float)((double)v[i] * inv);
}

// SPO+ (Sec. 3.4): c' = 2 c_hat - c_true; per instance k (one block),
// loss_k = -c'_k^T x~_k + 2 c_hat_k^T x*_k - z*_k and grad_k = 2 (x*_k - x~_k),
// fixed-order FP64 sums (Elmachtoub and Grigas 2022).
__global__ void k_spo_costs2(const double* __restrict__ c_hat, const double* __restrict__ c_true,
                             size_t len, double* __restrict__ out) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < len;
       t += (size_t)gridDim.x * blockDim.x)
    out[t] = 2.0 * c_hat[t] - c_true[t];
}
__global__ void k_spo_loss2(int n, const double* __restrict__ cp, const double* __restrict__ c_hat,
                            const double* __restrict__ x_true, const double* __restrict__ z_true,
                            const double* __restrict__ x_tl, double* __restrict__ loss,
                            double* __restrict__ grad) {
  __shared__ double sh[32];
  const size_t j0 = (size_t)blockIdx.x * n;
  double v = 0.0, t = 0.0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const double xt = x_tl[j0 + j], xs = x_true[j0 + j];
    v += cp[j0 + j] * xt;
    t += c_hat[j0 + j] * xs;
    grad[j0 + j] = 2.0 * (xs - xt);
  }
  v = block_sum(v, sh);
  __syncthreads();
  t = block_sum(t, sh);
  if (threadIdx.x == 0) loss[blockIdx.x] = -v + 2.0 * t - z_true[blockIdx.x];
}
__global__ void k_inst_pobj(const Inst* __restrict__ inst, int B, double* __restrict__ v) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < B) v[k] = inst[k].pobj;
}

}  // namespace
}  // namespace mpax

using namespace mpax;

struct mpax_shared {
  int m = 0, n = 0, B = 0;
  cudaStream_t user = nullptr, s = nullptr;
  float* A0 = nullptr;   // original FP32, row-major m x n
  float* As = nullptr;   // scaled FP32
  __nv_bfloat16 *Ahi = nullptr, *Alo = nullptr;
  double *C0 = nullptr, *lc = nullptr, *uc = nullptr, *l = nullptr, *u = nullptr;
  double *Dr = nullptr, *Dc = nullptr, *red_m = nullptr, *red_n = nullptr, *scal = nullptr;
  float *ct = nullptr, *lf = nullptr, *uf = nullptr, *lcf = nullptr, *ucf = nullptr;
  float *w = nullptr, *xa = nullptr, *xhat = nullptr, *T = nullptr, *xprev = nullptr;
  float *y = nullptr, *ya = nullptr, *yhat = nullptr, *S = nullptr, *yprev = nullptr;
  __nv_bfloat16 *xh_hi = nullptr, *xh_lo = nullptr, *y_hi = nullptr, *y_lo = nullptr;
  double *part = nullptr, *cn = nullptr, *cns = nullptr;
  Inst* inst = nullptr;
  double *Xout = nullptr, *Yout = nullptr;
  bool solved = false;
  double solve_seconds = 0.0, norm_A = 0.0;
  long long launches = 0, gemms = 0;
  double gemm_flops = 0.0;
  long long switch_iter = -1;  // last solve: iteration of the switch to FP32 products
  int switch_active = 0;       // last solve: instances still running at the switch
  std::vector<Inst> h_inst;
  // B = 1: partial sums of the A^T y product over gemv_chunks row chunks and of
  // the A w product over gemv_nchunks column chunks
  float* gpart = nullptr;
  float* gpart_n = nullptr;
  double* spo = nullptr;  // SPO+ staging of host arguments: 3 n B + B doubles
  // tensor-core products: BF16 splits are stored with row strides n8, m8 (n, m
  // rounded up to 8, as TMA wants 16-byte strides; the pad columns stay zero)
  long long n8 = 0, m8 = 0;
  UmmaPlan plan_dual, plan_primal;  // S = A~ X (K = n), T = A~^T Y (K = m)
  int* uerr = nullptr;              // set by a bounded wait of the product kernel
  float shape_ms[2][2] = {{0, 0}, {0, 0}};  // tuner: [dual, primal][K block 64, 32] ms
  double prep_seconds = 0.0;   // last solve: scaling, splits, plans, power iteration
  int power_rounds = 0;        // last solve: rounds of the power iteration
  // profile_kernels: event pairs of the iteration products and their sums
  struct ProdEvent {
    cudaEvent_t e0, e1;
    int trans;
  };
  bool profiling = false;
  std::vector<ProdEvent> prof_events;
  double prof_ms[2] = {0, 0};  // [primal (A~^T Y), dual (A~ X)]
  long long prof_n[2] = {0, 0};
  int gemv_chunks = 1, gemv_nchunks = 1;
  long long gemv_launches = 0;
};

namespace {

void free_shared(mpax_shared* sh) {
  if (!sh) return;
  if (sh->s) cudaStreamSynchronize(sh->s);
  void* bufs[] = {sh->A0,  sh->As,   sh->Ahi,   sh->Alo,   sh->C0,   sh->lc,   sh->uc,
                  sh->l,   sh->u,    sh->Dr,    sh->Dc,    sh->red_m, sh->red_n, sh->scal,
                  sh->ct,  sh->lf,   sh->uf,    sh->lcf,   sh->ucf,  sh->w,    sh->xa,
                  sh->xhat, sh->T,   sh->xprev, sh->y,     sh->ya,   sh->yhat, sh->S,
                  sh->yprev, sh->xh_hi, sh->xh_lo, sh->y_hi, sh->y_lo, sh->part, sh->cn,
                  sh->cns, sh->inst, sh->Xout, sh->Yout, sh->gpart, sh->gpart_n, sh->spo,
                  sh->uerr};
  for (void* b : bufs)
    if (b) cudaFree(b);
  if (sh->s) cudaStreamDestroy(sh->s);
  delete sh;
}

}  // namespace

// Template kernels sit in a named namespace: the host stubs generated for a
// template kernel name its enclosing unnamed namespace, which is ambiguous in
// this file (mpax's and the global one).
namespace mpax_gemv {

// ---- single instance (B = 1, FP32 products): the two matrix-vector products --------
// With one cost vector each product reads A once and is bound by HBM.  Both are
// plain FP32 sums in a fixed order (no atomics), so results do not depend on the
// schedule.  V = 4: float4 loads (n % 4 == 0 and 16-byte aligned rows), else 1.
constexpr int kGemvThreads = 256;

// part[s][j] = sum_{i in chunk s} A_ij y_i: block (bx, s) covers V * 256 columns
// from bx * V * 256 and the rows [s * rows_per, (s + 1) * rows_per), four rows
// in flight per thread.
template <int V>
__global__ void __launch_bounds__(kGemvThreads) k_gemv_t_part(const float* __restrict__ A, int m,
                                                              int n, const float* __restrict__ y,
                                                              int rows_per,
                                                              float* __restrict__ part) {
  const int j0 = (blockIdx.x * kGemvThreads + threadIdx.x) * V;
  if (j0 >= n) return;
  const int r0 = blockIdx.y * rows_per, r1 = min(m, r0 + rows_per);
  float acc[V];
#pragma unroll
  for (int v = 0; v < V; ++v) acc[v] = 0.0f;
  int i = r0;
  for (; i + 4 <= r1; i += 4) {
    float a[4][V];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float* row = A + (size_t)(i + k) * n + j0;
      if constexpr (V == 4) {
        const float4 q = __ldcs(reinterpret_cast<const float4*>(row));
        a[k][0] = q.x;
        a[k][1] = q.y;
        a[k][2] = q.z;
        a[k][3] = q.w;
      } else {
        a[k][0] = __ldcs(row);
      }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float yk = __ldg(y + i + k);
#pragma unroll
      for (int v = 0; v < V; ++v) acc[v] = fmaf(a[k][v], yk, acc[v]);
    }
  }
  for (; i < r1; ++i) {
    const float yk = __ldg(y + i);
    const float* row = A + (size_t)i * n + j0;
#pragma unroll
    for (int v = 0; v < V; ++v) acc[v] = fmaf(__ldcs(row + v), yk, acc[v]);
  }
  float* out = part + (size_t)blockIdx.y * n + j0;
#pragma unroll
  for (int v = 0; v < V; ++v) out[v] = acc[v];
}

// T_j = sum_s part[s][j], s in order.
__global__ void k_gemv_t_sum(const float* __restrict__ part, int chunks, int n,
                             float* __restrict__ T) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    float t = 0.0f;
    for (int c = 0; c < chunks; ++c) t += part[(size_t)c * n + j];
    T[j] = t;
  }
}

// part[c][i] = sum_{j in column chunk c} A_ij w_j for R rows per block: block
// (bx, c) covers rows [bx R, bx R + R) and the columns [c cols_per, (c + 1)
// cols_per) (cols_per a multiple of 4).  Each float4 of w is loaded once and used
// for the R rows, so every thread keeps R independent loads of A in flight; the
// R sums are reduced over the block in a fixed order.
constexpr int kGemvRows = 8;
template <int V>
__global__ void __launch_bounds__(kGemvThreads) k_gemv_n_part(const float* __restrict__ A, int m,
                                                              int n, const float* __restrict__ w,
                                                              int cols_per,
                                                              float* __restrict__ part) {
  constexpr int R = kGemvRows;
  __shared__ float sh[R][kGemvThreads / 32];
  const int r0 = blockIdx.x * R;
  const int j0 = blockIdx.y * cols_per, j1 = min(n, j0 + cols_per);
  float acc[R];
#pragma unroll
  for (int r = 0; r < R; ++r) acc[r] = 0.0f;
  const float* rows[R];
#pragma unroll
  for (int r = 0; r < R; ++r) rows[r] = A + (size_t)min(r0 + r, m - 1) * n;  // valid row
  if constexpr (V == 4) {
    for (int q = j0 / 4 + threadIdx.x; q < j1 / 4; q += kGemvThreads) {
      const float4 wv = __ldg(reinterpret_cast<const float4*>(w) + q);
      float4 a[R];
#pragma unroll
      for (int r = 0; r < R; ++r) a[r] = __ldcs(reinterpret_cast<const float4*>(rows[r]) + q);
#pragma unroll
      for (int r = 0; r < R; ++r)
        acc[r] = fmaf(a[r].x, wv.x, fmaf(a[r].y, wv.y, fmaf(a[r].z, wv.z, fmaf(a[r].w, wv.w, acc[r]))));
    }
  } else {
    for (int j = j0 + threadIdx.x; j < j1; j += kGemvThreads) {
      const float wv = __ldg(w + j);
      float a[R];
#pragma unroll
      for (int r = 0; r < R; ++r) a[r] = __ldcs(rows[r] + j);
#pragma unroll
      for (int r = 0; r < R; ++r) acc[r] = fmaf(a[r], wv, acc[r]);
    }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const float t = mpax::warp_sum(acc[r]);
    if (lane == 0) sh[r][wid] = t;
  }
  __syncthreads();
  if (threadIdx.x < R && r0 + threadIdx.x < m) {
    float t = 0.0f;
#pragma unroll
    for (int k = 0; k < kGemvThreads / 32; ++k) t += sh[threadIdx.x][k];
    part[(size_t)blockIdx.y * m + r0 + threadIdx.x] = t;
  }
}

// ---- B > 1, FP32 products on the CUDA cores ----------------------------------------
// C[n][m] = sum_k A_op[m][k] V[n][k] for the B instances' vectors V (rows of ldv):
// A_op = A~ stored [M][K] (A_MN = 0, the dual step's A~ X) or A~^T of an A~ stored
// [K][M] (A_MN = 1, the primal step's A~^T Y).  CTA tile 128 (M) x 128 (N) x 8 (K),
// 256 threads of 8 x 8 outputs each, accumulated in FP32 in increasing k (one
// fixed order per output).  The next k-slab is read from global memory into
// registers while the current one is multiplied, then stored into the other of
// two shared-memory buffers (one barrier per slab).
constexpr int kSgBM = 128, kSgBN = 128, kSgBK = 8;

template <int A_MN>
__device__ __forceinline__ void sg_load_a(const float* __restrict__ A, long long lda, int M, int K,
                                          int m0, int k0, int tid, float* ra) {
  // 128 x 8 values, 4 per thread
  if (A_MN) {  // rows k0..k0+7 of 128 contiguous m values: thread -> (k, 4 m)
    const int kk = tid / 32, mm = (tid % 32) * 4;
    const int gk = k0 + kk;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int gm = m0 + mm + t;
      ra[t] = (gk < K && gm < M) ? A[(long long)gk * lda + gm] : 0.0f;
    }
  } else {     // 128 rows m of 8 contiguous k values: thread -> (m, 4 k)
    const int r = tid / 2, kq = (tid % 2) * 4;
    const int gm = m0 + r;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int gk = k0 + kq + t;
      ra[t] = (gm < M && gk < K) ? A[(long long)gm * lda + gk] : 0.0f;
    }
  }
}

template <int A_MN>
__device__ __forceinline__ void sg_store_a(float (*As)[kSgBM + 4], int tid, const float* ra) {
  if (A_MN) {
    const int kk = tid / 32, mm = (tid % 32) * 4;
#pragma unroll
    for (int t = 0; t < 4; ++t) As[kk][mm + t] = ra[t];
  } else {
    const int r = tid / 2, kq = (tid % 2) * 4;
#pragma unroll
    for (int t = 0; t < 4; ++t) As[kq + t][r] = ra[t];
  }
}

template <int A_MN>
__global__ void __launch_bounds__(256) k_sgemm(const float* __restrict__ A, long long lda,
                                               const float* __restrict__ V, long long ldv,
                                               float* __restrict__ Cm, long long ldc, int M,
                                               int N, int K) {
  __shared__ __align__(16) float As[2][kSgBK][kSgBM + 4];
  __shared__ __align__(16) float Vs[2][kSgBK][kSgBN + 4];
  const int tid = threadIdx.x;
  const int tm = tid % 16, tn = tid / 16;  // 8 rows (m) and 8 instances (n) each
  const int m0 = blockIdx.x * kSgBM, n0 = blockIdx.y * kSgBN;
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;
  // V slab: 128 rows n of 8 contiguous k values: thread -> (n, 4 k)
  const int vr = tid / 2, vq = (tid % 2) * 4;
  float ra[4], rv[4];
  auto load_v = [&](int k0) {
    const int gn = n0 + vr;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int gk = k0 + vq + t;
      rv[t] = (gn < N && gk < K) ? V[(long long)gn * ldv + gk] : 0.0f;
    }
  };
  sg_load_a<A_MN>(A, lda, M, K, m0, 0, tid, ra);
  load_v(0);
  sg_store_a<A_MN>(As[0], tid, ra);
#pragma unroll
  for (int t = 0; t < 4; ++t) Vs[0][vq + t][vr] = rv[t];
  __syncthreads();
  int buf = 0;
  for (int k0 = 0; k0 < K; k0 += kSgBK) {
    const bool more = k0 + kSgBK < K;
    if (more) {
      sg_load_a<A_MN>(A, lda, M, K, m0, k0 + kSgBK, tid, ra);
      load_v(k0 + kSgBK);
    }
#pragma unroll
    for (int kk = 0; kk < kSgBK; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][tm * 8]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][tm * 8 + 4]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Vs[buf][kk][tn * 8]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Vs[buf][kk][tn * 8 + 4]);
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    if (more) {
      sg_store_a<A_MN>(As[buf ^ 1], tid, ra);
#pragma unroll
      for (int t = 0; t < 4; ++t) Vs[buf ^ 1][vq + t][vr] = rv[t];
    }
    __syncthreads();
    buf ^= 1;
  }
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int gn = n0 + tn * 8 + j;
    if (gn >= N) continue;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int gm = m0 + tm * 8 + i;
      if (gm < M) Cm[(long long)gn * ldc + gm] = acc[i][j];
    }
  }
}

}  // namespace mpax_gemv

namespace {

using namespace mpax_gemv;

// B = 1, FP32 products: the partial-sum kernel of one product, trans = 1: A v
// into gpart_n (column chunks), trans = 0: A^T v into gpart (row chunks).
void gemv_part(mpax_shared* sh, int trans, const float* vf, const float* Mf) {
  const int m = sh->m, n = sh->n;
  const bool v4 = (n % 4 == 0) && ((reinterpret_cast<uintptr_t>(Mf) & 15) == 0) &&
                  ((reinterpret_cast<uintptr_t>(vf) & 15) == 0);
  if (trans) {
    const dim3 grid((m + kGemvRows - 1) / kGemvRows, sh->gemv_nchunks);
    const int cols_per = ((n + sh->gemv_nchunks - 1) / sh->gemv_nchunks + 3) / 4 * 4;
    if (v4) k_gemv_n_part<4><<<grid, kGemvThreads, 0, sh->s>>>(Mf, m, n, vf, cols_per, sh->gpart_n);
    else k_gemv_n_part<1><<<grid, kGemvThreads, 0, sh->s>>>(Mf, m, n, vf, cols_per, sh->gpart_n);
  } else {
    const int V = v4 ? 4 : 1;
    const dim3 grid((n + V * kGemvThreads - 1) / (V * kGemvThreads), sh->gemv_chunks);
    const int rows_per = (m + sh->gemv_chunks - 1) / sh->gemv_chunks;
    if (v4) k_gemv_t_part<4><<<grid, kGemvThreads, 0, sh->s>>>(Mf, m, n, vf, rows_per, sh->gpart);
    else k_gemv_t_part<1><<<grid, kGemvThreads, 0, sh->s>>>(Mf, m, n, vf, rows_per, sh->gpart);
  }
  sh->gemv_launches += 1;
  sh->gemms += 1;
  sh->gemm_flops += 2.0 * m * (double)n;
}

// C (rows x B, col-major) = op(M) V, M the stored column-major n x m matrix
// (A row-major).  trans = 1: C = M^T V (= A V, rows = m, K = n); trans = 0:
// C = M V (= A^T V, rows = n, K = m).  BF16x3 or FP32.
cudaError_t product_impl(mpax_shared* sh, int trans, const __nv_bfloat16* vhi,
                         const __nv_bfloat16* vlo, const float* vf, float* C, bool bf16x3,
                         const float* Mf);

// With profile_kernels set, every iteration product is bracketed by CUDA events
// on the solve's stream; the host sums the times after each check block.
cudaError_t product(mpax_shared* sh, int trans, const __nv_bfloat16* vhi,
                    const __nv_bfloat16* vlo, const float* vf, float* C, bool bf16x3,
                    const float* Mf) {
  if (!sh->profiling) return product_impl(sh, trans, vhi, vlo, vf, C, bf16x3, Mf);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, sh->s);
  const cudaError_t e = product_impl(sh, trans, vhi, vlo, vf, C, bf16x3, Mf);
  cudaEventRecord(e1, sh->s);
  sh->prof_events.push_back({e0, e1, trans});
  return e;
}

void collect_product_times(mpax_shared* sh) {
  for (const auto& pe : sh->prof_events) {
    float ms = 0.f;
    cudaEventSynchronize(pe.e1);
    cudaEventElapsedTime(&ms, pe.e0, pe.e1);
    sh->prof_ms[pe.trans] += ms;
    sh->prof_n[pe.trans] += 1;
    cudaEventDestroy(pe.e0);
    cudaEventDestroy(pe.e1);
  }
  sh->prof_events.clear();
}

cudaError_t product_impl(mpax_shared* sh, int trans, const __nv_bfloat16* vhi,
                         const __nv_bfloat16* vlo, const float* vf, float* C, bool bf16x3,
                         const float* Mf) {
  const int m = sh->m, n = sh->n, B = sh->B;
  const int rows = trans ? m : n, K = trans ? n : m;
  if (!bf16x3 && B == 1) {
    gemv_part(sh, trans, vf, Mf);
    if (trans) k_gemv_t_sum<<<g1(m), 256, 0, sh->s>>>(sh->gpart_n, sh->gemv_nchunks, m, C);
    else k_gemv_t_sum<<<g1(n), 256, 0, sh->s>>>(sh->gpart, sh->gemv_chunks, n, C);
    sh->gemv_launches += 1;
    return cudaGetLastError();
  }
  if (!bf16x3) {
    // FP32 on the CUDA cores: trans = 1 is A~ V (A~ [m][n] K-major), trans = 0
    // is A~^T V (the same storage read M-major)
    const dim3 grid((rows + kSgBM - 1) / kSgBM, (B + kSgBN - 1) / kSgBN);
    if (trans) k_sgemm<0><<<grid, 256, 0, sh->s>>>(Mf, n, vf, K, C, rows, rows, B, K);
    else k_sgemm<1><<<grid, 256, 0, sh->s>>>(Mf, n, vf, K, C, rows, rows, B, K);
    sh->gemms += 1;
    sh->gemm_flops += 2.0 * rows * (double)B * K;
    return cudaGetLastError();
  }
  // A_hi V_lo + A_lo V_hi + A_hi V_hi in one tensor-core kernel (umma.cuh); the
  // plan of this direction holds the split buffers (vhi, vlo) and the output C
  (void)vhi;
  (void)vlo;
  const UmmaPlan& p = trans ? sh->plan_dual : sh->plan_primal;
  const cudaError_t e = umma_run(p, sh->s);
  sh->gemms += 1;
  sh->gemm_flops += p.flops;
  return e;
}

// The two products' plans.  Their pipeline shape (K block 64 with two stages,
// or 32 with four; the same sums in the same order) is chosen per direction by
// timing both on this solve's own buffers, once per (m, n, B) for the process.
std::mutex& shape_mutex() {
  static std::mutex mu;
  return mu;
}
std::map<std::tuple<int, int, int>, std::pair<int, int>>& shape_cache() {
  static std::map<std::tuple<int, int, int>, std::pair<int, int>> c;
  return c;
}

cudaError_t plan_products(mpax_shared* sh, bool tune) {
  const int m = sh->m, n = sh->n, B = sh->B;
  auto make = [&](UmmaPlan* p, int dir, int bk) {
    return dir == 0 ? umma_plan(p, sh->Ahi, sh->Alo, sh->n8, 0, sh->xh_hi, sh->xh_lo, sh->n8, m,
                                B, n, sh->S, m, sh->uerr, bk)
                    : umma_plan(p, sh->Ahi, sh->Alo, sh->n8, 1, sh->y_hi, sh->y_lo, sh->m8, n,
                                B, m, sh->T, n, sh->uerr, bk);
  };
  const auto key = std::make_tuple(m, n, B);
  std::pair<int, int> bk(32, 32);
  bool have;
  {
    std::lock_guard<std::mutex> g(shape_mutex());
    auto it = shape_cache().find(key);
    have = it != shape_cache().end();
    if (have) bk = it->second;
  }
  cudaError_t e;
  if (!have && tune) {
    // the products write S and T, scratch until the iteration starts
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int best[2] = {32, 32};
    for (int dir = 0; dir < 2; ++dir) {
      float tbest = INFINITY;
      for (int cand : {64, 32}) {
        UmmaPlan p;
        if ((e = make(&p, dir, cand))) return e;
        if ((e = umma_run(p, sh->s))) return e;
        cudaEventRecord(e0, sh->s);
        for (int r = 0; r < 2; ++r) umma_run(p, sh->s);
        cudaEventRecord(e1, sh->s);
        if ((e = cudaEventSynchronize(e1))) return e;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        sh->shape_ms[dir][cand == 64 ? 0 : 1] = ms / 2;
        if (ms < tbest) {
          tbest = ms;
          best[dir] = cand;
        }
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    bk = std::make_pair(best[0], best[1]);
    std::lock_guard<std::mutex> g(shape_mutex());
    shape_cache()[key] = bk;
  }
  if ((e = make(&sh->plan_dual, 0, bk.first))) return e;
  return make(&sh->plan_primal, 1, bk.second);
}

}  // namespace

extern "C" {

mpax_status mpax_lp_shared_create(int32_t m, int32_t n, int32_t B, const float* A,
                                  const double* C, const double* lc, const double* uc,
                                  const double* l, const double* u, mpax_mem_kind kind,
                                  void* cuda_stream, mpax_shared** out) {
  if (!out) return sfail(MPAX_ERR_INVALID_ARGUMENT, "out must not be NULL");
  *out = nullptr;
  if (m < 1 || n < 1 || B < 1) return sfail(MPAX_ERR_INVALID_ARGUMENT, "m, n, B must be >= 1");
  if (!A || !C || !lc || !uc || !l || !u)
    return sfail(MPAX_ERR_INVALID_ARGUMENT, "a required array pointer is NULL");
  mpax_shared* sh = new mpax_shared();
  sh->m = m;
  sh->n = n;
  sh->B = B;
  sh->user = (cudaStream_t)cuda_stream;
  const size_t mn = (size_t)m * n, nB = (size_t)n * B, mB = (size_t)m * B;
  cudaError_t e = cudaStreamCreateWithFlags(&sh->s, cudaStreamNonBlocking);
  auto al = [&](auto** p, size_t cnt) {
    if (!e) e = cudaMalloc((void**)p, sizeof(**p) * std::max<size_t>(cnt, 1));
  };
  al(&sh->A0, mn);
  al(&sh->As, mn);
  sh->n8 = ((long long)n + 7) / 8 * 8;
  sh->m8 = ((long long)m + 7) / 8 * 8;
  al(&sh->Ahi, (size_t)m * sh->n8);
  al(&sh->Alo, (size_t)m * sh->n8);
  al(&sh->C0, nB);
  al(&sh->lc, m);
  al(&sh->uc, m);
  al(&sh->l, n);
  al(&sh->u, n);
  al(&sh->Dr, m);
  al(&sh->Dc, n);
  al(&sh->red_m, m);
  al(&sh->red_n, n);
  al(&sh->scal, 8);
  al(&sh->ct, nB);
  al(&sh->lf, n);
  al(&sh->uf, n);
  al(&sh->lcf, m);
  al(&sh->ucf, m);
  for (float** p : {&sh->w, &sh->xa, &sh->xhat, &sh->T, &sh->xprev}) al(p, nB);
  for (float** p : {&sh->y, &sh->ya, &sh->yhat, &sh->S, &sh->yprev}) al(p, mB);
  al(&sh->xh_hi, (size_t)B * sh->n8);
  al(&sh->xh_lo, (size_t)B * sh->n8);
  al(&sh->y_hi, (size_t)B * sh->m8);
  al(&sh->y_lo, (size_t)B * sh->m8);
  al(&sh->uerr, 1);
  al(&sh->part, 16 * (size_t)B);
  al(&sh->cn, B);
  al(&sh->cns, B);
  al(&sh->inst, B);
  al(&sh->Xout, nB);
  al(&sh->Yout, mB);
  {
    // (every B: the power iteration's matrix-vector products use them too)
    // row chunks of the A^T y product: about four blocks per SM in all
    const long long tiles = (n + 4LL * kGemvThreads - 1) / (4LL * kGemvThreads);
    const long long want = (4LL * 152 + tiles - 1) / tiles;
    sh->gemv_chunks = (int)std::max(1LL, std::min(want, std::max(1LL, (long long)m / 16)));
    al(&sh->gpart, (size_t)sh->gemv_chunks * n);
    // column chunks of the A w product (multiples of 1024 columns)
    const long long groups = (m + kGemvRows - 1) / kGemvRows;
    const long long want_n = (4LL * 152 + groups - 1) / groups;
    sh->gemv_nchunks = (int)std::max(1LL, std::min(want_n, (n + 1023LL) / 1024));
    al(&sh->gpart_n, (size_t)sh->gemv_nchunks * m);
  }
  const cudaMemcpyKind k = kind == MPAX_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  for (void* q : {(void*)sh->xh_hi, (void*)sh->xh_lo})
    if (!e) e = cudaMemset(q, 0, sizeof(__nv_bfloat16) * (size_t)B * sh->n8);
  for (void* q : {(void*)sh->y_hi, (void*)sh->y_lo})
    if (!e) e = cudaMemset(q, 0, sizeof(__nv_bfloat16) * (size_t)B * sh->m8);
  if (!e) e = cudaMemset(sh->uerr, 0, sizeof(int));
  if (!e) e = cudaMemcpy(sh->A0, A, sizeof(float) * mn, k);
  if (!e) e = cudaMemcpy(sh->C0, C, sizeof(double) * nB, k);
  if (!e) e = cudaMemcpy(sh->lc, lc, sizeof(double) * m, k);
  if (!e) e = cudaMemcpy(sh->uc, uc, sizeof(double) * m, k);
  if (!e) e = cudaMemcpy(sh->l, l, sizeof(double) * n, k);
  if (!e) e = cudaMemcpy(sh->u, u, sizeof(double) * n, k);
  if (e) {
    free_shared(sh);
    return sfail(e == cudaErrorMemoryAllocation ? MPAX_ERR_OUT_OF_MEMORY : MPAX_ERR_CUDA,
                 cudaGetErrorString(e));
  }
*out = sh;
  return MPAX_OK;
}

mpax_status mpax_shared_solve(mpax_shared* sh, const mpax_options* o, int32_t fp32_products) {
  if (!sh || !o) return sfail(MPAX_ERR_INVALID_ARGUMENT, "NULL argument");
  if (o->reflection_gamma != 1.0 || o->check_every < 1 || o->iteration_limit < 1 ||
      !(o->time_limit >= 0) || o->power_max_iter < 0 ||
      (o->power_max_iter == 0 && !o->pock_chambolle))
    return sfail(MPAX_ERR_INVALID_ARGUMENT, "invalid options (reflection_gamma must be 1)");
  const auto t0 = std::chrono::steady_clock::now();
  const int m = sh->m, n = sh->n, B = sh->B;
  const size_t mn = (size_t)m * n, nB = (size_t)n * B, mB = (size_t)m * B;
  cudaStream_t s = sh->s;
  cudaEvent_t ev;
  cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  cudaEventRecord(ev, sh->user);
  cudaStreamWaitEvent(s, ev, 0);
  long long L = 0;
  sh->gemms = 0;
  sh->profiling = o->profile_kernels != 0;
  sh->prof_ms[0] = sh->prof_ms[1] = 0.0;
  sh->prof_n[0] = sh->prof_n[1] = 0;
  sh->gemm_flops = 0.0;
  sh->gemv_launches = 0;
  // ---- scaling of the shared matrix (Ruiz, Pock-Chambolle) ----------------------
  auto fill1 = [&](double* p, int cnt) {
    std::vector<double> ones(cnt, 1.0);
    cudaMemcpyAsync(p, ones.data(), sizeof(double) * cnt, cudaMemcpyHostToDevice, s);
    cudaStreamSynchronize(s);
  };
  fill1(sh->Dr, m);
  fill1(sh->Dc, n);
  cudaMemcpyAsync(sh->As, sh->A0, sizeof(float) * mn, cudaMemcpyDeviceToDevice, s);
  for (int t = 0; t < o->ruiz_iters; ++t) {
    k_row_red<<<std::min(m, 4096), 256, 0, s>>>(sh->As, m, n, 0, sh->red_m);
    k_col_red<<<(n + 255) / 256, 256, 0, s>>>(sh->As, m, n, 0, sh->red_n);
    k_factor<<<(m + 255) / 256, 256, 0, s>>>(sh->red_m, m, sh->Dr);
    k_factor<<<(n + 255) / 256, 256, 0, s>>>(sh->red_n, n, sh->Dc);
    k_scale_dense<<<g1(mn), 256, 0, s>>>(sh->As, sh->As, m, n, sh->red_m, sh->red_n);
    L += 5;
  }
  if (o->pock_chambolle) {
    k_row_red<<<std::min(m, 4096), 256, 0, s>>>(sh->As, m, n, 1, sh->red_m);
    k_col_red<<<(n + 255) / 256, 256, 0, s>>>(sh->As, m, n, 1, sh->red_n);
    k_factor<<<(m + 255) / 256, 256, 0, s>>>(sh->red_m, m, sh->Dr);
    k_factor<<<(n + 255) / 256, 256, 0, s>>>(sh->red_n, n, sh->Dc);
    L += 4;
  }
  k_scale_dense<<<g1(mn), 256, 0, s>>>(sh->A0, sh->As, m, n, sh->Dr, sh->Dc);
  split_rows(sh->As, m, n, n, sh->Ahi, sh->Alo, sh->n8, s);
  {
    cudaError_t pe = plan_products(sh, !fp32_products);
    if (pe) {
      cudaEventDestroy(ev);
      return sfail(MPAX_ERR_CUDA, std::string("tensor-core product plan: ") +
                                      cudaGetErrorString(pe));
    }
  }
  k_scale_costs<<<g1(nB), 256, 0, s>>>(sh->C0, sh->Dc, n, nB, sh->ct);
  k_scale_vec<<<(n + 255) / 256, 256, 0, s>>>(sh->l, sh->Dc, 1, n, sh->lf);
  k_scale_vec<<<(n + 255) / 256, 256, 0, s>>>(sh->u, sh->Dc, 1, n, sh->uf);
  k_scale_vec<<<(m + 255) / 256, 256, 0, s>>>(sh->lc, sh->Dr, 0, m, sh->lcf);
  k_scale_vec<<<(m + 255) / 256, 256, 0, s>>>(sh->uc, sh->Dr, 0, m, sh->ucf);
  L += 7;
  // ---- ||A~||_2 by power iteration (FP32 products, FP64 norms) --------------------
  {
    float* v = sh->T;    // n (first column of T as scratch)
    float* wv = sh->S;   // m
    std::vector<float> v0(n);  // the common start vector (power_start_raw), normalised
    double ss = 0.0;
    for (int j = 0; j < n; ++j) ss += power_start_raw(j) * power_start_raw(j);
    const double inv = 1.0 / std::sqrt(ss > 0.0 ? ss : 1.0);
    for (int j = 0; j < n; ++j) v0[j] = (float)(power_start_raw(j) * inv);
    cudaMemcpyAsync(v, v0.data(), sizeof(float) * n, cudaMemcpyHostToDevice, s);
    double prev = 0.0, nu = 0.0, d_prev = 0.0;
    sh->power_rounds = 0;
    for (int t = 1; t <= o->power_max_iter; ++t) {
      sh->power_rounds = t;
      // wv = A~ v, v = A~^T wv with this file's matrix-vector kernels
      gemv_part(sh, 1, v, sh->As);
      k_gemv_t_sum<<<g1(m), 256, 0, s>>>(sh->gpart_n, sh->gemv_nchunks, m, wv);
      gemv_part(sh, 0, wv, sh->As);
      k_gemv_t_sum<<<g1(n), 256, 0, s>>>(sh->gpart, sh->gemv_chunks, n, v);
      k_vec_norm_part<<<1, 512, 0, s>>>(v, n, sh->scal);
      double nrm = 0.0;
      cudaMemcpyAsync(&nrm, sh->scal, sizeof(double), cudaMemcpyDeviceToHost, s);
      cudaStreamSynchronize(s);
      k_scale_f<<<g1(n), 256, 0, s>>>(v, n, sh->scal);
      L += 4;
      if (nrm == 0.0) break;
      nu = std::sqrt(nrm);
      double est = nu;
      const double cap = o->pock_chambolle ? 1.0 : INFINITY;
      if (t > 1 && power_stop(nu, prev, &d_prev, o->power_tol, cap, &est)) {
        nu = est;
        break;
      }
      if (t == o->power_max_iter && std::isfinite(cap)) nu = cap;
      prev = nu;
    }
    if (o->power_max_iter == 0) nu = 1.0;  // the bound of the Pock-Chambolle round
    sh->norm_A = nu;
  }
  const double eta = sh->norm_A > 0 ? o->step_safety / sh->norm_A : 1.0;
  cudaStreamSynchronize(s);
  sh->prep_seconds =
      std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  // ---- per-instance initial state --------------------------------------------------
  k_colnorm<<<B, 256, 0, s>>>(sh->C0, sh->Dc, n, sh->cns);
  k_colnorm<<<B, 256, 0, s>>>(sh->C0, nullptr, n, sh->cn);
  k_bound_norm<<<1, 512, 0, s>>>(sh->lc, sh->uc, sh->Dr, m, sh->scal);
  double bn[2];
  cudaMemcpyAsync(bn, sh->scal, sizeof(bn), cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  k_init_inst<<<(B + 255) / 256, 256, 0, s>>>(sh->inst, B, sh->cns, sh->cn, bn[1], eta);
  for (void* p : {(void*)sh->w, (void*)sh->xa, (void*)sh->xhat})
    cudaMemsetAsync(p, 0, sizeof(float) * nB, s);
  for (void* p : {(void*)sh->y, (void*)sh->ya, (void*)sh->yhat})
    cudaMemsetAsync(p, 0, sizeof(float) * mB, s);
  cudaMemsetAsync(sh->xh_hi, 0, sizeof(__nv_bfloat16) * B * sh->n8, s);
  cudaMemsetAsync(sh->xh_lo, 0, sizeof(__nv_bfloat16) * B * sh->n8, s);
  cudaMemsetAsync(sh->y_hi, 0, sizeof(__nv_bfloat16) * B * sh->m8, s);
  cudaMemsetAsync(sh->y_lo, 0, sizeof(__nv_bfloat16) * B * sh->m8, s);
  cudaMemsetAsync(sh->uerr, 0, sizeof(int), s);
  L += 4;
  bool bf = !fp32_products;
  long long switch_iter = -1;  // iteration at which BF16x3 gave way to FP32 products
  int switch_active = 0;
  Vecs V{m, n, B, sh->ct, sh->lf, sh->uf, sh->lcf, sh->ucf, sh->w, sh->xa, sh->xhat, sh->T,
         sh->y, sh->ya, sh->yhat, sh->S, sh->xh_hi, sh->xh_lo, sh->y_hi, sh->y_lo, sh->part,
         sh->inst, sh->n8, sh->m8};
  KktArgs K{m, n, B, sh->xhat, sh->yhat, sh->S, sh->T, nullptr, sh->xa, nullptr, sh->ya,
            sh->Dr, sh->Dc, sh->C0, sh->lc, sh->uc, sh->l, sh->u, sh->part};
  long long done_iters = 0;
  int check_no = 0;
  // time limit, checked at each KKT check against the host clock
  const long long tl_ns = o->time_limit >= 9.0e9 ? LLONG_MAX : (long long)(o->time_limit * 1e9);
  std::vector<Inst> hi(B);
  mpax_status result = MPAX_OK;
  while (true) {
    const int len = (int)std::min<long long>(o->check_every, o->iteration_limit - done_iters);
    for (int it = 0; it < len; ++it) {
      const int chk = (it == len - 1);
      if (chk) {  // the iterate before the check step, for the fixed-point residual
        k_rebuild_x<<<grid2d(n, B), 256, 0, s>>>(sh->w, sh->xa, sh->xprev, n, B, sh->inst);
        k_copy_f<<<g1(mB), 256, 0, s>>>(sh->y, sh->yprev, mB);
        L += 2;
      }
      if (B == 1 && !bf) {
        // one instance, FP32: GEMV partials, summed inside the update kernels
        gemv_part(sh, 0, sh->y, sh->As);
        k_primal<<<grid2d(n, B), 256, 0, s>>>(V, chk, sh->gpart, sh->gemv_chunks);
        gemv_part(sh, 1, sh->w, sh->As);
        k_dual<<<grid2d(m, B), 256, 0, s>>>(V, chk, sh->gpart_n, sh->gemv_nchunks);
        k_advance<<<(B + 255) / 256, 256, 0, s>>>(sh->inst, B);
        L += 3;
        continue;
      }
      if (product(sh, 0, sh->y_hi, sh->y_lo, sh->y, sh->T, bf, sh->As)) {
        result = sfail(MPAX_ERR_CUDA, "matrix product launch failed");
        break;
      }
      k_primal<<<grid2d(n, B), 256, 0, s>>>(V, chk, nullptr, 0);
      // the dual product reads the reflected point w (FP32) or its BF16 split
      if (product(sh, 1, sh->xh_hi, sh->xh_lo, sh->w, sh->S, bf, sh->As)) {
        result = sfail(MPAX_ERR_CUDA, "matrix product launch failed");
        break;
      }
      k_dual<<<grid2d(m, B), 256, 0, s>>>(V, chk, nullptr, 0);
      k_advance<<<(B + 255) / 256, 256, 0, s>>>(sh->inst, B);
      L += 3;
    }
    if (result) break;
    done_iters += len;
    ++check_no;
    // KKT products at (x^, y^): S = A~ x^, T = A~^T y^ (the x^/y^ splits reuse the
    // BF16 buffers; the iteration rewrites them before its next product)
    split_rows(sh->xhat, B, n, n, sh->xh_hi, sh->xh_lo, sh->n8, s);
    split_rows(sh->yhat, B, m, m, sh->y_hi, sh->y_lo, sh->m8, s);
    product(sh, 1, sh->xh_hi, sh->xh_lo, sh->xhat, sh->S, bf, sh->As);
    product(sh, 0, sh->y_hi, sh->y_lo, sh->yhat, sh->T, bf, sh->As);
    k_kkt_cols<<<B, 256, 0, s>>>(K, sh->inst);
    k_fixed_point_cols<<<B, 256, 0, s>>>(sh->xhat, sh->xprev, sh->xa, sh->yhat, sh->yprev,
                                         sh->ya, m, n, B, sh->inst, sh->part);
    CheckParams cp{o->eps_abs, o->eps_rel, o->restart_sufficient, o->restart_necessary,
                   o->restart_artificial, o->primal_weight_smoothing, eta, bn[0],
                   o->iteration_limit,
                   (long long)std::chrono::duration_cast<std::chrono::nanoseconds>(
                       std::chrono::steady_clock::now() - t0).count(),
                   tl_ns, B, check_no, (bf && o->fp64_continuation) ? o->stall_checks : 0};
    k_check_finalize<<<(B + 255) / 256, 256, 0, s>>>(sh->inst, sh->part, cp);
    // the BF16 splits of the iterates are rebuilt (restart copies x^, y^ into them)
    split_rows(sh->w, B, n, n, sh->xh_hi, sh->xh_lo, sh->n8, s);
    split_rows(sh->y, B, m, m, sh->y_hi, sh->y_lo, sh->m8, s);
    k_restart_apply<<<grid2d(n + m, B), 256, 0, s>>>(V);
    L += 8;
    cudaMemcpyAsync(hi.data(), sh->inst, sizeof(Inst) * B, cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    if (sh->profiling) collect_product_times(sh);
    int active = 0, stalled = 0;
    for (const Inst& I : hi) {
      active += !I.done;
      stalled += !I.done && I.stalled;
    }
    if (!active) break;
    if (bf && stalled) {
      // an instance reached the BF16x3 floor: the rest of the solve forms its
      // products in FP32 (the iterates are FP32 throughout, so nothing converts)
      bf = false;
      switch_iter = done_iters;
      switch_active = active;
    }
  }
  if (sh->profiling) collect_product_times(sh);
  cudaError_t e = cudaGetLastError();
  if (!result && e) result = sfail(MPAX_ERR_CUDA, cudaGetErrorString(e));
  {
    int herr = 0;
    cudaMemcpyAsync(&herr, sh->uerr, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    if (!result && herr)
      result = sfail(MPAX_ERR_DEVICE_TIMEOUT, "a bounded wait of the tensor-core product gave up");
  }
  k_unscale_out<<<g1(nB), 256, 0, s>>>(sh->xhat, sh->Dc, n, nB, sh->Xout);
  k_unscale_out<<<g1(mB), 256, 0, s>>>(sh->yhat, sh->Dr, m, mB, sh->Yout);
  L += 2;
  cudaStreamSynchronize(s);
  cudaEventRecord(ev, s);
  cudaStreamWaitEvent(sh->user, ev, 0);
  cudaEventDestroy(ev);
  sh->h_inst = hi;
  sh->launches = L + sh->gemv_launches;
  sh->switch_iter = switch_iter;
  sh->switch_active = switch_active;
  sh->solved = !result;
  sh->solve_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return result;
}

mpax_status mpax_shared_get_solution(const mpax_shared* sh, double* X, double* Y,
                                     mpax_mem_kind kind) {
  if (!sh) return sfail(MPAX_ERR_INVALID_ARGUMENT, "NULL argument");
  if (!sh->solved) return sfail(MPAX_ERR_NOT_SOLVED, "call mpax_shared_solve first");
  const cudaMemcpyKind k = kind == MPAX_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  cudaError_t e = cudaSuccess;
  if (X) e = cudaMemcpy(X, sh->Xout, sizeof(double) * (size_t)sh->n * sh->B, k);
  if (!e && Y) e = cudaMemcpy(Y, sh->Yout, sizeof(double) * (size_t)sh->m * sh->B, k);
  if (e) return sfail(MPAX_ERR_CUDA, cudaGetErrorString(e));
  return MPAX_OK;
}

mpax_status mpax_shared_get_stats(const mpax_shared* sh, mpax_batch_stats* stats,
                                  int32_t* status, int64_t* iterations, double* rel_kkt,
                                  double* primal_obj, double* seconds, double* gemm_info) {
  if (!sh || !stats) return sfail(MPAX_ERR_INVALID_ARGUMENT, "NULL argument");
  if (!sh->solved) return sfail(MPAX_ERR_NOT_SOLVED, "call mpax_shared_solve first");
  std::memset(stats, 0, sizeof(*stats));
  stats->B = sh->B;
  std::vector<double> secs(sh->B);
  for (int k = 0; k < sh->B; ++k) {
    const Inst& I = sh->h_inst[k];
    stats->n_optimal += I.status == MPAX_TERM_OPTIMAL;
    stats->iterations_total += I.total;
    stats->iterations_max = std::max<long long>(stats->iterations_max, I.total);
    stats->restarts_total += I.restarts;
    stats->rel_kkt_max = std::max(stats->rel_kkt_max, I.rel);
    secs[k] = I.done_at * 1e-9;
    if (status) status[k] = I.status;
    if (iterations) iterations[k] = I.total;
    if (rel_kkt) rel_kkt[k] = I.rel;
    if (primal_obj) primal_obj[k] = I.pobj;
    if (seconds) seconds[k] = secs[k];
  }
  std::vector<double> so = secs;
  std::sort(so.begin(), so.end());
  auto pct = [&](double q) {
    const size_t i = std::min<size_t>(so.size() - 1, (size_t)std::ceil(q * so.size()) - 1);
    return so[i];
  };
  stats->instance_seconds_p50 = pct(0.5);
  stats->instance_seconds_p99 = pct(0.99);
  stats->instance_seconds_max = so.back();
  stats->solve_seconds = sh->solve_seconds;
  stats->kernel_launches = sh->launches;
  stats->fp64_instances = sh->switch_active;
  if (gemm_info) {
    gemm_info[0] = (double)sh->gemms;
    gemm_info[1] = sh->gemm_flops;
    gemm_info[2] = sh->norm_A;
    gemm_info[3] = sh->plan_dual.bk;
    gemm_info[4] = sh->plan_primal.bk;
    gemm_info[5] = sh->prof_n[1] ? sh->prof_ms[1] / sh->prof_n[1] : 0.0;
    gemm_info[6] = sh->prof_n[0] ? sh->prof_ms[0] / sh->prof_n[0] : 0.0;
    gemm_info[7] = sh->prep_seconds;
    gemm_info[8] = sh->power_rounds;
  }
  return MPAX_OK;
}

mpax_status mpax_shared_set_costs(mpax_shared* sh, const double* C, mpax_mem_kind kind) {
  if (!sh || !C) return sfail(MPAX_ERR_INVALID_ARGUMENT, "NULL argument");
  const cudaMemcpyKind k = kind == MPAX_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  cudaEvent_t ev;
  cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  cudaEventRecord(ev, sh->user);
  cudaStreamWaitEvent(sh->s, ev, 0);
  cudaError_t e = cudaMemcpyAsync(sh->C0, C, sizeof(double) * (size_t)sh->n * sh->B, k, sh->s);
  if (!e) e = cudaStreamSynchronize(sh->s);
  cudaEventDestroy(ev);
  if (e) return sfail(MPAX_ERR_CUDA, cudaGetErrorString(e));
  sh->solved = false;
  return MPAX_OK;
}

mpax_status mpax_shared_get_objective(const mpax_shared* sh, double* v, mpax_mem_kind kind) {
  if (!sh || !v) return sfail(MPAX_ERR_INVALID_ARGUMENT, "NULL argument");
  if (!sh->solved) return sfail(MPAX_ERR_NOT_SOLVED, "call mpax_shared_solve first");
  cudaError_t e;
  if (kind == MPAX_MEM_HOST) {
    for (int k = 0; k < sh->B; ++k) v[k] = sh->h_inst[k].pobj;
    return MPAX_OK;
  }
  k_inst_pobj<<<(sh->B + 255) / 256, 256, 0, sh->s>>>(sh->inst, sh->B, v);
  e = cudaGetLastError();
  if (!e) e = cudaStreamSynchronize(sh->s);
  if (e) return sfail(MPAX_ERR_CUDA, cudaGetErrorString(e));
  return MPAX_OK;
}

mpax_status mpax_shared_spo_plus(mpax_shared* sh, const mpax_options* o, int32_t fp32_products,
                                 const double* C_hat, const double* C_true, const double* X_true,
                                 const double* z_true, double* loss, double* grad,
                                 mpax_mem_kind kind) {
  if (!sh || !o || !C_hat || !C_true || !X_true || !z_true || !loss || !grad)
    return sfail(MPAX_ERR_INVALID_ARGUMENT, "NULL argument");
  const int B = sh->B, n = sh->n;
  const size_t nB = (size_t)n * B;
  cudaStream_t s = sh->s;
  cudaEvent_t ev;
  cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  cudaEventRecord(ev, sh->user);
  cudaStreamWaitEvent(s, ev, 0);
  cudaEventDestroy(ev);
  cudaError_t e = cudaSuccess;
  if (kind == MPAX_MEM_HOST) {
    if (!sh->spo) e = cudaMalloc(&sh->spo, sizeof(double) * (3 * nB + B));
    double* d = sh->spo;
    if (!e) e = cudaMemcpyAsync(d, C_hat, sizeof(double) * nB, cudaMemcpyHostToDevice, s);
    if (!e) e = cudaMemcpyAsync(d + nB, C_true, sizeof(double) * nB, cudaMemcpyHostToDevice, s);
    if (!e) e = cudaMemcpyAsync(d + 2 * nB, X_true, sizeof(double) * nB, cudaMemcpyHostToDevice, s);
    if (!e) e = cudaMemcpyAsync(d + 3 * nB, z_true, sizeof(double) * B, cudaMemcpyHostToDevice, s);
    C_hat = d;
    C_true = d + nB;
    X_true = d + 2 * nB;
    z_true = d + 3 * nB;
  }
  if (!e) {
    k_spo_costs2<<<g1(nB), 256, 0, s>>>(C_hat, C_true, nB, sh->C0);
    e = cudaGetLastError();
  }
  if (!e) e = cudaStreamSynchronize(s);
  if (e) return sfail(MPAX_ERR_CUDA, cudaGetErrorString(e));
  mpax_status st = mpax_shared_solve(sh, o, fp32_products);
  if (st) return st;
  double* dl = loss;
  double* dg = grad;
  if (kind == MPAX_MEM_HOST) {
    dg = sh->spo + nB;      // C_true is no longer read
    dl = sh->spo + 3 * nB;  // each block reads z_true[k] before writing loss[k]
  }
  k_spo_loss2<<<B, 256, 0, s>>>(n, sh->C0, C_hat, X_true, z_true, sh->Xout, dl, dg);
  e = cudaGetLastError();
  if (!e && kind == MPAX_MEM_HOST) {
    e = cudaMemcpyAsync(grad, dg, sizeof(double) * nB, cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaMemcpyAsync(loss, dl, sizeof(double) * B, cudaMemcpyDeviceToHost, s);
  }
  if (!e) e = cudaStreamSynchronize(s);
  if (e) return sfail(MPAX_ERR_CUDA, cudaGetErrorString(e));
  return MPAX_OK;
}

void mpax_shared_destroy(mpax_shared* sh) { free_shared(sh); }

}  // extern "C"
