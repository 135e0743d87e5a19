// Preprocessing on the device: Ruiz and Pock-Chambolle diagonal scaling
// (Sec. 3 names both and applies them by default), the rescaled problem data,
// and the norms that set the initial primal weight and the relative KKT test.
#include <algorithm>

#include "problem.cuh"

namespace mpax {

// out[row] = max_j |K_ij| (SUM = false) or sum_j |K_ij| (SUM = true); values
// read through `perm` when given (columns of A as rows of A^T).
template <bool SUM>
__global__ void row_absreduce(const int* __restrict__ rp, const double* __restrict__ val,
                              const int* __restrict__ perm, int rows, double* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < rows; i += nw) {
    double acc = 0.0;
    for (int p = rp[i] + lane; p < rp[i + 1]; p += 32) {
      const double v = fabs(perm ? val[perm[p]] : val[p]);
      acc = SUM ? acc + v : fmax(acc, v);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double t = __shfl_xor_sync(0xffffffffu, acc, o);
      acc = SUM ? acc + t : fmax(acc, t);
    }
    if (lane == 0) out[i] = acc;
  }
}

// One pass over the rows of A for a scaling round.  With the previous round's
// factors (dr, dc non-null) the values are first rescaled in place,
// v <- (v * dr_i) * dc_j; then |v| is reduced to its row norm (maximum, or sum
// when SUM, in a fixed-order warp tree) and, for the maximum, to its column
// maximum through an integer atomicMax on the bit patterns: non-negative
// doubles order like their bit patterns, so the result is exact and does not
// depend on the order of arrival.  colmax must start at +0.0 (all bits zero).
template <bool SUM>
__global__ void scale_pass(const int* __restrict__ rp, const int* __restrict__ col,
                           double* __restrict__ val, int rows, const double* __restrict__ dr,
                           const double* __restrict__ dc, double* __restrict__ rownorm,
                           unsigned long long* __restrict__ colmax) {
  const int lane = threadIdx.x & 31;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < rows; i += nw) {
    const double ri = dr ? dr[i] : 1.0;
    double acc = 0.0;
    for (int p = rp[i] + lane; p < rp[i + 1]; p += 32) {
      double v = val[p];
      const int j = col[p];
      if (dr) {
        v = (v * ri) * dc[j];
        val[p] = v;
      }
      const double a = fabs(v);
      acc = SUM ? acc + a : fmax(acc, a);
      if (colmax) atomicMax(colmax + j, (unsigned long long)__double_as_longlong(a));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double t = __shfl_xor_sync(0xffffffffu, acc, o);
      acc = SUM ? acc + t : fmax(acc, t);
    }
    if (lane == 0) rownorm[i] = acc;
  }
}

// d_i = 1/sqrt(norm_i) (1 for an empty row/column); D_i *= d_i.  d overwrites norm.
// With qdiag (QP columns) the current scaled diagonal D_i^2 qdiag_i joins the
// norm first: max with it (Ruiz, SUM = false) or added to it (Pock-Chambolle).
template <bool SUM>
__global__ void factor_update(double* __restrict__ norm, int k, double* __restrict__ D,
                              const double* __restrict__ qdiag) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= k) return;
  double v = norm[i];
  if (qdiag) {
    const double q = D[i] * D[i] * qdiag[i];
    v = SUM ? v + q : fmax(v, q);
  }
  const double d = (v > 0.0) ? 1.0 / sqrt(v) : 1.0;
  norm[i] = d;
  D[i] *= d;
}

// K_ij <- (K_ij * dr_i) * dc_j  (src may differ from dst: start from the original;
// dr or dc may be nullptr = all ones)
__global__ void apply_scale(const int* __restrict__ rp, const int* __restrict__ col,
                            const double* __restrict__ src, double* __restrict__ dst, int rows,
                            const double* __restrict__ dr, const double* __restrict__ dc) {
  const int lane = threadIdx.x & 31;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < rows; i += nw) {
    const double ri = dr ? dr[i] : 1.0;
    for (int p = rp[i] + lane; p < rp[i + 1]; p += 32)
      dst[p] = dc ? (src[p] * ri) * dc[col[p]] : src[p] * ri;
  }
}

// diag(Q)_j = D_j + sum_r F_jr^2 for Q = diag(D) + F F^T
__global__ void q_diagonal(const int* __restrict__ frp, const double* __restrict__ fval,
                           const double* __restrict__ D, int n, double* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double s = D[j];
  for (int p = frp[j]; p < frp[j + 1]; ++p) s += fval[p] * fval[p];
  out[j] = s;
}

// diag(Q)_j += Q_jj for a general sparse Q (entries of row j in column j)
__global__ void q_diagonal_add(const int* __restrict__ qrp, const int* __restrict__ qcol,
                               const double* __restrict__ qval, int n, double* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double s = 0.0;
  for (int p = qrp[j]; p < qrp[j + 1]; ++p)
    if (qcol[p] == j) s += qval[p];
  out[j] += s;
}

__global__ void fill_ones(double* a, int k) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < k) a[i] = 1.0;
}

__global__ void inv_vec(const double* __restrict__ a, double* __restrict__ b, int k) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < k) b[i] = 1.0 / a[i];
}

// D~ = (Dc * Dc) * D
__global__ void scale_diag(const double* __restrict__ D, const double* __restrict__ Dc, int k,
                           double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < k) out[i] = (Dc[i] * Dc[i]) * D[i];
}

static int grid_for(int k) { return std::max(1, (k + 255) / 256); }
// One warp per row (up to 2^21 warps, then grid-stride): every row's dependent
// load chain (row pointer, values and columns, the gathered factor) is in flight
// at once instead of walking rows one after another.
static int warp_grid(int rows) {
  const int warps = std::max(1, std::min(rows, 1 << 21));
  return (warps + 7) / 8;
}

cudaError_t compute_scaling(ProblemData& P, int ruiz_iters, bool pock_chambolle) {
  cudaStream_t s = P.s;
  const int m = P.m, n = P.n;
  if (m) fill_ones<<<grid_for(m), 256, 0, s>>>(P.Dr, m);
  if (n) fill_ones<<<grid_for(n), 256, 0, s>>>(P.Dc, n);
  if (P.nnz) cudaMemcpyAsync(P.val_s, P.val, sizeof(double) * P.nnz, cudaMemcpyDeviceToDevice, s);
  const bool have = (P.nnz > 0 && m > 0 && n > 0);
  const double* qd = nullptr;
  if (P.is_qp && n) {
    q_diagonal<<<grid_for(n), 256, 0, s>>>(P.F.rp, P.fval, P.D, n, P.qdiag);
    if (P.q_general)
      q_diagonal_add<<<grid_for(n), 256, 0, s>>>(P.Q.rp, P.Q.col, P.qval, n, P.qdiag);
    qd = P.qdiag;
  }
  // Round t's norms are taken in the pass that applies round t-1's factors, so a
  // round costs one pass over A: (rowred, colred) hold the factors of the last
  // finished round, (rowred2, colred2) receive the next round's norms.
  double *fr = P.rowred, *fc = P.colred, *nr = P.rowred2, *nc = P.colred2;
  bool pending = false;  // factors in (fr, fc) not yet applied to val_s
  for (int t = 0; (have || qd) && t < ruiz_iters; ++t) {
    cudaMemsetAsync(nc, 0, sizeof(double) * n, s);
    if (have)
      scale_pass<false><<<warp_grid(m), 256, 0, s>>>(
          P.A.rp, P.A.col, P.val_s, m, pending ? fr : nullptr, pending ? fc : nullptr, nr,
          reinterpret_cast<unsigned long long*>(nc));
    std::swap(fr, nr);
    std::swap(fc, nc);
    if (have) factor_update<false><<<grid_for(m), 256, 0, s>>>(fr, m, P.Dr, nullptr);
    factor_update<false><<<grid_for(n), 256, 0, s>>>(fc, n, P.Dc, qd);
    pending = have;
  }
  if ((have || qd) && pock_chambolle) {
    if (have) {
      // apply the last Ruiz factors while summing rows; columns through A^T
      scale_pass<true><<<warp_grid(m), 256, 0, s>>>(P.A.rp, P.A.col, P.val_s, m,
                                                    pending ? fr : nullptr,
                                                    pending ? fc : nullptr, nr, nullptr);
      row_absreduce<true><<<warp_grid(n), 256, 0, s>>>(P.At.rp, P.val_s, P.permT, n, nc);
      factor_update<true><<<grid_for(m), 256, 0, s>>>(nr, m, P.Dr, nullptr);
    } else {
      cudaMemsetAsync(nc, 0, sizeof(double) * n, s);
    }
    factor_update<true><<<grid_for(n), 256, 0, s>>>(nc, n, P.Dc, qd);
  }
  // the scaled matrix from the original values and the accumulated factors
  if (have)
    apply_scale<<<warp_grid(m), 256, 0, s>>>(P.A.rp, P.A.col, P.val, P.val_s, m, P.Dr, P.Dc);
  if (m) inv_vec<<<grid_for(m), 256, 0, s>>>(P.Dr, P.invDr, m);
  if (n) inv_vec<<<grid_for(n), 256, 0, s>>>(P.Dc, P.invDc, n);
  if (P.is_qp) {
    if (n) scale_diag<<<grid_for(n), 256, 0, s>>>(P.D, P.Dc, n, P.D_s);
    if (P.f_nnz)
      apply_scale<<<warp_grid(n), 256, 0, s>>>(P.F.rp, P.F.col, P.fval, P.fval_s, n, P.Dc,
                                                nullptr);  // F~ = diag(Dc) F
    if (P.q_general && P.Q.nnz)  // Q~ = diag(Dc) Q diag(Dc)
      apply_scale<<<warp_grid(n), 256, 0, s>>>(P.Q.rp, P.Q.col, P.qval, P.qval_s, n, P.Dc,
                                                P.Dc);
  }
  return cudaGetLastError();
}

// ---- norms of the cost and of the row-bound vector, scaled and unscaled ----

__device__ __forceinline__ double bound_of(double lo, double hi) {
  const bool fl = isfinite(lo), fu = isfinite(hi);
  if (fl && fu) return (fabs(lo) >= fabs(hi)) ? lo : hi;
  if (fl) return lo;
  if (fu) return hi;
  return 0.0;
}

__global__ void norms_partial(const double* __restrict__ c, const double* __restrict__ lc,
                              const double* __restrict__ uc, const double* __restrict__ Dr,
                              const double* __restrict__ Dc, int m, int n,
                              double* __restrict__ part) {
  __shared__ double sh[32];
  double s0 = 0, s1 = 0, s2 = 0, s3 = 0;
  const int stride = gridDim.x * blockDim.x;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
    const double cs = Dc[j] * c[j];
    s0 += cs * cs;
    s2 += c[j] * c[j];
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
    const double b = bound_of(lc[i], uc[i]);
    const double bs = bound_of(Dr[i] * lc[i], Dr[i] * uc[i]);
    s1 += bs * bs;
    s3 += b * b;
  }
  const double r0 = block_sum(s0, sh);
  const double r1 = block_sum(s1, sh);
  const double r2 = block_sum(s2, sh);
  const double r3 = block_sum(s3, sh);
  if (threadIdx.x == 0) {
    part[0 * gridDim.x + blockIdx.x] = r0;
    part[1 * gridDim.x + blockIdx.x] = r1;
    part[2 * gridDim.x + blockIdx.x] = r2;
    part[3 * gridDim.x + blockIdx.x] = r3;
  }
}

__global__ void finalize_sqrt_sums(const double* __restrict__ part, int nb, int nq,
                                   double* __restrict__ out) {
  __shared__ double sh[32];
  for (int q = 0; q < nq; ++q) {
    double v = 0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) v += part[q * nb + b];
    v = block_sum(v, sh);
    if (threadIdx.x == 0) out[q] = sqrt(v);
  }
}

cudaError_t bound_and_cost_norms(ProblemData& P) {
  norms_partial<<<kRedBlocks, 256, 0, P.s>>>(P.c, P.lc, P.uc, P.Dr, P.Dc, P.m, P.n, P.red);
  finalize_sqrt_sums<<<1, 256, 0, P.s>>>(P.red, kRedBlocks, 4, P.red_out);
  return cudaGetLastError();
}

// ---- casts ----

template <typename T>
__global__ void k_gather_cast(const double* __restrict__ src, const int* __restrict__ perm,
                              T* __restrict__ dst, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    dst[i] = (T)(perm ? src[perm[i]] : src[i]);
}

template <typename T>
__global__ void k_scale_cast(const double* __restrict__ src, const double* __restrict__ d,
                             bool divide, T* __restrict__ dst, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double v = src[i];
    if (d) v = divide ? v / d[i] : v * d[i];
    dst[i] = (T)v;
  }
}

template <typename T>
cudaError_t gather_cast(const double* src, const int* perm, T* dst, int n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_gather_cast<T><<<std::min(4096, grid_for(n)), 256, 0, s>>>(src, perm, dst, n);
  return cudaGetLastError();
}
template <typename T>
cudaError_t cast_vec(const double* src, T* dst, int n, cudaStream_t s) {
  return gather_cast<T>(src, nullptr, dst, n, s);
}
template <typename T>
cudaError_t scale_cast(const double* src, const double* d, bool divide, T* dst, int n,
                       cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_scale_cast<T><<<std::min(4096, grid_for(n)), 256, 0, s>>>(src, d, divide, dst, n);
  return cudaGetLastError();
}

template cudaError_t gather_cast<double>(const double*, const int*, double*, int, cudaStream_t);
template cudaError_t gather_cast<float>(const double*, const int*, float*, int, cudaStream_t);
template cudaError_t cast_vec<double>(const double*, double*, int, cudaStream_t);
template cudaError_t cast_vec<float>(const double*, float*, int, cudaStream_t);
template cudaError_t scale_cast<double>(const double*, const double*, bool, double*, int,
                                        cudaStream_t);
template cudaError_t scale_cast<float>(const double*, const double*, bool, float*, int,
                                       cudaStream_t);

}  // namespace mpax
