// mpax_lp_kkt_noalloc: the relative KKT evaluation of an LP on caller-owned
// device arrays, for callers that cannot allocate device memory (for example
// code running inside a memory pool it does not control, or a host process
// that must not call cudaMalloc while it holds a fixed device-memory budget).
//
// The per-block FP64 partial sums that mpax_kkt keeps in handle-owned scratch
// live here in one file-scope __device__ array instead.  Its size fixes the
// largest problem this entry point accepts: each of the m rows of A and the n
// rows of A^T is covered by blocks of kRowsPerBlock rows, and every block owns
// one slot per partial quantity, so m and n may not exceed
// kMaxSlots * kRowsPerBlock (16,777,216).  Every GPU that loads the library
// holds the array (3.5 MiB) until the process exits.
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <cmath>

#include "../../include/mpax.h"
#include "common.cuh"

namespace {

constexpr int kRowsPerBlock = 256;
constexpr int kMaxSlots = 65536;  // blocks per pass
// [0] r_p^2 [1] row dual terms [2] r_d^2 [3] c.x [4] bound terms [5] c^2 [6] b^2
constexpr int kQuant = 7;
constexpr int kMaxDevices = 64;

// The scratch: kQuant slots per block, FP64.  Shared by every call on this device.
static __device__ __align__(256) double g_scratch[kQuant * kMaxSlots];

// Device address of g_scratch per device, looked up on the first call on that
// device; concurrent first calls from several host threads store the same value.
std::atomic<double*> g_scratch_ptr[kMaxDevices];

__device__ __forceinline__ double bound_of(double lo, double hi) {
  const bool fl = isfinite(lo), fu = isfinite(hi);
  if (fl && fu) return (fabs(lo) >= fabs(hi)) ? lo : hi;
  if (fl) return lo;
  if (fu) return hi;
  return 0.0;
}

// One warp per row of A: (A x)_i, r_p = Ax - proj_[lc,uc](Ax), lc y^+ - uc y^-.
__global__ void k_rows(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                       const double* __restrict__ val, int m, const double* __restrict__ lc,
                       const double* __restrict__ uc, const double* __restrict__ x,
                       const double* __restrict__ y, double* __restrict__ scratch) {
  __shared__ double sh[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  double a0 = 0.0, a1 = 0.0, a6 = 0.0;
  const int r_end = min(m, (int)(blockIdx.x + 1) * kRowsPerBlock);
  for (int i = blockIdx.x * kRowsPerBlock + w; i < r_end; i += blockDim.x >> 5) {
    double s = 0.0;
    for (int64_t p = rp[i] + lane; p < rp[i + 1]; p += 32) s += val[p] * x[col[p]];
    s = mpax::warp_sum(s);
    if (lane == 0) {
      const double lo = lc[i], hi = uc[i];
      const double r = s - fmin(fmax(s, lo), hi);
      a0 += r * r;
      const double yi = y[i];
      if (yi > 0.0 && isfinite(lo)) a1 += lo * yi;
      if (yi < 0.0 && isfinite(hi)) a1 += hi * yi;
      const double b = bound_of(lo, hi);
      a6 += b * b;
    }
  }
  const double r0 = mpax::block_sum(a0, sh);
  const double r1 = mpax::block_sum(a1, sh);
  const double r6 = mpax::block_sum(a6, sh);
  if (threadIdx.x == 0) {
    scratch[0 * kMaxSlots + blockIdx.x] = r0;
    scratch[1 * kMaxSlots + blockIdx.x] = r1;
    scratch[6 * kMaxSlots + blockIdx.x] = r6;
  }
}

// One warp per row of A^T: lam = c - (A^T y), r_d = lam - proj_Lambda(lam),
// c x, l lh^+ - u lh^-.
__global__ void k_cols(const int64_t* __restrict__ rpt, const int32_t* __restrict__ colt,
                       const double* __restrict__ valt, int n, const double* __restrict__ c,
                       const double* __restrict__ l, const double* __restrict__ u,
                       const double* __restrict__ x, const double* __restrict__ y,
                       double* __restrict__ scratch) {
  __shared__ double sh[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  double a2 = 0.0, a3 = 0.0, a4 = 0.0, a5 = 0.0;
  const int r_end = min(n, (int)(blockIdx.x + 1) * kRowsPerBlock);
  for (int j = blockIdx.x * kRowsPerBlock + w; j < r_end; j += blockDim.x >> 5) {
    double t = 0.0;
    for (int64_t p = rpt[j] + lane; p < rpt[j + 1]; p += 32) t += valt[p] * y[colt[p]];
    t = mpax::warp_sum(t);
    if (lane == 0) {
      const double lam = c[j] - t;
      const double lo = l[j], hi = u[j];
      const bool lf = isfinite(lo), uf = isfinite(hi);
      double lh;
      if (lf && uf) lh = lam;
      else if (lf) lh = fmax(lam, 0.0);
      else if (uf) lh = fmin(lam, 0.0);
      else lh = 0.0;
      const double rd = lam - lh;
      a2 += rd * rd;
      a3 += c[j] * x[j];
      a5 += c[j] * c[j];
      a4 += (lf ? lo * fmax(lh, 0.0) : 0.0) + (uf ? hi * fmin(lh, 0.0) : 0.0);
    }
  }
  const double r2 = mpax::block_sum(a2, sh);
  const double r3 = mpax::block_sum(a3, sh);
  const double r4 = mpax::block_sum(a4, sh);
  const double r5 = mpax::block_sum(a5, sh);
  if (threadIdx.x == 0) {
    scratch[2 * kMaxSlots + blockIdx.x] = r2;
    scratch[3 * kMaxSlots + blockIdx.x] = r3;
    scratch[4 * kMaxSlots + blockIdx.x] = r4;
    scratch[5 * kMaxSlots + blockIdx.x] = r5;
  }
}

// The fixed-order reduction of every block slot (the norms of c and b included).
__global__ void k_finish(const double* __restrict__ scratch, int nbr, int nbc,
                         double* __restrict__ out) {
  __shared__ double sh[32];
  double v[kQuant];
  const int nb[kQuant] = {nbr, nbr, nbc, nbc, nbc, nbc, nbr};
  for (int q = 0; q < kQuant; ++q) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nb[q]; b += blockDim.x) s += scratch[q * kMaxSlots + b];
    v[q] = mpax::block_sum(s, sh);
  }
  const double nc = sqrt(v[5]);
  const double nbn = sqrt(v[6]);
  if (threadIdx.x == 0) {
    const double nrp = sqrt(v[0]), nrd = sqrt(v[2]);
    const double pobj = v[3];
    const double dobj = v[1] + v[4];
    const double gap = fabs(pobj - dobj);
    out[0] = nrp;
    out[1] = nrd;
    out[2] = pobj;
    out[3] = dobj;
    out[4] = gap;
    out[5] = fmax(fmax(nrp / (1.0 + nbn), nrd / (1.0 + nc)), gap / (1.0 + fabs(pobj) + fabs(dobj)));
  }
}

mpax_status noalloc_fail(mpax_status s, const char* msg) {
  mpax::set_last_error(msg);
  return s;
}

}  // namespace

extern "C" mpax_status mpax_lp_kkt_noalloc(int32_t m, int32_t n, int64_t nnz,
                                           const int64_t* row_ptr, const int32_t* col_idx,
                                           const double* val, const int64_t* row_ptr_t,
                                           const int32_t* col_idx_t, const double* val_t,
                                           const double* c, const double* lc, const double* uc,
                                           const double* l, const double* u, const double* x,
                                           const double* y, double* out, void* cuda_stream) {
  if (m < 0 || n < 0 || nnz < 0)
    return noalloc_fail(MPAX_ERR_INVALID_ARGUMENT, "sizes must be non-negative");
  if ((int64_t)m > (int64_t)kMaxSlots * kRowsPerBlock ||
      (int64_t)n > (int64_t)kMaxSlots * kRowsPerBlock)
    return noalloc_fail(MPAX_ERR_UNSUPPORTED,
                        "m and n must be at most 16777216 (size of the static scratch)");
  if (!out || !row_ptr || !row_ptr_t || (n > 0 && (!c || !l || !u || !x)) ||
      (m > 0 && (!lc || !uc || !y)) || (nnz > 0 && (!col_idx || !val || !col_idx_t || !val_t)))
    return noalloc_fail(MPAX_ERR_INVALID_ARGUMENT, "a required device pointer is NULL");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return noalloc_fail(MPAX_ERR_CUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices)
    return noalloc_fail(MPAX_ERR_UNSUPPORTED, "device index beyond the supported range");
  // Host code must not hand `g_scratch` itself to a kernel: on the host that name
  // is a stand-in, not a device address.  Look the address up once per device,
  // with that device current.
  double* scratch = g_scratch_ptr[dev].load(std::memory_order_relaxed);
  if (!scratch) {
    e = cudaGetSymbolAddress((void**)&scratch, g_scratch);
    if (e != cudaSuccess) return noalloc_fail(MPAX_ERR_CUDA, cudaGetErrorString(e));
    g_scratch_ptr[dev].store(scratch, std::memory_order_relaxed);
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const int nbr = (m + kRowsPerBlock - 1) / kRowsPerBlock;
  const int nbc = (n + kRowsPerBlock - 1) / kRowsPerBlock;
  if (nbr > 0) k_rows<<<nbr, 256, 0, s>>>(row_ptr, col_idx, val, m, lc, uc, x, y, scratch);
  if (nbc > 0) k_cols<<<nbc, 256, 0, s>>>(row_ptr_t, col_idx_t, val_t, n, c, l, u, x, y, scratch);
  k_finish<<<1, 256, 0, s>>>(scratch, nbr, nbc, out);
  e = cudaGetLastError();
  if (e != cudaSuccess) return noalloc_fail(MPAX_ERR_CUDA, cudaGetErrorString(e));
  return MPAX_OK;
}
