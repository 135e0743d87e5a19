// Sparse-structure kernels: exclusive scan, the warp-item schedule of a CSR
// matrix, and the device-built transpose A^T (the second CSR the SpMV^T of
// every primal half-step reads).
#include <algorithm>

#include "common.cuh"

namespace mpax {

unsigned long long sched_generation = 0;

// ---------------------------------------------------------------------------
// Exclusive scan (three passes: block sums, scan of block sums, block scans)
// ---------------------------------------------------------------------------

constexpr int kScanBlock = 1024;

__device__ __forceinline__ int block_exclusive_scan(int v, int* sh, int* total) {
  // sh: kScanBlock/32 ints.
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += t;
  }
  if (lane == 31) sh[w] = x;
  __syncthreads();
  if (w == 0) {
    int s = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int t = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += t;
    }
    sh[lane] = s;  // inclusive warp totals
  }
  __syncthreads();
  const int warp_off = (w > 0) ? sh[w - 1] : 0;
  if (total) *total = sh[(blockDim.x >> 5) - 1];
  return warp_off + x - v;
}

__global__ void scan_block_sums(const int* __restrict__ in, int n, int* __restrict__ bsum) {
  __shared__ int sh[32];
  const int i = blockIdx.x * kScanBlock + threadIdx.x;
  const int v = (i < n) ? in[i] : 0;
  int tot;
  block_exclusive_scan(v, sh, &tot);
  if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

// Single block: exclusive scan of nb block sums in place, total in bsum[nb].
__global__ void scan_bsums(int* bsum, int nb) {
  __shared__ int sh[32];
  const int per = (nb + kScanBlock - 1) / kScanBlock;
  const int lo = threadIdx.x * per;
  const int hi = min(nb, lo + per);
  int s = 0;
  for (int i = lo; i < hi; ++i) s += bsum[i];
  int tot;
  int off = block_exclusive_scan(s, sh, &tot);
  for (int i = lo; i < hi; ++i) {
    const int v = bsum[i];
    bsum[i] = off;
    off += v;
  }
  if (threadIdx.x == 0) bsum[nb] = tot;
}

__global__ void scan_apply(const int* __restrict__ in, int n, const int* __restrict__ bsum,
                           int* __restrict__ out) {
  __shared__ int sh[32];
  const int i = blockIdx.x * kScanBlock + threadIdx.x;
  const int v = (i < n) ? in[i] : 0;
  const int ex = block_exclusive_scan(v, sh, nullptr) + bsum[blockIdx.x];
  if (i < n) out[i] = ex;
  if (i == n - 1) out[n] = ex + v;
}

size_t scan_tmp_ints(int n) { return (size_t)(n + kScanBlock - 1) / kScanBlock + 2; }

cudaError_t scan_exclusive(const int* in, int* out, int n, int* tmp, cudaStream_t s) {
  if (n <= 0) return cudaMemsetAsync(out, 0, sizeof(int), s);
  const int nb = (n + kScanBlock - 1) / kScanBlock;
  scan_block_sums<<<nb, kScanBlock, 0, s>>>(in, n, tmp);
  scan_bsums<<<1, kScanBlock, 0, s>>>(tmp, nb);
  scan_apply<<<nb, kScanBlock, 0, s>>>(in, n, tmp, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Warp-item schedule
// ---------------------------------------------------------------------------
// Rows longer than kLongRow become ceil(len / kSliceNnz) slice items.  Runs of
// short rows are packed into one item; a new item starts at row i when the
// previous row was long, when rp[i] falls into another kSliceNnz-aligned bin
// than rp[i-1], or when i is a multiple of kItemRows.  Every row of an item
// therefore starts inside one bin, so an item holds fewer than
// kSliceNnz + kLongRow nonzeros and at most kItemRows rows.

__global__ void sched_count(const int* __restrict__ rp, int rows, int* __restrict__ cnt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows) return;
  const int len = rp[i + 1] - rp[i];
  int c;
  if (len > kLongRow) {
    c = (len + kSliceNnz - 1) / kSliceNnz;
  } else if (i == 0 || (i % kItemRows) == 0) {
    c = 1;
  } else {
    const int plen = rp[i] - rp[i - 1];
    c = (plen > kLongRow || (rp[i] / kSliceNnz) != (rp[i - 1] / kSliceNnz)) ? 1 : 0;
  }
  cnt[i] = c;
}

__global__ void sched_fill(const int* __restrict__ rp, int rows, const int* __restrict__ cnt,
                           const int* __restrict__ off, int4* __restrict__ items,
                           int* __restrict__ err) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows) return;
  const int c = cnt[i];
  if (c == 0) return;
  const int b = rp[i], len = rp[i + 1] - b;
  const int o = off[i];
  if (len > kLongRow) {
    if (c > 0xffff) {  // slice index and count are packed in 16 bits each
      atomicOr(err, 1);
      return;
    }
    for (int s = 0; s < c; ++s) {
      const int p0 = b + s * kSliceNnz;
      items[o + s] = make_int4(-(i + 1), p0, min(p0 + kSliceNnz, b + len), (s << 16) | c);
    }
  } else {
    items[o] = make_int4(i, -1, b, -1);
  }
}

// A packed item ends where the next item begins.
__global__ void sched_fix(int4* __restrict__ items, int n_items, int rows,
                          const int* __restrict__ rp) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_items) return;
  int4 it = items[k];
  if (it.x >= 0) {
    int next = rows;
    if (k + 1 < n_items) {
      // only the .x field of the next item is read; this kernel never writes it
      const int nx = reinterpret_cast<const int*>(items + k + 1)[0];
      next = nx >= 0 ? nx : -(nx + 1);
    }
    it.y = next;
    it.w = rp[next];
    items[k] = it;
  }
}

void free_schedule(Sched& sc) {
  if (sc.items) cudaFree(sc.items);
  if (sc.cnt) cudaFree(sc.cnt);
  if (sc.carry) cudaFree(sc.carry);
  if (sc.part) cudaFree(sc.part);
  sc = Sched();
}

cudaError_t build_schedule(const Csr& A, Sched& sc, cudaStream_t s, int* tmp_rows,
                           int* tmp_scan) {
  // tmp_rows: rows + 2 ints.  Buffers of an existing schedule with the same
  // item count are reused, so device pointers captured in CUDA graphs stay valid.
  sc.rows = A.rows;
  cudaError_t e;
  if (A.rows == 0) {
    free_schedule(sc);
    return cudaSuccess;
  }
  int* cnt = tmp_rows;
  int* off = nullptr;
  int* err = nullptr;
  if ((e = cudaMallocAsync(&off, sizeof(int) * (A.rows + 2), s))) return e;
  err = off + A.rows + 1;
  if ((e = cudaMemsetAsync(err, 0, sizeof(int), s))) return e;
  const int g = (A.rows + 255) / 256;
  sched_count<<<g, 256, 0, s>>>(A.rp, A.rows, cnt);
  if ((e = scan_exclusive(cnt, off, A.rows, tmp_scan, s))) return e;
  int n_items = 0;
  if ((e = cudaMemcpyAsync(&n_items, off + A.rows, sizeof(int), cudaMemcpyDeviceToHost, s)))
    return e;
  if ((e = cudaStreamSynchronize(s))) return e;
  if (sc.items == nullptr || sc.n_items != n_items) {
    free_schedule(sc);
    sc.rows = A.rows;
    sc.n_items = n_items;
    if ((e = cudaMalloc(&sc.items, sizeof(int4) * std::max(n_items, 1)))) return e;
    if ((e = cudaMalloc(&sc.cnt, sizeof(int) * (n_items + 1)))) return e;
    if ((e = cudaMalloc(&sc.carry, sizeof(double) * std::max(n_items, 1)))) return e;
    if ((e = cudaMalloc(&sc.part, sizeof(double) * kPartQ * std::max(n_items, 1)))) return e;
    cudaMemsetAsync(sc.cnt, 0, sizeof(int) * (n_items + 1), s);
    cudaMemsetAsync(sc.part, 0, sizeof(double) * kPartQ * std::max(n_items, 1), s);
    ++sched_generation;
  }
  sched_fill<<<g, 256, 0, s>>>(A.rp, A.rows, cnt, off, sc.items, err);
  if (n_items > 0)
    sched_fix<<<(n_items + 255) / 256, 256, 0, s>>>(sc.items, n_items, A.rows, A.rp);
  int herr = 0;
  if ((e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s))) return e;
  if ((e = cudaStreamSynchronize(s))) return e;
  cudaFreeAsync(off, s);
  if (herr) return cudaErrorInvalidValue;  // a row longer than 65535 slices
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Transpose
// ---------------------------------------------------------------------------
// 1. column counts (integer atomics, order independent)
// 2. exclusive scan -> A^T row pointers
// 3. scatter (row index, A position) into the A^T rows with atomic cursors
// 4. sort every A^T row by row index of A (unique within a column), which
//    makes the result independent of the atomic order: entries of each A^T
//    row end up in increasing A-row order, as in a sequential transpose.

__global__ void tr_count(const int* __restrict__ col, int nnz, int* __restrict__ cnt) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += gridDim.x * blockDim.x)
    atomicAdd(cnt + col[p], 1);
}

// one warp per A row
__global__ void tr_scatter(const int* __restrict__ rp, const int* __restrict__ col, int rows,
                           int* __restrict__ cursor, int* __restrict__ colT,
                           int* __restrict__ perm) {
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int i = w; i < rows; i += nw) {
    for (int p = rp[i] + lane; p < rp[i + 1]; p += 32) {
      const int pos = atomicAdd(cursor + col[p], 1);
      colT[pos] = i;
      perm[pos] = p;
    }
  }
}

__device__ __forceinline__ unsigned long long pack_key(int key, int val) {
  return ((unsigned long long)(unsigned)key << 32) | (unsigned)val;
}

// Rows of A^T with at most 32 entries: one thread, insertion sort.
__global__ void tr_sort_short(const int* __restrict__ rpT, int rowsT, int* __restrict__ colT,
                              int* __restrict__ perm) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= rowsT) return;
  const int b = rpT[j], e = rpT[j + 1];
  const int L = e - b;
  if (L <= 1 || L > 32) return;
  unsigned long long k[32];
  for (int t = 0; t < L; ++t) k[t] = pack_key(colT[b + t], perm[b + t]);
  for (int t = 1; t < L; ++t) {
    const unsigned long long v = k[t];
    int q = t - 1;
    while (q >= 0 && k[q] > v) {
      k[q + 1] = k[q];
      --q;
    }
    k[q + 1] = v;
  }
  for (int t = 0; t < L; ++t) {
    colT[b + t] = (int)(k[t] >> 32);
    perm[b + t] = (int)(k[t] & 0xffffffffull);
  }
}

// In-place ascending bitonic sort of L keys by one CTA (power-of-two network of
// size N >= L; every comparison that touches a position >= L compares with a
// virtual +inf and is a no-op, so no padding storage is needed).
__device__ void cta_bitonic(unsigned long long* d, int L) {
  int N = 1;
  while (N < L) N <<= 1;
  for (int k = 2; k <= N; k <<= 1) {
    const int h = k >> 1;
    for (int i = threadIdx.x; i < N / 2; i += blockDim.x) {  // flip step
      const int blk = i / h, off = i % h;
      const int a = blk * k + off, b = blk * k + k - 1 - off;
      if (b < L) {
        const unsigned long long x = d[a], y = d[b];
        if (x > y) { d[a] = y; d[b] = x; }
      }
    }
    __syncthreads();
    for (int j = h >> 1; j >= 1; j >>= 1) {
      for (int i = threadIdx.x; i < N / 2; i += blockDim.x) {
        const int a = (i / j) * 2 * j + (i % j), b = a + j;
        if (b < L) {
          const unsigned long long x = d[a], y = d[b];
          if (x > y) { d[a] = y; d[b] = x; }
        }
      }
      __syncthreads();
    }
  }
}

constexpr int kSortSmem = 4096;

// Rows of A^T with more than 32 entries: one CTA per row; shared memory when
// the row fits, else in place in `scratch` (a global buffer of nnz keys).
__global__ void tr_sort_long(const int* __restrict__ rpT, int rowsT, int* __restrict__ colT,
                             int* __restrict__ perm, unsigned long long* __restrict__ scratch,
                             int rows_per_cta) {
  __shared__ unsigned long long sk[kSortSmem];
  __shared__ int todo[kBlock];
  __shared__ int ntodo;
  const int r0 = blockIdx.x * rows_per_cta;
  const int r1 = min(rowsT, r0 + rows_per_cta);
  for (int base = r0; base < r1; base += blockDim.x) {
    if (threadIdx.x == 0) ntodo = 0;
    __syncthreads();
    const int j = base + threadIdx.x;
    if (j < r1 && rpT[j + 1] - rpT[j] > 32) todo[atomicAdd(&ntodo, 1)] = j;
    __syncthreads();
    const int nt = ntodo;
    // deterministic order of processing does not matter: each row is sorted independently
    for (int t = 0; t < nt; ++t) {
      const int row = todo[t];
      const int b = rpT[row], L = rpT[row + 1] - b;
      unsigned long long* d = (L <= kSortSmem) ? sk : scratch + b;
      for (int q = threadIdx.x; q < L; q += blockDim.x) d[q] = pack_key(colT[b + q], perm[b + q]);
      __syncthreads();
      cta_bitonic(d, L);
      for (int q = threadIdx.x; q < L; q += blockDim.x) {
        colT[b + q] = (int)(d[q] >> 32);
        perm[b + q] = (int)(d[q] & 0xffffffffull);
      }
      __syncthreads();
    }
    __syncthreads();
  }
}

cudaError_t transpose_csr(const Csr& A, Csr& At, int* perm, int* tmp_cnt, int* tmp_scan,
                          cudaStream_t s) {
  cudaError_t e;
  At.rows = A.cols;
  At.cols = A.rows;
  At.nnz = A.nnz;
  const int n = A.cols;
  if ((e = cudaMemsetAsync(tmp_cnt, 0, sizeof(int) * (n + 1), s))) return e;
  if (A.nnz > 0) {
    tr_count<<<std::min(4096, (A.nnz + 255) / 256), 256, 0, s>>>(A.col, A.nnz, tmp_cnt);
  }
  if ((e = scan_exclusive(tmp_cnt, At.rp, n, tmp_scan, s))) return e;
  if (n == 0) return cudaGetLastError();
  if (A.nnz == 0) return cudaGetLastError();
  // cursors start at the row pointers
  if ((e = cudaMemcpyAsync(tmp_cnt, At.rp, sizeof(int) * n, cudaMemcpyDeviceToDevice, s)))
    return e;
  const int warps = std::max(1, std::min(A.rows, 152 * 64));
  tr_scatter<<<(warps * 32 + 255) / 256, 256, 0, s>>>(A.rp, A.col, A.rows, tmp_cnt, At.col,
                                                      perm);
  tr_sort_short<<<(n + 255) / 256, 256, 0, s>>>(At.rp, n, At.col, perm);
  unsigned long long* scratch = nullptr;
  if ((e = cudaMallocAsync(&scratch, sizeof(unsigned long long) * A.nnz, s))) return e;
  const int rows_per_cta = 2048;
  tr_sort_long<<<(n + rows_per_cta - 1) / rows_per_cta, kBlock, 0, s>>>(At.rp, n, At.col, perm,
                                                                        scratch, rows_per_cta);
  cudaFreeAsync(scratch, s);
  return cudaGetLastError();
}

}  // namespace mpax
