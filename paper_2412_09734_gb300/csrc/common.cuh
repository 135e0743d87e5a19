// Internal definitions shared by the library's translation units.
//
// Layout in HBM (one problem):
//   A    : CSR, int32 row_ptr (m+1), int32 col (nnz), values (FP64 original +
//          scaled copy in the iteration precision)
//   A^T  : second CSR built on the device (int32 row_ptr (n+1), int32 col,
//          int32 perm mapping each A^T entry to its A entry), values in the
//          iteration precision
//   work items of each CSR (int4 each, see Sched), partial-sum slots (FP64)
//   vectors: originals in FP64; scaled data and iterates in the iteration
//          precision; scaling factors in FP64
//   DevState: scalars of the restarted iteration (step sizes, primal weight,
//          counters, Halpern coefficient table), device resident
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

namespace mpax {

constexpr int kWarp = 32;
constexpr int kWarpsPerBlock = 8;
constexpr int kBlock = kWarp * kWarpsPerBlock;

// Launch shape of the fused SpMV kernels: warps per CTA and the minimum number
// of resident CTAs per SM asked of the register allocator.  Small CTAs retire
// as soon as their few warp items are done, so an SM refills at warp grain.
// Measured on the 500k x 1M Zipf LP (FP32): 2-warp CTAs with at least 20 resident
// per SM (a 48-register cap) took the primal/dual launches from 61/79 us (8-warp
// CTAs, the allocator's choice) to 52/66 us.
#ifndef MPAX_SPMV_WARPS
#define MPAX_SPMV_WARPS 2
#endif
#ifndef MPAX_SPMV_MINB
#define MPAX_SPMV_MINB 20  // 0: the register allocator's own choice
#endif
// 1: sliced long rows are completed through acquire/release atomics on the
//    row's counter; 0: through __threadfence() around a relaxed atomic.
// 1: lane 0 of each warp item issues a TMA bulk prefetch into L2 of the values
//    and column indices of the item one resident wave ahead.
#ifndef MPAX_SPMV_PREFETCH
#define MPAX_SPMV_PREFETCH 1
#endif
// 1: the fused SpMVs are launched with programmatic stream serialization and
//    overlap their matrix loads with the previous launch's tail.  Measured on the
//    500k x 1M LP it does not pay (time to 1e-4 0.311 s against 0.299 s; the
//    primal launch 58 against 52 us: early CTAs hold SM slots while they wait).
#ifndef MPAX_SPMV_PDL
#define MPAX_SPMV_PDL 0
#endif
#ifndef MPAX_LONG_ACQREL
#define MPAX_LONG_ACQREL 1
#endif
constexpr int kSpmvWarps = MPAX_SPMV_WARPS;
constexpr int kSpmvBlock = kWarp * kSpmvWarps;
#if MPAX_SPMV_MINB > 0
#define MPAX_SPMV_BOUNDS __launch_bounds__(kSpmvBlock, MPAX_SPMV_MINB)
#else
#define MPAX_SPMV_BOUNDS __launch_bounds__(kSpmvBlock)
#endif
// Work decomposition of a CSR matrix into warp items.
#ifndef MPAX_SLICE_NNZ
#define MPAX_SLICE_NNZ 256
#endif
constexpr int kSliceNnz = MPAX_SLICE_NNZ;  // nonzeros of one slice of a long row
constexpr int kLongRow = 64;    // rows longer than this are cut into slices
constexpr int kItemRows = 64;   // at most this many short rows per item
constexpr int kShortCap = kSliceNnz + kLongRow;  // nonzeros of a packed item, upper bound
constexpr int kMaxCheckEvery = 1024;
constexpr int kRestartLog = 256;  // restarts whose iteration and weight are kept

// Number of FP64 partial-sum quantities kept per work item.
constexpr int kPartQ = 10;

// Work item encoding (int4):
//   packed short rows:   {r0, r1, base, end}        rows [r0, r1), nonzeros [base, end),
//                                                    every row <= kLongRow nonzeros
//   slice of a long row: {-(r+1), p0, p1, s<<16|S}  nonzeros [p0, p1) of row r, slice s
//                                                    of S; slice 0 is item (this - s)
struct Sched {
  int rows = 0;
  int n_items = 0;
  int4* items = nullptr;
  int* cnt = nullptr;      // arrival counters of sliced rows (self-resetting), then
                           // one error word (cnt[n_items]) of the pipelined kernel
  void* carry = nullptr;   // per-item partial row sums of sliced rows (8 bytes each)
  double* part = nullptr;  // kPartQ * n_items FP64 partials
  // Kernel that runs the items: 0 = spmv_fused (one warp per item), 1 =
  // spmv_pipe (persistent warps, TMA-staged matrix), 2 = spmv_fused with more
  // registers per thread.  All give identical bits; the choice is the
  // autotuner's (or the caller's).
  int kind = 0;
};
// Kernel kinds of a schedule: spmv_fused with the default launch shape, spmv_pipe,
// spmv_fused with the wide register budget (kSpmvWideMinB CTAs per SM).
constexpr int kSpmvItem = 0, kSpmvPipe = 1, kSpmvItemWide = 2, kSpmvKinds = 3;
constexpr int kSpmvWideMinB = 10;

struct Csr {
  int rows = 0, cols = 0, nnz = 0;
  int* rp = nullptr;
  int* col = nullptr;
};

// Scalars of the iteration, device resident.  Written by the finalize kernel
// at every check, read by every fused kernel.
struct DevState {
  double tau, sigma, inv_sigma, omega, eta, gamma;
  double norm_A, norm_Q, step_safety;
  double r_anchor, r_prev;
  double eps_abs, eps_rel, r_suff, r_nec, r_art, pw_smooth;
  double b_norm, c_norm;
  double primal_res, dual_res, pobj, dobj, gap, rel_kkt;
  double last_restart_metric;
  double pw_scale, pw_nu;  // power iteration: 1/||g|| of the last round, estimate
  double pw_d;             // power iteration: last increment of the estimate
  long long total, k_base, restarts, checks, iter_limit;
  long long tape_cursor;  // unrolled differentiation: the record the backward pass is on
  int pw_done, pw_iters, stall_limit, stall_count;
  double best_rel;
  double eps_pi, eps_di;  // infeasibility tolerances (LP; <= 0 turns a test off)
  int feas_mode;          // 0: KKT test; 1 / 2: primal / dual residual alone (polishing)
  int tape_err;           // a taped block found no record to write
  int done, restart_flag, termination, have_anchor;
  int check_every, is_qp, nan_seen, pad;
  // Restart log of the run: iteration count and primal weight after each of the
  // first kRestartLog restarts (rs_count counts them all).
  int rs_count, rs_pad;
  long long rs_iter[kRestartLog];
  double rs_omega[kRestartLog];
  // Halpern / averaging coefficient table for the current block:
  // coef_a[i], coef_b[i] for inner counter k' = k_base - 1 + i (i = 0..block).
  double coef_a[kMaxCheckEvery + 2];
  double coef_b[kMaxCheckEvery + 2];
};

// ---- power iteration: start vector and stopping rule ---------------------------
// Start vector: v_j = 2 u_j - 1, u_j the top 53 bits of SplitMix64(kPowerSeed + j)
// (Steele, Lea and Flood, 2014) over 2^53, normalised.  Entries of both signs
// and no structure give a component along every singular vector (the all-ones
// vector can be nearly orthogonal to the top one, and the iteration then
// settles on the second singular value first).
constexpr unsigned long long kPowerSeed = 0x6D706178ull;

__host__ __device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
  unsigned long long z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__host__ __device__ __forceinline__ double power_start_raw(long long j) {
  const unsigned long long z = splitmix64(kPowerSeed + (unsigned long long)j);
  return 2.0 * ((double)(z >> 11) * 1.1102230246251565e-16) - 1.0;  // (z >> 11) / 2^53
}

// Stopping rule: the estimates rise towards the norm with increments d that
// shrink geometrically (ratio q = d / d_prev), so about d q / (1 - q) is still
// to go.  Stop when d and that remainder are both <= tol * nu; the estimate is
// then nu + remainder.  With a certified upper bound `cap` on the norm (1 after
// the Pock-Chambolle round, by Schur's test), stop as soon as the increments are
// small (d <= 100 tol nu) and the extrapolated estimate is within 10 tol of the
// cap, and use the cap; an estimate never exceeds the cap.  d_prev (0 before
// the second estimate) is updated.
__host__ __device__ __forceinline__ bool power_stop(double nu, double nu_prev, double* d_prev,
                                                    double tol, double cap, double* est) {
  const double d = nu - nu_prev;
  const double dp = *d_prev;
  *d_prev = d;
  *est = nu;
  if (d <= 0.0) {
    *est = nu < cap ? nu : cap;
    return true;
  }
  const double q = dp > 0.0 ? d / dp : 1.0;
  if (q >= 1.0) return false;
  const double rem = d * q / (1.0 - q);
  if (d <= 100.0 * tol * nu && nu + rem >= (1.0 - 10.0 * tol) * cap) {
    *est = cap;
    return true;
  }
  if (d <= tol * nu && rem <= tol * nu) {
    *est = nu + rem < cap ? nu + rem : cap;
    return true;
  }
  return false;
}

// Termination recorded when a mixed-precision run stops improving and the
// solve continues in FP64 (internal; never reported to callers).
constexpr int kTermStalled = 100;

// Host-visible mirror written by the finalize kernel (pinned, mapped).
struct HostStatus {
  volatile long long total;
  volatile long long restarts;
  volatile long long checks;
  volatile int done;
  volatile int termination;
  volatile double rel_kkt;
  volatile double pobj, dobj, primal_res, dual_res, gap, omega;
};

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------

template <typename T>
__device__ __forceinline__ T clampv(T v, T lo, T hi) {
  return fmin(fmax(v, lo), hi);
}
template <>
__device__ __forceinline__ float clampv<float>(float v, float lo, float hi) {
  return fminf(fmaxf(v, lo), hi);
}

// Which value clampv(v, lo, hi) returned: 0 v itself (lo < v < hi), 1 lo, 2 hi.
template <typename T>
__device__ __forceinline__ unsigned char clamp_code(T v, T lo, T hi) {
  if (v > lo && v < hi) return 0;
  return (v > lo) ? 2 : 1;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__device__ __forceinline__ T ld_stream(const T* p) {
  return __ldcs(p);
}
template <typename T>
__device__ __forceinline__ T ld_ro(const T* p) {
  return __ldg(p);
}

// ---------------------------------------------------------------------------
// host-side launch helpers (defined in the .cu files)
// ---------------------------------------------------------------------------

// Message returned by mpax_last_error() for the calling thread.
void set_last_error(const char* msg);

// Exclusive scan of `n` int32 counts into out[0..n] (out[n] = total).
// `tmp` must hold scan_tmp_ints(n) ints.
size_t scan_tmp_ints(int n);
cudaError_t scan_exclusive(const int* in, int* out, int n, int* tmp, cudaStream_t s);

// Build the warp-item schedule of a CSR (device); sched.items etc. allocated here.
cudaError_t build_schedule(const Csr& A, Sched& sched, cudaStream_t s, int* tmp_rows,
                           int* tmp_scan);
void free_schedule(Sched& sched);
// Incremented whenever schedule buffers are (re)allocated; CUDA graphs that
// captured older buffers must be rebuilt.
extern unsigned long long sched_generation;
// Elements of padding allocated past the end of every value and column array
// (the L2 bulk prefetch rounds its range out to 16 bytes).
constexpr int kPad = 16;

// Device transpose: At.rp/At.col/perm allocated by the caller (n+1, nnz, nnz).
cudaError_t transpose_csr(const Csr& A, Csr& At, int* perm, int* tmp_cnt, int* tmp_scan,
                          cudaStream_t s);

}  // namespace mpax

namespace mpax {

// Fixed-order block reduction (result valid in thread 0).  `sh` holds 32 values.
template <typename T>
__device__ __forceinline__ T block_sum(T v, T* sh) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  if (w == 0) {
    v = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : T(0);
    v = warp_sum(v);
  }
  return v;
}

}  // namespace mpax
