// Fused CSR SpMV kernels of the restarted PDHG iteration.
//
// One kernel launch computes s = K v for a CSR matrix K (A or A^T) and hands
// each finished row sum to an epilogue that performs the elementwise part of
// the half-step (projection, reflection, Halpern or averaging update) and, on
// check iterations, accumulates FP64 partial sums for the KKT and restart
// tests.  Work is split into warp items (see Sched): packed runs of short rows
// and fixed-size slices of long rows.  A sliced row is finished by whichever
// warp arrives last at its counter; it sums the slices' partials in slice
// order, so every result is independent of scheduling.  No floating-point
// atomics are used anywhere: every reduction has a fixed order.
//
// Latency: a warp issues every independent load of its item at once (item
// descriptor, state scalars, row pointers and epilogue operands of its rows,
// all matrix values and column indices), then the gathers of the input vector,
// then computes.  Lane 0 also issues a TMA bulk prefetch into L2
// (cp.async.bulk.prefetch.L2) of the values and column indices of the item one
// resident wave ahead, so most matrix loads of later waves hit L2.
#pragma once

#include "common.cuh"

namespace mpax {

constexpr int kShortLoads = (kShortCap + kWarp - 1) / kWarp;  // per lane, packed rows
constexpr int kSliceLoads = kSliceNnz / kWarp;                // per lane, one slice

template <typename T>
struct SpmvArgs {
  const int4* items;
  int n_items;
  int pf_dist;  // prefetch distance in items (0 = off)
  const int* rp;
  const int* col;
  const T* val;
  int* cnt;
  T* carry;
  double* part;  // kPartQ * n_items
  int q0;        // first partial slot used by this launch
};

// Input gathers.
template <typename T>
struct InPlain {
  const T* x;
  __device__ __forceinline__ void load() {}
  __device__ __forceinline__ T operator()(int j) const { return ld_ro(x + j); }
};

// x_md = xavg + beta (x - xavg), beta = coef_a[it] (rAPDHG momentum point, eq. 6)
template <typename T>
struct InMomentum {
  const T* x;
  const T* xavg;
  const DevState* st;
  int it;
  T beta;
  __device__ __forceinline__ void load() { beta = (T)st->coef_a[it]; }
  __device__ __forceinline__ T operator()(int j) const {
    const T a = ld_ro(xavg + j);
    return a + beta * (ld_ro(x + j) - a);
  }
};

__device__ __forceinline__ int item_row(const int4& it) { return it.x >= 0 ? it.x : -(it.x + 1); }

__device__ __forceinline__ void item_range(const int4& it, int& p0, int& p1) {
  if (it.x >= 0) {
    p0 = it.z;
    p1 = it.w;
  } else {
    p0 = it.y;
    p1 = it.z;
  }
}

// Programmatic dependent launch (sm_90+ griddepcontrol).  launch_dependents lets
// the next kernel of the stream start its CTAs once every CTA of this grid has
// issued it or exited; wait returns when the previous grid has completed and its
// memory operations are visible.  Without the launch attribute both are no-ops.
__device__ __forceinline__ void pdl_launch_dependents() {
#if MPAX_SPMV_PDL
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
#endif
}
__device__ __forceinline__ void pdl_wait() {
#if MPAX_SPMV_PDL
  asm volatile("griddepcontrol.wait;" ::: "memory");
#endif
}

// TMA bulk prefetch of [p, p + bytes) into L2 (16-byte aligned, rounded out;
// arrays carry at least 16 bytes of padding past their end).
__device__ __forceinline__ void prefetch_l2(const void* p, size_t bytes) {
  if (bytes == 0) return;
  const unsigned long long a0 = (unsigned long long)p & ~15ull;
  const unsigned long long a1 = ((unsigned long long)p + bytes + 15ull) & ~15ull;
  const unsigned size = (unsigned)(a1 - a0);
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a0), "r"(size) : "memory");
}

template <typename T, class In, class Epi>
__global__ void MPAX_SPMV_BOUNDS spmv_fused(SpmvArgs<T> a, In in, Epi epi) {
  __shared__ T sbuf[kSpmvWarps][kShortCap];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int item = blockIdx.x * kSpmvWarps + wib;
  // The next launch may start its CTAs as this grid drains (programmatic
  // dependent launch); it reads only the constant matrix arrays before its wait.
  pdl_launch_dependents();
  if (item >= a.n_items) return;
  const int4 it = a.items[item];
  const bool do_pf = (lane == 0) && a.pf_dist > 0 && item + a.pf_dist < a.n_items;

  if (it.x >= 0) {
    // ---- packed short rows [r0, r1), nonzeros [base, end) ----------------
    const int r0 = it.x, r1 = it.y, base = it.z, end = it.w;
    const int ra = r0 + lane, rb = r0 + kWarp + lane;
    const bool ha = ra < r1, hb = rb < r1;
    const int sa = ha ? ra : r0, sb = hb ? rb : r0;  // always-valid rows
    const int pa0 = a.rp[sa], pa1 = a.rp[sa + 1];
    const int pb0 = a.rp[sb], pb1 = a.rp[sb + 1];
    T v[kShortLoads];
    int c[kShortLoads];
#pragma unroll
    for (int u = 0; u < kShortLoads; ++u) {
      const int q = base + lane + u * kWarp;
      if (q < end) {
        v[u] = ld_stream(a.val + q);
        c[u] = ld_stream(a.col + q);
      }
    }
    int4 ft;
    if (do_pf) ft = a.items[item + a.pf_dist];
    // everything below reads or writes state of the previous launches
    pdl_wait();
    if (epi.skip()) return;
    in.load();
    epi.load();
    double acc[Epi::NQ];
#pragma unroll
    for (int q = 0; q < Epi::NQ; ++q) acc[q] = 0.0;
    typename Epi::Pre pra, prb;
    epi.pre(sa, pra);
    epi.pre(sb, prb);
    T* buf = sbuf[wib];
#pragma unroll
    for (int u = 0; u < kShortLoads; ++u) {
      const int q = base + lane + u * kWarp;
      if (q < end) buf[q - base] = v[u] * in(c[u]);
    }
    if (do_pf) {
      int q0, q1;
      item_range(ft, q0, q1);
      prefetch_l2(a.val + q0, sizeof(T) * (size_t)(q1 - q0));
      prefetch_l2(a.col + q0, sizeof(int) * (size_t)(q1 - q0));
    }
    __syncwarp();
    if (ha) {
      T s = 0;
      for (int q = pa0; q < pa1; ++q) s += buf[q - base];
      epi.row(ra, s, pra, acc);
    }
    if (hb) {
      T s = 0;
      for (int q = pb0; q < pb1; ++q) s += buf[q - base];
      epi.row(rb, s, prb, acc);
    }
    if (Epi::NQ > 0 && epi.check) {
#pragma unroll
      for (int q = 0; q < Epi::NQ; ++q) {
        const double t = warp_sum(acc[q]);
        if (lane == 0) a.part[(a.q0 + q) * a.n_items + item] = t;
      }
    }
    return;
  }

  // ---- slice s of S of the long row r: nonzeros [p0, p1) ------------------
  const int r = -(it.x + 1), p0 = it.y, p1 = it.z;
  const int si = it.w >> 16, S = it.w & 0xffff;
  const int first = item - si;
  T v[kSliceLoads];
  int c[kSliceLoads];
#pragma unroll
  for (int u = 0; u < kSliceLoads; ++u) {
    const int q = p0 + lane + u * kWarp;
    if (q < p1) {
      v[u] = ld_stream(a.val + q);
      c[u] = ld_stream(a.col + q);
    }
  }
  int4 ft;
  if (do_pf) ft = a.items[item + a.pf_dist];
  pdl_wait();
  if (epi.skip()) return;
  in.load();
  epi.load();
  double acc[Epi::NQ];
#pragma unroll
  for (int q = 0; q < Epi::NQ; ++q) acc[q] = 0.0;
  typename Epi::Pre pr;
  epi.pre(r, pr);
  T s = 0;
#pragma unroll
  for (int u = 0; u < kSliceLoads; ++u) {
    const int q = p0 + lane + u * kWarp;
    if (q < p1) s += v[u] * in(c[u]);
  }
  if (do_pf) {
    int q0, q1;
    item_range(ft, q0, q1);
    prefetch_l2(a.val + q0, sizeof(T) * (size_t)(q1 - q0));
    prefetch_l2(a.col + q0, sizeof(int) * (size_t)(q1 - q0));
  }
  s = warp_sum(s);
  if (S == 1) {
    if (lane == 0) {
      epi.row(r, s, pr, acc);
      if (Epi::NQ > 0 && epi.check) {
#pragma unroll
        for (int q = 0; q < Epi::NQ; ++q) a.part[(a.q0 + q) * a.n_items + item] = acc[q];
      }
    }
    return;
  }
  if (lane == 0) {
    a.carry[item] = s;
#if MPAX_LONG_ACQREL
    // release: this slice's carry is visible to whoever observes the count;
    // acquire: the last arriver sees every earlier slice's carry
    int prev;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;"
                 : "=r"(prev)
                 : "l"(a.cnt + first)
                 : "memory");
    const bool last = (prev == S - 1);
#else
    __threadfence();
    const int prev = atomicAdd(a.cnt + first, 1);
    const bool last = (prev == S - 1);
    if (last) __threadfence();
#endif
    if (last) {
      T tot = 0;
      for (int t = 0; t < S; ++t) tot += __ldcg(a.carry + first + t);
      a.cnt[first] = 0;  // ready for the next launch
      epi.row(r, tot, pr, acc);
    }
    if (Epi::NQ > 0 && epi.check) {
      // the finished row's contribution always lands in slot `first`; the
      // other slices' slots hold zero
      if (si != 0) {
#pragma unroll
        for (int q = 0; q < Epi::NQ; ++q) a.part[(a.q0 + q) * a.n_items + item] = 0.0;
      }
      if (last) {
#pragma unroll
        for (int q = 0; q < Epi::NQ; ++q) a.part[(a.q0 + q) * a.n_items + first] = acc[q];
      }
    }
  }
}

}  // namespace mpax
