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
#pragma once

#include "common.cuh"

namespace mpax {

template <typename T>
struct SpmvArgs {
  const int4* items;
  int n_items;
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

// x_md = (1 - beta) xavg + beta x, beta = coef_a[it] (rAPDHG momentum point, eq. 6)
template <typename T>
struct InMomentum {
  const T* x;
  const T* xavg;
  const DevState* st;
  int it;
  T beta;
  __device__ __forceinline__ void load() { beta = (T)st->coef_a[it]; }
  __device__ __forceinline__ T operator()(int j) const {
    return ((T)1 - beta) * ld_ro(xavg + j) + beta * ld_ro(x + j);
  }
};

template <typename T, class In, class Epi>
__global__ void __launch_bounds__(kBlock) spmv_fused(SpmvArgs<T> a, In in, Epi epi) {
  __shared__ T sbuf[kWarpsPerBlock][kShortCap];
  if (epi.skip()) return;
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int item = blockIdx.x * kWarpsPerBlock + wib;
  if (item >= a.n_items) return;
  in.load();
  epi.load();
  double acc[Epi::NQ];
#pragma unroll
  for (int q = 0; q < Epi::NQ; ++q) acc[q] = 0.0;
  const int4 it = a.items[item];
  if (it.z < 0) {
    // packed short rows [r0, r1): stage the products, then one lane per row
    const int r0 = it.x, r1 = it.y;
    const int base = a.rp[r0], end = a.rp[r1];
    T* buf = sbuf[wib];
    for (int p = base + lane; p < end; p += 4 * kWarp) {
      T v[4];
      int c[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int q = p + u * kWarp;
        if (q < end) {
          v[u] = ld_stream(a.val + q);
          c[u] = ld_stream(a.col + q);
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int q = p + u * kWarp;
        if (q < end) buf[q - base] = v[u] * in(c[u]);
      }
    }
    __syncwarp();
    for (int r = r0 + lane; r < r1; r += kWarp) {
      const int q0 = a.rp[r] - base, q1 = a.rp[r + 1] - base;
      T s = 0;
      for (int q = q0; q < q1; ++q) s += buf[q];
      epi.row(r, s, acc);
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
  // slice s of S of the long row r
  const int r = it.x, si = it.y, S = it.z, first = it.w;
  const int rb = a.rp[r];
  const int p0 = rb + si * kSliceNnz;
  const int p1 = min(p0 + kSliceNnz, a.rp[r + 1]);
  T v[kSliceNnz / kWarp];
  int c[kSliceNnz / kWarp];
#pragma unroll
  for (int u = 0; u < kSliceNnz / kWarp; ++u) {
    const int q = p0 + lane + u * kWarp;
    if (q < p1) {
      v[u] = ld_stream(a.val + q);
      c[u] = ld_stream(a.col + q);
    }
  }
  T s = 0;
#pragma unroll
  for (int u = 0; u < kSliceNnz / kWarp; ++u) {
    const int q = p0 + lane + u * kWarp;
    if (q < p1) s += v[u] * in(c[u]);
  }
  s = warp_sum(s);
  if (S == 1) {
    if (lane == 0) {
      epi.row(r, s, acc);
      if (Epi::NQ > 0 && epi.check) {
#pragma unroll
        for (int q = 0; q < Epi::NQ; ++q) a.part[(a.q0 + q) * a.n_items + item] = acc[q];
      }
    }
    return;
  }
  if (lane == 0) {
    a.carry[item] = s;
    __threadfence();
    const int prev = atomicAdd(a.cnt + first, 1);
    bool last = (prev == S - 1);
    if (last) {
      __threadfence();
      T tot = 0;
      for (int t = 0; t < S; ++t) tot += __ldcg(a.carry + first + t);
      a.cnt[first] = 0;  // ready for the next launch
      epi.row(r, tot, acc);
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
