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
#include "sync.cuh"

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

// Row sums of packed short rows.  FP32: the products are formed lane-parallel
// into the warp's buffer and one lane adds a row's products in order.  FP64 runs
// at a small fraction of the FP32 rate on this GPU (two FP64 lane operations per
// SM and cycle: a warp-wide FP64 instruction holds the pipe for 16 cycles
// however many of its lanes are active, so the FP64 pipe, not memory, bounds
// these kernels).  There the buffer holds the values and, kShortCap further,
// the gathered inputs, and the sums are fused multiply-add chains that keep
// every lane busy (packed_rows_fma).
template <typename T>
constexpr bool kFmaRows = sizeof(T) == 8;

// Shared-memory words of the row-start bit mask of an FP64 packed item (one bit
// per nonzero position, kShortCap positions, plus a word read past the last).
constexpr int kRowWords = (kShortCap + 31) / 32 + 1;

// FP32 row sum: buf holds the products.
template <typename T>
__device__ __forceinline__ T packed_row_sum(const T* buf, int q0, int q1) {
  T s = 0;
  for (int q = q0; q < q1; ++q) s += buf[q];
  return s;
}

// Sum of row [s, e) after the chunk walk of packed_rows_fma: a row inside one
// chunk was stored whole at buf[s]; otherwise its pieces are added in chunk
// order: its piece of chunk a (that chunk's last segment, at the chunk's last
// position of bx), the whole chunks strictly between (their single segment, at
// their first position), and its piece of chunk b (that chunk's first segment).
template <typename T>
__device__ __forceinline__ T packed_row_total(const T* buf, const T* bx, int L, int s, int e) {
  if (s >= e) return T(0);
  const int a = s / L, b = (e - 1) / L;
  if (a == b) return buf[s];
  T tot = bx[(a + 1) * L - 1];
  for (int l = a + 1; l < b; ++l) tot += bx[l * L];
  return tot + bx[b * L];
}

// FP64 row sums of a packed item with every lane busy.  The item's cnt
// nonzeros (values in buf, gathered inputs in bx, both at offsets 0..cnt-1) are
// cut into 32 chunks of L = ceil(cnt / 32) consecutive positions, chunk l
// walked by lane l as one fused multiply-add chain that restarts at each row
// start.  Every chain segment that is a whole row is stored at buf[its first
// position]; the chunk's first and last segments are stored in bx at the
// chunk's first and last position (positions the lane has already read; no
// other lane reads them).  packed_row_total then assembles each row.  The
// order of every sum depends only on the item, so all kernel kinds that stage
// an item give the same bits.  The FP64 instructions per item are L chain steps
// plus the chunk pieces of the longest row sum, against the longest row pair
// of a lane when each lane sums its own rows.
// Rows [a0, a1) and [b0, b1) (offsets from the item's first nonzero) are this
// lane's two rows when ha / hb; words: kRowWords words of the warp's shared
// memory.  Called by the whole warp.
template <typename T>
__device__ __forceinline__ void packed_rows_fma(T* buf, T* bx, unsigned* words, int cnt, int lane,
                                                bool ha, int a0, int a1, bool hb, int b0, int b1,
                                                T& sa, T& sb) {
  if (lane < kRowWords) words[lane] = 0u;
  __syncwarp();
  if (ha && a0 < cnt) atomicOr(words + (a0 >> 5), 1u << (a0 & 31));
  if (hb && b0 < cnt) atomicOr(words + (b0 >> 5), 1u << (b0 & 31));
  __syncwarp();
  const int L = (cnt + kWarp - 1) / kWarp;
  const int c0 = lane * L, c1 = min(c0 + L, cnt);
  if (c0 < c1) {
    // bit t: position c0 + t starts a row (t <= L <= kShortCap / 32)
    const unsigned long long two = (unsigned long long)words[c0 >> 5] |
                                   ((unsigned long long)words[(c0 >> 5) + 1] << 32);
    const unsigned m = (unsigned)(two >> (c0 & 31));
    T acc = 0;
    int s = c0;  // first position of the open segment
#pragma unroll
    for (int t = 0; t < kShortLoads; ++t) {
      const int q = c0 + t;
      if (q < c1) {
        if (t > 0 && ((m >> t) & 1u)) {  // a row starts at q: close [s, q)
          if (s == c0) bx[c0] = acc;
          if ((m >> (s - c0)) & 1u) buf[s] = acc;  // [s, q) is a whole row
          acc = 0;
          s = q;
        }
        acc = fma(buf[q], bx[q], acc);
      }
    }
    // the last segment [s, c1): a whole row if a row starts at s and the
    // next row (or the item's end) at c1
    if (((m >> (s - c0)) & 1u) && (c1 == cnt || ((m >> (c1 - c0)) & 1u))) buf[s] = acc;
    if (s == c0) bx[c0] = acc;
    bx[c1 - 1] = acc;
  }
  __syncwarp();
  sa = ha ? packed_row_total(buf, bx, L, a0, a1) : T(0);
  sb = hb ? packed_row_total(buf, bx, L, b0, b1) : T(0);
}

// The CTA's staging buffer: one row per warp; FP64 keeps values and gathered
// inputs apart (kFmaRows), twice the length, followed by the row-start mask
// (kRowWords words, rounded up to whole elements).
template <typename T>
constexpr int kSpmvBufLen = kFmaRows<T> ? 2 * kShortCap + (kRowWords * 4 + 7) / 8 : kShortCap;
template <typename T>
using SpmvBuf = T[kSpmvWarps][kSpmvBufLen<T>];

// The work of CTA `cta` of a spmv_fused launch over the items of `a`: one item
// per warp.
template <typename T, class In, class Epi>
__device__ __forceinline__ void spmv_fused_cta(const SpmvArgs<T>& a, In& in, Epi& epi, int cta,
                                               SpmvBuf<T>& sbuf) {
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int item = cta * kSpmvWarps + wib;
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
    T* bufx = buf + kShortCap;  // FP64 only: the gathered inputs
#pragma unroll
    for (int u = 0; u < kShortLoads; ++u) {
      const int q = base + lane + u * kWarp;
      if (q < end) {
        if constexpr (kFmaRows<T>) {
          buf[q - base] = v[u];
          bufx[q - base] = in(c[u]);
        } else {
          buf[q - base] = v[u] * in(c[u]);
        }
      }
    }
    if (do_pf) {
      int q0, q1;
      item_range(ft, q0, q1);
      prefetch_l2(a.val + q0, sizeof(T) * (size_t)(q1 - q0));
      prefetch_l2(a.col + q0, sizeof(int) * (size_t)(q1 - q0));
    }
    __syncwarp();
    if constexpr (kFmaRows<T>) {
      T sa, sb;
      packed_rows_fma<T>(buf, bufx, reinterpret_cast<unsigned*>(bufx + kShortCap), end - base,
                         lane, ha, pa0 - base, pa1 - base, hb, pb0 - base, pb1 - base, sa, sb);
      if (ha) epi.row(ra, sa, pra, acc);
      if (hb) epi.row(rb, sb, prb, acc);
    } else {
      if (ha) epi.row(ra, packed_row_sum<T>(buf, pa0 - base, pa1 - base), pra, acc);
      if (hb) epi.row(rb, packed_row_sum<T>(buf, pb0 - base, pb1 - base), prb, acc);
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

// MINB: resident CTAs per SM asked of the register allocator (the default
// shape's MPAX_SPMV_MINB, or kSpmvWideMinB: more registers per thread, fewer
// warps; the FP64 instances of the default shape spill at its 48-register cap).
template <typename T, class In, class Epi, int MINB = MPAX_SPMV_MINB>
__global__ void __launch_bounds__(kSpmvBlock, MINB) spmv_fused(SpmvArgs<T> a, In in, Epi epi) {
  __shared__ SpmvBuf<T> sbuf;
  spmv_fused_cta<T, In, Epi>(a, in, epi, blockIdx.x, sbuf);
}

// Two independent products in one launch: CTAs [0, grid1) take the items of
// (a1, in1, epi1), the others those of (a2, in2, epi2), each item exactly as
// spmv_fused computes it.  Saves a launch where the second product need not
// wait for the first (the QP momentum product of the next step beside the dual
// half-step of this one).
template <typename T, class In1, class Epi1, class In2, class Epi2, int MINB = MPAX_SPMV_MINB>
__global__ void __launch_bounds__(kSpmvBlock, MINB)
    spmv_fused_pair(SpmvArgs<T> a1, In1 in1, Epi1 epi1, int grid1, SpmvArgs<T> a2, In2 in2,
                    Epi2 epi2) {
  __shared__ SpmvBuf<T> sbuf;
  if ((int)blockIdx.x < grid1) spmv_fused_cta<T, In1, Epi1>(a1, in1, epi1, blockIdx.x, sbuf);
  else spmv_fused_cta<T, In2, Epi2>(a2, in2, epi2, blockIdx.x - grid1, sbuf);
}


// ---------------------------------------------------------------------------
// Pipelined schedule of the same work items (spmv_pipe)
// ---------------------------------------------------------------------------
// Warps are persistent and own contiguous ranges of the item list.  Lane 0
// stages the values and column indices of each item in the warp's shared
// memory with TMA bulk copies (cp.async.bulk, completion on an mbarrier), two
// items ahead of the one being computed, so a warp's gathers of item i overlap
// the matrix loads of items i+1 and i+2, and no register holds a value in
// flight.  The arithmetic is that of spmv_fused item by item (the same products,
// the same order of every sum), so both kernels return identical bits:
//   * packed rows: products rounded to T in shared memory, then one lane per
//     row sums them left to right;
//   * slices of a long row: each lane's strided products accumulated (FMA),
//     then the xor tree; the slices' sums are added in slice order.  A warp that
//     holds every slice of a row keeps that running sum in a register; a row
//     whose slices span two or more warps is finished, as in spmv_fused, by the
//     warp that arrives last at the row's counter, which adds the slices'
//     carries in slice order.
// Every wait on a copy is bounded (kWaitNs of the device clock); a wait
// that gives up sets the schedule's error word, waits (again bounded) for the
// warp's other copy and returns.

constexpr int kPipeWarps = 8;  // warps per CTA

// Elements copied per staged array: an item's range rounded out to 16 bytes.
template <typename T>
struct PipeLayout {
  static constexpr int kValV = 16 / (int)sizeof(T);  // elements per 16 bytes
  static constexpr int kValCap = kShortCap + 2 * kValV;
  static constexpr int kColCap = kShortCap + 8;
  static constexpr int kStageBytes = kValCap * (int)sizeof(T) + kColCap * 4;
  // FP64: the gathered inputs of the current item and the row-start mask (see
  // packed_rows_fma)
  static constexpr int kXBytes = kFmaRows<T> ? kShortCap * (int)sizeof(T) + kRowWords * 4 + 4 : 0;
  // two stages, the input buffer, two mbarriers
  static constexpr int kWarpBytes = 2 * kStageBytes + kXBytes + 16;
  static_assert(kStageBytes % 16 == 0, "stage size must keep 16-byte alignment");
  static_assert(kXBytes % 16 == 0, "input buffer must keep 16-byte alignment");
};

// Lane 0: stage the values and columns of item `it` (nonzeros [p0, p1)),
// rounded out to 16-byte boundaries, into one stage; returns nothing, the
// offsets are recomputed by the consumer from p0.
template <typename T>
__device__ __forceinline__ void pipe_issue(const SpmvArgs<T>& a, const int4& it,
                                           unsigned char* stage, unsigned long long* bar) {
  using L = PipeLayout<T>;
  int p0, p1;
  item_range(it, p0, p1);
  const int v0 = p0 & ~(L::kValV - 1), v1 = (p1 + L::kValV - 1) & ~(L::kValV - 1);
  const int c0 = p0 & ~3, c1 = (p1 + 3) & ~3;
  const unsigned vb = (unsigned)((v1 - v0) * (int)sizeof(T)), cb = (unsigned)((c1 - c0) * 4);
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(vb + cb)
               : "memory");
  if (vb)
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_addr(stage)),
        "l"(a.val + v0), "r"(vb), "r"(smem_addr(bar))
        : "memory");
  if (cb)
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_addr(stage + L::kValCap * sizeof(T))),
        "l"(a.col + c0), "r"(cb), "r"(smem_addr(bar))
        : "memory");
}

// Items of warp gw (of W): [lo, hi), contiguous, balanced by count.
__device__ __forceinline__ void pipe_range(int n_items, int gw, int W, int& lo, int& hi) {
  lo = (int)((long long)gw * n_items / W);
  hi = (int)((long long)(gw + 1) * n_items / W);
}

template <typename T, class In, class Epi>
__global__ void __launch_bounds__(kWarp* kPipeWarps, sizeof(T) == 4 ? 5 : 3)
    spmv_pipe(SpmvArgs<T> a, In in, Epi epi, int* err) {
  using L = PipeLayout<T>;
  extern __shared__ __align__(128) unsigned char pipe_smem[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int W = gridDim.x * kPipeWarps;
  int lo, hi;
  pipe_range(a.n_items, blockIdx.x * kPipeWarps + wib, W, lo, hi);
  if (lo >= hi) return;
  if (epi.skip()) return;  // read before any copy is issued
  if (*(volatile int*)err) return;  // an earlier wait gave up: the solve reports it
  unsigned char* wsm = pipe_smem + (size_t)wib * L::kWarpBytes;
  T* xbuf = reinterpret_cast<T*>(wsm + 2 * L::kStageBytes);  // FP64 only
  unsigned long long* bar =
      reinterpret_cast<unsigned long long*>(wsm + 2 * L::kStageBytes + L::kXBytes);
  unsigned pending = 0;  // bit s: stage s has a copy in flight (lane 0's view)
  if (lane == 0) {
    mbar_init(bar);
    mbar_init(bar + 1);
    mbar_init_fence();
    pipe_issue<T>(a, a.items[lo], wsm, bar);
    pending = 1u;
    if (lo + 1 < hi) {
      pipe_issue<T>(a, a.items[lo + 1], wsm + L::kStageBytes, bar + 1);
      pending |= 2u;
    }
  }
  __syncwarp();
  in.load();
  epi.load();
  unsigned phase = 0;  // bit s: parity of stage s's next completion
  bool failed = false;
  T run = 0;  // running sum of the long row whose slices this warp is walking
  int4 it = a.items[lo];
  for (int i = lo; i < hi; ++i) {
    const int sidx = (i - lo) & 1;
    unsigned char* stage = wsm + sidx * L::kStageBytes;
    T* sval = reinterpret_cast<T*>(stage);
    const int* scol = reinterpret_cast<const int*>(stage + L::kValCap * sizeof(T));
    const int4 it_next = (i + 1 < hi) ? a.items[i + 1] : it;
    int4 nx = make_int4(0, 0, 0, 0);
    if (lane == 0 && i + 2 < hi) nx = a.items[i + 2];
    double acc[Epi::NQ];
#pragma unroll
    for (int q = 0; q < Epi::NQ; ++q) acc[q] = 0.0;
    // operands of the item's rows, requested before waiting for its matrix
    int r = 0, pa0 = 0, pa1 = 0, pb0 = 0, pb1 = 0, ra = 0, rb = 0;
    bool ha = false, hb = false;
    typename Epi::Pre pra, prb;
    if (it.x >= 0) {
      ra = it.x + lane;
      rb = it.x + kWarp + lane;
      ha = ra < it.y;
      hb = rb < it.y;
      const int sa = ha ? ra : it.x, sb = hb ? rb : it.x;
      pa0 = a.rp[sa];
      pa1 = a.rp[sa + 1];
      pb0 = a.rp[sb];
      pb1 = a.rp[sb + 1];
      epi.pre(sa, pra);
      epi.pre(sb, prb);
    } else {
      r = -(it.x + 1);
      epi.pre(r, pra);
    }
    // lane 0 waits (bounded) and tells the warp; the others then find the phase
    // complete, which also makes the staged bytes visible to them
    const unsigned par = (phase >> sidx) & 1u;
    bool ok = true;
    if (lane == 0) ok = mbar_wait(bar + sidx, par);
    ok = __shfl_sync(0xffffffffu, ok, 0);
    if (!ok) {
      failed = true;
      break;
    }
    if (lane != 0) mbar_wait(bar + sidx, par);
    phase ^= 1u << sidx;
    pending &= ~(1u << sidx);
    if (it.x >= 0) {
      // ---- packed short rows [r0, r1), nonzeros [base, end) ----------------
      const int base = it.z;
      const int cnt = it.w - base;
      T* buf = sval + (base & (L::kValV - 1));  // buf[q - base] = product q
      const int* cb = scol + (base & 3);
      // xbuf is rewritten for every item: the previous item's sums have read it
      if constexpr (kFmaRows<T>) __syncwarp();
#pragma unroll
      for (int u = 0; u < kShortLoads; ++u) {
        const int q = lane + u * kWarp;
        if (q < cnt) {
          if constexpr (kFmaRows<T>) xbuf[q] = in(cb[q]);
          else buf[q] = buf[q] * in(cb[q]);
        }
      }
      __syncwarp();
      if constexpr (kFmaRows<T>) {
        T sa, sb;
        packed_rows_fma<T>(buf, xbuf, reinterpret_cast<unsigned*>(xbuf + kShortCap), cnt, lane,
                           ha, pa0 - base, pa1 - base, hb, pb0 - base, pb1 - base, sa, sb);
        if (ha) epi.row(ra, sa, pra, acc);
        if (hb) epi.row(rb, sb, prb, acc);
      } else {
        if (ha) epi.row(ra, packed_row_sum<T>(buf, pa0 - base, pa1 - base), pra, acc);
        if (hb) epi.row(rb, packed_row_sum<T>(buf, pb0 - base, pb1 - base), prb, acc);
      }
      if (Epi::NQ > 0 && epi.check) {
#pragma unroll
        for (int q = 0; q < Epi::NQ; ++q) {
          const double t = warp_sum(acc[q]);
          if (lane == 0) a.part[(a.q0 + q) * a.n_items + i] = t;
        }
      }
    } else {
      // ---- slice si of S of the long row r: nonzeros [p0, p1) --------------
      const int p0 = it.y, cnt = it.z - it.y;
      const int si = it.w >> 16, S = it.w & 0xffff;
      const int first = i - si;
      const T* vb = sval + (p0 & (L::kValV - 1));
      const int* cb = scol + (p0 & 3);
      T s = 0;
#pragma unroll
      for (int u = 0; u < kSliceLoads; ++u) {
        const int q = lane + u * kWarp;
        if (q < cnt) s += vb[q] * in(cb[q]);
      }
      s = warp_sum(s);
      // the row's sum in slice order, as spmv_fused forms it: a one-slice row
      // is its slice's sum; otherwise 0 + c_0 + c_1 + ...  A warp whose range
      // begins inside the row starts a partial (it goes through the carries).
      if (si == 0 || i == lo) run = (S == 1) ? s : (T)0 + s;
      else run += s;
      const bool whole = first >= lo && first + S <= hi;  // every slice in this warp
      if (whole) {
        if (si == S - 1 && lane == 0) {
          epi.row(r, run, pra, acc);
          if (Epi::NQ > 0 && epi.check) {
#pragma unroll
            for (int q = 0; q < Epi::NQ; ++q) a.part[(a.q0 + q) * a.n_items + first] = acc[q];
          }
        }
      } else if (lane == 0) {
        // the row's slices span warps: every slice leaves its carry; the warp's
        // last slice of the row arrives at the counter with this warp's count
        a.carry[i] = s;
        if (si == S - 1 || i == hi - 1) {
          const int mine = i - max(first, lo) + 1;  // this warp's slices of the row
          int prev;
          asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;"
                       : "=r"(prev)
                       : "l"(a.cnt + first), "r"(mine)
                       : "memory");
          if (prev + mine == S) {
            T tot = 0;
            for (int t = 0; t < S; ++t) tot += __ldcg(a.carry + first + t);
            a.cnt[first] = 0;  // ready for the next launch
            epi.row(r, tot, pra, acc);
            if (Epi::NQ > 0 && epi.check) {
#pragma unroll
              for (int q = 0; q < Epi::NQ; ++q) a.part[(a.q0 + q) * a.n_items + first] = acc[q];
            }
          }
        }
      }
      // the finished row's contribution lands in slot `first`; the other
      // slices' slots hold zero
      if (Epi::NQ > 0 && epi.check && si != 0 && lane == 0) {
#pragma unroll
        for (int q = 0; q < Epi::NQ; ++q) a.part[(a.q0 + q) * a.n_items + i] = 0.0;
      }
    }
    // the stage is free again: order this warp's generic accesses to it before
    // the next bulk copy into it (async proxy), then refill it
    if (i + 2 < hi) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) {
        pipe_issue<T>(a, nx, stage, bar + sidx);
        pending |= 1u << sidx;
      }
    }
    it = it_next;
  }
  if (failed && lane == 0) {
    atomicOr(err, 1);
    // copies still in flight land in this warp's shared memory: wait for them
    // (bounded) before the CTA may exit
    for (int t = 0; t < 2; ++t)
      if (pending & (1u << t)) mbar_wait(bar + t, (phase >> t) & 1u);
  }
  __syncwarp();
}

}  // namespace mpax
