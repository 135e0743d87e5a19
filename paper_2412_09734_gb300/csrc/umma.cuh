// Dense BF16x3 products of the shared-matrix batch on the fifth-generation tensor
// cores: tcgen05.mma with the accumulator in tensor memory (TMEM), operand tiles
// staged in shared memory by TMA (cp.async.bulk.tensor) with the 128-byte swizzle,
// one elected thread issuing the MMAs.
//
// D (M x N, FP32) = A_op (M x K) . V^T, V (N x K) the instances' vectors, with the
// split x = x_hi + x_lo, x_hi = bf16(x), x_lo = bf16(x - x_hi), of both operands:
//   D = A_hi V_lo + A_lo V_hi + A_hi V_hi,
// the three products accumulated in one FP32 accumulator, k-block by k-block,
// small terms first within each k-block.  Each A_hi tile is read once for the two
// products it feeds.  A_op is either A (stored [M][K], K contiguous: the product
// A~ X of the dual step) or A^T (A stored [K][M], M contiguous: the product A~^T Y
// of the primal step); the MMA reads the latter as an MN-major operand.
//
// CTA: 6 warps.  Warp 0 (one lane) issues the TMA loads of a two- or four-stage
// pipeline (UmmaShape);
// warp 1 allocates TMEM and (one lane) issues the MMAs, releasing each stage
// with tcgen05.commit; warps 2-5 read the accumulator (tcgen05.ld, one 32-lane
// quarter each) and store D.  Every mbarrier wait is bounded; a wait that gives
// up sets the error word, the other roles drain what is in flight, and TMEM is
// freed on every path.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "sync.cuh"
#include "umma_host.h"

namespace mpax {

constexpr int kUmmaBM = 128;      // rows (M) of an output tile: TMEM lanes
constexpr int kUmmaBNMax = 256;   // instances (N) of an output tile, at most
constexpr int kUmmaThreads = 192;

// Two pipeline shapes with the same 192 KB of stages: K blocks of 64 (128-byte
// rows, 128-byte swizzle) in 2 stages, or K blocks of 32 (64-byte rows of the
// K-major operands, 64-byte swizzle) in 4 stages, which keeps three stages in
// flight while the MMAs read the fourth.
template <int BK>
struct UmmaShape {
  static_assert(BK == 64 || BK == 32, "K block of 64 or 32");
  static constexpr int kStages = BK == 64 ? 2 : 4;
  static constexpr int kATile = kUmmaBM * BK * 2;     // 16 / 8 KB
  static constexpr int kVTile = kUmmaBNMax * BK * 2;  // 32 / 16 KB
  static constexpr int kStage = 2 * kATile + 2 * kVTile;
  static constexpr int kSmem = kStages * kStage + 1024 + 256;  // + alignment, barriers
  // K-major operands: rows of BK elements; 8-row atoms of 8 * 2 BK bytes
  static constexpr uint32_t kKSwizzle = BK == 64 ? 2u : 4u;  // 128- / 64-byte swizzle
  static constexpr uint32_t kKAtom = 8u * 2u * BK;
};

// Shared-memory matrix descriptor of a tcgen05 operand: start address, leading-
// and stride-dimension byte offsets (all >> 4), descriptor version 1, swizzle
// mode (2: 128-byte, 4: 64-byte).  Tiles start on 1024-byte boundaries (base
// offset 0).
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo,
                                              uint32_t swizzle) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46) | ((uint64_t)swizzle << 61);
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, A K-major
// (0) or MN-major (1), B K-major, N / 8 and M / 16.
__host__ __device__ constexpr uint32_t umma_idesc(int M, int N, int a_mn) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)a_mn << 15) |
         ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void umma_commit(unsigned long long* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::
                   "r"(smem_addr(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* tm, int c0, int c1,
                                            unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(c0), "r"(c1), "r"(smem_addr(bar))
      : "memory");
}
// 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

template <int BK>
__global__ void __launch_bounds__(kUmmaThreads, 1)
    umma_bf16x3(const __grid_constant__ CUtensorMap tAh, const __grid_constant__ CUtensorMap tAl,
                const __grid_constant__ CUtensorMap tVh, const __grid_constant__ CUtensorMap tVl,
                UmmaArgs g) {
  using S = UmmaShape<BK>;
  constexpr int kUmmaStages = S::kStages, kUmmaStage = S::kStage;
  constexpr int kUmmaATile = S::kATile, kUmmaVTile = S::kVTile, kUmmaBK = BK;
  extern __shared__ unsigned char umma_raw[];
  __shared__ int s_fail;
  // the swizzled tiles need 1024-byte alignment in the shared window
  const uint32_t raw = smem_addr(umma_raw);
  unsigned char* sm = umma_raw + ((1024u - (raw & 1023u)) & 1023u);
  unsigned long long* full = reinterpret_cast<unsigned long long*>(sm + kUmmaStages * kUmmaStage);
  unsigned long long* empty = full + kUmmaStages;
  unsigned long long* accf = empty + kUmmaStages;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(accf + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // instance tiles vary fastest: the CTAs that share an A tile run together, so
  // all but the first read it from L2 (A is larger than L2 and streams from HBM)
  const int m0 = blockIdx.y * kUmmaBM, n0 = blockIdx.x * g.bn;
  const int KB = (g.K + kUmmaBK - 1) / kUmmaBK;
  const uint32_t ncols = (uint32_t)g.bn;
  if (threadIdx.x == 0) {
    s_fail = 0;
    for (int s = 0; s < kUmmaStages; ++s) {
      mbar_init(full + s);
      mbar_init(empty + s);
    }
    mbar_init(accf);
    mbar_init_fence();
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(tslot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  if (warp == 0) {
    if (lane == 0) {
      const uint32_t tx = 2u * kUmmaATile + 2u * (uint32_t)g.bn * kUmmaBK * 2u;
      int issued = 0;
      for (int kb = 0; kb < KB; ++kb) {
        const int s = kb % kUmmaStages;
        if (kb >= kUmmaStages && !mbar_wait(empty + s, ((kb / kUmmaStages) - 1) & 1)) {
          s_fail = 1;
          break;
        }
        if (*(volatile int*)&s_fail) break;
        unsigned char* st = sm + s * kUmmaStage;
        const int k0 = kb * kUmmaBK;
        mbar_expect_tx(full + s, tx);
        if (!g.a_mn_major) {
          tma_load_2d(st, &tAh, k0, m0, full + s);
          tma_load_2d(st + kUmmaATile, &tAl, k0, m0, full + s);
        } else {
          // two 64 (M) x 64 (K) boxes per operand: M atoms 8 KB apart
          tma_load_2d(st, &tAh, m0, k0, full + s);
          tma_load_2d(st + kUmmaATile / 2, &tAh, m0 + 64, k0, full + s);
          tma_load_2d(st + kUmmaATile, &tAl, m0, k0, full + s);
          tma_load_2d(st + kUmmaATile + kUmmaATile / 2, &tAl, m0 + 64, k0, full + s);
        }
        tma_load_2d(st + 2 * kUmmaATile, &tVh, k0, n0, full + s);
        tma_load_2d(st + 2 * kUmmaATile + kUmmaVTile, &tVl, k0, n0, full + s);
        issued = kb + 1;
      }
      // copies still in flight land in this CTA's shared memory: wait for them
      // (bounded) before the CTA may exit
      for (int kb = issued > kUmmaStages ? issued - kUmmaStages : 0; kb < issued; ++kb)
        mbar_wait(full + (kb % kUmmaStages), (kb / kUmmaStages) & 1);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = umma_idesc(kUmmaBM, g.bn, g.a_mn_major);
      for (int kb = 0; kb < KB; ++kb) {
        const int s = kb % kUmmaStages;
        if (!mbar_wait(full + s, (kb / kUmmaStages) & 1)) {
          s_fail = 1;
          break;
        }
        tc_fence_after();
        const uint32_t st = smem_addr(sm + s * kUmmaStage);
        const uint32_t ah = st, al = st + kUmmaATile;
        const uint32_t vh = st + 2 * kUmmaATile, vl = vh + kUmmaVTile;
#pragma unroll
        for (int ks = 0; ks < kUmmaBK / 16; ++ks) {
          // K = 16 per MMA: 32 bytes along a K-major row (8-row atoms of S::kKAtom
          // bytes); two 8-row atoms (2 KB) of an MN-major tile (128-byte swizzle),
          // whose two 64-row halves sit half an A tile apart
          uint64_t dah, dal;
          if (!g.a_mn_major) {
            dah = umma_desc(ah + 32 * ks, 16, S::kKAtom, S::kKSwizzle);
            dal = umma_desc(al + 32 * ks, 16, S::kKAtom, S::kKSwizzle);
          } else {
            dah = umma_desc(ah + 2048 * ks, kUmmaATile / 2, 1024, 2u);
            dal = umma_desc(al + 2048 * ks, kUmmaATile / 2, 1024, 2u);
          }
          const uint64_t dvh = umma_desc(vh + 32 * ks, 16, S::kKAtom, S::kKSwizzle);
          const uint64_t dvl = umma_desc(vl + 32 * ks, 16, S::kKAtom, S::kKSwizzle);
          umma_mma(tmem, dah, dvl, idesc, (kb | ks) ? 1u : 0u);
          umma_mma(tmem, dal, dvh, idesc, 1u);
          umma_mma(tmem, dah, dvh, idesc, 1u);
        }
        umma_commit(empty + s);  // the stage is free once these MMAs have read it
      }
      umma_commit(accf);  // the accumulator is complete once every MMA above is
      if (!mbar_wait(accf, 0)) s_fail = 1;
    }
  } else {
    // warps 2-5: warp w reads TMEM lanes 32 (w % 4) .. +31, i.e. rows of the tile
    const int q = warp & 3;
    const bool ok = mbar_wait(accf, 0);
    tc_fence_after();
    if (ok) {
      const int row = m0 + q * 32 + lane;
      for (int c0 = 0; c0 < g.bn; c0 += 32) {
        float v[32];
        tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, v);
        if (row < g.M) {
#pragma unroll
          for (int c = 0; c < 32; ++c) {
            const int n = n0 + c0 + c;
            if (n < g.N) g.D[(size_t)n * g.ldd + row] = v[c];
          }
        }
      }
    } else {
      s_fail = 1;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols)
                 : "memory");
  }
  if (threadIdx.x == 0 && s_fail) atomicOr(g.err, 1);
}

}  // namespace mpax
