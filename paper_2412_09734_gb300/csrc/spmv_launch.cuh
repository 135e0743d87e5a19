// Launch of the fused SpMV kernels of kernels.cuh on a row schedule: the
// schedule's kernel kind (one warp per item, the pipelined kernel, or one warp
// per item with the wide register budget) and each kind's launch shape.
#pragma once

#include <algorithm>

#include "common.cuh"
#include "kernels.cuh"

namespace mpax {

// Warps of spmv_fused<T, In, Epi, MINB> resident on the whole GPU (one wave).
template <typename T, class In, class Epi, int MINB>
int resident_warps() {
  static int w = -1;
  if (w < 0) {
    int blocks = 0, dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, spmv_fused<T, In, Epi, MINB>,
                                                  kSpmvBlock, 0);
    w = std::max(1, blocks) * sms * kSpmvWarps;
  }
  return w;
}

// Launch shape of spmv_pipe<T, In, Epi>: CTAs resident on the whole GPU and the
// dynamic shared memory of one CTA (two stages per warp).
struct PipeShape {
  int grid = -1;
  size_t smem = 0;
};
template <typename T, class In, class Epi>
const PipeShape& pipe_shape() {
  static PipeShape sh;
  if (sh.grid < 0) {
    const size_t smem = (size_t)kPipeWarps * PipeLayout<T>::kWarpBytes;
    cudaFuncSetAttribute(spmv_pipe<T, In, Epi>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    int blocks = 0, dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, spmv_pipe<T, In, Epi>,
                                                  kWarp * kPipeWarps, smem);
    sh.smem = smem;
    sh.grid = std::max(1, blocks) * sms;
  }
  return sh;
}
// Items per warp below which spmv_pipe launches fewer warps than fit (a warp
// needs a few items for its copies to run ahead of its gathers).
constexpr int kPipeMinItems = 4;

template <typename T, class In, class Epi>
void launch_spmv(const Sched& sc, const Csr& K, const T* val, In in, Epi epi, int q0,
                 cudaStream_t s) {
  if (sc.n_items == 0) return;
  if (sc.kind == kSpmvPipe) {
    SpmvArgs<T> a;
    a.items = sc.items;
    a.n_items = sc.n_items;
    a.pf_dist = 0;
    a.rp = K.rp;
    a.col = K.col;
    a.val = val;
    a.cnt = sc.cnt;
    a.carry = reinterpret_cast<T*>(sc.carry);
    a.part = sc.part;
    a.q0 = q0;
    const PipeShape& sh = pipe_shape<T, In, Epi>();
    const int want = (sc.n_items + kPipeMinItems * kPipeWarps - 1) / (kPipeMinItems * kPipeWarps);
    const int grid = std::max(1, std::min(sh.grid, want));
    spmv_pipe<T, In, Epi><<<grid, kWarp * kPipeWarps, sh.smem, s>>>(a, in, epi,
                                                                     sc.cnt + sc.n_items);
    return;
  }
  SpmvArgs<T> a;
  a.items = sc.items;
  a.n_items = sc.n_items;
  const bool wide = sc.kind == kSpmvItemWide;
  a.pf_dist = !MPAX_SPMV_PREFETCH ? 0
              : wide ? resident_warps<T, In, Epi, kSpmvWideMinB>()
                     : resident_warps<T, In, Epi, MPAX_SPMV_MINB>();
  a.rp = K.rp;
  a.col = K.col;
  a.val = val;
  a.cnt = sc.cnt;
  a.carry = reinterpret_cast<T*>(sc.carry);
  a.part = sc.part;
  a.q0 = q0;
  const int grid = (sc.n_items + kSpmvWarps - 1) / kSpmvWarps;
  if (wide) {
    spmv_fused<T, In, Epi, kSpmvWideMinB><<<grid, kSpmvBlock, 0, s>>>(a, in, epi);
    return;
  }
#if MPAX_SPMV_PDL
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(kSpmvBlock);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, spmv_fused<T, In, Epi>, a, in, epi);
#else
  spmv_fused<T, In, Epi><<<grid, kSpmvBlock, 0, s>>>(a, in, epi);
#endif
}

// The arguments of a spmv_fused launch over schedule sc (no prefetch).
template <typename T>
SpmvArgs<T> fused_args(const Sched& sc, const Csr& K, const T* val, int q0) {
  SpmvArgs<T> a;
  a.items = sc.items;
  a.n_items = sc.n_items;
  a.pf_dist = 0;
  a.rp = K.rp;
  a.col = K.col;
  a.val = val;
  a.cnt = sc.cnt;
  a.carry = reinterpret_cast<T*>(sc.carry);
  a.part = sc.part;
  a.q0 = q0;
  return a;
}

// Two independent products in one spmv_fused_pair launch, with the first
// schedule's register budget.  Returns false, launching nothing, when either
// schedule runs the pipelined kernel or has no items: the caller then launches
// the two apart.  Every item is computed as launch_spmv computes it, so the
// results are the same bits.
template <typename T, class In1, class Epi1, class In2, class Epi2>
bool launch_spmv_pair(const Sched& s1, const Csr& K1, const T* v1, In1 in1, Epi1 e1,
                      const Sched& s2, const Csr& K2, const T* v2, In2 in2, Epi2 e2,
                      cudaStream_t s) {
  if (s1.n_items == 0 || s2.n_items == 0 || s1.kind == kSpmvPipe || s2.kind == kSpmvPipe)
    return false;
  const SpmvArgs<T> a1 = fused_args<T>(s1, K1, v1, 0), a2 = fused_args<T>(s2, K2, v2, 0);
  const int g1 = (s1.n_items + kSpmvWarps - 1) / kSpmvWarps;
  const int g2 = (s2.n_items + kSpmvWarps - 1) / kSpmvWarps;
  if (s1.kind == kSpmvItemWide)
    spmv_fused_pair<T, In1, Epi1, In2, Epi2, kSpmvWideMinB>
        <<<g1 + g2, kSpmvBlock, 0, s>>>(a1, in1, e1, g1, a2, in2, e2);
  else
    spmv_fused_pair<T, In1, Epi1, In2, Epi2><<<g1 + g2, kSpmvBlock, 0, s>>>(a1, in1, e1, g1, a2,
                                                                          in2, e2);
  return true;
}

}  // namespace mpax
