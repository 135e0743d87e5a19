// Host interface of the tensor-core BF16x3 product (umma.cu).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace mpax {

// Arguments of one product kernel (umma.cuh).
struct UmmaArgs {
  int M, N, K;
  int a_mn_major;  // 0: A_op stored [M][K]; 1: stored [K][M]
  int bn;          // instances per tile: 32, 64, 128 or 256 (TMEM columns)
  float* D;        // D[n * ldd + m]
  long long ldd;
  int* err;        // set to 1 when a bounded wait gave up
};

// One product D = A_op V^T with fixed operand buffers: its four tensor maps,
// arguments and grid, built once and launched many times.
struct UmmaPlan {
  CUtensorMap ah, al, vh, vl;
  UmmaArgs args;
  dim3 grid;
  double flops;  // 3 * 2 M N K
  int bk;        // K block of the pipeline: 64 (2 stages) or 32 (4 stages)
};

// Instances per output tile for N instances: 32, 64, 128 or 256.
int umma_tile_n(int N);
// A_op (M x K) is A stored [M][lda] (a_mn_major = 0) or [K][lda] (= 1), V is
// [N][ldv] (K used), D[n * ldd + m].  lda and ldv must be multiples of 8 and the
// buffers 16-byte aligned.  err: device int set when a bounded wait gives up.
// bk: K block of the pipeline, 64 (2 stages) or 32 (4 stages).
cudaError_t umma_plan(UmmaPlan* p, const __nv_bfloat16* Ahi, const __nv_bfloat16* Alo,
                      long long lda, int a_mn_major, const __nv_bfloat16* Vhi,
                      const __nv_bfloat16* Vlo, long long ldv, int M, int N, int K, float* D,
                      long long ldd, int* err, int bk);
cudaError_t umma_run(const UmmaPlan& p, cudaStream_t s);
// BF16 split of a rows x cols FP32 matrix (row stride lds) into row stride ldd.
cudaError_t split_rows(const float* src, long long rows, long long cols, long long lds,
                       __nv_bfloat16* hi, __nv_bfloat16* lo, long long ldd, cudaStream_t s);

}  // namespace mpax
