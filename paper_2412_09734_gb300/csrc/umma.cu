// Host side of the tensor-core BF16x3 product (umma.cuh): TMA tensor maps,
// launch, and the C-ABI entry point mpax_dense_bf16x3 that splits FP32 operands
// and forms one product (the product of the shared-matrix batch on its own).
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>
#include <string>

#include "../../include/mpax.h"
#include "common.cuh"
#include "umma.cuh"
#include "umma_host.h"

namespace mpax {

namespace {

typedef CUresult (*EncodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// cuTensorMapEncodeTiled from the driver through the runtime (no -lcuda link).
EncodeTiled encode_tiled() {
  static EncodeTiled fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(p);
  }
  return fn;
}

// 2-D BF16 tensor map: inner dimension `inner` (contiguous), `outer` rows of
// `ld` elements, box {box_inner, box_rows} (box_inner 64: 128-byte swizzle, 32:
// 64-byte swizzle), out-of-range reads zero.
cudaError_t make_map(CUtensorMap* m, const __nv_bfloat16* base, long long inner, long long outer,
                     long long ld, int box_inner, int box_rows) {
  EncodeTiled fn = encode_tiled();
  if (!fn) return cudaErrorNotSupported;
  if ((ld * 2) % 16 != 0 || (reinterpret_cast<uintptr_t>(base) & 15) != 0)
    return cudaErrorInvalidValue;
  const cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
  const cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
  const cuuint32_t box[2] = {(cuuint32_t)box_inner, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1u, 1u};
  const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                        const_cast<__nv_bfloat16*>(base), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE,
                        box_inner == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// x -> (bf16(x), bf16(x - bf16(x))) of a rows x cols FP32 matrix (row stride
// lds) into BF16 matrices of row stride ldd; columns [cols, ldd) are zero.
__global__ void k_split_rows(const float* __restrict__ src, long long rows, long long cols,
                             long long lds, __nv_bfloat16* __restrict__ hi,
                             __nv_bfloat16* __restrict__ lo, long long ldd) {
  const long long total = rows * ldd;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long r = e / ldd, c = e - r * ldd;
    const float v = c < cols ? src[r * lds + c] : 0.0f;
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    hi[e] = h;
    lo[e] = __float2bfloat16_rn(v - __bfloat162float(h));
  }
}

}  // namespace

int umma_tile_n(int N) {
  int bn = 32;
  while (bn < N && bn < kUmmaBNMax) bn *= 2;
  return bn;
}

cudaError_t umma_plan(UmmaPlan* p, const __nv_bfloat16* Ahi, const __nv_bfloat16* Alo,
                      long long lda, int a_mn_major, const __nv_bfloat16* Vhi,
                      const __nv_bfloat16* Vlo, long long ldv, int M, int N, int K, float* D,
                      long long ldd, int* err, int bk) {
  std::memset(p, 0, sizeof(*p));
  if (M < 1 || N < 1 || K < 1 || (bk != 64 && bk != 32)) return cudaErrorInvalidValue;
  const int bn = umma_tile_n(N);
  cudaError_t e;
  if (!a_mn_major) {
    if ((e = make_map(&p->ah, Ahi, K, M, lda, bk, kUmmaBM))) return e;
    if ((e = make_map(&p->al, Alo, K, M, lda, bk, kUmmaBM))) return e;
  } else {  // MN-major: 64 rows of M per box (128-byte swizzle), bk rows of K
    if ((e = make_map(&p->ah, Ahi, M, K, lda, 64, bk))) return e;
    if ((e = make_map(&p->al, Alo, M, K, lda, 64, bk))) return e;
  }
  if ((e = make_map(&p->vh, Vhi, K, N, ldv, bk, bn))) return e;
  if ((e = make_map(&p->vl, Vlo, K, N, ldv, bk, bn))) return e;
  p->bk = bk;
  p->args = UmmaArgs{M, N, K, a_mn_major, bn, D, ldd, err};
  p->grid = dim3((unsigned)((N + bn - 1) / bn), (unsigned)((M + kUmmaBM - 1) / kUmmaBM));
  p->flops = 3.0 * 2.0 * (double)M * N * K;
  return cudaSuccess;
}

template <int BK>
cudaError_t umma_launch(const UmmaPlan& p, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(umma_bf16x3<BK>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         UmmaShape<BK>::kSmem);
    if (e) return e;
    attr = true;
  }
  umma_bf16x3<BK><<<p.grid, kUmmaThreads, UmmaShape<BK>::kSmem, s>>>(p.ah, p.al, p.vh, p.vl,
                                                                     p.args);
  return cudaGetLastError();
}

cudaError_t umma_run(const UmmaPlan& p, cudaStream_t s) {
  return p.bk == 32 ? umma_launch<32>(p, s) : umma_launch<64>(p, s);
}

cudaError_t split_rows(const float* src, long long rows, long long cols, long long lds,
                       __nv_bfloat16* hi, __nv_bfloat16* lo, long long ldd, cudaStream_t s) {
  const long long total = rows * ldd;
  if (total == 0) return cudaSuccess;
  const int g = (int)std::min<long long>(8192, (total + 255) / 256);
  k_split_rows<<<g, 256, 0, s>>>(src, rows, cols, lds, hi, lo, ldd);
  return cudaGetLastError();
}

}  // namespace mpax

using namespace mpax;

extern "C" {

mpax_status mpax_dense_bf16x3(int32_t M, int32_t N, int32_t K, int32_t a_mn_major,
                              int32_t tile_k, const float* A, const float* V, float* D,
                              mpax_mem_kind kind, void* cuda_stream) {
  if (M < 1 || N < 1 || K < 1 || !A || !V || !D) {
    set_last_error("M, N, K must be >= 1 and A, V, D non-NULL");
    return MPAX_ERR_INVALID_ARGUMENT;
  }
  if (tile_k != 0 && tile_k != 32 && tile_k != 64) {
    set_last_error("tile_k must be 0 (default), 32 or 64");
    return MPAX_ERR_INVALID_ARGUMENT;
  }
  const int bk = tile_k == 64 ? 64 : 32;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const long long arows = a_mn_major ? K : M, acols = a_mn_major ? M : K;
  const long long lda = (acols + 7) / 8 * 8, ldv = ((long long)K + 7) / 8 * 8;
  const cudaMemcpyKind kin = kind == MPAX_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  float *dA = nullptr, *dV = nullptr, *dD = nullptr;
  __nv_bfloat16 *ah = nullptr, *al = nullptr, *vh = nullptr, *vl = nullptr;
  int* err = nullptr;
  cudaError_t e = cudaSuccess;
  if (kind == MPAX_MEM_HOST) {
    e = cudaMalloc(&dA, sizeof(float) * arows * acols);
    if (!e) e = cudaMalloc(&dV, sizeof(float) * (size_t)N * K);
    if (!e) e = cudaMalloc(&dD, sizeof(float) * (size_t)N * M);
    if (!e) e = cudaMemcpyAsync(dA, A, sizeof(float) * arows * acols, kin, s);
    if (!e) e = cudaMemcpyAsync(dV, V, sizeof(float) * (size_t)N * K, kin, s);
  }
  const float* Ad = kind == MPAX_MEM_HOST ? dA : A;
  const float* Vd = kind == MPAX_MEM_HOST ? dV : V;
  float* Dd = kind == MPAX_MEM_HOST ? dD : D;
  if (!e) e = cudaMalloc(&ah, sizeof(__nv_bfloat16) * arows * lda);
  if (!e) e = cudaMalloc(&al, sizeof(__nv_bfloat16) * arows * lda);
  if (!e) e = cudaMalloc(&vh, sizeof(__nv_bfloat16) * (size_t)N * ldv);
  if (!e) e = cudaMalloc(&vl, sizeof(__nv_bfloat16) * (size_t)N * ldv);
  if (!e) e = cudaMalloc(&err, sizeof(int));
  if (!e) e = cudaMemsetAsync(err, 0, sizeof(int), s);
  if (!e) e = split_rows(Ad, arows, acols, acols, ah, al, lda, s);
  if (!e) e = split_rows(Vd, N, K, K, vh, vl, ldv, s);
  UmmaPlan p;
  if (!e) e = umma_plan(&p, ah, al, lda, a_mn_major, vh, vl, ldv, M, N, K, Dd, M, err, bk);
  if (!e) e = umma_run(p, s);
  int herr = 0;
  if (!e) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (!e && kind == MPAX_MEM_HOST)
    e = cudaMemcpyAsync(D, dD, sizeof(float) * (size_t)N * M, cudaMemcpyDeviceToHost, s);
  if (!e) e = cudaStreamSynchronize(s);
  for (void* q : {(void*)dA, (void*)dV, (void*)dD, (void*)ah, (void*)al, (void*)vh, (void*)vl,
                  (void*)err})
    if (q) cudaFree(q);
  if (e) {
    set_last_error(cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? MPAX_ERR_OUT_OF_MEMORY : MPAX_ERR_CUDA;
  }
  if (herr) {
    set_last_error("a bounded wait of the tensor-core product gave up");
    return MPAX_ERR_DEVICE_TIMEOUT;
  }
  return MPAX_OK;
}

}  // extern "C"
