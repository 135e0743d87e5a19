// C ABI of the library (include/mpax.h): argument checks, device copies of the
// problem data, validation on the device, preprocessing and the solve routine.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "engine.cuh"

using namespace mpax;

namespace {

thread_local std::string g_err;

mpax_status fail(mpax_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

}  // namespace

void mpax::set_last_error(const char* msg) { g_err = msg; }

namespace {

mpax_status cuda_fail(cudaError_t e, const char* where) {
  if (e == cudaErrorMemoryAllocation)
    return fail(MPAX_ERR_OUT_OF_MEMORY, std::string(where) + ": out of device memory");
  if (e == cudaErrorTimeout)  // the library's own bounded device waits
    return fail(MPAX_ERR_DEVICE_TIMEOUT,
                std::string(where) + ": a bounded wait of a SpMV kernel gave up");
  return fail(MPAX_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define TRY_CUDA(expr, where)                    \
  do {                                           \
    cudaError_t e_ = (expr);                     \
    if (e_ != cudaSuccess) return cuda_fail(e_, where); \
  } while (0)

// ---- validation kernels -----------------------------------------------------
enum : int {
  V_ROWPTR = 1,
  V_COL_RANGE = 2,
  V_COL_ORDER = 4,
  V_VAL_NAN = 8,
  V_COST = 16,
  V_VBOUNDS = 32,
  V_RBOUNDS = 64,
  V_DIAG = 128,
};

__global__ void k_rowptr64_to_32(const long long* __restrict__ src, int* __restrict__ dst,
                                 int rows, long long nnz, int* flags) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > rows) return;
  const long long v = src[i];
  if (v < 0 || v > nnz || (i == 0 && v != 0) || (i == rows && v != nnz) ||
      (i < rows && src[i + 1] < v))
    atomicOr(flags, V_ROWPTR);
  dst[i] = (int)(v < 0 ? 0 : (v > nnz ? nnz : v));
}

__global__ void k_check_csr(const int* __restrict__ rp, const int* __restrict__ col,
                            const double* __restrict__ val, int rows, int cols, int* flags) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows) return;
  const int b = rp[i], e = rp[i + 1];
  int prev = -1;
  for (int p = b; p < e; ++p) {
    const int c = col[p];
    if (c < 0 || c >= cols) atomicOr(flags, V_COL_RANGE);
    if (c <= prev) atomicOr(flags, V_COL_ORDER);
    prev = c;
    if (!isfinite(val[p])) atomicOr(flags, V_VAL_NAN);
  }
}

// FP32 inputs widened to FP64 (mpax_lp_create_f32)
__global__ void k_widen(const float* __restrict__ a, double* __restrict__ b, size_t k) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < k;
       i += (size_t)gridDim.x * blockDim.x)
    b[i] = (double)a[i];
}

__global__ void k_check_vecs(const double* c, const double* l, const double* u, int n,
                             const double* lc, const double* uc, int m, const double* D,
                             int* flags) {
  const int stride = gridDim.x * blockDim.x;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
    if (!isfinite(c[j])) atomicOr(flags, V_COST);
    const double lo = l[j], hi = u[j];
    if (isnan(lo) || isnan(hi) || lo > hi || lo == INFINITY || hi == -INFINITY)
      atomicOr(flags, V_VBOUNDS);
    if (D && (!isfinite(D[j]) || D[j] < 0.0)) atomicOr(flags, V_DIAG);
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
    const double lo = lc[i], hi = uc[i];
    if (isnan(lo) || isnan(hi) || lo > hi || lo == INFINITY || hi == -INFINITY)
      atomicOr(flags, V_RBOUNDS);
  }
}

std::string flags_message(int f) {
  std::string s;
  if (f & V_ROWPTR) s += "row_ptr must start at 0, end at nnz and be non-decreasing; ";
  if (f & V_COL_RANGE) s += "column index out of range; ";
  if (f & V_COL_ORDER) s += "column indices must be strictly increasing within a row; ";
  if (f & V_VAL_NAN) s += "matrix values must be finite; ";
  if (f & V_COST) s += "c must be finite; ";
  if (f & V_VBOUNDS) s += "variable bounds must satisfy l <= u, l < +inf, u > -inf, no NaN; ";
  if (f & V_RBOUNDS) s += "row bounds must satisfy lc <= uc, lc < +inf, uc > -inf, no NaN; ";
  if (f & V_DIAG) s += "D must be finite and non-negative; ";
  return s;
}

template <typename T>
cudaError_t dmalloc(T** p, size_t n) {
  *p = nullptr;
  return cudaMalloc(p, sizeof(T) * std::max<size_t>(n, 1));
}

cudaError_t copy_in(void* dst, const void* src, size_t bytes, mpax_mem_kind kind,
                    cudaStream_t s) {
  if (bytes == 0) return cudaSuccess;
  return cudaMemcpyAsync(dst, src, bytes,
                         kind == MPAX_MEM_HOST ? cudaMemcpyHostToDevice
                                               : cudaMemcpyDeviceToDevice,
                         s);
}

cudaError_t copy_out(void* dst, const void* src, size_t bytes, mpax_mem_kind kind,
                     cudaStream_t s) {
  if (bytes == 0) return cudaSuccess;
  return cudaMemcpyAsync(dst, src, bytes,
                         kind == MPAX_MEM_HOST ? cudaMemcpyDeviceToHost
                                               : cudaMemcpyDeviceToDevice,
                         s);
}

void free_csr(Csr& c) {
  if (c.rp) cudaFree(c.rp);
  if (c.col) cudaFree(c.col);
  c = Csr();
}

}  // namespace

struct mpax_problem {
  ProblemData P;
  cudaStream_t user = nullptr;
  EngineBase* eng[2] = {nullptr, nullptr};
  int cur = -1;  // precision of the prepared engine
  bool prepared = false;
  bool solved = false;
  mpax_options last_opts;
  mpax_stats stats;
  double* dx = nullptr;  // n FP64 device scratch (host-kind inputs/outputs)
  double* dy = nullptr;  // m
  double* dxa = nullptr;
  double* dya = nullptr;
  double* d6 = nullptr;  // 8 doubles
  cudaEvent_t ev = nullptr;
  double* dxp = nullptr;  // polished x (n), allocated on the first polishing
  double* dyp = nullptr;  // polished y (m)
  bool polished = false;  // the last solve returned the polished pair
};

namespace {

cudaError_t order_after_user(mpax_problem* pb) {
  cudaError_t e = cudaEventRecord(pb->ev, pb->user);
  if (e) return e;
  return cudaStreamWaitEvent(pb->P.s, pb->ev, 0);
}

cudaError_t order_user_after(mpax_problem* pb) {
  cudaError_t e = cudaEventRecord(pb->ev, pb->P.s);
  if (e) return e;
  return cudaStreamWaitEvent(pb->user, pb->ev, 0);
}

void destroy_problem(mpax_problem* pb) {
  if (!pb) return;
  ProblemData& P = pb->P;
  if (P.s) cudaStreamSynchronize(P.s);
  for (auto& e : pb->eng) delete e;
  free_csr(P.A);
  free_csr(P.At);
  free_csr(P.F);
  free_csr(P.Ft);
  free_csr(P.Q);
  free_schedule(P.schedA);
  free_schedule(P.schedAt);
  free_schedule(P.schedF);
  free_schedule(P.schedFt);
  free_schedule(P.schedQ);
  if (P.qval) cudaFree(P.qval);
  if (P.qval_s) cudaFree(P.qval_s);
  double* ds[] = {P.val, P.c,     P.lc,    P.uc,    P.l,   P.u,      P.D,      P.fval,
                  P.Dr,  P.Dc,    P.invDr, P.invDc, P.val_s, P.fval_s, P.D_s,  P.rowred,
                  P.colred, P.rowred2, P.colred2, P.red, P.red_out, P.qdiag, pb->dx, pb->dy,
                  pb->dxa, pb->dya, pb->d6, pb->dxp, pb->dyp};
  for (double* d : ds)
    if (d) cudaFree(d);
  int* is[] = {P.permT, P.permF, P.tmp_rows, P.tmp_scan};
  for (int* d : is)
    if (d) cudaFree(d);
  if (pb->ev) cudaEventDestroy(pb->ev);
  if (P.s) cudaStreamDestroy(P.s);
  delete pb;
}

bool bad_ptr(const void* p, long long count) { return count > 0 && p == nullptr; }

mpax_status create_common(int32_t m, int32_t n, int64_t nnz, const int64_t* row_ptr,
                          const int32_t* col_idx, const double* val, const double* c,
                          const double* lc, const double* uc, const double* l,
                          const double* u, const double* D, int32_t r, int64_t f_nnz,
                          const int64_t* f_row_ptr, const int32_t* f_col_idx,
                          const double* f_val, bool is_qp, mpax_mem_kind kind,
                          void* cuda_stream, mpax_problem** out, int64_t q_nnz = 0,
                          const int64_t* q_row_ptr = nullptr, const int32_t* q_col_idx = nullptr,
                          const double* q_val = nullptr) {
  if (!out) return fail(MPAX_ERR_INVALID_ARGUMENT, "out must not be NULL");
  *out = nullptr;
  const bool q_general = q_row_ptr != nullptr;
  if (m < 0 || n < 0 || nnz < 0 || r < 0 || f_nnz < 0 || q_nnz < 0)
    return fail(MPAX_ERR_INVALID_ARGUMENT, "sizes must be non-negative");
  if (nnz >= (1LL << 31) || f_nnz >= (1LL << 31) || q_nnz >= (1LL << 31))
    return fail(MPAX_ERR_UNSUPPORTED, "nnz must be < 2^31");
  if (q_general && (bad_ptr(q_col_idx, q_nnz) || bad_ptr(q_val, q_nnz)))
    return fail(MPAX_ERR_INVALID_ARGUMENT, "a required Q array pointer is NULL");
  if (kind != MPAX_MEM_HOST && kind != MPAX_MEM_DEVICE)
    return fail(MPAX_ERR_INVALID_ARGUMENT, "kind must be MPAX_MEM_HOST or MPAX_MEM_DEVICE");
  if (bad_ptr(row_ptr, 1) || bad_ptr(col_idx, nnz) || bad_ptr(val, nnz) || bad_ptr(c, n) ||
      bad_ptr(l, n) || bad_ptr(u, n) || bad_ptr(lc, m) || bad_ptr(uc, m))
    return fail(MPAX_ERR_INVALID_ARGUMENT, "a required array pointer is NULL");
  if (is_qp && !q_general &&
      (bad_ptr(D, n) || bad_ptr(f_row_ptr, 1) || bad_ptr(f_col_idx, f_nnz) ||
       bad_ptr(f_val, f_nnz)))
    return fail(MPAX_ERR_INVALID_ARGUMENT, "a required QP array pointer is NULL");
  if (is_qp && r == 0 && f_nnz > 0)
    return fail(MPAX_ERR_INVALID_ARGUMENT, "F has entries but r = 0");

  mpax_problem* pb = new mpax_problem();
  ProblemData& P = pb->P;
  P.m = m;
  P.n = n;
  P.nnz = (int)nnz;
  P.is_qp = is_qp;
  P.r = r;
  P.f_nnz = (int)f_nnz;
  P.q_general = q_general;
  pb->user = (cudaStream_t)cuda_stream;
  mpax_options_default(&pb->last_opts);
  std::memset(&pb->stats, 0, sizeof(pb->stats));
  cudaError_t e = cudaStreamCreateWithFlags(&P.s, cudaStreamNonBlocking);
  if (!e) e = cudaEventCreateWithFlags(&pb->ev, cudaEventDisableTiming);
  if (!e) e = order_after_user(pb);
  const int big = std::max(std::max(m, n), r) + 2;
  if (!e) e = dmalloc(&P.A.rp, m + 1);
  if (!e) e = dmalloc(&P.A.col, nnz + kPad);
  if (!e) e = dmalloc(&P.val, nnz);
  if (!e) e = dmalloc(&P.c, n);
  if (!e) e = dmalloc(&P.l, n);
  if (!e) e = dmalloc(&P.u, n);
  if (!e) e = dmalloc(&P.lc, m);
  if (!e) e = dmalloc(&P.uc, m);
  if (!e) e = dmalloc(&P.Dr, m);
  if (!e) e = dmalloc(&P.Dc, n);
  if (!e) e = dmalloc(&P.invDr, m);
  if (!e) e = dmalloc(&P.invDc, n);
  if (!e) e = dmalloc(&P.val_s, nnz);
  if (!e) e = dmalloc(&P.rowred, m);
  if (!e) e = dmalloc(&P.colred, n);
  if (!e) e = dmalloc(&P.rowred2, m);
  if (!e) e = dmalloc(&P.colred2, n);
  // (also the 32-bin row-length histogram of the kernel autotuner)
  if (!e) e = dmalloc(&P.tmp_rows, std::max<size_t>(big, 64));
  if (!e) e = dmalloc(&P.tmp_scan, scan_tmp_ints(big));
  if (!e) e = dmalloc(&P.red, kRedBlocks * 8);
  if (!e) e = dmalloc(&P.red_out, 16);
  if (!e) e = dmalloc(&P.At.rp, n + 1);
  if (!e) e = dmalloc(&P.At.col, nnz + kPad);
  if (!e) e = dmalloc(&P.permT, nnz);
  if (!e) e = dmalloc(&pb->dx, n);
  if (!e) e = dmalloc(&pb->dy, m);
  if (!e) e = dmalloc(&pb->dxa, n);
  if (!e) e = dmalloc(&pb->dya, m);
  if (!e) e = dmalloc(&pb->d6, 8);
  if (is_qp) {
    if (!e) e = dmalloc(&P.D, n);
    if (!e) e = dmalloc(&P.D_s, n);
    if (!e) e = dmalloc(&P.qdiag, n);
    if (!e) e = dmalloc(&P.F.rp, n + 1);
    if (!e) e = dmalloc(&P.F.col, f_nnz + kPad);
    if (!e) e = dmalloc(&P.fval, f_nnz);
    if (!e) e = dmalloc(&P.fval_s, f_nnz);
    if (!e) e = dmalloc(&P.Ft.rp, r + 1);
    if (!e) e = dmalloc(&P.Ft.col, f_nnz + kPad);
    if (!e) e = dmalloc(&P.permF, f_nnz);
  }
  if (q_general) {
    if (!e) e = dmalloc(&P.Q.rp, n + 1);
    if (!e) e = dmalloc(&P.Q.col, q_nnz + kPad);
    if (!e) e = dmalloc(&P.qval, q_nnz);
    if (!e) e = dmalloc(&P.qval_s, q_nnz);
  }
  P.Q.rows = n;
  P.Q.cols = n;
  P.Q.nnz = (int)q_nnz;
  P.A.rows = m;
  P.A.cols = n;
  P.A.nnz = (int)nnz;
  P.F.rows = n;
  P.F.cols = r;
  P.F.nnz = (int)f_nnz;
  long long* rp64 = nullptr;
  int* flags = nullptr;
  if (!e) e = dmalloc(&rp64, (size_t)std::max(m, n) + 1);
  if (!e) e = dmalloc(&flags, 1);
  if (!e) e = cudaMemsetAsync(flags, 0, sizeof(int), P.s);
  cudaStream_t s = P.s;
  if (!e) e = copy_in(rp64, row_ptr, sizeof(int64_t) * (m + 1), kind, s);
  if (!e)
    k_rowptr64_to_32<<<(m + 256) / 256, 256, 0, s>>>(rp64, P.A.rp, m, nnz, flags);
  if (!e) e = copy_in(P.A.col, col_idx, sizeof(int32_t) * nnz, kind, s);
  if (!e) e = copy_in(P.val, val, sizeof(double) * nnz, kind, s);
  if (!e) e = copy_in(P.c, c, sizeof(double) * n, kind, s);
  if (!e) e = copy_in(P.l, l, sizeof(double) * n, kind, s);
  if (!e) e = copy_in(P.u, u, sizeof(double) * n, kind, s);
  if (!e) e = copy_in(P.lc, lc, sizeof(double) * m, kind, s);
  if (!e) e = copy_in(P.uc, uc, sizeof(double) * m, kind, s);
  if (is_qp && !q_general) {
    if (!e) e = copy_in(P.D, D, sizeof(double) * n, kind, s);
    if (!e) e = cudaStreamSynchronize(s);  // rp64 reused below
    if (!e) e = copy_in(rp64, f_row_ptr, sizeof(int64_t) * (n + 1), kind, s);
    if (!e)
      k_rowptr64_to_32<<<(n + 256) / 256, 256, 0, s>>>(rp64, P.F.rp, n, f_nnz, flags);
    if (!e) e = copy_in(P.F.col, f_col_idx, sizeof(int32_t) * f_nnz, kind, s);
    if (!e) e = copy_in(P.fval, f_val, sizeof(double) * f_nnz, kind, s);
  }
  if (q_general) {
    // D = 0 and an empty F: the diagonal-plus-low-rank terms vanish
    if (!e) e = cudaMemsetAsync(P.D, 0, sizeof(double) * std::max(n, 1), s);
    if (!e) e = cudaMemsetAsync(P.F.rp, 0, sizeof(int) * (n + 1), s);
    if (!e) e = cudaStreamSynchronize(s);  // rp64 reused below
    if (!e) e = copy_in(rp64, q_row_ptr, sizeof(int64_t) * (n + 1), kind, s);
    if (!e)
      k_rowptr64_to_32<<<(n + 256) / 256, 256, 0, s>>>(rp64, P.Q.rp, n, q_nnz, flags);
    if (!e) e = copy_in(P.Q.col, q_col_idx, sizeof(int32_t) * q_nnz, kind, s);
    if (!e) e = copy_in(P.qval, q_val, sizeof(double) * q_nnz, kind, s);
  }
  if (!e && m > 0) k_check_csr<<<(m + 255) / 256, 256, 0, s>>>(P.A.rp, P.A.col, P.val, m, n, flags);
  if (!e && is_qp && n > 0)
    k_check_csr<<<(n + 255) / 256, 256, 0, s>>>(P.F.rp, P.F.col, P.fval, n, r, flags);
  if (!e && q_general && n > 0)
    k_check_csr<<<(n + 255) / 256, 256, 0, s>>>(P.Q.rp, P.Q.col, P.qval, n, n, flags);
  if (!e)
    k_check_vecs<<<std::max(1, std::min(4096, (std::max(m, n) + 255) / 256)), 256, 0, s>>>(
        P.c, P.l, P.u, n, P.lc, P.uc, m, is_qp ? P.D : nullptr, flags);
  int hflags = 0;
  if (!e) e = cudaGetLastError();
  if (!e) e = cudaMemcpyAsync(&hflags, flags, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (!e) e = cudaStreamSynchronize(s);
  if (rp64) cudaFree(rp64);
  if (flags) cudaFree(flags);
  if (e) {
    destroy_problem(pb);
    return cuda_fail(e, "create");
  }
  if (hflags) {
    destroy_problem(pb);
    return fail(MPAX_ERR_INVALID_ARGUMENT, "invalid problem data: " + flags_message(hflags));
  }
  *out = pb;
  return MPAX_OK;
}

mpax_status check_options(const mpax_options* o) {
  if (!o) return fail(MPAX_ERR_INVALID_ARGUMENT, "opts must not be NULL");
  if (o->check_every < 1 || o->check_every > kMaxCheckEvery)
    return fail(MPAX_ERR_INVALID_ARGUMENT, "check_every must be in [1, 1024]");
  if (o->precision != MPAX_PREC_FP64 && o->precision != MPAX_PREC_MIXED)
    return fail(MPAX_ERR_INVALID_ARGUMENT, "precision must be MPAX_PREC_FP64 or MPAX_PREC_MIXED");
  if (!(o->eps_abs >= 0) || !(o->eps_rel >= 0))
    return fail(MPAX_ERR_INVALID_ARGUMENT, "tolerances must be non-negative");
  if (o->iteration_limit < 1)
    return fail(MPAX_ERR_INVALID_ARGUMENT, "iteration_limit must be >= 1");
  if (!(o->reflection_gamma >= 0.0 && o->reflection_gamma <= 1.0))
    return fail(MPAX_ERR_INVALID_ARGUMENT, "reflection_gamma must be in [0, 1]");
  if (o->ruiz_iters < 0) return fail(MPAX_ERR_INVALID_ARGUMENT, "ruiz_iters must be >= 0");
  if (!(o->step_safety > 0.0 && o->step_safety < 1.0))
    return fail(MPAX_ERR_INVALID_ARGUMENT, "step_safety must be in (0, 1)");
  if (o->power_max_iter < 0) return fail(MPAX_ERR_INVALID_ARGUMENT, "power_max_iter must be >= 0");
  if (o->power_max_iter == 0 && !o->pock_chambolle)
    return fail(MPAX_ERR_INVALID_ARGUMENT,
                "power_max_iter = 0 takes the bound ||A~||_2 <= 1 of the Pock-Chambolle round");
  if (o->feasibility_polishing && !(o->eps_feas_polish > 0.0))
    return fail(MPAX_ERR_INVALID_ARGUMENT, "eps_feas_polish must be > 0");
  if (!(o->time_limit >= 0)) return fail(MPAX_ERR_INVALID_ARGUMENT, "time_limit must be >= 0");
  if (o->fp64_continuation && o->stall_checks < 1)
    return fail(MPAX_ERR_INVALID_ARGUMENT, "stall_checks must be >= 1");
  if (o->spmv_kernel < -1 || o->spmv_kernel >= kSpmvKinds)
    return fail(MPAX_ERR_INVALID_ARGUMENT, "spmv_kernel must be -1, 0, 1 or 2");
  if (o->batch_stage != 0 && o->batch_stage != 1)
    return fail(MPAX_ERR_INVALID_ARGUMENT, "batch_stage must be 0 or 1");
  if (o->record_tape && o->precision != MPAX_PREC_FP64)
    return fail(MPAX_ERR_UNSUPPORTED, "record_tape needs precision FP64");
  return MPAX_OK;
}

mpax_status do_prepare(mpax_problem* pb, const mpax_options* o, long long* launches) {
  ProblemData& P = pb->P;
  cudaStream_t s = P.s;
  if (P.is_qp && o->power_max_iter == 0)
    return fail(MPAX_ERR_INVALID_ARGUMENT, "power_max_iter = 0 is for LPs (||Q~|| has no bound)");
  // structure: transpose(s) and work-item schedules
  TRY_CUDA(transpose_csr(P.A, P.At, P.permT, P.tmp_rows, P.tmp_scan, s), "transpose");
  *launches += 6;
  if (P.is_qp) {
    TRY_CUDA(transpose_csr(P.F, P.Ft, P.permF, P.tmp_rows, P.tmp_scan, s), "transpose F");
    *launches += 6;
  }
  P.transposed = true;
  TRY_CUDA(build_schedule(P.A, P.schedA, s, P.tmp_rows, P.tmp_scan), "schedule A");
  TRY_CUDA(build_schedule(P.At, P.schedAt, s, P.tmp_rows, P.tmp_scan), "schedule A^T");
  *launches += 12;
  if (P.is_qp) {
    TRY_CUDA(build_schedule(P.F, P.schedF, s, P.tmp_rows, P.tmp_scan), "schedule F");
    TRY_CUDA(build_schedule(P.Ft, P.schedFt, s, P.tmp_rows, P.tmp_scan), "schedule F^T");
    *launches += 12;
  }
  if (P.q_general) {
    TRY_CUDA(build_schedule(P.Q, P.schedQ, s, P.tmp_rows, P.tmp_scan), "schedule Q");
    *launches += 6;
  }
  P.scheduled = true;
  TRY_CUDA(compute_scaling(P, o->ruiz_iters, o->pock_chambolle != 0), "scaling");
  *launches += 5 * o->ruiz_iters + 8;
  TRY_CUDA(bound_and_cost_norms(P), "norms");
  *launches += 2;
  const int prec = o->precision;
  if (!pb->eng[prec]) {
    cudaError_t e;
    pb->eng[prec] = make_engine(&P, prec, &e);
    if (!pb->eng[prec]) return cuda_fail(e, "engine allocation");
  }
  EngineBase* eng = pb->eng[prec];
  TRY_CUDA(eng->load_values(), "load values");
  *launches += 9;
  TRY_CUDA(eng->tune(*o, launches), "kernel tuning");
  TRY_CUDA(eng->init_state(*o, launches), "init state");
  pb->cur = prec;
  pb->prepared = true;
  pb->last_opts = *o;
  return MPAX_OK;
}

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

}  // namespace

namespace mpax {
ProblemData* problem_data(mpax_problem* p) { return &p->P; }
void problem_order_after_user(mpax_problem* p) { order_after_user(p); }
void problem_order_user_after(mpax_problem* p) { order_user_after(p); }
}  // namespace mpax

// ============================================================================
// exported functions
// ============================================================================

extern "C" {

const char* mpax_version(void) { return "mpax-gb300 0.1.0 (sm_103a)"; }

const char* mpax_last_error(void) { return g_err.c_str(); }

const char* mpax_status_string(mpax_status s) {
  switch (s) {
    case MPAX_OK: return "ok";
    case MPAX_ERR_INVALID_ARGUMENT: return "invalid argument";
    case MPAX_ERR_CUDA: return "CUDA error";
    case MPAX_ERR_OUT_OF_MEMORY: return "out of device memory";
    case MPAX_ERR_NOT_SOLVED: return "not solved";
    case MPAX_ERR_DEVICE_TIMEOUT: return "device timeout";
    case MPAX_ERR_NUMERICAL: return "numerical error";
    case MPAX_ERR_UNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

void mpax_options_default(mpax_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->verbose = 0;
  o->display_frequency = 10;
  o->warm_start = 0;
  o->feasibility_polishing = 0;
  o->eps_abs = 1e-4;
  o->eps_rel = 1e-4;
  o->eps_primal_infeasible = 1e-8;
  o->eps_dual_infeasible = 1e-8;
  o->eps_feas_polish = 1e-6;
  o->iteration_limit = INT64_MAX;
  o->time_limit = INFINITY;
  o->precision = MPAX_PREC_FP64;
  o->check_every = 64;
  o->ruiz_iters = 10;
  o->pock_chambolle = 1;
  o->reflection_gamma = 1.0;
  o->restart_sufficient = 0.2;
  o->restart_necessary = 0.8;
  o->restart_artificial = 0.36;
  o->primal_weight_smoothing = 0.5;
  o->step_safety = 0.998;
  o->power_max_iter = 1000;
  o->power_tol = 1e-4;
  o->use_graphs = 1;
  o->profile_kernels = 0;
  o->fp64_continuation = 1;
  o->stall_checks = 8;
  o->record_tape = 0;
  o->spmv_kernel = -1;
  o->batch_stage = 1;
}

mpax_status mpax_lp_create(int32_t m, int32_t n, int64_t nnz, const int64_t* row_ptr,
                           const int32_t* col_idx, const double* val, const double* c,
                           const double* lc, const double* uc, const double* l,
                           const double* u, mpax_mem_kind kind, void* cuda_stream,
                           mpax_problem** out) {
  return create_common(m, n, nnz, row_ptr, col_idx, val, c, lc, uc, l, u, nullptr, 0, 0,
                       nullptr, nullptr, nullptr, false, kind, cuda_stream, out);
}

mpax_status mpax_qp_create_diag_lowrank(
    int32_t m, int32_t n, int64_t nnz, const int64_t* row_ptr, const int32_t* col_idx,
    const double* val, const double* c, const double* lc, const double* uc, const double* l,
    const double* u, const double* D, int32_t r, int64_t f_nnz, const int64_t* f_row_ptr,
    const int32_t* f_col_idx, const double* f_val, mpax_mem_kind kind, void* cuda_stream,
    mpax_problem** out) {
  return create_common(m, n, nnz, row_ptr, col_idx, val, c, lc, uc, l, u, D, r, f_nnz,
                       f_row_ptr, f_col_idx, f_val, true, kind, cuda_stream, out);
}

mpax_status mpax_lp_create_f32(int32_t m, int32_t n, int64_t nnz, const int64_t* row_ptr,
                               const int32_t* col_idx, const float* val, const float* c,
                               const float* lc, const float* uc, const float* l,
                               const float* u, mpax_mem_kind kind, void* cuda_stream,
                               mpax_problem** out) {
  if (m < 0 || n < 0 || nnz < 0) return fail(MPAX_ERR_INVALID_ARGUMENT, "sizes must be non-negative");
  if (kind != MPAX_MEM_HOST && kind != MPAX_MEM_DEVICE)
    return fail(MPAX_ERR_INVALID_ARGUMENT, "kind must be MPAX_MEM_HOST or MPAX_MEM_DEVICE");
  if (bad_ptr(val, nnz) || bad_ptr(c, n) || bad_ptr(l, n) || bad_ptr(u, n) || bad_ptr(lc, m) ||
      bad_ptr(uc, m))
    return fail(MPAX_ERR_INVALID_ARGUMENT, "a required array pointer is NULL");
  const float* src[6] = {val, c, lc, uc, l, u};
  const size_t len[6] = {(size_t)nnz, (size_t)n, (size_t)m, (size_t)m, (size_t)n, (size_t)n};
  if (kind == MPAX_MEM_HOST) {
    std::vector<double> w[6];
    for (int q = 0; q < 6; ++q) w[q].assign(src[q], src[q] + len[q]);
    return create_common(m, n, nnz, row_ptr, col_idx, w[0].data(), w[1].data(), w[2].data(),
                         w[3].data(), w[4].data(), w[5].data(), nullptr, 0, 0, nullptr, nullptr,
                         nullptr, false, kind, cuda_stream, out);
  }
  // device inputs: widen into temporaries on the caller's stream, then copy in
  double* buf = nullptr;
  const size_t tot = len[0] + len[1] + len[2] + len[3] + len[4] + len[5];
  TRY_CUDA(cudaMalloc(&buf, sizeof(double) * std::max<size_t>(tot, 1)), "f32 widening");
  double* dst[6];
  size_t off = 0;
  for (int q = 0; q < 6; ++q) {
    dst[q] = buf + off;
    off += len[q];
    if (len[q])
      k_widen<<<(int)std::min<size_t>(4096, (len[q] + 255) / 256), 256, 0,
                (cudaStream_t)cuda_stream>>>(src[q], dst[q], len[q]);
  }
  cudaError_t e = cudaGetLastError();
  mpax_status st = MPAX_ERR_CUDA;
  if (!e)
    st = create_common(m, n, nnz, row_ptr, col_idx, dst[0], dst[1], dst[2], dst[3], dst[4],
                       dst[5], nullptr, 0, 0, nullptr, nullptr, nullptr, false, kind,
                       cuda_stream, out);
  cudaStreamSynchronize((cudaStream_t)cuda_stream);
  cudaFree(buf);
  if (e) return cuda_fail(e, "f32 widening");
  return st;
}

mpax_status mpax_qp_create(int32_t m, int32_t n, int64_t nnz, const int64_t* row_ptr,
                           const int32_t* col_idx, const double* val, const double* c,
                           const double* lc, const double* uc, const double* l,
                           const double* u, int64_t q_nnz, const int64_t* q_row_ptr,
                           const int32_t* q_col_idx, const double* q_val, mpax_mem_kind kind,
                           void* cuda_stream, mpax_problem** out) {
  if (!q_row_ptr) return fail(MPAX_ERR_INVALID_ARGUMENT, "q_row_ptr must not be NULL");
  return create_common(m, n, nnz, row_ptr, col_idx, val, c, lc, uc, l, u, nullptr, 1, 0,
                       nullptr, nullptr, nullptr, true, kind, cuda_stream, out, q_nnz,
                       q_row_ptr, q_col_idx, q_val);
}

mpax_status mpax_prepare(mpax_problem* pb, const mpax_options* opts) {
  if (!pb) return fail(MPAX_ERR_INVALID_ARGUMENT, "problem is NULL");
  mpax_status st = check_options(opts);
  if (st) return st;
  TRY_CUDA(order_after_user(pb), "stream order");
  long long launches = 0;
  st = do_prepare(pb, opts, &launches);
  if (st) return st;
  TRY_CUDA(cudaStreamSynchronize(pb->P.s), "prepare");
  TRY_CUDA(order_user_after(pb), "stream order");
  return MPAX_OK;
}

mpax_status mpax_solve(mpax_problem* pb, const mpax_options* opts, const double* x0,
                       const double* y0, mpax_mem_kind kind) {
  if (!pb) return fail(MPAX_ERR_INVALID_ARGUMENT, "problem is NULL");
  mpax_status st = check_options(opts);
  if (st) return st;
  if (kind != MPAX_MEM_HOST && kind != MPAX_MEM_DEVICE)
    return fail(MPAX_ERR_INVALID_ARGUMENT, "bad memory kind");
  ProblemData& P = pb->P;
  if (opts->record_tape && !P.is_qp)
    return fail(MPAX_ERR_INVALID_ARGUMENT, "record_tape is for QPs");
  const double t0 = now_s();
  TRY_CUDA(order_after_user(pb), "stream order");
  long long launches = 0;
  st = do_prepare(pb, opts, &launches);
  if (st) return st;
  TRY_CUDA(cudaStreamSynchronize(P.s), "prepare");
  const double t1 = now_s();
  const double* x0d = nullptr;
  const double* y0d = nullptr;
  if (x0) {
    if (kind == MPAX_MEM_HOST) {
      TRY_CUDA(copy_in(pb->dx, x0, sizeof(double) * P.n, kind, P.s), "copy x0");
      x0d = pb->dx;
    } else {
      x0d = x0;
    }
  }
  if (y0) {
    if (kind == MPAX_MEM_HOST) {
      TRY_CUDA(copy_in(pb->dy, y0, sizeof(double) * P.m, kind, P.s), "copy y0");
      y0d = pb->dy;
    } else {
      y0d = y0;
    }
  }
  EngineBase* eng = pb->eng[pb->cur];
  TRY_CUDA(eng->init_iterate(x0d, y0d), "init iterate");
  launches += 15;
  RunInfo info;
  cudaError_t e = eng->run(*opts, &info);
  if (e) return cuda_fail(e, "solve");
  long long fp64_iters = 0;
  if (info.termination == kTermStalled) {
    // FP64 continuation from the FP32 point (unscaled), with the remaining budget
    TRY_CUDA(eng->get_solution(pb->dxa, pb->dya), "fp32 point");
    mpax_options o64 = *opts;
    o64.precision = MPAX_PREC_FP64;
    o64.iteration_limit = std::max<long long>(1, opts->iteration_limit - info.iterations);
    st = do_prepare(pb, &o64, &launches);
    if (st) return st;
    eng = pb->eng[pb->cur];
    TRY_CUDA(eng->init_iterate(pb->dxa, pb->dya), "fp64 start");
    RunInfo info64;
    e = eng->run(o64, &info64);
    if (e) return cuda_fail(e, "fp64 continuation");
    fp64_iters = info64.iterations;
    info64.iterations += info.iterations;
    info64.restarts += info.restarts;
    info64.checks += info.checks;
    info64.launches += info.launches;
    for (int i = 0; i < 5; ++i) {
      info64.profile_ms[i] += info.profile_ms[i];
      info64.profile_launches[i] += info.profile_launches[i];
    }
    info = info64;
  }
  pb->polished = false;
  long long polish_iters = 0;
  if (opts->feasibility_polishing && !P.is_qp && info.termination == MPAX_TERM_OPTIMAL) {
    // Feasibility polishing (Sec. 3.3), in FP64: the zero-objective problem from
    // (x^, 0) until the primal residual meets eps_feas_polish, then the problem
    // with every finite bound at zero from (0, y^) until the dual residual does.
    if (!pb->dxp) TRY_CUDA(cudaMalloc(&pb->dxp, sizeof(double) * std::max(P.n, 1)), "alloc");
    if (!pb->dyp) TRY_CUDA(cudaMalloc(&pb->dyp, sizeof(double) * std::max(P.m, 1)), "alloc");
    TRY_CUDA(eng->get_solution(pb->dxa, pb->dya), "point to polish");
    mpax_options op = *opts;
    op.precision = MPAX_PREC_FP64;
    op.eps_abs = op.eps_rel = opts->eps_feas_polish;
    op.eps_primal_infeasible = op.eps_dual_infeasible = 0.0;
    op.fp64_continuation = 0;
    st = do_prepare(pb, &op, &launches);
    if (st) return st;
    eng = pb->eng[pb->cur];
    for (int phase = 1; phase <= 2; ++phase) {
      if (phase == 2) TRY_CUDA(eng->load_values(), "reload");
      TRY_CUDA(eng->set_feasibility(phase), "polishing data");
      TRY_CUDA(eng->init_state(op, &launches), "polishing state");
      TRY_CUDA(eng->init_iterate(phase == 1 ? pb->dxa : nullptr, phase == 2 ? pb->dya : nullptr),
               "polishing start");
      RunInfo ip;
      e = eng->run(op, &ip);
      if (e) return cuda_fail(e, "feasibility polishing");
      polish_iters += ip.iterations;
      info.launches += ip.launches;
      TRY_CUDA(eng->get_solution(phase == 1 ? pb->dxp : pb->dx, phase == 1 ? pb->dy : pb->dyp),
               "polished point");
    }
    TRY_CUDA(eng->load_values(), "restore");
    TRY_CUDA(eng->kkt_at(pb->dxp, pb->dyp, pb->d6), "polished kkt");
    pb->polished = true;
  }
  DevState h;
  TRY_CUDA(eng->read_state(&h), "read state");
  TRY_CUDA(order_user_after(pb), "stream order");
  mpax_stats& S = pb->stats;
  std::memset(&S, 0, sizeof(S));
  S.termination = info.termination;
  S.precision = opts->precision;
  S.iterations = info.iterations;
  S.restarts = info.restarts;
  S.kkt_checks = info.checks;
  S.primal_obj = h.pobj;
  S.dual_obj = h.dobj;
  S.gap = h.gap;
  S.primal_res = h.primal_res;
  S.dual_res = h.dual_res;
  S.rel_kkt = h.rel_kkt;
  S.omega = h.omega;
  S.eta = h.eta;
  S.norm_A = h.norm_A;
  S.norm_Q = h.norm_Q;
  S.prepare_seconds = t1 - t0;
  S.solve_seconds = now_s() - t0;
  S.kernel_launches = launches + info.launches;
  for (int i = 0; i < 4; ++i) {
    S.profile_ms[i] = info.profile_ms[i];
    S.profile_launches[i] = info.profile_launches[i];
  }
  S.profile_ms_aux = info.profile_ms[4];
  S.profile_launches_aux = info.profile_launches[4];
  S.fp64_iterations = fp64_iters;
  S.polish_iterations = polish_iters;
  eng->tune_info(S.spmv_kernel, S.spmv_tune_us);
  if (pb->polished) {
    double k6[6];
    TRY_CUDA(cudaMemcpyAsync(k6, pb->d6, sizeof(k6), cudaMemcpyDeviceToHost, P.s), "kkt");
    TRY_CUDA(cudaStreamSynchronize(P.s), "kkt");
    S.primal_res = k6[0];
    S.dual_res = k6[1];
    S.primal_obj = k6[2];
    S.dual_obj = k6[3];
    S.gap = k6[4];
    S.rel_kkt = k6[5];
  }
  pb->solved = true;
  pb->last_opts = *opts;
  if (info.termination == MPAX_TERM_NUMERICAL_ERROR)
    return fail(MPAX_ERR_NUMERICAL, "NaN or Inf appeared in the iteration");
  return MPAX_OK;
}

mpax_status mpax_get_solution(const mpax_problem* cpb, double* x, double* y,
                              mpax_mem_kind kind) {
  mpax_problem* pb = const_cast<mpax_problem*>(cpb);
  if (!pb) return fail(MPAX_ERR_INVALID_ARGUMENT, "problem is NULL");
  if (!pb->solved) return fail(MPAX_ERR_NOT_SOLVED, "call mpax_solve first");
  const ProblemData& P = pb->P;
  EngineBase* eng = pb->eng[pb->cur];
  const double* sx = pb->dx;
  const double* sy = pb->dy;
  if (pb->polished) {
    sx = pb->dxp;
    sy = pb->dyp;
  } else {
    TRY_CUDA(eng->get_solution(pb->dx, pb->dy), "get solution");
  }
  if (x) TRY_CUDA(copy_out(x, sx, sizeof(double) * P.n, kind, P.s), "copy x");
  if (y) TRY_CUDA(copy_out(y, sy, sizeof(double) * P.m, kind, P.s), "copy y");
  TRY_CUDA(cudaStreamSynchronize(P.s), "get solution");
  return MPAX_OK;
}

mpax_status mpax_qp_unrolled_grad(mpax_problem* pb, const double* gx, const double* gy,
                                  double* dc, double* dlc, double* duc, double* dl,
                                  double* du, double* dD, mpax_mem_kind kind) {
  if (!pb || !gx) return fail(MPAX_ERR_INVALID_ARGUMENT, "NULL argument");
  if (kind != MPAX_MEM_HOST && kind != MPAX_MEM_DEVICE)
    return fail(MPAX_ERR_INVALID_ARGUMENT, "bad memory kind");
  ProblemData& P = pb->P;
  if (!P.is_qp) return fail(MPAX_ERR_INVALID_ARGUMENT, "mpax_qp_unrolled_grad needs a QP");
  if (!pb->solved || !pb->last_opts.record_tape || pb->cur != MPAX_PREC_FP64)
    return fail(MPAX_ERR_NOT_SOLVED, "solve with record_tape = 1 (FP64) first");
  const int n = P.n, m = P.m;
  cudaStream_t s = P.s;
  TRY_CUDA(order_after_user(pb), "stream order");
  // device buffers: the loss gradients in, the six gradients out
  double* buf = nullptr;
  const size_t N = (size_t)n, M = (size_t)m;
  TRY_CUDA(cudaMalloc(&buf, sizeof(double) * (6 * N + 4 * M + 8)), "unrolled buffers");
  double* dgx = buf;
  double* dgy = dgx + N;
  double* ogc = dgy + M;
  double* ogl = ogc + N;
  double* ogu = ogl + N;
  double* ogD = ogu + N;
  double* oglc = ogD + N;
  double* oguc = oglc + M;
  const cudaMemcpyKind kin =
      kind == MPAX_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  const cudaMemcpyKind kout =
      kind == MPAX_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  cudaError_t e = cudaMemcpyAsync(dgx, gx, sizeof(double) * N, kin, s);
  if (!e && gy && m) e = cudaMemcpyAsync(dgy, gy, sizeof(double) * M, kin, s);
  long long launches = 0;
  if (!e)
    e = pb->eng[pb->cur]->unrolled_backward(dgx, gy ? dgy : nullptr, ogc, oglc, oguc, ogl, ogu,
                                            ogD, pb->last_opts.use_graphs != 0, &launches);
  if (e == cudaErrorNotReady) {
    cudaFree(buf);
    cudaGetLastError();
    return fail(MPAX_ERR_NOT_SOLVED, "no tape: solve with record_tape = 1 (FP64) first");
  }
  struct {
    double* dst;
    const double* src;
    size_t k;
  } outs[] = {{dc, ogc, N}, {dl, ogl, N}, {du, ogu, N}, {dD, ogD, N}, {dlc, oglc, M}, {duc, oguc, M}};
  for (auto& o : outs)
    if (!e && o.dst && o.k) e = cudaMemcpyAsync(o.dst, o.src, sizeof(double) * o.k, kout, s);
  if (!e) e = cudaStreamSynchronize(s);
  cudaFree(buf);
  if (e) return cuda_fail(e, "unrolled gradient");
  TRY_CUDA(order_user_after(pb), "stream order");
  pb->stats.backward_launches = launches;
  return MPAX_OK;
}

mpax_status mpax_get_stats(const mpax_problem* pb, mpax_stats* stats) {
  if (!pb || !stats) return fail(MPAX_ERR_INVALID_ARGUMENT, "NULL argument");
  *stats = pb->stats;
  if (!pb->solved) return fail(MPAX_ERR_NOT_SOLVED, "call mpax_solve first");
  return MPAX_OK;
}

mpax_status mpax_get_restart_history(const mpax_problem* cpb, int32_t cap, int64_t* iters,
                                     double* omega, int32_t* count) {
  mpax_problem* pb = const_cast<mpax_problem*>(cpb);
  if (!pb || !count || cap < 0) return fail(MPAX_ERR_INVALID_ARGUMENT, "bad argument");
  if (!pb->solved) return fail(MPAX_ERR_NOT_SOLVED, "call mpax_solve first");
  DevState h;
  TRY_CUDA(pb->eng[pb->cur]->read_state(&h), "read state");
  *count = h.rs_count;
  const int k = std::min(std::min(h.rs_count, cap), kRestartLog);
  for (int i = 0; i < k; ++i) {
    if (iters) iters[i] = h.rs_iter[i];
    if (omega) omega[i] = h.rs_omega[i];
  }
  return MPAX_OK;
}

void mpax_destroy(mpax_problem* pb) { destroy_problem(pb); }

mpax_status mpax_get_scaling(const mpax_problem* cpb, double* Dr, double* Dc, double* info,
                             mpax_mem_kind kind) {
  mpax_problem* pb = const_cast<mpax_problem*>(cpb);
  if (!pb) return fail(MPAX_ERR_INVALID_ARGUMENT, "problem is NULL");
  if (!pb->prepared) return fail(MPAX_ERR_NOT_SOLVED, "call mpax_prepare first");
  const ProblemData& P = pb->P;
  if (Dr) TRY_CUDA(copy_out(Dr, P.Dr, sizeof(double) * P.m, kind, P.s), "copy Dr");
  if (Dc) TRY_CUDA(copy_out(Dc, P.Dc, sizeof(double) * P.n, kind, P.s), "copy Dc");
  if (info) {
    DevState h;
    TRY_CUDA(pb->eng[pb->cur]->read_state(&h), "read state");
    const double v[4] = {h.norm_A, h.norm_Q, h.eta, h.omega};
    if (kind == MPAX_MEM_HOST) std::memcpy(info, v, sizeof(v));
    else TRY_CUDA(cudaMemcpyAsync(info, v, sizeof(v), cudaMemcpyHostToDevice, P.s), "copy info");
  }
  TRY_CUDA(cudaStreamSynchronize(P.s), "get scaling");
  return MPAX_OK;
}

mpax_status mpax_get_transpose(const mpax_problem* cpb, int64_t* rowptr_t, int32_t* col_t,
                               double* val_t, mpax_mem_kind kind) {
  mpax_problem* pb = const_cast<mpax_problem*>(cpb);
  if (!pb) return fail(MPAX_ERR_INVALID_ARGUMENT, "problem is NULL");
  if (!pb->P.transposed) return fail(MPAX_ERR_NOT_SOLVED, "call mpax_prepare first");
  const ProblemData& P = pb->P;
  cudaStream_t s = P.s;
  double* v = nullptr;
  cudaError_t e = dmalloc(&v, P.nnz);
  if (!e && P.nnz > 0) e = gather_cast<double>(P.val, P.permT, v, P.nnz, s);
  if (!e) {
    // widen the row pointers on the host side of the copy
    std::vector<int> h(P.n + 1);
    e = cudaMemcpyAsync(h.data(), P.At.rp, sizeof(int) * (P.n + 1), cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaStreamSynchronize(s);
    std::vector<long long> h64(h.begin(), h.end());
    if (!e && rowptr_t) {
      if (kind == MPAX_MEM_HOST) std::memcpy(rowptr_t, h64.data(), sizeof(long long) * (P.n + 1));
      else e = cudaMemcpyAsync(rowptr_t, h64.data(), sizeof(long long) * (P.n + 1), cudaMemcpyHostToDevice, s);
    }
  }
  if (!e && col_t) e = copy_out(col_t, P.At.col, sizeof(int) * P.nnz, kind, s);
  if (!e && val_t) e = copy_out(val_t, v, sizeof(double) * P.nnz, kind, s);
  if (!e) e = cudaStreamSynchronize(s);
  if (v) cudaFree(v);
  if (e) return cuda_fail(e, "get transpose");
  return MPAX_OK;
}

mpax_status mpax_set_iterate(mpax_problem* pb, const double* x, const double* y,
                             const double* x_aux, const double* y_aux, int64_t k, double tau,
                             double sigma, mpax_mem_kind kind) {
  if (!pb) return fail(MPAX_ERR_INVALID_ARGUMENT, "problem is NULL");
  if (!pb->prepared) return fail(MPAX_ERR_NOT_SOLVED, "call mpax_prepare first");
  if (k < 0 || !(tau > 0) || !(sigma > 0))
    return fail(MPAX_ERR_INVALID_ARGUMENT, "k >= 0, tau > 0 and sigma > 0 required");
  const ProblemData& P = pb->P;
  if (bad_ptr(x, P.n) || bad_ptr(x_aux, P.n) || bad_ptr(y, P.m) || bad_ptr(y_aux, P.m))
    return fail(MPAX_ERR_INVALID_ARGUMENT, "NULL iterate array");
  TRY_CUDA(copy_in(pb->dx, x, sizeof(double) * P.n, kind, P.s), "copy x");
  TRY_CUDA(copy_in(pb->dxa, x_aux, sizeof(double) * P.n, kind, P.s), "copy x_aux");
  TRY_CUDA(copy_in(pb->dy, y, sizeof(double) * P.m, kind, P.s), "copy y");
  TRY_CUDA(copy_in(pb->dya, y_aux, sizeof(double) * P.m, kind, P.s), "copy y_aux");
  TRY_CUDA(pb->eng[pb->cur]->set_iterate(pb->dx, pb->dy, pb->dxa, pb->dya, k, tau, sigma,
                                         pb->last_opts.reflection_gamma),
           "set iterate");
  TRY_CUDA(cudaStreamSynchronize(P.s), "set iterate");
  return MPAX_OK;
}

mpax_status mpax_iterate(mpax_problem* pb, int64_t iters) {
  if (!pb) return fail(MPAX_ERR_INVALID_ARGUMENT, "problem is NULL");
  if (!pb->prepared) return fail(MPAX_ERR_NOT_SOLVED, "call mpax_prepare first");
  if (iters < 0) return fail(MPAX_ERR_INVALID_ARGUMENT, "iters must be >= 0");
  TRY_CUDA(pb->eng[pb->cur]->iterate(iters), "iterate");
  TRY_CUDA(cudaStreamSynchronize(pb->P.s), "iterate");
  return MPAX_OK;
}

mpax_status mpax_get_iterate(const mpax_problem* cpb, double* x, double* y, double* x_hat,
                             double* y_hat, mpax_mem_kind kind) {
  mpax_problem* pb = const_cast<mpax_problem*>(cpb);
  if (!pb) return fail(MPAX_ERR_INVALID_ARGUMENT, "problem is NULL");
  if (!pb->prepared) return fail(MPAX_ERR_NOT_SOLVED, "call mpax_prepare first");
  const ProblemData& P = pb->P;
  TRY_CUDA(pb->eng[pb->cur]->get_iterate(pb->dx, pb->dy, pb->dxa, pb->dya), "get iterate");
  if (x) TRY_CUDA(copy_out(x, pb->dx, sizeof(double) * P.n, kind, P.s), "copy");
  if (y) TRY_CUDA(copy_out(y, pb->dy, sizeof(double) * P.m, kind, P.s), "copy");
  if (x_hat) TRY_CUDA(copy_out(x_hat, pb->dxa, sizeof(double) * P.n, kind, P.s), "copy");
  if (y_hat) TRY_CUDA(copy_out(y_hat, pb->dya, sizeof(double) * P.m, kind, P.s), "copy");
  TRY_CUDA(cudaStreamSynchronize(P.s), "get iterate");
  return MPAX_OK;
}

mpax_status mpax_kkt(mpax_problem* pb, const double* x, const double* y, mpax_mem_kind kind,
                     double* out) {
  if (!pb || !out) return fail(MPAX_ERR_INVALID_ARGUMENT, "NULL argument");
  if (!pb->prepared) return fail(MPAX_ERR_NOT_SOLVED, "call mpax_prepare first");
  const ProblemData& P = pb->P;
  if (bad_ptr(x, P.n) || bad_ptr(y, P.m)) return fail(MPAX_ERR_INVALID_ARGUMENT, "NULL x or y");
  TRY_CUDA(copy_in(pb->dx, x, sizeof(double) * P.n, kind, P.s), "copy x");
  TRY_CUDA(copy_in(pb->dy, y, sizeof(double) * P.m, kind, P.s), "copy y");
  TRY_CUDA(pb->eng[pb->cur]->kkt_at(pb->dx, pb->dy, pb->d6), "kkt");
  TRY_CUDA(copy_out(out, pb->d6, sizeof(double) * 6, kind, P.s), "copy kkt");
  TRY_CUDA(cudaStreamSynchronize(P.s), "kkt");
  return MPAX_OK;
}

}  // extern "C"
