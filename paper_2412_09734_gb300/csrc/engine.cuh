// Iteration engine interface (one instance per problem and precision).
#pragma once

#include "../../include/mpax.h"
#include "problem.cuh"

namespace mpax {

struct RunInfo {
  int termination = 0;
  long long iterations = 0, restarts = 0, checks = 0;
  long long launches = 0;
  // [0] primal, [1] dual, [2] KKT SpMV, [3] KKT SpMV^T, [4] QP product ahead of
  // the primal half-step
  double profile_ms[5] = {0, 0, 0, 0, 0};
  long long profile_launches[5] = {0, 0, 0, 0, 0};
  bool time_limit_hit = false;
};

class EngineBase {
 public:
  virtual ~EngineBase() = default;
  // Scaled matrix values and vectors in the iteration precision (after
  // compute_scaling and bound_and_cost_norms).
  virtual cudaError_t load_values() = 0;
  // Power iterations for ||A~|| (and ||Q~||), initial primal weight, step
  // sizes, counters; Halpern/averaging tables for the first block.
  virtual cudaError_t init_state(const mpax_options& o, long long* launches) = 0;
  // Kernel of the A and A^T schedules: o.spmv_kernel when >= 0, else the
  // faster of the kinds timed on this matrix (cached by matrix signature).
  // kind[0], kind[1]: A, A^T; us[2 * s + k]: average microseconds of kind k on
  // schedule s (0 where not timed in this call).
  virtual cudaError_t tune(const mpax_options& o, long long* launches) = 0;
  virtual void tune_info(int* kind, double* us) const = 0;
  // Starting point from unscaled FP64 device vectors (nullable = zeros).
  virtual cudaError_t init_iterate(const double* x0, const double* y0) = 0;
  virtual cudaError_t run(const mpax_options& o, RunInfo* info) = 0;
  // Lower-level access (scaled space, FP64 device vectors).
  virtual cudaError_t set_iterate(const double* x, const double* y, const double* xa,
                                  const double* ya, long long k, double tau, double sigma,
                                  double gamma) = 0;
  virtual cudaError_t iterate(long long iters) = 0;
  virtual cudaError_t get_iterate(double* x, double* y, double* xh, double* yh) = 0;
  virtual cudaError_t get_solution(double* x, double* y) = 0;  // unscaled
  virtual cudaError_t kkt_at(const double* x, const double* y, double* out6) = 0;  // unscaled
  virtual cudaError_t read_state(DevState* h) = 0;
  // Feasibility polishing (LP): 1 = objective set to zero, the run ends on the
  // primal residual; 2 = every finite bound set to zero, the run ends on the
  // dual residual; 0 = the problem as loaded.  Call init_state afterwards.
  virtual cudaError_t set_feasibility(int mode) = 0;
  // Unrolled differentiation (QP, FP64) of the last run, which had
  // record_tape set: gradients of gx . x + gy . y at its returned point along
  // its path.  Device vectors; gy nullable; gc, gl, gu, gD have n entries,
  // glc, guc m.  use_graphs: replay each block's launches as one CUDA graph.
  // cudaErrorNotReady: no tape.
  virtual cudaError_t unrolled_backward(const double* gx, const double* gy, double* gc,
                                        double* glc, double* guc, double* gl, double* gu,
                                        double* gD, bool use_graphs, long long* launches) = 0;
};

EngineBase* make_engine(ProblemData* P, int precision, cudaError_t* err);

}  // namespace mpax
