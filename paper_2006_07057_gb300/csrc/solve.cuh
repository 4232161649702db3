// Host helpers shared by the solvers: argument checks, workspace start, one pass.
#pragma once

#include "pass.cuh"

namespace lsf {

#define LSF_TRY(expr)              \
  do {                             \
    int _rc = (expr);              \
    if (_rc != LSF_OK) return _rc; \
  } while (0)

int check_theta(const lsf_theta* th);
int check_cloud(const lsf_cloud* c, int mode, const char* name);
int check_scalings(const lsf_scalings* s, const char* name);

// One fused pass (pmode, nrhs right-hand sides) over one cloud in solver mode `mode`.
int run_pass(int mode, const lsf_theta* th, const lsf_cloud* cl, int pmode, int nrhs,
             const PassRhs* rhs, const Workspace& ws, int* status, cudaStream_t st);

// Eq. (6) for up to three solves in one reduction launch: W_t = eps (w_x^T log u +
// w_y^T log v) from the shifted scalings of each term (is_log: they hold logs);
// *combined (if not NULL) = sum_t coef[t] W_t (coef NULL: all 1).
int launch_divergence(const lsf_theta* th, int nterms, const lsf_cloud* const* xs,
                      const lsf_cloud* const* ys, const lsf_scalings* const* s,
                      lsf_result* const* res, const double* coef, double* combined,
                      const Workspace& ws, cudaStream_t st, int is_log);

// Carve the workspace, zero the result records and the workspace counters.
int start_solve(void* workspace, size_t ws_bytes, int ldr, lsf_result* result, int nres,
                Workspace* ws, cudaStream_t st);

}  // namespace lsf
