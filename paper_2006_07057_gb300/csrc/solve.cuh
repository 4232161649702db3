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

// Carve the workspace, zero the result records and the workspace counters.
int start_solve(void* workspace, size_t ws_bytes, int ldr, lsf_result* result, int nres,
                Workspace* ws, cudaStream_t st);

}  // namespace lsf
