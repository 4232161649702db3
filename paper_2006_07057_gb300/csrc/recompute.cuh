// Fused Sinkhorn pass that recomputes the features in registers (recompute variant).
#pragma once

#include "pass.cuh"

namespace lsf {

struct RecomputeArgs {
  const float* X;      // n x d points
  const float* shift;  // n row log-shifts
  int64_t n;
  const float* U;      // r x d anchors
  const float* c;      // r anchor log-constants
  int r, ldr, d;
  float two_over_eps;
  PassRhs rhs[2];
  float* part;
  float* gpart;
  double* rpart;
  unsigned* counter;
  int* status;
};

int launch_recompute_pass(int mode, int nrhs, RecomputeArgs a, cudaStream_t st);

}  // namespace lsf
