// Cluster-persistent Sinkhorn solve for problems whose features stay in L2.
#pragma once

#include "common.cuh"

namespace lsf {

// One W(a,b) problem for the cluster solver. Side 0 is the u side (rows of F[0]
// are scaled by u~), side 1 the v side. The scalings are written to s[0], s[1],
// the final r-vectors t_u = F[0]^T u~ and t_v = F[1]^T v~ to t[0], t[1], and
// log_scale, residual, status and iters to *result (zeroed by the caller).
struct SProb {
  const float* F[2];
  const float* w[2];
  const float* shift[2];
  float* s[2];
  float* t[2];
  lsf_result* result;
  int64_t n[2];
};

constexpr int kSmallMaxProblems = 3;

// Whether the cluster solver takes a stored-feature problem of this shape under
// the current policy (lsf_set_small_solver).
bool small_solver_takes(int64_t n, int64_t m, int ldr);

// Launch the cluster solver for `count` (<= kSmallMaxProblems) problems of
// common row stride ldr: init v~ = exp(shift_y - M), `iters` iterations of
// Alg. 1, then the residual. One launch, one cluster per problem.
int small_solve(const SProb* probs, int count, int ldr, int iters, cudaStream_t st);

// As small_solve for a batch: `count` problems from a device table (any count),
// one 8-CTA cluster each, rows read from L2. The kernel also clears each
// problem's result record (W, residual, status) before solving it.
int small_solve_table(const SProb* table, int count, int ldr, int iters, cudaStream_t st);

}  // namespace lsf
