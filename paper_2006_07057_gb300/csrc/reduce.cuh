// End of a fused pass: CTA partials to the workspace, then a fixed-order sum by
// the last CTA to arrive (so results do not depend on scheduling).
#pragma once

#include "pass.cuh"

namespace lsf {

// All threads of the CTA call this once the per-group partial r-vectors are in
// shared memory (red: [ngroups][NRHS * ldr]) and the per-group residual sums in
// rres ([ngroups][2]). flag: status bits gathered by this CTA.
template <int NRHS, bool ACC>
__device__ __forceinline__ void finish_pass(const float* red, int ngroups, const double* rres,
                                            int ldr, const PassRhs* rhs, float* part,
                                            double* rpart, unsigned* counter, int* status,
                                            int flag, int* s_last) {
  const unsigned G = gridDim.x;
  const int nv = NRHS * ldr;
  if (ACC) {
    for (int idx = threadIdx.x; idx < nv; idx += blockDim.x) {
      float sum = 0.f;
      for (int g = 0; g < ngroups; ++g) sum += red[static_cast<size_t>(g) * nv + idx];
      part[static_cast<size_t>(blockIdx.x) * nv + idx] = sum;
    }
  }
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NRHS; ++k) {
      double r = 0.0;
      for (int g = 0; g < ngroups; ++g) r += rres[g * 2 + k];
      rpart[static_cast<size_t>(blockIdx.x) * NRHS + k] = r;
    }
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    *s_last = (atomicAdd(counter, 1u) == G - 1u) ? 1 : 0;
    if (flag) atomicOr(status, flag);
  }
  __syncthreads();
  if (!*s_last) return;
  __threadfence();
  if (ACC) {
    for (int idx = threadIdx.x; idx < nv; idx += blockDim.x) {
      double s0 = 0.0, s1 = 0.0;
      unsigned g = 0;
      for (; g + 1 < G; g += 2) {
        s0 += __ldcg(part + static_cast<size_t>(g) * nv + idx);
        s1 += __ldcg(part + static_cast<size_t>(g + 1) * nv + idx);
      }
      if (g < G) s0 += __ldcg(part + static_cast<size_t>(g) * nv + idx);
      const int k = idx / ldr;
      const int col = idx - k * ldr;
      float* to = rhs[k].t_out;
      if (to) to[col] = static_cast<float>(s0 + s1);
    }
  }
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NRHS; ++k) {
      if (!rhs[k].res_out) continue;
      double r = 0.0;
      for (unsigned g = 0; g < G; ++g) r += __ldcg(rpart + static_cast<size_t>(g) * NRHS + k);
      *rhs[k].res_out = r;
    }
    *counter = 0u;
  }
}

// Log-domain merge of (max, sum) pairs: (m1, s1) (+) (m2, s2) represents
// log(s1 e^m1 + s2 e^m2) = M + log(s1 e^(m1-M) + s2 e^(m2-M)), M = max(m1, m2).
__device__ __forceinline__ void lse_merge(float& m, float& s, float m2, float s2) {
  if (m2 == -INFINITY) return;
  if (m == -INFINITY) {
    m = m2;
    s = s2;
    return;
  }
  const float M = fmaxf(m, m2);
  s = s * __expf(m - M) + s2 * __expf(m2 - M);
  m = M;
}

// As finish_pass for the log-domain passes: red holds [ngroups][NRHS][2][ldr]
// (per-group maxima then sums per column); the r-vector written is
// t_out[k] = m + log(s) (-inf where no mass), merged in group then CTA order.
template <int NRHS, bool ACC>
__device__ __forceinline__ void finish_pass_log(const float* red, int ngroups, const double* rres,
                                                int ldr, const PassRhs* rhs, float* part,
                                                double* rpart, unsigned* counter, int* status,
                                                int flag, int* s_last) {
  const unsigned G = gridDim.x;
  const int nv = NRHS * ldr;
  if (ACC) {
    for (int idx = threadIdx.x; idx < nv; idx += blockDim.x) {
      const int k = idx / ldr, col = idx - k * ldr;
      float m = -INFINITY, s = 0.f;
      for (int g = 0; g < ngroups; ++g) {
        const float* rg = red + (static_cast<size_t>(g) * NRHS + k) * 2 * ldr;
        lse_merge(m, s, rg[col], rg[ldr + col]);
      }
      float* pp = part + (static_cast<size_t>(blockIdx.x) * NRHS + k) * 2 * ldr;
      pp[col] = m;
      pp[ldr + col] = s;
    }
  }
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NRHS; ++k) {
      double r = 0.0;
      for (int g = 0; g < ngroups; ++g) r += rres[g * 2 + k];
      rpart[static_cast<size_t>(blockIdx.x) * NRHS + k] = r;
    }
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    *s_last = (atomicAdd(counter, 1u) == G - 1u) ? 1 : 0;
    if (flag) atomicOr(status, flag);
  }
  __syncthreads();
  if (!*s_last) return;
  __threadfence();
  if (ACC) {
    for (int idx = threadIdx.x; idx < nv; idx += blockDim.x) {
      const int k = idx / ldr, col = idx - k * ldr;
      float m = -INFINITY, s = 0.f;
      for (unsigned g = 0; g < G; ++g) {
        const float* pp = part + (static_cast<size_t>(g) * NRHS + k) * 2 * ldr;
        lse_merge(m, s, __ldcg(pp + col), __ldcg(pp + ldr + col));
      }
      float* to = rhs[k].t_out;
      if (to) to[col] = (s > 0.f) ? m + logf(s) : -INFINITY;
    }
  }
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NRHS; ++k) {
      if (!rhs[k].res_out) continue;
      double r = 0.0;
      for (unsigned g = 0; g < G; ++g) r += __ldcg(rpart + static_cast<size_t>(g) * NRHS + k);
      *rhs[k].res_out = r;
    }
    *counter = 0u;
  }
}

}  // namespace lsf
