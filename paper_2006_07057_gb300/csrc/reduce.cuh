// End of a fused pass: CTA partials to the workspace, then fixed-order sums in
// two levels by the last CTAs to arrive (so results do not depend on scheduling).
#pragma once

#include "pass.cuh"

namespace lsf {

// Compensated FP32 sum (Neumaier): the rounding error of every addition is
// carried in c, so a short fixed-order sum of positive partials is accurate to
// about one rounding of the result. FP64 is not used here: its throughput on
// this GPU is a small fraction of FP32's.
struct CompSum {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float t = s + x;
    c += (fabsf(s) >= fabsf(x)) ? (s - t) + x : (x - t) + s;
    s = t;
  }
  __device__ __forceinline__ float value() const { return s + c; }
};

// Cross-CTA reduction of a pass, in two fixed-order levels so that no single CTA
// walks all partials: CTA b writes its partial to part[b]; the last CTA to arrive
// in group b / kReduceGroup sums that group's partials (CTA order) into
// gpart[group]; the last group to finish sums the group partials (group order)
// into t_out, and the residual partials. The order of every sum is fixed by the
// CTA indices, not by arrival, so the result is deterministic.
// counter: [0] groups finished, [1 + g] CTAs of group g arrived (all zero
// between launches; each level resets what it used).
//
// All threads of the CTA call this once the per-warp partial r-vectors are in
// shared memory (red: [ngroups][NRHS * ldr]) and the per-warp residual sums in
// rres ([ngroups][2]). flag: status bits gathered by this CTA.
template <int NRHS, bool ACC>
__device__ __forceinline__ void finish_pass(const float* red, int ngroups, const double* rres,
                                            int ldr, const PassRhs* rhs, float* part, float* gpart,
                                            double* rpart, unsigned* counter, int* status,
                                            int flag, int* s_last) {
  const unsigned G = gridDim.x;
  const int nv = NRHS * ldr;
  const int nv4 = nv >> 2;
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
  const unsigned grp = blockIdx.x / kReduceGroup;
  const unsigned b0 = grp * kReduceGroup;
  const unsigned b1 = min(G, b0 + kReduceGroup);
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    *s_last = (atomicAdd(counter + 1 + grp, 1u) == b1 - b0 - 1u) ? 1 : 0;
    if (flag) atomicOr(status, flag);
  }
  __syncthreads();
  if (!*s_last) return;
  __threadfence();
  if (ACC) {
    for (int i4 = threadIdx.x; i4 < nv4; i4 += blockDim.x) {
      CompSum a0, a1, a2, a3;
#pragma unroll
      for (int q = 0; q < kReduceGroup; ++q) {
        const unsigned b = b0 + q;
        if (b < b1) {
          const float4 v = __ldcg(reinterpret_cast<const float4*>(part + static_cast<size_t>(b) * nv) + i4);
          a0.add(v.x); a1.add(v.y); a2.add(v.z); a3.add(v.w);
        }
      }
      reinterpret_cast<float4*>(gpart + static_cast<size_t>(grp) * nv)[i4] =
          make_float4(a0.value(), a1.value(), a2.value(), a3.value());
    }
  }
  __threadfence();
  __syncthreads();
  const unsigned NG = (G + kReduceGroup - 1) / kReduceGroup;
  if (threadIdx.x == 0) {
    counter[1 + grp] = 0u;
    *s_last = (atomicAdd(counter, 1u) == NG - 1u) ? 1 : 0;
  }
  __syncthreads();
  if (!*s_last) return;
  __threadfence();
  if (ACC) {
    for (int i4 = threadIdx.x; i4 < nv4; i4 += blockDim.x) {
      CompSum a0, a1, a2, a3;
      for (unsigned g = 0; g < NG; ++g) {
        const float4 v = __ldcg(reinterpret_cast<const float4*>(gpart + static_cast<size_t>(g) * nv) + i4);
        a0.add(v.x); a1.add(v.y); a2.add(v.z); a3.add(v.w);
      }
      const int idx = 4 * i4;
      const int k = idx / ldr;  // ldr is a multiple of 4: a float4 never straddles two r-vectors
      const int col = idx - k * ldr;
      float* to = rhs[k].t_out;
      if (to) *reinterpret_cast<float4*>(to + col) = make_float4(a0.value(), a1.value(), a2.value(), a3.value());
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
  // A partial without mass is skipped: a real partial with finite m2 has s2 >= 1
  // (its maximum contributes exp(0)), and a slot no CTA wrote holds (0, 0).
  if (m2 == -INFINITY || !(s2 > 0.f)) return;
  if (m == -INFINITY) {
    m = m2;
    s = s2;
    return;
  }
  const float M = fmaxf(m, m2);
  s = s * __expf(m - M) + s2 * __expf(m2 - M);
  m = M;
}

// Online log-sum-exp: (m, s) represents log(s e^m); adding one term y gives
// (max(m, y), s e^(m - max) + e^(y - max)). One of the two exponentials is
// e^0 = 1, so one ex2 per term suffices. The empty sum is (kLogFloor, 0): a
// finite floor far below any log-domain value, so a term y = -inf (no mass)
// adds e^-inf = 0 without a branch, and merges skip partials with s = 0.
constexpr float kLogFloor = -1e30f;
__device__ __forceinline__ void lse_push(float& m, float& s, float y) {
  const float d = y - m;
  const float e = ex2_approx(-fabsf(d) * kLog2e);
  s = (d > 0.f) ? fmaf(s, e, 1.f) : s + e;
  m = fmaxf(m, y);
}

// As finish_pass for the log-domain passes: red holds [ngroups][NRHS][2][ldr]
// (per-group maxima then sums per column); the r-vector written is
// t_out[k] = m + log(s) (-inf where no mass). The same two fixed-order levels
// (CTA order within a group of kReduceGroup CTAs, then group order) merge the
// (max, sum) pairs.
template <int NRHS, bool ACC>
__device__ __forceinline__ void finish_pass_log(const float* red, int ngroups, const double* rres,
                                                int ldr, const PassRhs* rhs, float* part,
                                                float* gpart, double* rpart, unsigned* counter,
                                                int* status, int flag, int* s_last) {
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
  const unsigned grp = blockIdx.x / kReduceGroup;
  const unsigned b0 = grp * kReduceGroup;
  const unsigned b1 = min(G, b0 + kReduceGroup);
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    *s_last = (atomicAdd(counter + 1 + grp, 1u) == b1 - b0 - 1u) ? 1 : 0;
    if (flag) atomicOr(status, flag);
  }
  __syncthreads();
  if (!*s_last) return;
  __threadfence();
  if (ACC) {
    for (int idx = threadIdx.x; idx < nv; idx += blockDim.x) {
      const int k = idx / ldr, col = idx - k * ldr;
      float m = -INFINITY, s = 0.f;
#pragma unroll
      for (int q = 0; q < kReduceGroup; ++q) {
        const unsigned b = b0 + q;
        if (b < b1) {
          const float* pp = part + (static_cast<size_t>(b) * NRHS + k) * 2 * ldr;
          lse_merge(m, s, __ldcg(pp + col), __ldcg(pp + ldr + col));
        }
      }
      float* gp = gpart + (static_cast<size_t>(grp) * NRHS + k) * 2 * ldr;
      gp[col] = m;
      gp[ldr + col] = s;
    }
  }
  __threadfence();
  __syncthreads();
  const unsigned NG = (G + kReduceGroup - 1) / kReduceGroup;
  if (threadIdx.x == 0) {
    counter[1 + grp] = 0u;
    *s_last = (atomicAdd(counter, 1u) == NG - 1u) ? 1 : 0;
  }
  __syncthreads();
  if (!*s_last) return;
  __threadfence();
  if (ACC) {
    for (int idx = threadIdx.x; idx < nv; idx += blockDim.x) {
      const int k = idx / ldr, col = idx - k * ldr;
      float m = -INFINITY, s = 0.f;
      for (unsigned g = 0; g < NG; ++g) {
        const float* gp = gpart + (static_cast<size_t>(g) * NRHS + k) * 2 * ldr;
        lse_merge(m, s, __ldcg(gp + col), __ldcg(gp + ldr + col));
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
