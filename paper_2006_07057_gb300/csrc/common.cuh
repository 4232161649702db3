// Shared device helpers and host bookkeeping of libsinkhorn_pf (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstdio>
#include <string>

#include "sinkhorn_pf.h"

namespace lsf {

// ---------------------------------------------------------------- host side

void set_error(const char* fmt, ...);
int fail(int status, const char* fmt, ...);

// Number of SMs and opt-in shared memory per block of the current device.
struct DeviceInfo {
  int device = -1;
  int sms = 0;
  int smem_optin = 0;
};
const DeviceInfo& device_info();

// Every launch goes through this so that it is counted and (optionally) timed
// and named on the host timeline (tracing level 2).
struct LaunchScope {
  LaunchScope(cudaStream_t s, int kernel_class, double bytes);
  ~LaunchScope();
  cudaStream_t stream;
  int cls;
  double bytes;
  int slot;
  bool traced;
};

// An NVTX range named `name` for the life of the object (tracing level >= 1).
struct TraceRange {
  explicit TraceRange(const char* name);
  ~TraceRange();
  bool on;
};

int check_launch(const char* what);

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// Workspace layout shared by the solver entry points (all offsets 256-aligned).
struct Workspace {
  float* part;          // [grid][2][2][ldr] per-CTA partial r-vectors (log passes: max and sum)
  float* gpart;         // [groups][2][2][ldr] per-group partials of the two-level reduction
  double* rpart;        // [grid][2] per-CTA partial residuals
  double* dpart;        // [grid][3] per-block partial divergences
  unsigned* counters;   // arrival counters: [1] divergence, [kPassCounter ...] passes
  unsigned* keys;       // [8] order-preserving float keys of running maxima
  size_t bytes;
};
size_t workspace_bytes(int ldr);
int carve_workspace(void* base, size_t bytes, int ldr, Workspace* ws);

// Lemma 1 on the device (no host round trip): q, sigma from the device radius R
// into qs = {q, sigma}; and anchors U = sigma Z with their log-constants from qs.
int launch_params_device(const float* R, double eps, int d, double* qs, cudaStream_t st);
int launch_anchors_device(const float* Z, int r, int d, const double* qs, double eps, float* U,
                          float* c, cudaStream_t st);

// Most CTAs any pass may launch: the workspace holds one partial r-vector slot per
// CTA, so every pass launcher clamps its grid to this.
int max_pass_ctas();
constexpr int kMaxPassCtasPerSm = 3;

// Two-level pass reduction: CTAs are summed in groups of kReduceGroup, then the
// groups. The pass counters start at counters[kPassCounter]: one for the groups,
// then one per group.
constexpr int kReduceGroup = 16;
constexpr int kPassCounter = 8;
inline int reduce_groups(int grid) { return (grid + kReduceGroup - 1) / kReduceGroup; }
int workspace_counters();  // unsigned counters in the workspace

// The divergence reduction runs one block per partial slot, at most max_pass_ctas().

// ---------------------------------------------------------------- device side

constexpr int kConsumerWarps = 11;  // + 1 producer warp: 3 warps per SMSP, up to 168 registers
constexpr int kPassThreads = (kConsumerWarps + 1) * 32;
constexpr unsigned long long kWaitLimitNs = 4000000000ull;  // 4 s per bounded wait

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void fence_mbarrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t tx) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(tx)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for the phase of the given parity to complete; false if limit_ns
// (default kWaitLimitNs) ran out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  unsigned long long limit_ns = kWaitLimitNs) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer_ns();
  while (true) {
#pragma unroll 1
    for (int i = 0; i < 32; ++i)
      if (mbar_try_wait(bar, parity)) return true;
    if (globaltimer_ns() - t0 > limit_ns) return false;
  }
}

// One bulk (non-tensor) TMA copy global -> shared, completing on an mbarrier.
// dst and src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes,
                                              uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// 4-byte asynchronous copy global -> shared (tracked with cp_async_mbar_arrive).
__device__ __forceinline__ void cp_async_4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src)
               : "memory");
}

// Close the thread's current group of cp.async copies.
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

// Wait until at most N of the thread's committed cp.async groups are still in
// flight (their copies then visible to this thread).
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// The mbarrier receives one arrival once all prior cp.async of this thread landed.
__device__ __forceinline__ void cp_async_mbar_arrive(uint64_t* bar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__device__ __forceinline__ float warp_min(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Hardware base-2 exponential (MUFU ex2, flushes subnormal results to zero).
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

constexpr float kLog2e = 1.4426950408889634f;

// Order-preserving map float -> unsigned (0 sorts below every finite float).
__device__ __forceinline__ unsigned float_key(float f) {
  unsigned b = __float_as_uint(f);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float key_float(unsigned k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// Neumaier-compensated FP64 accumulation.
struct KahanSum {
  double s = 0.0, c = 0.0;
  __device__ __forceinline__ void add(double x) {
    double t = s + x;
    if (fabs(s) >= fabs(x))
      c += (s - t) + x;
    else
      c += (x - t) + s;
    s = t;
  }
  __device__ __forceinline__ double value() const { return s + c; }
};

}  // namespace lsf
