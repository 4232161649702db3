// Pipe-rate probe: the issue rates the recompute and hybrid passes are bound by,
// measured on the device instead of taken from nominal lane counts. One CTA of
// 1024 threads per SM (a shared-memory request keeps a second CTA off the SM)
// runs eight independent dependency chains per thread of one instruction kind;
// the SM's cycle counter around the loop gives results per clock per SM:
//   - FP32 lane operations with the packed two-lane FMA (fma.rn.f32x2),
//   - FP32 lane operations with the scalar FMA,
//   - ex2.approx results (the special-function unit).
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"

namespace lsf {
namespace {

constexpr int kProbeThreads = 1024;
constexpr int kProbeIters = 2048;
constexpr int kProbeMaxCtas = 1024;
constexpr size_t kProbeSmem = 120 * 1024;  // more than half an SM's shared memory

__device__ unsigned long long g_probe_cycles[3][kProbeMaxCtas];
__device__ float g_probe_sink[kProbeMaxCtas];

template <int KIND>
__global__ void __launch_bounds__(kProbeThreads, 1) probe_kernel(float a, float b) {
  extern __shared__ float s_pad[];
  float2 acc[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) acc[j] = make_float2(a + j, b - j);
  const float2 m2 = make_float2(a, a), c2 = make_float2(b, b);
  __syncthreads();
  const unsigned long long t0 = clock64();
#pragma unroll 4
  for (int it = 0; it < kProbeIters; ++it) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      if (KIND == 0) {
        acc[j] = __ffma2_rn(acc[j], m2, c2);
      } else if (KIND == 1) {
        acc[j].x = fmaf(acc[j].x, a, b);
      } else {
        acc[j].x = ex2_approx(-acc[j].x);
      }
    }
  }
  __syncthreads();
  const unsigned long long t1 = clock64();
  float sum = 0.f;
#pragma unroll
  for (int j = 0; j < 8; ++j) sum += acc[j].x + acc[j].y;
  if (threadIdx.x == 0) g_probe_cycles[KIND][blockIdx.x] = t1 - t0;
  if (sum == 1234.5678f) {  // never true in practice; keeps the chains live
    s_pad[threadIdx.x] = sum;
    g_probe_sink[blockIdx.x] = s_pad[(threadIdx.x + 1) % kProbeThreads];
  }
}

}  // namespace
}  // namespace lsf

using namespace lsf;

extern "C" int lsf_probe_pipe_rates(double* ffma2_lane_ops, double* ffma_lane_ops, double* ex2_ops,
                                    void* stream) {
  if (!ffma2_lane_ops || !ffma_lane_ops || !ex2_ops) return fail(LSF_ERR_ARG, "lsf_probe_pipe_rates: NULL output");
  cudaStream_t st = as_stream(stream);
  const int grid = std::min(device_info().sms, kProbeMaxCtas);
  void (*kern[3])(float, float) = {probe_kernel<0>, probe_kernel<1>, probe_kernel<2>};
  for (int k = 0; k < 3; ++k) {
    if (cudaFuncSetAttribute(kern[k], cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(kProbeSmem)) != cudaSuccess)
      return fail(LSF_ERR_CUDA, "lsf_probe_pipe_rates: shared-memory attribute");
    for (int rep = 0; rep < 2; ++rep) {  // the first launch warms the clocks up
      LaunchScope ls(st, LSF_KERNEL_OTHER, 0.0);
      kern[k]<<<grid, kProbeThreads, kProbeSmem, st>>>(0.999f, 0.001f);
    }
    int rc = check_launch("probe_kernel");
    if (rc != LSF_OK) return rc;
  }
  unsigned long long cyc[3][kProbeMaxCtas];
  if (cudaMemcpyFromSymbolAsync(cyc, g_probe_cycles, sizeof(cyc), 0, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return fail(LSF_ERR_CUDA, "lsf_probe_pipe_rates: read-back failed");
  // per instruction kind: lane results per thread, and the slowest SM's cycles
  const double per_thread[3] = {2.0 * 8 * kProbeIters, 1.0 * 8 * kProbeIters, 1.0 * 8 * kProbeIters};
  double rate[3];
  for (int k = 0; k < 3; ++k) {
    unsigned long long worst = 1;
    for (int b = 0; b < grid; ++b) worst = std::max(worst, cyc[k][b]);
    rate[k] = per_thread[k] * kProbeThreads / static_cast<double>(worst);
  }
  *ffma2_lane_ops = rate[0];
  *ffma_lane_ops = rate[1];
  *ex2_ops = rate[2];
  return LSF_OK;
}
