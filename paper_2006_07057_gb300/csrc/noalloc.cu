// lsf_solve_noalloc: the solver for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all: code that runs inside a framework
// whose memory pool owns every byte of the device (an allocation outside the
// pool breaks its accounting and, through the implicit device synchronisation
// of cudaMalloc, stalls every other stream), or latency-bound serving loops that
// must never block on the allocator. They still own their inputs and outputs,
// but they cannot provide the solver's scratch workspace. This entry point runs
// the same solve with its scratch taken from a fixed-size array that lives in
// the library's own device image.
#include <cuda_runtime.h>

#include <mutex>

#include "common.cuh"

namespace {

// Largest scratch this entry point can use. One solve needs
// lsf_workspace_bytes(ldr): about 52 * SMs * ldr bytes, i.e. ~8 MB at
// ldr = 1024 on a 152-SM GB300. Every GPU that loads the library keeps this
// array until the process exits.
constexpr size_t kNoAllocScratchBytes = size_t(12) << 20;  // 12 MiB

// In host code this name is only a stand-in for the device array: its device
// address must be fetched with cudaGetSymbolAddress on each device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once per
// device, with that device current).
int scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return lsf::fail(LSF_ERR_CUDA, "lsf_solve_noalloc: cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices)
    return lsf::fail(LSF_ERR_UNSUPPORTED, "lsf_solve_noalloc: device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return lsf::fail(LSF_ERR_CUDA, "lsf_solve_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return LSF_OK;
}

}  // namespace

extern "C" int lsf_solve_noalloc(const lsf_theta* theta, const lsf_cloud* x, const lsf_cloud* y,
                                 int iters, int mode, const lsf_scalings* out, lsf_result* result,
                                 void* stream) {
  if (!theta) return lsf::fail(LSF_ERR_ARG, "lsf_solve_noalloc: theta is NULL");
  size_t need = 0;
  int rc = lsf_workspace_bytes(theta->ldr, &need);
  if (rc != LSF_OK) return rc;
  if (need > kNoAllocScratchBytes)
    return lsf::fail(LSF_ERR_UNSUPPORTED,
                     "lsf_solve_noalloc: this problem needs %zu bytes of scratch, more than the "
                     "%zu-byte built-in array; use lsf_solve with a caller workspace",
                     need, kNoAllocScratchBytes);
  void* ws = nullptr;
  rc = scratch_address(&ws);
  if (rc != LSF_OK) return rc;
  // lsf_solve clears the counters and keys it needs at the start of every call.
  return lsf_solve(theta, x, y, iters, mode, out, result, ws, kNoAllocScratchBytes, stream);
}
