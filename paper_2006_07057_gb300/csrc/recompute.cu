#include "recompute.cuh"

namespace lsf {

int launch_recompute_pass(int, int, RecomputeArgs, cudaStream_t) {
  return fail(LSF_ERR_UNSUPPORTED, "recompute mode is not built yet");
}

}  // namespace lsf
