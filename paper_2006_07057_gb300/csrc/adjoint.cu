#include "common.cuh"

using namespace lsf;

extern "C" int lsf_gradient(const lsf_theta*, const lsf_cloud*, const lsf_cloud*,
                            const lsf_scalings*, const lsf_scalings*, const lsf_scalings*,
                            const lsf_result*, int, float*, float*, float*, float*, void*) {
  return fail(LSF_ERR_UNSUPPORTED, "gradient is not built yet");
}
