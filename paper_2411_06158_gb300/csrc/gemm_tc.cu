// Tensor-core (tcgen05) query projection: placeholder until the sm_103a kernel lands.
#include "common.cuh"

namespace mrq {

bool tc_available() { return false; }

void project_tc(const float*, const float*, const __nv_bfloat16*, const __nv_bfloat16*, int, int,
                int, bool, __nv_bfloat16*, float*, float*, cudaStream_t) {
  fail(MRQ_EINVAL, "tensor-core projection not built");
}

}  // namespace mrq
