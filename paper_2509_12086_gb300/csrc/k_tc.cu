// k_tc.cu -- tensor-core projection (tcgen05 + TMA).  Not yet enabled.
#include "saq_internal.h"

namespace saq {

bool tc_supported(const saq_model *) { return false; }

saq_status model_build_tc(saq_model *, int, cudaStream_t) {
    return set_error(SAQ_ERR_UNSUPPORTED, "tensor-core projection not built");
}

saq_status launch_project_tc(const saq_model *, const float *, int64_t, float *, int64_t,
                             float *, int64_t, cudaStream_t) {
    return set_error(SAQ_ERR_UNSUPPORTED, "tensor-core projection not built");
}

}  // namespace saq
