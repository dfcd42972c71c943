// Mixed-precision transforms (placeholder until the float32 path lands).
#include "internal.h"

namespace mlsdc {
mlsdc_status mp_init(sh_plan_t) { return MLSDC_ERR_INVALID; }
void mp_free(sh_plan_t) {}
mlsdc_status rhs_explicit_mp(sh_plan_t, const swe_params*, const double*, double*, cudaStream_t, int64_t*, int) {
    return MLSDC_ERR_INVALID;
}
}  // namespace mlsdc
