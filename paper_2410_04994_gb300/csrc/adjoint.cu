// Adjoint (reverse) sweep of the discrete split-step map.
#include "plan.h"

namespace shg {
void free_adjoint(shg_plan*) {}
}  // namespace shg

extern "C" shg_status_t shg_propagate_adjoint(shg_plan_t* p, double, double*, double*, double*,
                                              float*, shg_stream_t) {
    if (!p) return SHG_ERR_INVALID_ARG;
    return SHG_ERR_STATE;
}
