// Heat solve (red-black SOR) and the self-consistent loop.
#include "plan.h"

extern "C" shg_status_t shg_heat_solve(shg_plan_t* p, int, double, double*, int*, shg_stream_t) {
    if (!p) return SHG_ERR_INVALID_ARG;
    return SHG_ERR_STATE;
}
extern "C" shg_status_t shg_thermal_loop(shg_plan_t* p, int, int, double, double*, double*,
                                         shg_stream_t) {
    if (!p) return SHG_ERR_INVALID_ARG;
    return SHG_ERR_STATE;
}
extern "C" shg_status_t shg_get_heat(shg_plan_t* p, double*, float*, shg_stream_t) {
    if (!p) return SHG_ERR_INVALID_ARG;
    return SHG_ERR_STATE;
}
