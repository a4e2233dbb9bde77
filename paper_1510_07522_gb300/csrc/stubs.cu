// Temporary: the projection and reduced-solve stages are not built yet.
#include "internal.h"
namespace rsrr {
int project_run(rsrr_nep, double) { return set_error(RSRR_EUNSUPPORTED, "rsrr_project not built yet"); }
int solve_run(rsrr_nep, int, int, double, int, double*, double*, double*, int32_t*) {
    return set_error(RSRR_EUNSUPPORTED, "rsrr_solve not built yet");
}
}  // namespace rsrr
