// fused2d.cu -- placeholder until the single-pass FP32 kernel lands.
#include "hyb_internal.cuh"

namespace hyb {
struct FusedPlan {};
bool fused_supported(const hyb_grid_desc&) { return false; }
hyb_status fused_create(hyb_grid*) { set_error("fused path unavailable"); return HYB_EINVAL; }
void fused_destroy(hyb_grid* g) { delete g->fused; g->fused = nullptr; }
hyb_status fused_advance(hyb_grid*, int) { set_error("fused path unavailable"); return HYB_EINVAL; }
int fused_launches_per_step(const hyb_grid*) { return 0; }
}  // namespace hyb
