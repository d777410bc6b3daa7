// Shared-memory tiled forward kernel of the explicit DOM step (arXiv 2306.14181, Sec. 4).
#include "bte_tiled.h"

namespace bte {

bool tiled_plan(int, const int *, int, int, int, const int *, TiledPlan &plan, std::string &why) {
    plan = TiledPlan();
    why = "not built yet";
    return false;
}
bool tiled_setup(TiledPlan &, void *, void *, size_t, std::string &why) {
    why = "not built yet";
    return false;
}
void tiled_free(TiledPlan &) {}
cudaError_t launch_step_tiled(const StepArgs &, const TiledPlan &, int, int, int, cudaStream_t) {
    return cudaErrorNotSupported;
}
cudaError_t launch_finalize_tiled(const StepArgs &, const TiledPlan &, float *, cudaStream_t) {
    return cudaErrorNotSupported;
}

}  // namespace bte
