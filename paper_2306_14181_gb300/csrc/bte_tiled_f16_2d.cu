// Instances of the tiled forward kernel: F16 codes rounded to nearest, 2-D grids.
#include "bte_tiled_kernel.cuh"

namespace bte {
namespace tiled {
StepKernel pick_f16_2d(int lim, int nx, bool sr) {
    return sr ? pick_f16sr_2d(lim, nx) : pick_instance<kStoreF16, 2, false>(lim, nx);
}
}  // namespace tiled
}  // namespace bte
