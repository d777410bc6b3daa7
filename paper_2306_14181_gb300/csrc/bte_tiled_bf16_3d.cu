// Instances of the tiled forward kernel: BF16 codes rounded to nearest, 3-D grids.
#include "bte_tiled_kernel.cuh"

namespace bte {
namespace tiled {
StepKernel pick_bf16_3d(int lim, int nx, bool sr) {
    return sr ? pick_bf16sr_3d(lim, nx) : pick_instance<kStoreBF16, 3, false>(lim, nx);
}
}  // namespace tiled
}  // namespace bte
