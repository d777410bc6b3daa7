// Instances of the tiled forward kernel: BF16 codes rounded to nearest, 2-D grids.
#include "bte_tiled_kernel.cuh"

namespace bte {
namespace tiled {
StepKernel pick_bf16_2d(int lim, int nx, bool sr) {
    return sr ? pick_bf16sr_2d(lim, nx) : pick_instance<kStoreBF16, 2, false>(lim, nx);
}
}  // namespace tiled
}  // namespace bte
