// Instances of the tiled forward kernel: FP32 storage, 2-D grids.
#include "bte_tiled_kernel.cuh"

namespace bte {
namespace tiled {
StepKernel pick_f32_2d(int lim, int nx) { return pick_instance<kStoreF32, 2, false>(lim, nx); }
}  // namespace tiled
}  // namespace bte
