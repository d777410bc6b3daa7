// Instances of the tiled forward kernel: FP32 storage, 3-D grids.
#include "bte_tiled_kernel.cuh"

namespace bte {
namespace tiled {
StepKernel pick_f32_3d(int lim, int nx) { return pick_instance<kStoreF32, 3, false>(lim, nx); }
}  // namespace tiled
}  // namespace bte
