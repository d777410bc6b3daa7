// Instances of the tiled forward kernel: BF16 storage, 3-D grids.
#include "bte_tiled_kernel.cuh"

namespace bte {
namespace tiled {
StepKernel pick_bf16_3d(int lim, int nx) { return pick_instance<kStoreBF16, 3>(lim, nx); }
}  // namespace tiled
}  // namespace bte
