// Instances of the tiled forward kernel: BF16 codes rounded stochastically, 3-D grids.
#include "bte_tiled_kernel.cuh"

namespace bte {
namespace tiled {
StepKernel pick_bf16sr_3d(int lim, int nx) { return pick_instance<kStoreBF16, 3, true>(lim, nx); }
}  // namespace tiled
}  // namespace bte
