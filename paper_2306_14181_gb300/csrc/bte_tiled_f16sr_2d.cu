// Instances of the tiled forward kernel: F16 codes rounded stochastically, 2-D grids.
#include "bte_tiled_kernel.cuh"

namespace bte {
namespace tiled {
StepKernel pick_f16sr_2d(int lim, int nx) { return pick_instance<kStoreF16, 2, true>(lim, nx); }
}  // namespace tiled
}  // namespace bte
