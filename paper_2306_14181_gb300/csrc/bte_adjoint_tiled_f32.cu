// Instances of the tiled adjoint kernel: FP32 storage, 2-D and 3-D grids.
#include "bte_adjoint_tiled.cuh"

namespace bte {
namespace tiled {
AdjKernel adj_pick_f32(int lim, int nx, int dim) { return adj_pick_instance<kStoreF32>(lim, nx, dim); }
}  // namespace tiled
}  // namespace bte
