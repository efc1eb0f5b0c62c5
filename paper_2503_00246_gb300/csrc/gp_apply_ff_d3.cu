// Instantiations of the face and cell kernels: float-float on FP64 data, dimension 3, degrees 1..8.
#include "gp_launch.h"

namespace gp {
cudaError_t apply_ff_d3(const ApplyArgs& a, cudaStream_t st) { GP_DISPATCH_K(3, ArFF, a, st) }
BatchOps batch_ops_ff_d3() { GP_BATCH_OPS(3, ArFF) }
CellsFn cells_ff_d3() { GP_CELLS_FN(3, ArFF) }
TileOps tile_ops_ff_d3() { GP_TILE_OPS(3, ArFF) }
}  // namespace gp
