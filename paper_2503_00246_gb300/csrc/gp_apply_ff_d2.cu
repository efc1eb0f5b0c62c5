// Instantiations of the face and cell kernels: float-float on FP64 data, dimension 2, degrees 1..8.
#include "gp_launch.h"

namespace gp {
cudaError_t apply_ff_d2(const ApplyArgs& a, cudaStream_t st) { GP_DISPATCH_K(2, ArFF, a, st) }
BatchOps batch_ops_ff_d2() { GP_BATCH_OPS(2, ArFF) }
CellsFn cells_ff_d2() { GP_CELLS_FN(2, ArFF) }
TileOps tile_ops_ff_d2() { GP_TILE_OPS(2, ArFF) }
}  // namespace gp
