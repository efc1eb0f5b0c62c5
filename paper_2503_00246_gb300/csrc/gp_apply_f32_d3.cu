// Instantiations of the face and cell kernels: FP32, dimension 3, degrees 1..8.
#include "gp_launch.h"

namespace gp {
cudaError_t apply_f32_d3(const ApplyArgs& a, cudaStream_t st) { GP_DISPATCH_K(3, ArF32, a, st) }
BatchOps batch_ops_f32_d3() { GP_BATCH_OPS(3, ArF32) }
CellsFn cells_f32_d3() { GP_CELLS_FN(3, ArF32) }
TileOps tile_ops_f32_d3() { GP_TILE_OPS(3, ArF32) }
}  // namespace gp
