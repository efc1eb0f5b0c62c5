// Instantiations of the face and cell kernels: FP32, dimension 2, degrees 1..8.
#include "gp_launch.h"

namespace gp {
cudaError_t apply_f32_d2(const ApplyArgs& a, cudaStream_t st) { GP_DISPATCH_K(2, ArF32, a, st) }
BatchOps batch_ops_f32_d2() { GP_BATCH_OPS(2, ArF32) }
CellsFn cells_f32_d2() { GP_CELLS_FN(2, ArF32) }
TileOps tile_ops_f32_d2() { GP_TILE_OPS(2, ArF32) }
}  // namespace gp
