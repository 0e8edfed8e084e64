// Instantiations of the row-tiled SG operator kernel in FP32 (a translation unit of its own so the
// two precisions compile in parallel).
#include <algorithm>

#include "k_apply_tile.cuh"

namespace sg {

int launch_tile_op_f32(const System& s, const TileOp& op, const float* X, float* Y, float alpha,
                      const float* B, float beta, cudaStream_t st, const int* done) {
  if (!tile_variant_ok(sizeof(float), op.kappa, op.ctas))
    return fail(SG_ERR_ARG, "tile operator: kernel variant not built");
  const bool two = op.ctas == 2;
  switch (op.kappa) {
    case 1: return two ? launch_tile_k<float, 1, 2>(s, op, X, Y, alpha, B, beta, st, done)
                       : launch_tile_k<float, 1, 1>(s, op, X, Y, alpha, B, beta, st, done);
    case 2: return two ? launch_tile_k<float, 2, 2>(s, op, X, Y, alpha, B, beta, st, done)
                       : launch_tile_k<float, 2, 1>(s, op, X, Y, alpha, B, beta, st, done);
    default: return two ? launch_tile_k<float, 4, 2>(s, op, X, Y, alpha, B, beta, st, done)
                        : launch_tile_k<float, 4, 1>(s, op, X, Y, alpha, B, beta, st, done);
  }
}

}  // namespace sg
