// Instantiations of the row-tiled SG operator kernel in FP64 (a translation unit of its own so the
// two precisions compile in parallel).
#include <algorithm>

#include "k_apply_tile.cuh"

namespace sg {

int launch_tile_op_f64(const System& s, const TileOp& op, const double* X, double* Y, double alpha,
                      const double* B, double beta, cudaStream_t st, const int* done) {
  if (!tile_variant_ok(sizeof(double), op.kappa, op.ctas))
    return fail(SG_ERR_ARG, "tile operator: kernel variant not built");
  const bool two = op.ctas == 2;
  switch (op.kappa) {
    case 1: return two ? launch_tile_k<double, 1, 2>(s, op, X, Y, alpha, B, beta, st, done)
                       : launch_tile_k<double, 1, 1>(s, op, X, Y, alpha, B, beta, st, done);
    default: return two ? launch_tile_k<double, 2, 2>(s, op, X, Y, alpha, B, beta, st, done)
                        : launch_tile_k<double, 2, 1>(s, op, X, Y, alpha, B, beta, st, done);
  }
}

}  // namespace sg
