// Instantiations of the row-tiled SG operator kernel in FP32 (a translation unit of its own so the
// two precisions compile in parallel).
#include <algorithm>

#include "k_apply_tile.cuh"

namespace sg {

namespace {

template <int KAPPA, int MINB>
int by_apw(const System& s, const TileOp& op, const float* X, float* Y, float alpha, const float* B,
           float beta, cudaStream_t st, const int* done) {
  const int b = tile_apw_bucket(op.apw);
  if (b == 8) return launch_tile_k<float, KAPPA, 8, MINB>(s, op, X, Y, alpha, B, beta, st, done);
  if constexpr (MINB == 1 || true) {
    if (b == 16) return launch_tile_k<float, KAPPA, 16, MINB>(s, op, X, Y, alpha, B, beta, st, done);
  }
  if constexpr (MINB == 1) return launch_tile_k<float, KAPPA, 32, MINB>(s, op, X, Y, alpha, B, beta, st, done);
  return fail(SG_ERR_ARG, "tile operator: kernel variant not built");
}

}  // namespace

int launch_tile_op_f32(const System& s, const TileOp& op, const float* X, float* Y, float alpha,
                      const float* B, float beta, cudaStream_t st, const int* done) {
  if (!tile_variant_ok(sizeof(float), op.kappa, op.apw, op.ctas))
    return fail(SG_ERR_ARG, "tile operator: kernel variant not built");
  const bool two = op.ctas == 2;
  switch (op.kappa) {
    case 1: return two ? by_apw<1, 2>(s, op, X, Y, alpha, B, beta, st, done)
                       : by_apw<1, 1>(s, op, X, Y, alpha, B, beta, st, done);
    case 2: return two ? by_apw<2, 2>(s, op, X, Y, alpha, B, beta, st, done)
                       : by_apw<2, 1>(s, op, X, Y, alpha, B, beta, st, done);
    default: return two ? by_apw<4, 2>(s, op, X, Y, alpha, B, beta, st, done)
                        : by_apw<4, 1>(s, op, X, Y, alpha, B, beta, st, done);
  }
}

}  // namespace sg
