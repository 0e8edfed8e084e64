// The SG operator Y = sum_k A_k X G_k^T (Eqs. stochastic_matrix and K_matrix): a shared-pattern
// CSR SpMM over the stacked stiffness values fused with the sparse contraction over the
// triple-product tensor, row by row, so the N x L x P intermediate never exists in memory.
//
// For node row i with stencil entries e (column j_e):
//   T[k,b] = sum_e A[e,k] X[j_e, b]       for the (k,b) pairs that meet a nonzero G_k[a,b]
//   Y[i,a] = sum_{(k,b)} G_k[a,b] T[k,b]
// which costs 9 U + nnz_G fused multiply-adds per row (U = number of such pairs), the fewest of
// the orderings: building the dense L x P product first costs 9 L P, building K_ab first 9 nnz_G.
//
// One CTA works on one row at a time (persistent over rows).  The row's stencil values of a k
// range and the 9 neighbour rows of X are staged in shared memory; T lives in shared memory for
// one chunk of pairs; each warp owns output columns a and reduces its entries with shuffles, so
// the result does not depend on scheduling.
#include "sg_internal.h"

namespace sg {

namespace {

template <typename TA, typename TV>
__device__ __forceinline__ TA cvt(const TV* p);
template <> __device__ __forceinline__ double cvt<double, double>(const double* p) { return *p; }
template <> __device__ __forceinline__ float cvt<float, float>(const float* p) { return *p; }
template <> __device__ __forceinline__ float cvt<float, __nv_bfloat16>(const __nv_bfloat16* p) {
  return __bfloat162float(*p);
}

template <typename TA>
__device__ __forceinline__ TA warp_sum(TA v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Rows per tile: the pair and entry tables are read once per tile instead of once per row.
constexpr int kRows = 4;
constexpr int kTs = kChunkPairs + 1;  // row stride of T in shared memory

template <typename TA, typename TV>
__global__ void __launch_bounds__(256) sg_apply_kernel(
    int N, int P, int L, const int* __restrict__ rowptr, const int* __restrict__ col,
    const TV* __restrict__ stack, const int* __restrict__ pair_kb, const int2* __restrict__ chunks,
    const int2* __restrict__ chunks_k, int nchunks, const int* __restrict__ ent_ptr,
    const int* __restrict__ ent_u, const TA* __restrict__ ent_g, const TA* __restrict__ X,
    TA* __restrict__ Y, TA alpha, const TA* __restrict__ B, TA beta, const int* __restrict__ done) {
  if (done != nullptr && *done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // stencil slots are padded to 9 per row with zeros, so every row runs the same unrolled loop
  TA* As = reinterpret_cast<TA*>(smem_raw);   // kRows x 9 x kChunkK
  TA* Xs = As + kRows * 9 * kChunkK;          // kRows x 9 x P
  TA* Ts = Xs + kRows * 9 * P;                // kRows x kTs (padded against bank conflicts)
  TA* Ys = Ts + kRows * kTs;                  // kRows x P
  __shared__ int rs_e0[kRows], rs_ne[kRows];
  const int tid = threadIdx.x, nth = blockDim.x;
  const int ntiles = (N + kRows - 1) / kRows;

  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int row0 = tile * kRows;
    const int nr = min(kRows, N - row0);
    if (tid < kRows) {
      int r = row0 + tid;
      rs_e0[tid] = tid < nr ? rowptr[r] : 0;
      rs_ne[tid] = tid < nr ? rowptr[r + 1] - rowptr[r] : 0;
    }
    __syncthreads();
    // one warp per (row, slot), lanes over chaos index: no runtime division
    for (int re = tid >> 5; re < kRows * 9; re += nth >> 5) {
      const int r = re / 9, e = re - r * 9;
      const bool have = e < rs_ne[r];
      const TA* xr = have ? X + (size_t)col[rs_e0[r] + e] * P : nullptr;
      for (int b = tid & 31; b < P; b += 32) Xs[re * P + b] = have ? xr[b] : TA(0);
    }
    for (int t = tid; t < kRows * P; t += nth) Ys[t] = TA(0);
    for (int c = 0; c < nchunks; ++c) {
      const int2 uu = chunks[c];
      const int2 kr = chunks_k[c];
      const int kw = kr.y - kr.x;
      static_assert((kChunkK & (kChunkK - 1)) == 0, "chunk width must be a power of two");
      for (int t = tid; t < kRows * 9 * kChunkK; t += nth) {
        const int re = t / kChunkK, kk = t & (kChunkK - 1);
        if (kk >= kw) continue;
        const int r = re / 9, e = re - r * 9;
        TA v = TA(0);
        if (e < rs_ne[r]) v = cvt<TA, TV>(stack + (size_t)(rs_e0[r] + e) * L + kr.x + kk);
        As[re * kChunkK + kk] = v;
      }
      __syncthreads();
      int kb = (uu.x + tid < uu.y) ? pair_kb[uu.x + tid] : 0;
      for (int u = uu.x + tid; u < uu.y; u += nth) {
        const int kbn = (u + nth < uu.y) ? pair_kb[u + nth] : 0;  // next pair, loaded early
        const int kk = (kb >> 16) - kr.x, b = kb & 0xffff;
        kb = kbn;
#pragma unroll
        for (int r = 0; r < kRows; ++r) {
          const TA* a = As + r * 9 * kChunkK + kk;
          const TA* x = Xs + r * 9 * P + b;
          TA s = a[0] * x[0];
#pragma unroll
          for (int e = 1; e < 9; ++e) s = fma(a[e * kChunkK], x[e * P], s);
          Ts[r * kTs + (u - uu.x)] = s;
        }
      }
      __syncthreads();
      // one thread per (a, row): a sequential sum, no cross-lane reduction (on this GPU an FP64
      // warp instruction costs the same whatever its active lanes, so shuffle trees are dear)
      const int* ep = ent_ptr + (size_t)c * (P + 1);
      for (int t = tid; t < kRows * P; t += nth) {
        const int a = t / kRows, r = t - a * kRows;
        TA acc = TA(0);
        for (int q = ep[a]; q < ep[a + 1]; ++q) acc = fma(ent_g[q], Ts[r * kTs + ent_u[q]], acc);
        Ys[r * P + a] += acc;
      }
      __syncthreads();
    }
    for (int t = tid; t < nr * P; t += nth) {
      size_t o = (size_t)row0 * P + t;
      TA v = alpha * Ys[t];
      if (B != nullptr) v = fma(beta, B[o], v);
      Y[o] = v;
    }
    __syncthreads();
  }
}

template <typename TA>
size_t apply_smem(int P) {
  return sizeof(TA) * ((size_t)kRows * 9 * kChunkK + (size_t)kRows * 9 * P +
                       (size_t)kRows * kTs + (size_t)kRows * P);
}

int num_sms() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 152;
  }
  return sms;
}

template <typename TA, typename TV>
int launch_apply(const System& s, const TV* stack, const TA* eg, const TA* X, TA* Y, TA alpha,
                 const TA* B, TA beta, cudaStream_t st, const int* done) {
  size_t smem = apply_smem<TA>(s.P);
  auto kern = sg_apply_kernel<TA, TV>;
  SG_TRY(ensure_smem((const void*)kern, smem));
  int per_sm = (int)std::max<size_t>(1, std::min<size_t>(8, (220 * 1024) / smem));
  int grid = std::min((s.N + kRows - 1) / kRows, num_sms() * per_sm);
  TimeScope ts(s.timer, sizeof(TA) == 8 ? K_APPLY_F64 : K_APPLY_LOWP, st);
  kern<<<grid, 256, smem, st>>>(s.N, s.P, s.L, s.rowptr.p, s.col.p, stack, s.pair_kb.p, s.chunks.p,
                                s.chunks_k.p, s.op.nchunks, s.ent_ptr.p, s.ent_u.p, eg, X, Y, alpha,
                                B, beta, done);
  return check_launch("sg_apply");
}

}  // namespace

int launch_matvec_f64(const System& s, const double* X, double* Y, double alpha, const double* B,
                      double beta, cudaStream_t st, const int* done) {
  if (s.tile64.ready) return launch_tile_op<double>(s, s.tile64, X, Y, alpha, B, beta, st, done);
  return launch_apply<double, double>(s, s.stack.p, s.ent_g.p, X, Y, alpha, B, beta, st, done);
}

int launch_matvec_f32(const System& s, const float* X, float* Y, float alpha, const float* B,
                      float beta, cudaStream_t st, const int* done) {
  if (s.tile32.ready && s.prm.precision == SG_MIXED_FP32)
    return launch_tile_op<float>(s, s.tile32, X, Y, alpha, B, beta, st, done);
  if (s.prm.precision == SG_MIXED_BF16)
    return launch_apply<float, __nv_bfloat16>(s, s.stack_bf16.p, s.ent_g_f32.p, X, Y, alpha, B,
                                              beta, st, done);
  return launch_apply<float, float>(s, s.stack_f32.p, s.ent_g_f32.p, X, Y, alpha, B, beta, st,
                                    done);
}

}  // namespace sg
