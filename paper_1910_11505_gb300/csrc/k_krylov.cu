// Krylov kernels of restarted GMRES (Sec. 3) on the device: classical Gram-Schmidt applied twice
// (CGS2) with deterministic two-level reductions, the Givens least-squares update, the
// back-substitution and the solution update.  Every kernel of one Arnoldi step reads the
// system's ``done`` flag first and returns at once when the cycle has already converged, so a
// whole cycle can be queued without a host round trip.
//
// Reductions: each CTA writes its partial sums, the last CTA to arrive (atomic ticket) adds the
// partials in CTA order and resets the ticket, so results are bitwise reproducible.
#include "sg_internal.h"

namespace sg {

constexpr int kRedBlocks = 304;   // 2 CTAs per SM on 152 SMs
constexpr int kRedThreads = 256;
constexpr int kMaxBasis = 1025;   // restart <= 1024 -> at most 1025 basis vectors
constexpr int kLT = 8;            // basis vectors per register tile

namespace {

__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += sh[i];
  return s;  // valid in thread 0
}

// Partial dot products of w with basis vectors [0, nv) for this CTA's grid-stride slice.
__device__ void partial_dots(size_t n, const double* __restrict__ V, int nv,
                             const double* __restrict__ w, double* __restrict__ partial,
                             double* sh) {
  for (int l0 = 0; l0 < nv; l0 += kLT) {
    double acc[kLT];
#pragma unroll
    for (int q = 0; q < kLT; ++q) acc[q] = 0.0;
    int lc = min(kLT, nv - l0);
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
      double wi = w[i];
#pragma unroll
      for (int q = 0; q < kLT; ++q)
        if (q < lc) acc[q] = fma(V[(size_t)(l0 + q) * n + i], wi, acc[q]);
    }
#pragma unroll
    for (int q = 0; q < kLT; ++q) {
      if (q < lc) {
        double s = block_sum(acc[q], sh);
        if (threadIdx.x == 0) partial[(size_t)blockIdx.x * kMaxBasis + l0 + q] = s;
      }
    }
  }
}

// Returns true in every thread of the CTA that arrives last.
__device__ bool arrive_last(unsigned int* ticket) {
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  __syncthreads();
  return last;
}

__device__ void finish_sums(const double* partial, int nv, double* out, unsigned int* ticket) {
  __threadfence();
  for (int l = threadIdx.x; l < nv; l += blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < (int)gridDim.x; ++b) s += __ldcg(partial + (size_t)b * kMaxBasis + l);
    out[l] = s;
  }
  if (threadIdx.x == 0) *ticket = 0u;
}

// h = V[0:nv]^T w
__global__ void __launch_bounds__(kRedThreads) cgs_dots_kernel(
    size_t n, const double* __restrict__ V, int nv, const double* __restrict__ w,
    double* __restrict__ partial, unsigned int* ticket, double* __restrict__ h,
    const int* __restrict__ done) {
  if (*done) return;
  __shared__ double sh[32];
  partial_dots(n, V, nv, w, partial, sh);
  if (arrive_last(ticket)) finish_sums(partial, nv, h, ticket);
}

// w -= V[0:nv] h1, then h2 = V[0:nv]^T w
__global__ void __launch_bounds__(kRedThreads) cgs_update_dots_kernel(
    size_t n, const double* __restrict__ V, int nv, double* __restrict__ w,
    const double* __restrict__ h1, double* __restrict__ partial, unsigned int* ticket,
    double* __restrict__ h2, const int* __restrict__ done) {
  if (*done) return;
  __shared__ double sh[32];
  __shared__ double hs[kMaxBasis];
  for (int l = threadIdx.x; l < nv; l += blockDim.x) hs[l] = h1[l];
  __syncthreads();
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    double v = w[i];
    for (int l = 0; l < nv; ++l) v = fma(-V[(size_t)l * n + i], hs[l], v);
    w[i] = v;
  }
  // each thread re-reads only the entries it wrote itself
  partial_dots(n, V, nv, w, partial, sh);
  if (arrive_last(ticket)) finish_sums(partial, nv, h2, ticket);
}

// w -= V[0:nv] h2; column j = nv-1 of the Hessenberg matrix is h1 + h2 and ||w||; the last CTA
// applies the previous Givens rotations to it, makes the new one, updates g and the flags.
// state: [0] target (absolute), [1] beta, [2] ||F||, [3] 1/h_{j+1,j}
// flags: [0] done, [1] columns in this cycle, [2] status
__global__ void __launch_bounds__(kRedThreads) cgs_update_norm_kernel(
    size_t n, const double* __restrict__ V, int nv, double* __restrict__ w,
    const double* __restrict__ h1, const double* __restrict__ h2, double* __restrict__ partial,
    unsigned int* ticket, double* __restrict__ Hs, int ldh, double* __restrict__ cs,
    double* __restrict__ sn, double* __restrict__ g, double* __restrict__ state,
    int* __restrict__ flags, int last_col) {
  if (flags[0]) return;
  __shared__ double sh[32];
  __shared__ double hs[kMaxBasis];
  for (int l = threadIdx.x; l < nv; l += blockDim.x) hs[l] = h2[l];
  __syncthreads();
  double acc = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    double v = w[i];
    for (int l = 0; l < nv; ++l) v = fma(-V[(size_t)l * n + i], hs[l], v);
    w[i] = v;
    acc = fma(v, v, acc);
  }
  double s = block_sum(acc, sh);
  if (threadIdx.x == 0) partial[(size_t)blockIdx.x * kMaxBasis] = s;
  if (!arrive_last(ticket)) return;
  __threadfence();
  if (threadIdx.x != 0) return;
  double ss = 0.0;
  for (int b = 0; b < (int)gridDim.x; ++b) ss += __ldcg(partial + (size_t)b * kMaxBasis);
  *ticket = 0u;
  const int j = nv - 1;
  double hn = sqrt(ss);
  double* col = Hs + (size_t)j * ldh;
  for (int l = 0; l <= j; ++l) col[l] = __ldcg(h1 + l) + hs[l];
  for (int i = 0; i < j; ++i) {
    double t = cs[i] * col[i] + sn[i] * col[i + 1];
    col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
    col[i] = t;
  }
  double den = hypot(col[j], hn);
  if (!isfinite(den) || !isfinite(hn)) {
    flags[2] = SG_ERR_NAN;
    flags[0] = 1;
    return;
  }
  double c = den > 0.0 ? col[j] / den : 1.0;
  double sgn = den > 0.0 ? hn / den : 0.0;
  cs[j] = c;
  sn[j] = sgn;
  col[j] = den;
  g[j + 1] = -sgn * g[j];
  g[j] = c * g[j];
  flags[1] = j + 1;
  state[3] = hn > 0.0 ? 1.0 / hn : 0.0;
  if (fabs(g[j + 1]) <= state[0] || hn == 0.0 || den == 0.0 || j == last_col) flags[0] = 1;
}

// v *= state[3]  (normalise the new basis vector)
__global__ void scale_kernel(size_t n, double* __restrict__ v, const double* __restrict__ state,
                             const int* __restrict__ flags) {
  if (flags[0]) return;
  double sc = state[3];
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    v[i] *= sc;
}

// ||r||_2 -> out
__global__ void __launch_bounds__(kRedThreads) norm_kernel(size_t n, const double* __restrict__ r,
                                                           double* __restrict__ partial,
                                                           unsigned int* ticket,
                                                           double* __restrict__ out) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    acc = fma(r[i], r[i], acc);
  double s = block_sum(acc, sh);
  if (threadIdx.x == 0) partial[(size_t)blockIdx.x * kMaxBasis] = s;
  if (!arrive_last(ticket)) return;
  __threadfence();
  if (threadIdx.x != 0) return;
  double ss = 0.0;
  for (int b = 0; b < (int)gridDim.x; ++b) ss += __ldcg(partial + (size_t)b * kMaxBasis);
  *ticket = 0u;
  *out = sqrt(ss);
}

// Start of a cycle: V0 = r / beta, g = (beta, 0, ...), flags cleared.
__global__ void init_cycle_kernel(size_t n, const double* __restrict__ r, double* __restrict__ V0,
                                  const double* __restrict__ state, double* __restrict__ g,
                                  int glen, int* __restrict__ flags) {
  double beta = state[1];
  double inv = beta > 0.0 ? 1.0 / beta : 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    V0[i] = r[i] * inv;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    g[0] = beta;
    for (int i = 1; i < glen; ++i) g[i] = 0.0;
    flags[0] = 0;
    flags[1] = 0;
  }
}

// y = H(0:k,0:k)^{-1} g(0:k), k = flags[1]: column-oriented back substitution by one CTA;
// after y_i is known every thread removes H(l,i) y_i from its own right-hand-side entries l < i.
__global__ void __launch_bounds__(1024) backsolve_kernel(const double* __restrict__ Hs, int ldh,
                                                         const double* __restrict__ g,
                                                         double* __restrict__ y,
                                                         const int* __restrict__ flags) {
  __shared__ double rhs[kMaxBasis];
  __shared__ double yi;
  const int k = flags[1];
  for (int l = threadIdx.x; l < k; l += blockDim.x) rhs[l] = g[l];
  __syncthreads();
  for (int i = k - 1; i >= 0; --i) {
    const double* col = Hs + (size_t)i * ldh;
    if (threadIdx.x == 0) {
      yi = rhs[i] / col[i];
      y[i] = yi;
    }
    __syncthreads();
    const double v = yi;
    for (int l = threadIdx.x; l < i; l += blockDim.x) rhs[l] -= col[l] * v;
    __syncthreads();
  }
}

// x += sum_{l < k} Z_l y_l  (Z rows FP64 or FP32)
template <typename TZ>
__global__ void update_x_kernel(size_t n, const TZ* __restrict__ Z, const double* __restrict__ y,
                                const int* __restrict__ flags, double* __restrict__ x) {
  __shared__ double ys[kMaxBasis];
  int k = flags[1];
  for (int l = threadIdx.x; l < k; l += blockDim.x) ys[l] = y[l];
  __syncthreads();
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    double v = x[i];
    for (int l = 0; l < k; ++l) v = fma((double)Z[(size_t)l * n + i], ys[l], v);
    x[i] = v;
  }
}

// FP64 -> FP32 copy that honours the cycle flag
__global__ void to_f32_kernel(size_t n, const double* __restrict__ src, float* __restrict__ dst,
                              const int* __restrict__ flags) {
  if (flags != nullptr && flags[0]) return;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    dst[i] = (float)src[i];
}
__global__ void to_f64_kernel(size_t n, const float* __restrict__ src, double* __restrict__ dst,
                              const int* __restrict__ flags) {
  if (flags != nullptr && flags[0]) return;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    dst[i] = (double)src[i];
}

// *flag = 0 if any of x[0..n) is nonzero (the caller sets it nonzero beforehand).
__global__ void any_nonzero_kernel(size_t n, const double* __restrict__ x, int* __restrict__ flag) {
  bool nz = false;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n && !nz;
       i += (size_t)gridDim.x * blockDim.x)
    nz = x[i] != 0.0;
  if (__syncthreads_or(nz) && threadIdx.x == 0) *flag = 0;
}

}  // namespace

// ------------------------------------------------------------------ launchers used by the driver

int k_zero_flag(System& s, size_t n, const double* x, int* flag, cudaStream_t st) {
  TimeScope ts(s.timer, K_OTHER, st);
  SG_CUDA(cudaMemsetAsync(flag, 1, sizeof(int), st));
  any_nonzero_kernel<<<kRedBlocks, kRedThreads, 0, st>>>(n, x, flag);
  return check_launch("any_nonzero");
}

int k_norm(System& s, size_t n, const double* r, double* out, cudaStream_t st) {
  TimeScope ts(s.timer, K_OTHER, st);
  norm_kernel<<<kRedBlocks, kRedThreads, 0, st>>>(n, r, s.red.p, s.ticket.p, out);
  return check_launch("norm");
}

int k_init_cycle(System& s, size_t n, const double* r, cudaStream_t st) {
  TimeScope ts(s.timer, K_OTHER, st);
  init_cycle_kernel<<<kRedBlocks, kRedThreads, 0, st>>>(n, r, s.V.p, s.scal.p, s.g.p, s.m + 1,
                                                        s.flags.p);
  return check_launch("init_cycle");
}

// CGS2 on the new vector V[j+1] against V[0..j], Givens update, normalisation.
int k_arnoldi(System& s, size_t n, int j, int last_col, cudaStream_t st) {
  int nv = j + 1;
  double* w = s.V.p + (size_t)(j + 1) * n;
  double* h1 = s.y.p + kMaxBasis;       // scratch: two h vectors after y
  double* h2 = s.y.p + 2 * kMaxBasis;
  {
    TimeScope ts(s.timer, K_ARNOLDI, st);
    cgs_dots_kernel<<<kRedBlocks, kRedThreads, 0, st>>>(n, s.V.p, nv, w, s.red.p, s.ticket.p, h1,
                                                        s.flags.p);
  }
  SG_TRY(check_launch("cgs_dots"));
  {
  TimeScope ts(s.timer, K_ARNOLDI, st);
  cgs_update_dots_kernel<<<kRedBlocks, kRedThreads, 0, st>>>(n, s.V.p, nv, w, h1, s.red.p,
                                                             s.ticket.p, h2, s.flags.p);
  }
  SG_TRY(check_launch("cgs_update_dots"));
  {
    TimeScope ts(s.timer, K_ARNOLDI, st);
    cgs_update_norm_kernel<<<kRedBlocks, kRedThreads, 0, st>>>(
        n, s.V.p, nv, w, h1, h2, s.red.p, s.ticket.p, s.Hs.p, s.m + 1, s.cs.p, s.sn.p, s.g.p,
        s.scal.p, s.flags.p, last_col);
  }
  SG_TRY(check_launch("cgs_update_norm"));
  {
    TimeScope ts(s.timer, K_ARNOLDI, st);
    scale_kernel<<<kRedBlocks, kRedThreads, 0, st>>>(n, w, s.scal.p, s.flags.p);
  }
  return check_launch("scale");
}

int k_finish_cycle(System& s, size_t n, double* x, bool z32, cudaStream_t st) {
  TimeScope ts(s.timer, K_OTHER, st);
  backsolve_kernel<<<1, 1024, 0, st>>>(s.Hs.p, s.m + 1, s.g.p, s.y.p, s.flags.p);
  SG_TRY(check_launch("backsolve"));
  if (z32)
    update_x_kernel<float><<<kRedBlocks * 2, kRedThreads, 0, st>>>(n, s.Z32.p, s.y.p, s.flags.p, x);
  else
    update_x_kernel<double><<<kRedBlocks * 2, kRedThreads, 0, st>>>(n, s.Z.p, s.y.p, s.flags.p, x);
  return check_launch("update_x");
}

int k_to_f32(size_t n, const double* src, float* dst, const int* flags, cudaStream_t st) {
  to_f32_kernel<<<kRedBlocks * 2, kRedThreads, 0, st>>>(n, src, dst, flags);
  return check_launch("to_f32");
}
int k_to_f64(size_t n, const float* src, double* dst, const int* flags, cudaStream_t st) {
  to_f64_kernel<<<kRedBlocks * 2, kRedThreads, 0, st>>>(n, src, dst, flags);
  return check_launch("to_f64");
}

int krylov_red_blocks() { return kRedBlocks; }
int krylov_max_basis() { return kMaxBasis; }

}  // namespace sg
