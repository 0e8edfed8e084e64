// Preconditioners of the SG system.
//
//  * mean-based: Z[:,a] = ILU0(A_0)^{-1} R[:,a] for every chaos column a (block diagonal
//    I (x) A_0, the mean-based preconditioner the paper cites in Sec. 1);
//  * field split (Sec. 3, Eq. P_preconditioner): the block lower triangle of K, swept block by
//    block (Gauss-Seidel over the chaos modes), or its block diagonal (Jacobi); each diagonal
//    block K_aa approximated by its ILU(0) factors with ``inner_iters`` Richardson steps;
//  * both wrapped in ``outer_sweeps`` steps of the level solver of Eq. level_solver.
//
// The ILU(0) triangular solves are pipelined wavefronts.  With the 9-point Q1 pattern in natural
// order, row (x, y) of the lower factor depends on (x-1, y-1), (x, y-1), (x+1, y-1), (x-1, y).
// One CTA owns one chaos column; lane j of warp w owns grid row y = 32 w + j and walks it in x,
// two columns behind the lane below it: at step s it solves x = s - 2j.  The row below then
// finished x + 1 one step earlier, so inside a warp the lockstep order alone satisfies every
// dependency (a __syncwarp publishes the step's writes).  Only lane 0 depends on another warp:
// it needs column x + 1 of the last row of warp w - 1, i.e. that warp's step s + 63, which it
// reads from a progress counter in shared memory (a bounded spin: past the limit the kernel sets
// an error flag and carries on, it never hangs).  The upper factor runs the same scheme mirrored
// (rows top down, x from right to left).  No CTA-wide barrier sits inside a sweep, so each lane
// keeps the factors of its next AHEAD columns in flight in registers.
// The off-diagonal coupling of the Gauss-Seidel sweep, sum_{b<a} K_ab z_b, is pushed forward
// after each block b by a grid-wide kernel: T[k] = sum_e A[e,k] z_b[j_e] once per (row, k), then
// acc[:,a] += G_k[a,b] T[k] for every a > b.
#include "sg_internal.h"

namespace sg {

namespace {

constexpr long long kSpinLimit = 1ll << 26;   // polls of a progress counter before giving up
constexpr int kSolveThreads = 256;            // CTA size when one warp per grid row suffices

template <typename T>
__device__ __forceinline__ void cp_async_elem(T* dst, const T* src) {
  unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(sa), "l"(src), "n"(sizeof(T)));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int K>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(K)); }
__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ld.acquire.cta.shared::cta.u32 %0, [%1];\n" : "=r"(v) : "r"(a) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
  unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("st.release.cta.shared::cta.u32 [%0], %1;\n" ::"r"(a), "r"(v) : "memory");
}

// Factors are stored per factor set as 9 node-major slot arrays (slot (dy+1)*3 + (dx+1) of node
// x + m y; slot 4 holds 1/u_ii; absent neighbours 0).  Each lane copies the factors of its
// next AHEAD columns into a per-warp shared-memory ring with cp.async (loads held in registers
// would be drained by every release/acquire of the hand-off and cost an L2 round trip a step).
template <typename T, int AHEAD, bool UPPER>
__device__ __forceinline__ void pipe_sweep(T* w, T* ring, const T* __restrict__ lu, int m, int N,
                                           int* progress, int* err) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int yy = warp * 32 + lane;  // rank of this lane's row in sweep order
  const bool row_ok = yy < m;
  const int y = UPPER ? m - 1 - yy : yy;
  const int o0 = UPPER ? 1 : -m - 1, o1 = UPPER ? m - 1 : -m, o2 = UPPER ? m : -m + 1,
            o3 = UPPER ? m + 1 : -1;
  const int sbase = UPPER ? 5 : 0;
  const int nsteps = m + 62;
  T* myring = ring + (size_t)warp * AHEAD * 5 * 32 + lane;  // [d][q][lane]
  auto stage = [&](int st, int d) {
    const int xx = st - 2 * lane;
    if (row_ok && xx >= 0 && xx < m) {
      const int x = UPPER ? m - 1 - xx : xx;
      const size_t i = (size_t)x + (size_t)m * y;
      T* dst = myring + d * 5 * 32;
#pragma unroll
      for (int q = 0; q < 4; ++q) cp_async_elem(dst + q * 32, lu + (size_t)(sbase + q) * N + i);
      if (UPPER) cp_async_elem(dst + 4 * 32, lu + (size_t)4 * N + i);
    }
    cp_async_commit();
  };
#pragma unroll
  for (int d = 0; d < AHEAD; ++d) stage(d, d);
  for (int s0 = 0; s0 < nsteps; s0 += AHEAD) {
#pragma unroll
    for (int d = 0; d < AHEAD; ++d) {
      const int st = s0 + d;
      if (st < nsteps) {
        if (warp > 0) {
          const int need = min(st + 64, nsteps);
          long long spins = 0;
          while (ld_acquire(progress + warp - 1) < need) {
            if (++spins > kSpinLimit) {
              *err = 1;
              break;
            }
          }
        }
        cp_async_wait<AHEAD - 1>();
        const int xx = st - 2 * lane;
        if (row_ok && xx >= 0 && xx < m) {
          const int x = UPPER ? m - 1 - xx : xx;
          const int i = x + m * y;
          const T* f = myring + d * 5 * 32;
          T v = w[i];
          v -= f[0] * w[min(max(i + o0, 0), N - 1)];
          v -= f[32] * w[min(max(i + o1, 0), N - 1)];
          v -= f[64] * w[min(max(i + o2, 0), N - 1)];
          v -= f[96] * w[min(max(i + o3, 0), N - 1)];
          w[i] = UPPER ? v * f[128] : v;
        }
        __syncwarp();
        if (lane == 0) st_release(progress + warp, st + 1);
        stage(st + AHEAD, d);
      }
    }
  }
  cp_async_wait<0>();
}

// Both sweeps on the column in w; the first ceil(m/32) warps sweep, the others wait.
template <typename T, int AHEAD>
__device__ __forceinline__ void ilu_solve_column(T* w, T* ring, const T* __restrict__ lu, int m,
                                                 int N, int* progress, int* err) {
  const int nw = (m + 31) >> 5;
  const int warp = threadIdx.x >> 5;
  for (int q = threadIdx.x; q < nw; q += blockDim.x) progress[q] = 0;
  __syncthreads();
  if (warp < nw) pipe_sweep<T, AHEAD, false>(w, ring, lu, m, N, progress, err);
  __syncthreads();
  for (int q = threadIdx.x; q < nw; q += blockDim.x) progress[q] = 0;
  __syncthreads();
  if (warp < nw) pipe_sweep<T, AHEAD, true>(w, ring, lu, m, N, progress, err);
  __syncthreads();
}

// CTA c solves column a = a0 + c with factor set (fac_per_col ? a : 0):
//   z = ILU^{-1}(rhs), then inner-1 times z += ILU^{-1}(rhs - K_blk z), rhs = R[:,a] - acc[:,a].
template <typename T, bool SMEM, int MAXT, int AHEAD>
__global__ void __launch_bounds__(MAXT) ilu_block_solve_kernel(
    int m, int N, int P, int nnz, int a0, int fac_per_col, const T* __restrict__ lu9s,
    const int* __restrict__ rowptr, const int* __restrict__ col, const T* __restrict__ blks,
    const T* __restrict__ R, const T* __restrict__ acc, T* __restrict__ Z, T* __restrict__ wglob,
    int inner, const int* __restrict__ done, int* __restrict__ err) {
  if (done != nullptr && *done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int progress[32];
  const int a = a0 + blockIdx.x;
  const int fsel = fac_per_col ? a : 0;
  const T* lu = lu9s + (size_t)fsel * 9 * N;
  const T* blk = blks + (size_t)fsel * nnz;
  T* ring = reinterpret_cast<T*>(smem_raw);  // ceil(m/32) warps x AHEAD x 5 x 32
  T* w = SMEM ? ring + (size_t)((m + 31) >> 5) * AHEAD * 5 * 32 : wglob + (size_t)a * N;
#pragma unroll 4
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    T v = R[(size_t)i * P + a];
    if (acc != nullptr) v -= acc[(size_t)i * P + a];
    w[i] = v;
  }
  ilu_solve_column<T, AHEAD>(w, ring, lu, m, N, progress, err);
#pragma unroll 4
  for (int i = threadIdx.x; i < N; i += blockDim.x) Z[(size_t)i * P + a] = w[i];
  for (int it = 1; it < inner; ++it) {
    __syncthreads();
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
      T v = R[(size_t)i * P + a];
      if (acc != nullptr) v -= acc[(size_t)i * P + a];
      for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) v -= blk[e] * Z[(size_t)col[e] * P + a];
      w[i] = v;
    }
    ilu_solve_column<T, AHEAD>(w, ring, lu, m, N, progress, err);
    for (int i = threadIdx.x; i < N; i += blockDim.x) Z[(size_t)i * P + a] += w[i];
  }
}

constexpr int kScatterRows = 8;

// After block b of the Gauss-Seidel sweep: for every row i and every a > b,
// acc[i,a] += sum_k G_k[a,b] (A_k z_b)[i].
template <typename T, typename TV>
__global__ void __launch_bounds__(128) fs_scatter_kernel(
    int N, int P, int L, int b, const int* __restrict__ rowptr, const int* __restrict__ col,
    const TV* __restrict__ stack, const int* __restrict__ kptr, const int* __restrict__ klist,
    const int* __restrict__ eptr, const int* __restrict__ ek, const T* __restrict__ eg,
    const T* __restrict__ Z, T* __restrict__ acc, const int* __restrict__ done) {
  if (done != nullptr && *done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Ts = reinterpret_cast<T*>(smem_raw);
  const int k0 = kptr[b], klen = kptr[b + 1] - k0;
  const int r0 = blockIdx.x * kScatterRows;
  const int nr = min(kScatterRows, N - r0);
  for (int t = threadIdx.x; t < nr * klen; t += blockDim.x) {
    int rr = t / klen, kk = t - rr * klen;
    int i = r0 + rr;
    int k = klist[k0 + kk];
    T s = T(0);
    for (int e = rowptr[i]; e < rowptr[i + 1]; ++e)
      s += (T)stack[(size_t)e * L + k] * Z[(size_t)col[e] * P + b];
    Ts[rr * klen + kk] = s;
  }
  __syncthreads();
  const int na = P - 1 - b;
  const int* ep = eptr + (size_t)b * (P + 1);
  for (int t = threadIdx.x; t < nr * na; t += blockDim.x) {
    int rr = t / na, a = b + 1 + (t - rr * na);
    T s = T(0);
    for (int q = ep[a]; q < ep[a + 1]; ++q) s += eg[q] * Ts[rr * klen + ek[q]];
    acc[(size_t)(r0 + rr) * P + a] += s;
  }
}

template <typename T>
__global__ void axpy_kernel(size_t n, const T* __restrict__ x, T* __restrict__ y,
                            const int* __restrict__ done) {
  if (done != nullptr && *done) return;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (size_t)gridDim.x * blockDim.x)
    y[t] += x[t];
}

template <typename T>
struct PcBufs;
template <>
struct PcBufs<double> {
  static const double* lu9(const System& s) { return s.lu9.p; }
  static const double* blk(const System& s) { return s.blk.p; }
  static double* acc(System& s) { return s.acc.p; }
  static double* tmp(System& s) { return s.tmp.p; }
  static double* tmp2(System& s) { return s.tmp2.p; }
  static double* triw(System& s) { return s.tri_w.p; }
  static const double* eg(const System& s) { return s.gs_eg.p; }
  static bool smem(const System& s) { return s.tri_smem; }
};
template <>
struct PcBufs<float> {
  static const float* lu9(const System& s) { return s.lu9_f32.p; }
  static const float* blk(const System& s) { return s.blk_f32.p; }
  static float* acc(System& s) { return s.acc32.p; }
  static float* tmp(System& s) { return s.tmp32.p; }
  static float* tmp2(System& s) { return s.tmp232.p; }
  static float* triw(System& s) { return s.tri_w32.p; }
  static const float* eg(const System& s) { return s.gs_eg_f32.p; }
  static bool smem(const System& s) { return s.tri_smem32; }
};

template <typename T, bool SMEM, int MAXT, int AHEAD>
int launch_block_solve_t(System& s, int a0, int ncols, int fac_per_col, const T* R, const T* acc,
                         T* Z, cudaStream_t st, const int* done) {
  using B = PcBufs<T>;
  const int m = s.pat.m;
  const int threads = std::max(kSolveThreads, (m + 31) / 32 * 32);
  size_t smem = sizeof(T) * ((size_t)((m + 31) / 32) * AHEAD * 5 * 32 + (SMEM ? (size_t)s.N : 0));
  auto kern = ilu_block_solve_kernel<T, SMEM, MAXT, AHEAD>;
  SG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  TimeScope ts(s.timer, K_ILU_SOLVE, st);
  kern<<<ncols, threads, smem, st>>>(m, s.N, s.P, s.pat.nnz, a0, fac_per_col, B::lu9(s),
                                     s.rowptr.p, s.col.p, B::blk(s), R, acc, Z,
                                     SMEM ? nullptr : B::triw(s), std::max(1, s.prm.inner_iters),
                                     done, s.flags.p + 3);
  return check_launch("ilu_block_solve");
}

template <typename T>
int launch_block_solve(System& s, int a0, int ncols, int fac_per_col, const T* R, const T* acc,
                       T* Z, cudaStream_t st, const int* done) {
  using B = PcBufs<T>;
  const int m = s.pat.m;
  if (B::smem(s)) {
    if (m <= 256) return launch_block_solve_t<T, true, 256, 8>(s, a0, ncols, fac_per_col, R, acc, Z, st, done);
    if (m <= 512) return launch_block_solve_t<T, true, 512, 4>(s, a0, ncols, fac_per_col, R, acc, Z, st, done);
    return launch_block_solve_t<T, true, 1024, 2>(s, a0, ncols, fac_per_col, R, acc, Z, st, done);
  }
  if (m <= 256) return launch_block_solve_t<T, false, 256, 8>(s, a0, ncols, fac_per_col, R, acc, Z, st, done);
  if (m <= 512) return launch_block_solve_t<T, false, 512, 4>(s, a0, ncols, fac_per_col, R, acc, Z, st, done);
  return launch_block_solve_t<T, false, 1024, 2>(s, a0, ncols, fac_per_col, R, acc, Z, st, done);
}

template <typename T>
int launch_scatter(System& s, int b, const T* Z, T* acc, cudaStream_t st, const int* done);
template <>
int launch_scatter<double>(System& s, int b, const double* Z, double* acc, cudaStream_t st,
                           const int* done) {
  size_t smem = sizeof(double) * kScatterRows * std::max(1, s.gs_max_klen);
  auto kern = fs_scatter_kernel<double, double>;
  SG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int grid = (s.N + kScatterRows - 1) / kScatterRows;
  TimeScope ts(s.timer, K_GS_SCATTER, st);
  kern<<<grid, 128, smem, st>>>(s.N, s.P, s.L, b, s.rowptr.p, s.col.p, s.stack.p, s.gs_kptr.p,
                                s.gs_k.p, s.gs_eptr.p, s.gs_ea.p, s.gs_eg.p, Z, acc, done);
  return check_launch("fs_scatter");
}
template <>
int launch_scatter<float>(System& s, int b, const float* Z, float* acc, cudaStream_t st,
                          const int* done) {
  size_t smem = sizeof(float) * kScatterRows * std::max(1, s.gs_max_klen);
  int grid = (s.N + kScatterRows - 1) / kScatterRows;
  TimeScope ts(s.timer, K_GS_SCATTER, st);
  if (s.prm.precision == SG_MIXED_BF16) {
    auto kern = fs_scatter_kernel<float, __nv_bfloat16>;
    SG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<grid, 128, smem, st>>>(s.N, s.P, s.L, b, s.rowptr.p, s.col.p, s.stack_bf16.p,
                                  s.gs_kptr.p, s.gs_k.p, s.gs_eptr.p, s.gs_ea.p, s.gs_eg_f32.p, Z,
                                  acc, done);
  } else {
    auto kern = fs_scatter_kernel<float, float>;
    SG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<grid, 128, smem, st>>>(s.N, s.P, s.L, b, s.rowptr.p, s.col.p, s.stack_f32.p,
                                  s.gs_kptr.p, s.gs_k.p, s.gs_eptr.p, s.gs_ea.p, s.gs_eg_f32.p, Z,
                                  acc, done);
  }
  return check_launch("fs_scatter");
}

// One application of P^{-1} (no outer sweeps): D = P^{-1} R.
template <typename T>
int apply_once(System& s, const T* R, T* D, cudaStream_t st, const int* done) {
  using B = PcBufs<T>;
  switch (s.prm.precond) {
    case SG_PC_MEAN:
      return launch_block_solve<T>(s, 0, s.P, 0, R, nullptr, D, st, done);
    case SG_PC_FS_JACOBI:
      return launch_block_solve<T>(s, 0, s.P, 1, R, nullptr, D, st, done);
    case SG_PC_FS_GS: {
      T* acc = B::acc(s);
      SG_CUDA(cudaMemsetAsync(acc, 0, sizeof(T) * (size_t)s.N * s.P, st));
      for (int a = 0; a < s.P; ++a) {
        SG_TRY(launch_block_solve<T>(s, a, 1, 1, R, a > 0 ? acc : nullptr, D, st, done));
        if (a + 1 < s.P) SG_TRY(launch_scatter<T>(s, a, D, acc, st, done));
      }
      return SG_OK;
    }
    default: {
      SG_CUDA(cudaMemcpyAsync(D, R, sizeof(T) * (size_t)s.N * s.P, cudaMemcpyDeviceToDevice, st));
      return SG_OK;
    }
  }
}

template <typename T>
int matvec_t(const System& s, const T* X, T* Y, T alpha, const T* Bv, T beta, cudaStream_t st,
             const int* done);
template <>
int matvec_t<double>(const System& s, const double* X, double* Y, double alpha, const double* Bv,
                     double beta, cudaStream_t st, const int* done) {
  return launch_matvec_f64(s, X, Y, alpha, Bv, beta, st, done);
}
template <>
int matvec_t<float>(const System& s, const float* X, float* Y, float alpha, const float* Bv,
                    float beta, cudaStream_t st, const int* done) {
  return launch_matvec_f32(s, X, Y, alpha, Bv, beta, st, done);
}

// Eq. level_solver from zero: Z = D_0; for i >= 1: Z += P^{-1}(R - K Z).
template <typename T>
int precond_apply_t(System& s, const T* R, T* Z, cudaStream_t st, const int* done) {
  using B = PcBufs<T>;
  SG_TRY(apply_once<T>(s, R, Z, st, done));
  size_t n = (size_t)s.N * s.P;
  for (int sw = 1; sw < s.prm.outer_sweeps; ++sw) {
    SG_TRY(matvec_t<T>(s, Z, B::tmp(s), T(-1), R, T(1), st, done));
    SG_TRY(apply_once<T>(s, B::tmp(s), B::tmp2(s), st, done));
    TimeScope ts(s.timer, K_OTHER, st);
    axpy_kernel<T><<<1216, 256, 0, st>>>(n, B::tmp2(s), Z, done);
    SG_TRY(check_launch("axpy"));
  }
  return SG_OK;
}

}  // namespace

int fs_gs_apply_f64_with(System& s, const double* R, double* Z, double* acc, cudaStream_t st) {
  SG_CUDA(cudaMemsetAsync(acc, 0, sizeof(double) * (size_t)s.N * s.P, st));
  for (int a = 0; a < s.P; ++a) {
    SG_TRY(launch_block_solve<double>(s, a, 1, 1, R, a > 0 ? acc : nullptr, Z, st, nullptr));
    if (a + 1 < s.P) SG_TRY(launch_scatter<double>(s, a, Z, acc, st, nullptr));
  }
  return SG_OK;
}

int precond_apply_f64(System& s, const double* R, double* Z, cudaStream_t st, const int* done) {
  return precond_apply_t<double>(s, R, Z, st, done);
}
int precond_apply_f32(System& s, const float* R, float* Z, cudaStream_t st, const int* done) {
  return precond_apply_t<float>(s, R, Z, st, done);
}

}  // namespace sg
