// Preconditioners of the SG system.
//
//  * mean-based: Z[:,a] = ILU0(A_0)^{-1} R[:,a] for every chaos column a (block diagonal
//    I (x) A_0, the mean-based preconditioner the paper cites in Sec. 1);
//  * field split (Sec. 3, Eq. P_preconditioner): the block lower triangle of K, swept block by
//    block (Gauss-Seidel over the chaos modes), or its block diagonal (Jacobi); each diagonal
//    block K_aa approximated by its ILU(0) factors with ``inner_iters`` Richardson steps;
//  * both wrapped in ``outer_sweeps`` steps of the level solver of Eq. level_solver.
//
// The ILU(0) triangular solves run as wavefronts: rows of one level of the lower (upper) graph
// of the pattern depend only on rows of earlier levels.  One CTA owns one chaos column and walks
// all levels with a CTA barrier in between, holding the column in shared memory when it fits.
// The off-diagonal coupling of the Gauss-Seidel sweep, sum_{b<a} K_ab z_b, is pushed forward
// after each block b by a grid-wide kernel: T[k] = sum_e A[e,k] z_b[j_e] once per (row, k), then
// acc[:,a] += G_k[a,b] T[k] for every a > b.
#include "sg_internal.h"

namespace sg {

namespace {

// Wavefront schedule of the 9-point Q1 pattern in natural order: row (x, y) of the lower factor
// depends on (x-1, y-1), (x, y-1), (x+1, y-1), (x-1, y), so the rows with x + 2y = l form level l
// (3m - 2 levels); the upper factor uses the same levels in reverse.  Factors are stored per
// factor set as 9 slot arrays in level-major row order (slot (dy+1)*3 + (dx+1); slot 4 holds
// 1/u_ii; absent neighbours hold 0), so a level needs no index loads and its factors can be
// fetched one level ahead.
__device__ __forceinline__ void level_range(int l, int m, int& ylo, int& cnt) {
  ylo = max(0, (l - (m - 1) + 1) >> 1);
  int yhi = min(m - 1, l >> 1);
  cnt = yhi - ylo + 1;
}

// Factors of the next kAhead levels are copied into a shared-memory ring with cp.async while the
// current level is computed.  Ordinary loads cannot run ahead like this: the level barrier waits
// for every load the thread has in flight, so each level would pay a full L2 round trip.  Each
// thread copies and later reads only its own rows' factors, so the ring needs no barrier of its
// own; cp.async.wait_group orders the copy before the read.
#ifndef SG_TRI_AHEAD
#define SG_TRI_AHEAD 8
#endif
#ifndef SG_TRI_THREADS
#define SG_TRI_THREADS 256
#endif
constexpr int kAhead = SG_TRI_AHEAD;
constexpr int kTriThreads = SG_TRI_THREADS;

template <typename T>
__device__ __forceinline__ void cp_async_elem(T* dst, const T* src) {
  unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(sa), "l"(src), "n"(sizeof(T)));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// Copy the factors of level l (4 off-diagonal slots, plus 1/u_ii for the upper sweep) of the rows
// this thread owns into ring slot ``slot``; always commits one group (possibly empty).
template <typename T, int RPT, bool UPPER>
__device__ __forceinline__ void stage_level(T* ring, int slot, int W, int l, int nlev, int m,
                                            int N, const T* __restrict__ lu, const int* lev_off_s) {
  if (l >= 0 && l < nlev) {
    int ylo, cnt;
    level_range(l, m, ylo, cnt);
    const int base = lev_off_s[l];
    const int s0 = UPPER ? 5 : 0;
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      int t = threadIdx.x + r * blockDim.x;
      if (t < cnt) {
        T* d = ring + (size_t)slot * 5 * W + t;
#pragma unroll
        for (int q = 0; q < 4; ++q) cp_async_elem(d + q * W, lu + (size_t)(s0 + q) * N + base + t);
        if (UPPER) cp_async_elem(d + 4 * W, lu + (size_t)4 * N + base + t);
      }
    }
  }
  cp_async_commit();
}

// Barrier among the first ``nact`` threads only (the warps that own rows of some level).
#ifndef SG_TRI_NAMED_BARRIER
#define SG_TRI_NAMED_BARRIER 0
#endif
__device__ __forceinline__ void level_barrier(int nact) {
#if SG_TRI_NAMED_BARRIER
  asm volatile("bar.sync 1, %0;\n" ::"r"(nact) : "memory");
#else
  (void)nact;
  __syncthreads();
#endif
}

template <typename T, int RPT, bool UPPER>
__device__ __forceinline__ void ilu9_sweep(T* w, T* ring, int W, const T* __restrict__ lu, int m,
                                           int N, const int* lev_off_s, int nlev, int nact) {
  const int o0 = UPPER ? 1 : -m - 1, o1 = UPPER ? m - 1 : -m, o2 = UPPER ? m : -m + 1,
            o3 = UPPER ? m + 1 : -1;
  auto lev = [&](int it) { return UPPER ? nlev - 1 - it : it; };
#pragma unroll
  for (int d = 0; d < kAhead - 1; ++d)
    stage_level<T, RPT, UPPER>(ring, d, W, d < nlev ? lev(d) : -1, nlev, m, N, lu, lev_off_s);
  for (int it = 0; it < nlev; ++it) {
    int ahead = it + kAhead - 1;
    stage_level<T, RPT, UPPER>(ring, ahead % kAhead, W, ahead < nlev ? lev(ahead) : -1, nlev, m,
                               N, lu, lev_off_s);
    cp_async_wait<kAhead - 1>();
    const int l = lev(it);
    int ylo, cnt;
    level_range(l, m, ylo, cnt);
    const T* f = ring + (size_t)(it % kAhead) * 5 * W;
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      int t = threadIdx.x + r * blockDim.x;
      if (t < cnt) {
        int y = ylo + t, x = l - 2 * y;
        int i = x + m * y;
        T s = w[i];
        s -= f[t] * w[min(max(i + o0, 0), N - 1)];
        s -= f[W + t] * w[min(max(i + o1, 0), N - 1)];
        s -= f[2 * W + t] * w[min(max(i + o2, 0), N - 1)];
        s -= f[3 * W + t] * w[min(max(i + o3, 0), N - 1)];
        w[i] = UPPER ? s * f[4 * W + t] : s;
      }
    }
    level_barrier(nact);
  }
  cp_async_wait<0>();
}

// Forward and backward sweeps: the level loops run in the first nact threads.
template <typename T, int RPT>
__device__ __forceinline__ void ilu9_solve(T* w, T* ring, int W, const T* __restrict__ lu, int m,
                                           int N, const int* lev_off_s, int nlev, int nact) {
#if SG_TRI_NAMED_BARRIER
  if ((int)threadIdx.x < nact) {
    ilu9_sweep<T, RPT, false>(w, ring, W, lu, m, N, lev_off_s, nlev, nact);
    ilu9_sweep<T, RPT, true>(w, ring, W, lu, m, N, lev_off_s, nlev, nact);
  }
#else
  ilu9_sweep<T, RPT, false>(w, ring, W, lu, m, N, lev_off_s, nlev, nact);
  ilu9_sweep<T, RPT, true>(w, ring, W, lu, m, N, lev_off_s, nlev, nact);
#endif
  __syncthreads();
}

// CTA c solves column a = a0 + c with factor set (fac_per_col ? a : 0):
//   z = ILU^{-1}(rhs), then inner-1 times z += ILU^{-1}(rhs - K_blk z), rhs = R[:,a] - acc[:,a].
template <typename T, bool SMEM, int RPT>
__global__ void __launch_bounds__(kTriThreads) ilu_block_solve_kernel(
    int m, int N, int P, int nnz, int a0, int fac_per_col, const int* __restrict__ lev_off,
    int nlev, int W, int nact, const T* __restrict__ lu9s, const int* __restrict__ rowptr,
    const int* __restrict__ col, const T* __restrict__ blks, const T* __restrict__ R,
    const T* __restrict__ acc, T* __restrict__ Z, T* __restrict__ wglob, int inner,
    const int* __restrict__ done) {
  if (done != nullptr && *done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int a = a0 + blockIdx.x;
  const int fsel = fac_per_col ? a : 0;
  const T* lu = lu9s + (size_t)fsel * 9 * N;
  const T* blk = blks + (size_t)fsel * nnz;
  T* w = SMEM ? reinterpret_cast<T*>(smem_raw) : wglob + (size_t)a * N;
  T* ring = reinterpret_cast<T*>(smem_raw + (SMEM ? sizeof(T) * (size_t)N : 0));
  int* lev_s = reinterpret_cast<int*>(ring + (size_t)kAhead * 5 * W);
  for (int l = threadIdx.x; l <= nlev; l += blockDim.x) lev_s[l] = lev_off[l];
#pragma unroll 4
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    T v = R[(size_t)i * P + a];
    if (acc != nullptr) v -= acc[(size_t)i * P + a];
    w[i] = v;
  }
  __syncthreads();
  ilu9_solve<T, RPT>(w, ring, W, lu, m, N, lev_s, nlev, nact);
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
    __syncthreads();
    ilu9_solve<T, RPT>(w, ring, W, lu, m, N, lev_s, nlev, nact);
    for (int i = threadIdx.x; i < N; i += blockDim.x) Z[(size_t)i * P + a] += w[i];
  }
}

constexpr int kScatterRows = 8;

// After block b of the Gauss-Seidel sweep: for every row i and every a > b,
// acc[i,a] += sum_k G_k[a,b] (A_k z_b)[i].  The stiffness values are read from the k-major copy
// of the stack (stack_km[k*nnz + e]): the block needs only the k of its list, and consecutive
// threads take consecutive rows of one k, so each k reads one contiguous run of entries.
template <typename T, typename TV>
__global__ void __launch_bounds__(128) fs_scatter_kernel(
    int N, int P, int nnz, int b, const int* __restrict__ rowptr, const int* __restrict__ col,
    const TV* __restrict__ stack_km, const int* __restrict__ kptr, const int* __restrict__ klist,
    const int* __restrict__ eptr, const int* __restrict__ ek, const T* __restrict__ eg,
    const T* __restrict__ Z, T* __restrict__ acc, const int* __restrict__ done) {
  if (done != nullptr && *done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Ts = reinterpret_cast<T*>(smem_raw);
  const int k0 = kptr[b], klen = kptr[b + 1] - k0;
  const int r0 = blockIdx.x * kScatterRows;
  const int nr = min(kScatterRows, N - r0);
  for (int t = threadIdx.x; t < kScatterRows * klen; t += blockDim.x) {
    const int rr = t % kScatterRows, kk = t / kScatterRows;
    T s = T(0);
    if (rr < nr) {
      const int i = r0 + rr;
      const TV* ak = stack_km + (size_t)klist[k0 + kk] * nnz;
      for (int e = rowptr[i]; e < rowptr[i + 1]; ++e)
        s += (T)ak[e] * Z[(size_t)col[e] * P + b];
    }
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

template <typename T, bool SMEM, int RPT>
int launch_block_solve_t(System& s, int a0, int ncols, int fac_per_col, const T* R, const T* acc,
                         T* Z, cudaStream_t st, const int* done) {
  using B = PcBufs<T>;
  const int W = s.pat.max_width;
  const int nact = std::min(kTriThreads, (W + 31) / 32 * 32);
  size_t smem = (SMEM ? sizeof(T) * (size_t)s.N : 0) + sizeof(T) * (size_t)kAhead * 5 * W +
                sizeof(int) * (size_t)(s.nlev9 + 1);
  auto kern = ilu_block_solve_kernel<T, SMEM, RPT>;
  SG_TRY(ensure_smem((const void*)kern, smem));
  TimeScope ts(s.timer, K_ILU_SOLVE, st);
  kern<<<ncols, kTriThreads, smem, st>>>(s.pat.m, s.N, s.P, s.pat.nnz, a0, fac_per_col, s.lev9_off.p,
                                 s.nlev9, W, nact, B::lu9(s), s.rowptr.p, s.col.p, B::blk(s), R, acc, Z,
                                 SMEM ? nullptr : B::triw(s), std::max(1, s.prm.inner_iters), done);
  return check_launch("ilu_block_solve");
}

template <typename T>
int launch_block_solve(System& s, int a0, int ncols, int fac_per_col, const T* R, const T* acc,
                       T* Z, cudaStream_t st, const int* done) {
  using B = PcBufs<T>;
  int rpt = (s.pat.max_width + kTriThreads - 1) / kTriThreads;
  if (B::smem(s)) {
    if (rpt <= 1) return launch_block_solve_t<T, true, 1>(s, a0, ncols, fac_per_col, R, acc, Z, st, done);
    return launch_block_solve_t<T, true, 4>(s, a0, ncols, fac_per_col, R, acc, Z, st, done);
  }
  if (rpt <= 1) return launch_block_solve_t<T, false, 1>(s, a0, ncols, fac_per_col, R, acc, Z, st, done);
  if (rpt <= 2) return launch_block_solve_t<T, false, 2>(s, a0, ncols, fac_per_col, R, acc, Z, st, done);
  return launch_block_solve_t<T, false, 4>(s, a0, ncols, fac_per_col, R, acc, Z, st, done);
}

template <typename T>
int launch_scatter(System& s, int b, const T* Z, T* acc, cudaStream_t st, const int* done);
template <>
int launch_scatter<double>(System& s, int b, const double* Z, double* acc, cudaStream_t st,
                           const int* done) {
  size_t smem = sizeof(double) * kScatterRows * std::max(1, s.gs_max_klen);
  auto kern = fs_scatter_kernel<double, double>;
  SG_TRY(ensure_smem((const void*)kern, smem));
  int grid = (s.N + kScatterRows - 1) / kScatterRows;
  TimeScope ts(s.timer, K_GS_SCATTER, st);
  kern<<<grid, 128, smem, st>>>(s.N, s.P, s.pat.nnz, b, s.rowptr.p, s.col.p, s.stack_km.p,
                                s.gs_kptr.p, s.gs_k.p, s.gs_eptr.p, s.gs_ea.p, s.gs_eg.p, Z, acc,
                                done);
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
    SG_TRY(ensure_smem((const void*)kern, smem));
    kern<<<grid, 128, smem, st>>>(s.N, s.P, s.pat.nnz, b, s.rowptr.p, s.col.p, s.stack_km16.p,
                                  s.gs_kptr.p, s.gs_k.p, s.gs_eptr.p, s.gs_ea.p, s.gs_eg_f32.p, Z,
                                  acc, done);
  } else {
    auto kern = fs_scatter_kernel<float, float>;
    SG_TRY(ensure_smem((const void*)kern, smem));
    kern<<<grid, 128, smem, st>>>(s.N, s.P, s.pat.nnz, b, s.rowptr.p, s.col.p, s.stack_km32.p,
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
