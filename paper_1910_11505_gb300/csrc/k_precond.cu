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

template <typename T>
__device__ __forceinline__ void ilu_sweeps(T* w, const T* __restrict__ fac,
                                           const int* __restrict__ rowptr,
                                           const int* __restrict__ col,
                                           const int* __restrict__ diag,
                                           const int* __restrict__ lf_ptr,
                                           const int* __restrict__ lf_rows, int nlf,
                                           const int* __restrict__ lb_ptr,
                                           const int* __restrict__ lb_rows, int nlb) {
  for (int l = 0; l < nlf; ++l) {
    for (int t = lf_ptr[l] + threadIdx.x; t < lf_ptr[l + 1]; t += blockDim.x) {
      int i = lf_rows[t];
      T s = w[i];
      for (int e = rowptr[i]; e < diag[i]; ++e) s -= fac[e] * w[col[e]];
      w[i] = s;
    }
    __syncthreads();
  }
  for (int l = 0; l < nlb; ++l) {
    for (int t = lb_ptr[l] + threadIdx.x; t < lb_ptr[l + 1]; t += blockDim.x) {
      int i = lb_rows[t];
      int d = diag[i];
      T s = w[i];
      for (int e = d + 1; e < rowptr[i + 1]; ++e) s -= fac[e] * w[col[e]];
      w[i] = s / fac[d];
    }
    __syncthreads();
  }
}

// CTA c solves column a = a0 + c with factor set fsel = (fac_stride ? a : 0):
//   z = ILU^{-1}(rhs), then inner-1 times z += ILU^{-1}(rhs - K_blk z), rhs = R[:,a] - acc[:,a].
template <typename T, bool SMEM>
__global__ void __launch_bounds__(256) ilu_block_solve_kernel(
    int N, int P, int nnz, int a0, int fac_per_col, const int* __restrict__ rowptr,
    const int* __restrict__ col, const int* __restrict__ diag, const int* __restrict__ lf_ptr,
    const int* __restrict__ lf_rows, int nlf, const int* __restrict__ lb_ptr,
    const int* __restrict__ lb_rows, int nlb, const T* __restrict__ facs,
    const T* __restrict__ blks, const T* __restrict__ R, const T* __restrict__ acc,
    T* __restrict__ Z, T* __restrict__ wglob, int inner, const int* __restrict__ done) {
  if (done != nullptr && *done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int a = a0 + blockIdx.x;
  const size_t fo = fac_per_col ? (size_t)a * nnz : 0;
  const T* fac = facs + fo;
  const T* blk = blks + fo;
  T* w = SMEM ? reinterpret_cast<T*>(smem_raw) : wglob + (size_t)a * N;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    T v = R[(size_t)i * P + a];
    if (acc != nullptr) v -= acc[(size_t)i * P + a];
    w[i] = v;
  }
  __syncthreads();
  ilu_sweeps<T>(w, fac, rowptr, col, diag, lf_ptr, lf_rows, nlf, lb_ptr, lb_rows, nlb);
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
    ilu_sweeps<T>(w, fac, rowptr, col, diag, lf_ptr, lf_rows, nlf, lb_ptr, lb_rows, nlb);
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
  static const double* fac(const System& s) { return s.fac.p; }
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
  static const float* fac(const System& s) { return s.fac_f32.p; }
  static const float* blk(const System& s) { return s.blk_f32.p; }
  static float* acc(System& s) { return s.acc32.p; }
  static float* tmp(System& s) { return s.tmp32.p; }
  static float* tmp2(System& s) { return s.tmp232.p; }
  static float* triw(System& s) { return s.tri_w32.p; }
  static const float* eg(const System& s) { return s.gs_eg_f32.p; }
  static bool smem(const System& s) { return s.tri_smem32; }
};

template <typename T>
int launch_block_solve(System& s, int a0, int ncols, int fac_per_col, const T* R, const T* acc,
                       T* Z, cudaStream_t st, const int* done) {
  using B = PcBufs<T>;
  int nlf = (int)s.pat.lev_f_ptr.size() - 1, nlb = (int)s.pat.lev_b_ptr.size() - 1;
  int inner = std::max(1, s.prm.inner_iters);
  TimeScope ts(s.timer, K_ILU_SOLVE, st);
  if (B::smem(s)) {
    size_t smem = sizeof(T) * (size_t)s.N;
    auto kern = ilu_block_solve_kernel<T, true>;
    SG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<ncols, 256, smem, st>>>(s.N, s.P, s.pat.nnz, a0, fac_per_col, s.rowptr.p, s.col.p,
                                   s.diag.p, s.lev_f_ptr.p, s.lev_f_rows.p, nlf, s.lev_b_ptr.p,
                                   s.lev_b_rows.p, nlb, B::fac(s), B::blk(s), R, acc, Z, nullptr,
                                   inner, done);
  } else {
    ilu_block_solve_kernel<T, false><<<ncols, 256, 0, st>>>(
        s.N, s.P, s.pat.nnz, a0, fac_per_col, s.rowptr.p, s.col.p, s.diag.p, s.lev_f_ptr.p,
        s.lev_f_rows.p, nlf, s.lev_b_ptr.p, s.lev_b_rows.p, nlb, B::fac(s), B::blk(s), R, acc, Z,
        B::triw(s), inner, done);
  }
  return check_launch("ilu_block_solve");
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

int precond_apply_f64(System& s, const double* R, double* Z, cudaStream_t st, const int* done) {
  return precond_apply_t<double>(s, R, Z, st, done);
}
int precond_apply_f32(System& s, const float* R, float* Z, cudaStream_t st, const int* done) {
  return precond_apply_t<float>(s, R, Z, st, done);
}

}  // namespace sg
