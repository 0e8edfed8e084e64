// Device-side setup of an SG system: Gauss-point table of the KL fields, assembly of the
// stiffness stack A_q (Eq. A_q) on the shared 9-point Q1 pattern, the load vector F
// (Eq. stochastic_matrix), the diagonal blocks used by the preconditioners and their ILU(0)
// factors, and precision casts.
#include <algorithm>

#include "sg_internal.h"

namespace sg {

namespace {

// 3-point Gauss-Legendre rule on [0, 1] (reading R1 of the element quadrature).
__device__ __forceinline__ double gl_t(int i) {
  const double r = 0.5 * sqrt(0.6);
  return i == 0 ? 0.5 - r : (i == 1 ? 0.5 : 0.5 + r);
}
__device__ __forceinline__ double gl_w(int i) { return i == 1 ? 8.0 / 18.0 : 5.0 / 18.0; }

// Bilinear shape function gradients on the reference square, local nodes (0,0), (1,0), (0,1),
// (1,1).
__device__ __forceinline__ void q1_grad(int a, double xi, double eta, double& gx, double& gy) {
  switch (a) {
    case 0: gx = eta - 1.0; gy = xi - 1.0; break;
    case 1: gx = 1.0 - eta; gy = -xi; break;
    case 2: gx = -eta; gy = 1.0 - xi; break;
    default: gx = eta; gy = xi; break;
  }
}
__device__ __forceinline__ double q1_val(int a, double xi, double eta) {
  double fx = (a & 1) ? xi : 1.0 - xi;
  double fy = (a & 2) ? eta : 1.0 - eta;
  return fx * fy;
}

__device__ __forceinline__ double kl_f(double w, double nrm, double odd, double x) {
  double t = x - 0.5;
  return (odd != 0.0 ? sin(w * t) : cos(w * t)) / nrm;
}

// qp[(cell*9 + gp)*(M+1)] = exp(mu + |g|^2/2), followed by g_1..g_M at that Gauss point, where
// g_n(x) = sqrt(lambda_n) f_i(x1) f_j(x2) (Eq. aKL).
__global__ void qp_table_kernel(int n, int M, double mu, const double* __restrict__ klp,
                                double* __restrict__ qp) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  int ncell = n * n;
  if (t >= ncell * 9) return;
  int cell = t / 9, gp = t % 9;
  int ex = cell % n, ey = cell / n;
  double h = 1.0 / n;
  double x1 = (ex + gl_t(gp % 3)) * h, x2 = (ey + gl_t(gp / 3)) * h;
  double s2 = 0.0;
  double* out = qp + (size_t)t * (M + 1);
  for (int k = 0; k < M; ++k) {
    const double* d = klp + 7 * k;
    double g = d[6] * kl_f(d[0], d[1], d[2], x1) * kl_f(d[3], d[4], d[5], x2);
    out[1 + k] = g;
    s2 += g * g;
  }
  out[0] = exp(mu + 0.5 * s2);
}

// One thread per (row r, chaos index k): the 9 entries of row r of A_k, summed over the cells
// around node r and their 9 Gauss points.  a_k(x) = exp(mu + |g|^2/2) prod g_n^{k_n} / sqrt(k_n!)
// (+ a_min for k = 0).  Dirichlet rows and columns are zeroed, with 1 on the diagonal of A_0.
__global__ void assemble_kernel(int n, int M, int L, double a_min, const int* __restrict__ rowptr,
                                const int* __restrict__ col, const int* __restrict__ Jq,
                                const double* __restrict__ cfac, const double* __restrict__ qp,
                                double* __restrict__ stack) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int m = n + 1;
  long long total = (long long)m * m * L;
  if (t >= total) return;
  int k = (int)(t % L);
  int r = (int)(t / L);
  int i = r % m, j = r / m;
  int e0 = rowptr[r], ne = rowptr[r + 1] - e0;
  double vals[9];
  for (int s = 0; s < 9; ++s) vals[s] = 0.0;
  bool rbnd = (i == 0 || j == 0 || i == n || j == n);
  if (!rbnd) {
    int kk[8];
    for (int d = 0; d < M; ++d) kk[d] = Jq[k * M + d];
    double ck = cfac[k];
    for (int cy = j - 1; cy <= j; ++cy)
      for (int cx = i - 1; cx <= i; ++cx) {
        if (cx < 0 || cy < 0 || cx >= n || cy >= n) continue;
        int cell = cx + n * cy;
        int aloc = (i - cx) + 2 * (j - cy);
        for (int gp = 0; gp < 9; ++gp) {
          const double* q = qp + (size_t)(cell * 9 + gp) * (M + 1);
          double ak = q[0] * ck;
          for (int d = 0; d < M; ++d)
            for (int pw = 0; pw < kk[d]; ++pw) ak *= q[1 + d];
          if (k == 0) ak += a_min;
          double xi = gl_t(gp % 3), eta = gl_t(gp / 3);
          double wq = gl_w(gp % 3) * gl_w(gp / 3) * ak;
          double gax, gay;
          q1_grad(aloc, xi, eta, gax, gay);
          for (int b = 0; b < 4; ++b) {
            int cnode = (cx + (b & 1)) + m * (cy + (b >> 1));
            double gbx, gby;
            q1_grad(b, xi, eta, gbx, gby);
            int slot = 0;
            for (int s = 0; s < ne; ++s)
              if (col[e0 + s] == cnode) slot = s;
            vals[slot] += wq * (gax * gbx + gay * gby);
          }
        }
      }
  }
  for (int s = 0; s < ne; ++s) {
    int c = col[e0 + s];
    int ci = c % m, cj = c / m;
    bool cbnd = (ci == 0 || cj == 0 || ci == n || cj == n);
    double v = vals[s];
    if (rbnd) v = (k == 0 && c == r) ? 1.0 : 0.0;
    else if (cbnd) v = 0.0;
    stack[(size_t)(e0 + s) * L + k] = v;
  }
}

// F[r*P + 0] = sum over cells around r of f h^2 sum_gp w phi_r(gp); other modes and boundary 0.
__global__ void rhs_kernel(int n, int P, double f, double* __restrict__ F) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  int m = n + 1;
  if (r >= m * m) return;
  int i = r % m, j = r / m;
  double h = 1.0 / n;
  double v = 0.0;
  bool bnd = (i == 0 || j == 0 || i == n || j == n);
  if (!bnd) {
    for (int cy = j - 1; cy <= j; ++cy)
      for (int cx = i - 1; cx <= i; ++cx) {
        int aloc = (i - cx) + 2 * (j - cy);
        double s = 0.0;
        for (int gp = 0; gp < 9; ++gp)
          s += gl_w(gp % 3) * gl_w(gp / 3) * q1_val(aloc, gl_t(gp % 3), gl_t(gp / 3));
        v += f * h * h * s;
      }
  }
  F[(size_t)r * P] = v;
  for (int a = 1; a < P; ++a) F[(size_t)r * P + a] = 0.0;
}

// blk[f*nnz + e] = sum over (k, g) in list f of g * stack[e*L + k]
__global__ void block_values_kernel(int nnz, int L, int nfac, const int* __restrict__ lptr,
                                    const int* __restrict__ lk, const double* __restrict__ lg,
                                    const double* __restrict__ stack, double* __restrict__ blk) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)nnz * nfac) return;
  int f = (int)(t / nnz), e = (int)(t % nnz);
  double s = 0.0;
  for (int q = lptr[f]; q < lptr[f + 1]; ++q) s += lg[q] * stack[(size_t)e * L + lk[q]];
  blk[t] = s;
}

// ILU(0) in the IKJ form, natural order, one CTA per factor set: rows of one wavefront level
// only depend on rows of earlier levels, which this CTA has finished before the barrier.
__global__ void ilu0_kernel(int nnz, const int* __restrict__ rowptr, const int* __restrict__ col,
                            const int* __restrict__ diag, const int* __restrict__ lptr,
                            const int* __restrict__ lrows, int nlev, double* __restrict__ fac) {
  double* v = fac + (size_t)blockIdx.x * nnz;
  for (int l = 0; l < nlev; ++l) {
    for (int t = lptr[l] + threadIdx.x; t < lptr[l + 1]; t += blockDim.x) {
      int i = lrows[t];
      int r0 = rowptr[i], r1 = rowptr[i + 1];
      for (int kk = r0; kk < diag[i]; ++kk) {
        int k = col[kk];
        double lik = v[kk] / v[diag[k]];
        v[kk] = lik;
        for (int kj = diag[k] + 1; kj < rowptr[k + 1]; ++kj) {
          int jc = col[kj];
          for (int s = r0; s < r1; ++s)
            if (col[s] == jc) {
              v[s] -= lik * v[kj];
              break;
            }
        }
      }
    }
    __syncthreads();
  }
}

// CSR ILU(0) factors -> 9-slot level-major layout used by the wavefront solves: the unit lower
// factor in slots 0-3 and the upper factor as D^{-1} U (slot 4 holds 1 / u_ii, slots 5-8 hold
// u_ij / u_ii), so that U z = w reads z = D^{-1} w - (D^{-1} U - I) z.
__global__ void lu9_kernel(int m, int N, int nnz, int nfac, const int* __restrict__ rowptr,
                           const int* __restrict__ col, const int* __restrict__ lev_off,
                           const double* __restrict__ fac, double* __restrict__ lu9) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)N * nfac) return;
  int f = (int)(t / N), i = (int)(t % N);
  int x = i % m, y = i / m;
  int l = x + 2 * y;
  int ylo = max(0, (l - (m - 1) + 1) >> 1);
  int pos = lev_off[l] + (y - ylo);
  double dinv = 0.0;
  for (int e = rowptr[i]; e < rowptr[i + 1]; ++e)
    if (col[e] == i) dinv = 1.0 / fac[(size_t)f * nnz + e];
  for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) {
    int c = col[e];
    int dx = c % m - x, dy = c / m - y;
    int slot = (dy + 1) * 3 + (dx + 1);
    double v = fac[(size_t)f * nnz + e];
    lu9[((size_t)f * 9 + slot) * N + pos] = slot == 4 ? dinv : slot > 4 ? v * dinv : v;
  }
}

// 32 x 32 tiles through shared memory (padded against bank conflicts).
__global__ void transpose_kernel(const double* __restrict__ src, double* __restrict__ dst,
                                 size_t rows, int cols) {
  __shared__ double tile[32][33];
  size_t r0 = (size_t)blockIdx.x * 32;  // rows can exceed the grid's y limit, columns cannot
  int c0 = blockIdx.y * 32;
  for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
    size_t r = r0 + dy;
    int c = c0 + threadIdx.x;
    tile[dy][threadIdx.x] = (r < rows && c < cols) ? src[r * cols + c] : 0.0;
  }
  __syncthreads();
  for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
    int c = c0 + dy;
    size_t r = r0 + threadIdx.x;
    if (r < rows && c < cols) dst[(size_t)c * rows + r] = tile[threadIdx.x][dy];
  }
}

template <typename S, typename D>
__global__ void cast_kernel(const S* __restrict__ src, D* __restrict__ dst, size_t n) {
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (size_t)gridDim.x * blockDim.x)
    dst[t] = (D)src[t];
}
template <>
__global__ void cast_kernel<double, __nv_bfloat16>(const double* __restrict__ src,
                                                   __nv_bfloat16* __restrict__ dst, size_t n) {
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (size_t)gridDim.x * blockDim.x)
    dst[t] = __double2bfloat16(src[t]);
}

inline unsigned blocks_for(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

}  // namespace

int launch_qp_table(System& s, double* qp, cudaStream_t st) {
  std::vector<double> klp;
  for (auto& t : s.kl) {
    double d[7] = {t.fx.w, t.fx.nrm, (double)t.fx.odd, t.fy.w, t.fy.nrm, (double)t.fy.odd,
                   t.sqrt_lam};
    klp.insert(klp.end(), d, d + 7);
  }
  DBuf<double> dk;
  SG_TRY(dk.alloc(klp.size()));
  SG_TRY(dk.upload(klp, st));
  int cnt = s.n * s.n * 9;
  qp_table_kernel<<<blocks_for(cnt, 256), 256, 0, st>>>(s.n, s.M, s.prm.mu, dk.p, qp);
  int rc = check_launch("qp_table");
  cudaStreamSynchronize(st);
  dk.release();
  return rc;
}

int launch_assemble(System& s, const double* qp, cudaStream_t st) {
  std::vector<int> Jq = total_degree_set(s.M, s.prm.q);
  std::vector<double> cfac(s.L);
  for (int k = 0; k < s.L; ++k) {
    double c = 1.0;
    for (int d = 0; d < s.M; ++d) {
      double fct = 1.0;
      for (int x = 2; x <= Jq[k * s.M + d]; ++x) fct *= x;
      c /= std::sqrt(fct);
    }
    cfac[k] = c;
  }
  DBuf<int> dJ;
  DBuf<double> dc;
  SG_TRY(dJ.alloc(Jq.size()));
  SG_TRY(dJ.upload(Jq, st));
  SG_TRY(dc.alloc(cfac.size()));
  SG_TRY(dc.upload(cfac, st));
  long long total = (long long)s.N * s.L;
  assemble_kernel<<<blocks_for(total, 128), 128, 0, st>>>(s.n, s.M, s.L, s.prm.a_min, s.rowptr.p,
                                                          s.col.p, dJ.p, dc.p, qp, s.stack.p);
  int rc = check_launch("assemble");
  cudaStreamSynchronize(st);
  dJ.release();
  dc.release();
  return rc;
}

int launch_rhs(System& s, double* F, cudaStream_t st) {
  rhs_kernel<<<blocks_for(s.N, 256), 256, 0, st>>>(s.n, s.P, s.prm.f, F);
  return check_launch("rhs");
}

// Diagonal blocks: A_0 for the mean preconditioner, K_aa = sum_k G_k[a,a] A_k for field split.
int launch_block_values(System& s, cudaStream_t st) {
  std::vector<int> lptr(1, 0), lk;
  std::vector<double> lg;
  if (s.pc_fac == SG_PC_MEAN) {
    lk.push_back(0);
    lg.push_back(1.0);
    lptr.push_back(1);
  } else {
    for (int a = 0; a < s.P; ++a) {
      for (auto& t : s.triples)
        if (t.a == a && t.b == a) {
          lk.push_back(t.k);
          lg.push_back(t.g);
        }
      lptr.push_back((int)lk.size());
    }
  }
  DBuf<int> dp, dk;
  DBuf<double> dg;
  SG_TRY(dp.alloc(lptr.size()));
  SG_TRY(dp.upload(lptr, st));
  SG_TRY(dk.alloc(lk.size()));
  SG_TRY(dk.upload(lk, st));
  SG_TRY(dg.alloc(lg.size()));
  SG_TRY(dg.upload(lg, st));
  long long total = (long long)s.pat.nnz * s.nfac;
  block_values_kernel<<<blocks_for(total, 256), 256, 0, st>>>(s.pat.nnz, s.L, s.nfac, dp.p, dk.p,
                                                              dg.p, s.stack.p, s.blk.p);
  int rc = check_launch("block_values");
  cudaStreamSynchronize(st);
  dp.release();
  dk.release();
  dg.release();
  return rc;
}

int launch_ilu0(System& s, cudaStream_t st) {
  SG_CUDA(cudaMemcpyAsync(s.fac.p, s.blk.p, sizeof(double) * s.blk.n, cudaMemcpyDeviceToDevice, st));
  int nlev = (int)s.pat.lev_f_ptr.size() - 1;
  ilu0_kernel<<<s.nfac, 256, 0, st>>>(s.pat.nnz, s.rowptr.p, s.col.p, s.diag.p, s.lev_f_ptr.p,
                                      s.lev_f_rows.p, nlev, s.fac.p);
  return check_launch("ilu0");
}

int launch_lu9(System& s, cudaStream_t st) {
  const int m = s.pat.m;
  s.nlev9 = 3 * m - 2;
  std::vector<int> off(s.nlev9 + 1, 0);
  int maxw = 0;
  for (int l = 0; l < s.nlev9; ++l) {
    int ylo = std::max(0, (l - (m - 1) + 1) >> 1);
    int yhi = std::min(m - 1, l >> 1);
    int cnt = yhi - ylo + 1;
    maxw = std::max(maxw, cnt);
    off[l + 1] = off[l] + cnt;
  }
  if (off[s.nlev9] != s.N) return fail(SG_ERR_ARG, "level schedule does not cover the mesh");
  s.pat.max_width = maxw;
  SG_TRY(s.lev9_off.alloc(off.size()));
  SG_TRY(s.lev9_off.upload(off, st));
  SG_TRY(s.lu9.alloc((size_t)s.nfac * 9 * s.N));
  SG_CUDA(cudaMemsetAsync(s.lu9.p, 0, sizeof(double) * s.lu9.n, st));
  long long total = (long long)s.N * s.nfac;
  lu9_kernel<<<blocks_for(total, 256), 256, 0, st>>>(m, s.N, s.pat.nnz, s.nfac, s.rowptr.p, s.col.p,
                                                     s.lev9_off.p, s.fac.p, s.lu9.p);
  return check_launch("lu9");
}

int launch_transpose(const double* src, double* dst, size_t rows, int cols, cudaStream_t st) {
  dim3 block(32, 8), grid((unsigned)((rows + 31) / 32), (cols + 31) / 32);
  transpose_kernel<<<grid, block, 0, st>>>(src, dst, rows, cols);
  return check_launch("transpose");
}

int launch_cast_f32(const double* src, float* dst, size_t n, cudaStream_t st) {
  cast_kernel<double, float><<<1216, 256, 0, st>>>(src, dst, n);
  return check_launch("cast_f32");
}
int launch_cast_bf16(const double* src, __nv_bfloat16* dst, size_t n, cudaStream_t st) {
  cast_kernel<double, __nv_bfloat16><<<1216, 256, 0, st>>>(src, dst, n);
  return check_launch("cast_bf16");
}
int launch_cast_f64(const float* src, double* dst, size_t n, cudaStream_t st) {
  cast_kernel<float, double><<<1216, 256, 0, st>>>(src, dst, n);
  return check_launch("cast_f64");
}

}  // namespace sg
