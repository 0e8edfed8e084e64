// Geometric multigrid for the SG system (Sec. 3: GMRES preconditioned by a multigrid V-cycle whose
// level solver is Eq. level_solver, with a direct solve on the coarsest level; Sec. 4: the
// midpoint-refined hierarchy that starts from a 2 x 2 mesh).
//
// Every level is the same SG problem assembled on its own mesh (its own stiffness stack, ILU(0)
// smoother factors and operator tables).  The coarse space is the nested Q1 space with the zero
// Dirichlet condition, so the prolongation is bilinear interpolation from the interior coarse
// nodes and the restriction is its transpose.  Both work on N x P nodal fields, chaos index
// fastest: one thread per (node, chaos index) value, consecutive threads on consecutive values.
// The coarsest interior system (nint = (nc - 1)^2 nodes, nint P unknowns) is inverted once on the
// host at setup (Gauss-Jordan with partial pivoting in FP64) and applied as a dense product.
#include <algorithm>
#include <cmath>

#include "sg_internal.h"

namespace sg {

namespace {

// Restriction b_c = P^T r_f: coarse node (I, J) gathers the fine nodes (2I + dx, 2J + dy),
// |dx|, |dy| <= 1, with weights (1 - |dx|/2)(1 - |dy|/2); coarse boundary nodes get zero.
template <typename T>
__global__ void restrict_kernel(const T* __restrict__ rf, T* __restrict__ bc, int nc, int P,
                                const int* __restrict__ done) {
  if (done != nullptr && *done) return;
  const int mc = nc + 1, mf = 2 * nc + 1;
  const long long total = (long long)mc * mc * P;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int a = (int)(t % P);
    const int c = (int)(t / P);
    const int I = c % mc, J = c / mc;
    T v = T(0);
    if (I > 0 && J > 0 && I < nc && J < nc) {
      const int i0 = 2 * I, j0 = 2 * J;
#pragma unroll
      for (int dy = -1; dy <= 1; ++dy) {
        const T wy = dy == 0 ? T(1) : T(0.5);
        const T* row = rf + ((size_t)(j0 + dy) * mf + i0) * P + a;
        T sx = T(0.5) * row[-P] + row[0] + T(0.5) * row[P];
        v += wy * sx;
      }
    }
    bc[t] = v;
  }
}

// Prolongation added into the fine iterate: u_f += P u_c, bilinear interpolation from the
// interior coarse nodes (coarse boundary values are taken as zero).
template <typename T>
__global__ void prolong_add_kernel(const T* __restrict__ uc, T* __restrict__ uf, int nc, int P,
                                   const int* __restrict__ done) {
  if (done != nullptr && *done) return;
  const int mc = nc + 1, mf = 2 * nc + 1;
  const long long total = (long long)mf * mf * P;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int a = (int)(t % P);
    const int f = (int)(t / P);
    const int i = f % mf, j = f / mf;
    const int I0 = i >> 1, J0 = j >> 1;
    const int nx = (i & 1) ? 2 : 1, ny = (j & 1) ? 2 : 1;
    const T w = T(1) / T(nx * ny);
    T v = T(0);
    for (int dy = 0; dy < ny; ++dy)
      for (int dx = 0; dx < nx; ++dx) {
        const int I = I0 + dx, J = J0 + dy;
        if (I > 0 && J > 0 && I < nc && J < nc) v += uc[((size_t)J * mc + I) * P + a];
      }
    uf[t] += w * v;
  }
}

// Coarsest level: u = K_int^{-1} b on the interior unknowns, zero on boundary rows.  One warp per
// output unknown, lanes over the inverse's row (coalesced), a fixed-order shuffle reduction.
template <typename T>
__global__ void coarse_solve_kernel(const T* __restrict__ inv, const int* __restrict__ nodes,
                                    int nint, int N, int P, const T* __restrict__ b,
                                    T* __restrict__ u, const int* __restrict__ done) {
  if (done != nullptr && *done) return;
  const int dim = nint * P;
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  // boundary rows (and every node not in the interior list) are zero
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < (long long)N * P;
       t += (long long)gridDim.x * blockDim.x) {
    const int node = (int)(t / P);
    bool interior = false;
    for (int q = 0; q < nint; ++q) interior |= nodes[q] == node;
    if (!interior) u[t] = T(0);
  }
  for (int r = warp; r < dim; r += nwarps) {
    const T* row = inv + (size_t)r * dim;
    T s = T(0);
    for (int c = lane; c < dim; c += 32) s += row[c] * b[(size_t)nodes[c / P] * P + (c % P)];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) u[(size_t)nodes[r / P] * P + (r % P)] = s;
  }
}

int grid_for(long long total) {
  long long g = (total + 255) / 256;
  return (int)std::max(1LL, std::min(g, 152LL * 16));
}

// Gauss-Jordan inversion with partial pivoting of a dense row-major dim x dim matrix (FP64).
int invert_dense(std::vector<double>& A, int dim) {
  std::vector<double> inv((size_t)dim * dim, 0.0);
  for (int i = 0; i < dim; ++i) inv[(size_t)i * dim + i] = 1.0;
  for (int c = 0; c < dim; ++c) {
    int piv = c;
    for (int r = c + 1; r < dim; ++r)
      if (std::fabs(A[(size_t)r * dim + c]) > std::fabs(A[(size_t)piv * dim + c])) piv = r;
    if (!(std::fabs(A[(size_t)piv * dim + c]) > 0.0))
      return fail(SG_ERR_ARG, "multigrid: the coarsest SG matrix is singular");
    if (piv != c)
      for (int k = 0; k < dim; ++k) {
        std::swap(A[(size_t)piv * dim + k], A[(size_t)c * dim + k]);
        std::swap(inv[(size_t)piv * dim + k], inv[(size_t)c * dim + k]);
      }
    const double d = 1.0 / A[(size_t)c * dim + c];
    for (int k = 0; k < dim; ++k) {
      A[(size_t)c * dim + k] *= d;
      inv[(size_t)c * dim + k] *= d;
    }
    for (int r = 0; r < dim; ++r) {
      if (r == c) continue;
      const double f = A[(size_t)r * dim + c];
      if (f == 0.0) continue;
      for (int k = 0; k < dim; ++k) {
        A[(size_t)r * dim + k] -= f * A[(size_t)c * dim + k];
        inv[(size_t)r * dim + k] -= f * inv[(size_t)c * dim + k];
      }
    }
  }
  A.swap(inv);
  return SG_OK;
}

// Dense inverse of the coarsest level's interior SG matrix K[(i,a),(j,b)] = sum_k G_k[a,b] A_k[i,j]
// from its assembled stack (copied to the host).
int build_coarse_inverse(System& c, cudaStream_t st) {
  const int m = c.pat.m;
  std::vector<int> nodes, pos(c.N, -1);
  for (int y = 1; y < m - 1; ++y)
    for (int x = 1; x < m - 1; ++x) {
      pos[x + m * y] = (int)nodes.size();
      nodes.push_back(x + m * y);
    }
  c.mg_nint = (int)nodes.size();
  const int dim = c.mg_nint * c.P;
  if (dim < 1 || dim > 4096)
    return fail(SG_ERR_ARG, "multigrid: the coarsest interior system has " + std::to_string(dim) +
                                " unknowns (limit 4096); choose a smaller mg_coarse");
  std::vector<double> stack((size_t)c.pat.nnz * c.L);
  SG_CUDA(cudaStreamSynchronize(st));
  SG_CUDA(cudaMemcpy(stack.data(), c.stack.p, sizeof(double) * stack.size(), cudaMemcpyDeviceToHost));
  std::vector<double> K((size_t)dim * dim, 0.0);
  for (int ti = 0; ti < c.mg_nint; ++ti) {
    const int i = nodes[ti];
    for (int e = c.pat.rowptr[i]; e < c.pat.rowptr[i + 1]; ++e) {
      const int tj = pos[c.pat.col[e]];
      if (tj < 0) continue;  // boundary columns are zero after the Dirichlet treatment
      for (const Triple& t : c.triples)
        K[((size_t)ti * c.P + t.a) * dim + (size_t)tj * c.P + t.b] += t.g * stack[(size_t)e * c.L + t.k];
    }
  }
  SG_TRY(invert_dense(K, dim));
  SG_TRY(c.mg_nodes.alloc(nodes.size()));
  SG_TRY(c.mg_nodes.upload(nodes, st));
  SG_TRY(c.mg_inv.alloc(K.size()));
  SG_TRY(c.mg_inv.upload(K, st));
  if (c.prm.precision != SG_FP64) {
    std::vector<float> k32(K.begin(), K.end());
    SG_TRY(c.mg_inv32.alloc(k32.size()));
    SG_TRY(c.mg_inv32.upload(k32, st));
  }
  return SG_OK;
}

}  // namespace

template <typename T>
int launch_restrict(const T* rf, T* bc, int nc, int P, cudaStream_t st, const int* done,
                    Timer* timer) {
  TimeScope ts(timer, K_OTHER, st);
  restrict_kernel<T><<<grid_for((long long)(nc + 1) * (nc + 1) * P), 256, 0, st>>>(rf, bc, nc, P, done);
  return check_launch("mg_restrict");
}

template <typename T>
int launch_prolong_add(const T* uc, T* uf, int nc, int P, cudaStream_t st, const int* done,
                       Timer* timer) {
  TimeScope ts(timer, K_OTHER, st);
  const long long mf = 2 * nc + 1;
  prolong_add_kernel<T><<<grid_for(mf * mf * P), 256, 0, st>>>(uc, uf, nc, P, done);
  return check_launch("mg_prolong");
}

template <typename T>
int launch_coarse_solve(const System& c, const T* b, T* u, cudaStream_t st, const int* done) {
  const T* inv;
  if constexpr (sizeof(T) == 8) inv = c.mg_inv.p;
  else inv = c.mg_inv32.p;
  if (inv == nullptr) return fail(SG_ERR_ARG, "multigrid: no coarsest inverse in this precision");
  TimeScope ts(c.timer, K_OTHER, st);
  const int dim = c.mg_nint * c.P;
  const int grid = std::max(1, std::min(152 * 4, (dim + 7) / 8));
  coarse_solve_kernel<T><<<grid, 256, 0, st>>>(inv, c.mg_nodes.p, c.mg_nint, c.N, c.P, b, u, done);
  return check_launch("mg_coarse_solve");
}

template int launch_restrict<double>(const double*, double*, int, int, cudaStream_t, const int*, Timer*);
template int launch_restrict<float>(const float*, float*, int, int, cudaStream_t, const int*, Timer*);
template int launch_prolong_add<double>(const double*, double*, int, int, cudaStream_t, const int*, Timer*);
template int launch_prolong_add<float>(const float*, float*, int, int, cudaStream_t, const int*, Timer*);
template int launch_coarse_solve<double>(const System&, const double*, double*, cudaStream_t, const int*);
template int launch_coarse_solve<float>(const System&, const float*, float*, cudaStream_t, const int*);

// Build the coarser levels of a multigrid system: meshes n/2, n/4, ..., mg_coarse, each set up as
// its own System (same stochastic data, the smoother's factors, no Krylov workspace), the V-cycle
// vectors of every level and the dense inverse on the coarsest one.
int mg_setup_levels(System& s, cudaStream_t st) {
  const sg_params& p = s.prm;
  std::vector<int> sizes;
  for (int nl = p.n / 2; nl >= p.mg_coarse; nl /= 2) {
    sizes.push_back(nl);
    if (nl == p.mg_coarse) break;
  }
  std::reverse(sizes.begin(), sizes.end());  // coarsest first
  const bool lowp = p.precision != SG_FP64;
  for (size_t li = 0; li < sizes.size(); ++li) {
    System* c = new System();
    s.mg.push_back(c);
    c->prm = p;
    c->prm.n = sizes[li];
    c->prm.precond = li == 0 ? SG_PC_NONE : p.mg_smoother;
    c->prm.outer_sweeps = 1;
    c->prm.graphs = 0;
    c->timer = s.timer;
    SG_TRY(setup_system_public(*c, st, false));
    const size_t NP = (size_t)c->N * c->P;
    SG_TRY(c->mg_b.alloc(NP));
    SG_TRY(c->mg_u.alloc(NP));
    if (li > 0) {
      SG_TRY(c->mg_r.alloc(NP));
      SG_TRY(c->mg_d.alloc(NP));
    }
    if (lowp) {
      SG_TRY(c->mg_b32.alloc(NP));
      SG_TRY(c->mg_u32.alloc(NP));
      if (li > 0) {
        SG_TRY(c->mg_r32.alloc(NP));
        SG_TRY(c->mg_d32.alloc(NP));
      }
    }
    if (li == 0) SG_TRY(build_coarse_inverse(*c, st));
  }
  const size_t NP = (size_t)s.N * s.P;
  SG_TRY(s.mg_r.alloc(NP));
  SG_TRY(s.mg_d.alloc(NP));
  if (lowp) {
    SG_TRY(s.mg_r32.alloc(NP));
    SG_TRY(s.mg_d32.alloc(NP));
  }
  return SG_OK;
}

}  // namespace sg
