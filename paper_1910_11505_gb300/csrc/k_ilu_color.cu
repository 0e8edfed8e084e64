// ILU(0) in the four-colour ordering (colour (x mod 2) + 2 (y mod 2) of the mesh node, colours in
// turn, natural order inside a colour).  No two nodes of one colour share a 9-point stencil, so
// the factorisation and both triangular sweeps proceed one colour at a time with every node of
// the colour independent: 4 dependent phases per sweep instead of the ~3m wavefront levels of
// the natural ordering, each phase a fully parallel pass.
//
// Factor layout per factor set: 9 slot arrays of N values in colour-major node order (slot
// (dy+1)*3 + (dx+1) for the neighbour at (x+dx, y+dy), absent neighbours 0): slots whose neighbour
// has a lower colour hold the unit lower factor l_ij, slots of a higher colour hold u_ij / u_ii,
// slot 4 holds 1 / u_ii.
#include "sg_internal.h"

namespace sg {

namespace {

__device__ __forceinline__ int node_colour(int x, int y) { return (x & 1) + 2 * (y & 1); }

// Position of node (x, y) in the colour-major order of an m x m grid.
__device__ __forceinline__ int colour_pos(int x, int y, int m, const int* __restrict__ cstart) {
  const int cx = x & 1, cy = y & 1;
  const int nx = (m - cx + 1) >> 1;  // nodes of this x parity on a line
  return cstart[cx + 2 * cy] + ((y - cy) >> 1) * nx + ((x - cx) >> 1);
}

// Node of position p of colour c.
__device__ __forceinline__ int colour_node(int c, int p, int m, const int* __restrict__ cstart) {
  const int cx = c & 1, cy = c >> 1;
  const int nx = (m - cx + 1) >> 1;
  const int q = p - cstart[c];
  const int y = cy + 2 * (q / nx), x = cx + 2 * (q % nx);
  return x + m * y;
}

// One colour of the IKJ factorisation for every factor set: row i (colour c) takes, in increasing
// colour-major position, each neighbour k of a lower colour: l_ik = a_ik / u_kk, then
// a_ij -= l_ik u_kj for every j after k in that order present in both rows.  Rows of lower
// colours are final when this colour runs.
__global__ void color_ilu0_kernel(int m, int nnz, int nfac, int c, const int* __restrict__ rowptr,
                                  const int* __restrict__ col, const int* __restrict__ diag,
                                  const int* __restrict__ cstart, double* __restrict__ fac) {
  const int ncol = cstart[c + 1] - cstart[c];
  const long long total = (long long)ncol * nfac;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int f = (int)(t / ncol);
    const int i = colour_node(c, cstart[c] + (int)(t % ncol), m, cstart);
    double* v = fac + (size_t)f * nnz;
    const int r0 = rowptr[i], r1 = rowptr[i + 1];
    // lower neighbours in increasing colour-major position (at most 8: selection order)
    int done_mask = 0;
    for (int step = 0; step < 8; ++step) {
      int best = -1, bpos = 0x7fffffff;
      for (int e = r0; e < r1; ++e) {
        const int k = col[e];
        if (k == i || (done_mask >> (e - r0) & 1)) continue;
        const int kx = k % m, ky = k / m;
        if (node_colour(kx, ky) >= c) continue;
        const int pk = colour_pos(kx, ky, m, cstart);
        if (pk < bpos) {
          bpos = pk;
          best = e;
        }
      }
      if (best < 0) break;
      done_mask |= 1 << (best - r0);
      const int k = col[best];
      const double lik = v[best] / v[diag[k]];
      v[best] = lik;
      // row k's entries after k in colour-major order
      for (int kj = rowptr[k]; kj < rowptr[k + 1]; ++kj) {
        const int j = col[kj];
        if (j == k) continue;
        const int jx = j % m, jy = j / m;
        if (colour_pos(jx, jy, m, cstart) <= bpos) continue;
        for (int s = r0; s < r1; ++s)
          if (col[s] == j) {
            v[s] -= lik * v[kj];
            break;
          }
      }
    }
  }
}

// CSR factors -> colour-major 9-slot layout (lower colours: l_ij; higher colours: u_ij / u_ii;
// slot 4: 1 / u_ii).
__global__ void color_slots_kernel(int m, int N, int nnz, int nfac, const int* __restrict__ rowptr,
                                   const int* __restrict__ col, const int* __restrict__ cstart,
                                   const double* __restrict__ fac, double* __restrict__ cf) {
  const long long total = (long long)N * nfac;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int f = (int)(t / N), i = (int)(t % N);
    const int x = i % m, y = i / m, c = node_colour(x, y);
    const int pos = colour_pos(x, y, m, cstart);
    const double* v = fac + (size_t)f * nnz;
    double* out = cf + (size_t)f * 9 * N;
    double dinv = 0.0;
    for (int e = rowptr[i]; e < rowptr[i + 1]; ++e)
      if (col[e] == i) dinv = 1.0 / v[e];
    for (int sl = 0; sl < 9; ++sl) out[(size_t)sl * N + pos] = 0.0;
    out[(size_t)4 * N + pos] = dinv;
    for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) {
      const int j = col[e];
      if (j == i) continue;
      const int jx = j % m, jy = j / m;
      const int sl = (jy - y + 1) * 3 + (jx - x + 1);
      out[(size_t)sl * N + pos] = node_colour(jx, jy) < c ? v[e] : v[e] * dinv;
    }
  }
}

// One phase of the triangular sweeps for ncols columns: lower (w_i -= sum l_ij w_j over lower
// colours) or upper (w_i = (w_i - sum over higher colours) / u_ii, i.e. w_i / u_ii minus the scaled
// couplings), colour c, in place on the column; the upper phases also store the result into Z.
template <typename T, bool UPPER>
__device__ __forceinline__ void color_phase_node(int pos, int i, int m, int N, const T* __restrict__ cf,
                                                 T* __restrict__ w) {
  const int x = i % m, y = i / m, c = node_colour(x, y);
  T v = w[i];
  if (UPPER) v *= cf[(size_t)4 * N + pos];
#pragma unroll
  for (int sl = 0; sl < 9; ++sl) {
    if (sl == 4) continue;
    const int dx = sl % 3 - 1, dy = sl / 3 - 1;
    const int jx = x + dx, jy = y + dy;
    if (jx < 0 || jy < 0 || jx >= m || jy >= m) continue;
    const int cj = node_colour(jx, jy);
    if (UPPER ? cj <= c : cj >= c) continue;
    v -= cf[(size_t)sl * N + pos] * w[jx + m * jy];
  }
  w[i] = v;
}

// All eight phases of one column in one CTA, the column in shared memory (meshes whose column
// fits): CTA b solves column a0 + b.
template <typename T>
__global__ void __launch_bounds__(1024) color_cta_kernel(int m, int N, int ldN, int P, int a0,
                                                        int fac_per_col, const int* __restrict__ cstart_g,
                                                        const T* __restrict__ cfs,
                                                        const T* __restrict__ Rt, T* __restrict__ Z,
                                                        const int* __restrict__ done) {
  if (done != nullptr && *done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* w = reinterpret_cast<T*>(smem_raw);
  __shared__ int cstart[5];
  const int a = a0 + blockIdx.x;
  const T* cf = cfs + (size_t)(fac_per_col ? a : 0) * 9 * N;
  const T* rhs = Rt + (size_t)a * ldN;
  if (threadIdx.x < 5) cstart[threadIdx.x] = cstart_g[threadIdx.x];
  for (int i = threadIdx.x; i < N; i += blockDim.x) w[i] = rhs[i];
  __syncthreads();
  for (int c = 0; c < 4; ++c) {
    for (int pos = cstart[c] + threadIdx.x; pos < cstart[c + 1]; pos += blockDim.x)
      color_phase_node<T, false>(pos, colour_node(c, pos, m, cstart), m, N, cf, w);
    __syncthreads();
  }
  for (int c = 3; c >= 0; --c) {
    for (int pos = cstart[c] + threadIdx.x; pos < cstart[c + 1]; pos += blockDim.x)
      color_phase_node<T, true>(pos, colour_node(c, pos, m, cstart), m, N, cf, w);
    __syncthreads();
  }
  for (int i = threadIdx.x; i < N; i += blockDim.x) Z[(size_t)i * P + a] = w[i];
}

// All eight phases of one column on a thread-block cluster of CL CTAs (grid = columns x CL): the
// column stays in global memory (L2), every CTA takes a share of each colour's nodes, and a
// cluster barrier (release / acquire at cluster scope) separates the phases.  Neighbour values
// are read at L2 (ld.global.cg) so no SM reads a stale L1 line written by another.
template <typename T, int CL>
__global__ void __launch_bounds__(1024) color_cluster_kernel(
    int m, int N, int ldN, int P, int a0, int fac_per_col, const int* __restrict__ cstart_g,
    const T* __restrict__ cfs, T* __restrict__ Rt, T* __restrict__ Z, const int* __restrict__ done) {
  if (done != nullptr && *done) return;  // uniform over the cluster: no barrier is skipped by some
  __shared__ int cstart[5];
  const int a = a0 + blockIdx.x / CL;
  const int rank = blockIdx.x % CL;
  const T* cf = cfs + (size_t)(fac_per_col ? a : 0) * 9 * N;
  T* w = Rt + (size_t)a * ldN;
  if (threadIdx.x < 5) cstart[threadIdx.x] = cstart_g[threadIdx.x];
  __syncthreads();
  const int stride = CL * blockDim.x;
  auto phase = [&](int c, bool upper) {
    for (int pos = cstart[c] + rank * blockDim.x + threadIdx.x; pos < cstart[c + 1]; pos += stride) {
      const int i = colour_node(c, pos, m, cstart);
      const int x = i % m, y = i / m;
      T v = __ldcg(w + i);
      if (upper) v *= cf[(size_t)4 * N + pos];
#pragma unroll
      for (int sl = 0; sl < 9; ++sl) {
        if (sl == 4) continue;
        const int jx = x + sl % 3 - 1, jy = y + sl / 3 - 1;
        if (jx < 0 || jy < 0 || jx >= m || jy >= m) continue;
        const int cj = node_colour(jx, jy);
        if (upper ? cj <= c : cj >= c) continue;
        v -= cf[(size_t)sl * N + pos] * __ldcg(w + jx + m * jy);
      }
      w[i] = v;
      if (upper) Z[(size_t)i * P + a] = v;
    }
    asm volatile("barrier.cluster.arrive.release.aligned;\n"
                 "barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
  };
  for (int c = 0; c < 4; ++c) phase(c, false);
  for (int c = 3; c >= 0; --c) phase(c, true);
}

template <typename T, int CL>
int launch_cluster(System& s, int a0, int ncols, int fac_per_col, const T* lu, T* Rt, T* Z,
                   cudaStream_t st, const int* done) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(ncols * CL), 1, 1);
  cfg.blockDim = dim3(1024, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  TimeScope ts(s.timer, K_ILU_SOLVE, st);
  SG_CUDA(cudaLaunchKernelEx(&cfg, color_cluster_kernel<T, CL>, s.pat.m, s.N, s.ldN, s.P, a0,
                             fac_per_col, (const int*)s.cstart.p, lu, Rt, Z, done));
  return check_launch("color_cluster");
}

}  // namespace

// Colour offsets, the factorisation and the slot layout (FP64); the system's ILU(0) factors.
int launch_color_ilu(System& s, cudaStream_t st) {
  const int m = s.pat.m;
  std::vector<int> cs(5, 0);
  for (int c = 0; c < 4; ++c) {
    const int cx = c & 1, cy = c >> 1;
    const int nx = (m - cx + 1) / 2, ny = (m - cy + 1) / 2;
    cs[c + 1] = cs[c] + nx * ny;
  }
  SG_TRY(s.cstart.alloc(5));
  SG_TRY(s.cstart.upload(cs, st));
  SG_CUDA(cudaMemcpyAsync(s.fac.p, s.blk.p, sizeof(double) * s.blk.n, cudaMemcpyDeviceToDevice, st));
  for (int c = 1; c < 4; ++c) {  // colour 0 has no lower neighbours: its rows are already final
    const long long total = (long long)(cs[c + 1] - cs[c]) * s.nfac;
    const int grid = (int)std::max(1LL, std::min((total + 255) / 256, 152LL * 32));
    color_ilu0_kernel<<<grid, 256, 0, st>>>(m, s.pat.nnz, s.nfac, c, s.rowptr.p, s.col.p, s.diag.p,
                                            s.cstart.p, s.fac.p);
    SG_TRY(check_launch("color_ilu0"));
  }
  SG_TRY(s.lu9.alloc((size_t)s.nfac * 9 * s.N));
  const long long total = (long long)s.N * s.nfac;
  const int grid = (int)std::max(1LL, std::min((total + 255) / 256, 152LL * 32));
  color_slots_kernel<<<grid, 256, 0, st>>>(m, s.N, s.pat.nnz, s.nfac, s.rowptr.p, s.col.p,
                                           s.cstart.p, s.fac.p, s.lu9.p);
  return check_launch("color_slots");
}

// Block solves of columns a0 .. a0 + ncols - 1 from Rt into Z (colour-ordered factors).
template <typename T>
int launch_color_solve(System& s, int a0, int ncols, int fac_per_col, const T* lu, T* Rt, T* Z,
                       cudaStream_t st, const int* done) {
  const int m = s.pat.m;
  const size_t smem = sizeof(T) * (size_t)s.ldN;
  // a cluster of CTAs once one CTA would hold more than ~1024 nodes per colour; one CTA with the
  // column in shared memory below that
  const int per_colour = (s.N + 3) / 4;
  if (per_colour > 2048) {
    if (per_colour > 4 * 2048) return launch_cluster<T, 8>(s, a0, ncols, fac_per_col, lu, Rt, Z, st, done);
    if (per_colour > 2 * 2048) return launch_cluster<T, 4>(s, a0, ncols, fac_per_col, lu, Rt, Z, st, done);
    return launch_cluster<T, 2>(s, a0, ncols, fac_per_col, lu, Rt, Z, st, done);
  }
  {
    auto kern = color_cta_kernel<T>;
    SG_TRY(ensure_smem((const void*)kern, smem));
    TimeScope ts(s.timer, K_ILU_SOLVE, st);
    kern<<<ncols, 1024, smem, st>>>(m, s.N, s.ldN, s.P, a0, fac_per_col, s.cstart.p, lu, Rt, Z, done);
    return check_launch("color_cta");
  }
  return fail(SG_ERR_ARG, "four-colour block solve: column larger than shared memory");
}

template int launch_color_solve<double>(System&, int, int, int, const double*, double*, double*,
                                        cudaStream_t, const int*);
template int launch_color_solve<float>(System&, int, int, int, const float*, float*, float*,
                                       cudaStream_t, const int*);

}  // namespace sg
