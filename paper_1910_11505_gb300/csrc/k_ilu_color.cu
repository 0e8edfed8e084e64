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

// Elements of padding after the slot arrays (lu9, gsn_cs): a bulk copy of the last column's
// array may run up to 16 bytes past its end.
constexpr size_t kColorPad = 8;
constexpr size_t kColorSmemMax = 200 * 1024;  // shared memory the one-CTA solve may take

// Shared-memory bytes that hold one 9-slot array of n nodes copied from any 16-byte-aligned
// start at or below it: the array plus up to 16 bytes either side, a multiple of 16.
__host__ __device__ constexpr size_t kColorSlotBuf(long long n, size_t elem) {
  return ((size_t)(9 * n) * elem + 32 + 15) & ~(size_t)15;
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

// Next-column coupling stencils: for every column a >= 1 and node i, slot sl of K_{a,a-1} =
// sum_k G_k[a,a-1] A_k (the G-weighted sum in the order of the next-column tables, in FP64, each
// A_k value first rounded to BF16 when the sweep couples in BF16), at the node's colour-major
// position; absent neighbours 0.
template <typename D>
__global__ void color_coupling_kernel(int m, int N, int nnz, int P, int round_bf16,
                                      const int* __restrict__ rowptr, const int* __restrict__ col,
                                      const int* __restrict__ cstart, const double* __restrict__ km,
                                      const int* __restrict__ kptr, const int* __restrict__ klist,
                                      const int* __restrict__ eptr, const int* __restrict__ ek,
                                      const double* __restrict__ eg, D* __restrict__ out) {
  const long long total = (long long)(P - 1) * N;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int a = 1 + (int)(t / N), i = (int)(t % N), b = a - 1;
    const int x = i % m, y = i / m;
    const int pos = colour_pos(x, y, m, cstart);
    D* o = out + (size_t)(a - 1) * 9 * N;
    for (int sl = 0; sl < 9; ++sl) o[(size_t)sl * N + pos] = D(0);
    const int q0 = eptr[(size_t)b * (P + 1) + a], q1 = eptr[(size_t)b * (P + 1) + a + 1];
    const int k0 = kptr[b];
    for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) {
      const int j = col[e];
      const int sl = (j / m - y + 1) * 3 + (j % m - x + 1);
      double v = 0.0;
      for (int q = q0; q < q1; ++q) {
        double av = km[(size_t)klist[k0 + ek[q]] * nnz + e];
        if (round_bf16) av = (double)__bfloat162float(__double2bfloat16(av));
        v += eg[q] * av;
      }
      o[(size_t)sl * N + pos] = (D)v;
    }
  }
}

// Node (x, y) of position p of colour C: q = p - cstart[C] splits into y = cy + 2 (q / nx),
// x = cx + 2 (q mod nx), the quotient taken in FP32 and corrected by one step (exact for
// q < 2^24, nx < 2^12).
template <int C>
__device__ __forceinline__ void colour_xy(int p, int m, const int* __restrict__ cstart, int& x, int& y) {
  constexpr int cx = C & 1, cy = C >> 1;
  const int nx = (m - cx + 1) >> 1;
  const int q = p - cstart[C];
  int r = (int)((float)q * __frcp_rn((float)nx));
  int rem = q - r * nx;
  if (rem < 0) {
    --r;
    rem += nx;
  } else if (rem >= nx) {
    ++r;
    rem -= nx;
  }
  y = cy + 2 * r;
  x = cx + 2 * rem;
}

// Colour of the neighbour (dx, dy) of a node of colour C.
__host__ __device__ constexpr int nb_colour(int C, int dx, int dy) {
  return ((C & 1) ^ (dx & 1)) + 2 * (((C >> 1) & 1) ^ (dy & 1));
}

// New value of node (x, y) (colour C, position pos) in one phase of the triangular sweeps: lower
// (w_i minus sum l_ij w_j over the lower colours; first, with ``corr``, minus the coupling
// corr[pos] = sum_j K_{a,a-1}[i, j] z_{a-1}[j] of the previous column) or upper (w_i / u_ii minus
// the scaled couplings of the higher colours).  Slots in increasing order; which slots a colour uses is fixed
// at compile time.  Neighbour indices are clamped into the mesh: an absent neighbour's slot holds
// 0, so it subtracts 0 * (a finite value).  CG reads the column at L2 (ld.global.cg: other SMs of
// the cluster wrote it).
template <typename T, int C, bool UPPER, bool CG>
__device__ __forceinline__ T color_node_value(int x, int y, int pos, int m, int N,
                                              const T* __restrict__ cf, const T* w,
                                              const T* __restrict__ corr) {
  const int i = x + m * y;
  const int xl = max(x - 1, 0), xr = min(x + 1, m - 1);
  const int yd = max(y - 1, 0) * m, yu = min(y + 1, m - 1) * m, yc = y * m;
  auto nb = [&](int dx, int dy) {
    return (dx < 0 ? xl : dx > 0 ? xr : x) + (dy < 0 ? yd : dy > 0 ? yu : yc);
  };
  T v = CG ? __ldcg(w + i) : w[i];
  if (UPPER) {
    v *= cf[(size_t)4 * N + pos];
  } else if (corr != nullptr) {
    v -= corr[pos];
  }
#pragma unroll
  for (int sl = 0; sl < 9; ++sl) {
    if (sl == 4) continue;
    const int dx = sl % 3 - 1, dy = sl / 3 - 1;
    const int cj = nb_colour(C, dx, dy);
    if (UPPER ? cj <= C : cj >= C) continue;
    const int j = nb(dx, dy);
    v -= cf[(size_t)sl * N + pos] * (CG ? __ldcg(w + j) : w[j]);
  }
  return v;
}

// One phase over the positions beg, beg + stride, ... < end of colour C, two nodes at a time:
// both nodes' loads are issued before either result is stored, so a thread waits for memory once
// per pair.  Nodes of one colour are independent, so the order of the stores does not matter.
// Z (optional, upper phases) receives the solution at column a of an N x P row-major array.
template <typename T, int C, bool UPPER, bool CG>
__device__ __forceinline__ void color_phase(int beg, int end, int stride, int m, int N, int P,
                                            int a, const int* __restrict__ cstart,
                                            const T* __restrict__ cf, T* w,
                                            const T* __restrict__ corr, T* __restrict__ Z) {
  for (int p0 = beg; p0 < end; p0 += 2 * stride) {
    const int p1 = p0 + stride;
    const bool two = p1 < end;
    int x0, y0, x1, y1;
    colour_xy<C>(p0, m, cstart, x0, y0);
    colour_xy<C>(two ? p1 : p0, m, cstart, x1, y1);
    const T v0 = color_node_value<T, C, UPPER, CG>(x0, y0, p0, m, N, cf, w, corr);
    const T v1 = two ? color_node_value<T, C, UPPER, CG>(x1, y1, p1, m, N, cf, w, corr) : T(0);
    const int i0 = x0 + m * y0, i1 = x1 + m * y1;
    w[i0] = v0;
    if (two) w[i1] = v1;
    if (UPPER && Z != nullptr) {
      Z[(size_t)i0 * P + a] = v0;
      if (two) Z[(size_t)i1 * P + a] = v1;
    }
  }
}

// Coupling of the next column for the positions beg, beg + stride, ... < end of colour C:
// corr[pos] = sum over slots of K_{a+1,a}[i, j] z_a[j] (slots in increasing order), z_a the
// completed column w; two nodes at a time as in color_phase.
template <typename T, int C, bool CG>
__device__ __forceinline__ void coupling_phase(int beg, int end, int stride, int m, int N,
                                               const int* __restrict__ cstart,
                                               const T* __restrict__ csn, const T* w,
                                               T* __restrict__ corr) {
  auto value = [&](int p) {
    int x, y;
    colour_xy<C>(p, m, cstart, x, y);
    const int xl = max(x - 1, 0), xr = min(x + 1, m - 1);
    const int yd = max(y - 1, 0) * m, yu = min(y + 1, m - 1) * m, yc = y * m;
    T s = T(0);
#pragma unroll
    for (int sl = 0; sl < 9; ++sl) {
      const int dx = sl % 3 - 1, dy = sl / 3 - 1;
      const int j = (dx < 0 ? xl : dx > 0 ? xr : x) + (dy < 0 ? yd : dy > 0 ? yu : yc);
      s += csn[(size_t)sl * N + p] * (CG ? __ldcg(w + j) : w[j]);
    }
    return s;
  };
  for (int p0 = beg; p0 < end; p0 += 2 * stride) {
    const int p1 = p0 + stride;
    const bool two = p1 < end;
    const T s0 = value(p0);
    const T s1 = two ? value(p1) : T(0);
    corr[p0] = s0;
    if (two) corr[p1] = s1;
  }
}

// The four lower phases (colours 0..3) then the four upper phases (3..0) of one column, with
// ``sync`` between phases; with ``csn``, then the next column's coupling into ``corr`` (no phase
// of this column reads corr after the last sync).
template <typename T, bool CG, typename Sync>
__device__ __forceinline__ void color_sweeps(int off, int stride, int m, int N, int P, int a,
                                             const int* __restrict__ cstart, const T* __restrict__ cf,
                                             T* w, const T* __restrict__ corr_in,
                                             const T* __restrict__ csn, T* __restrict__ corr,
                                             T* __restrict__ Z, Sync sync) {
  color_phase<T, 0, false, CG>(cstart[0] + off, cstart[1], stride, m, N, P, a, cstart, cf, w, corr_in, nullptr);
  sync();
  color_phase<T, 1, false, CG>(cstart[1] + off, cstart[2], stride, m, N, P, a, cstart, cf, w, corr_in, nullptr);
  sync();
  color_phase<T, 2, false, CG>(cstart[2] + off, cstart[3], stride, m, N, P, a, cstart, cf, w, corr_in, nullptr);
  sync();
  color_phase<T, 3, false, CG>(cstart[3] + off, cstart[4], stride, m, N, P, a, cstart, cf, w, corr_in, nullptr);
  sync();
  color_phase<T, 3, true, CG>(cstart[3] + off, cstart[4], stride, m, N, P, a, cstart, cf, w, nullptr, Z);
  sync();
  color_phase<T, 2, true, CG>(cstart[2] + off, cstart[3], stride, m, N, P, a, cstart, cf, w, nullptr, Z);
  sync();
  color_phase<T, 1, true, CG>(cstart[1] + off, cstart[2], stride, m, N, P, a, cstart, cf, w, nullptr, Z);
  sync();
  color_phase<T, 0, true, CG>(cstart[0] + off, cstart[1], stride, m, N, P, a, cstart, cf, w, nullptr, Z);
  sync();
  if (csn != nullptr) {
    coupling_phase<T, 0, CG>(cstart[0] + off, cstart[1], stride, m, N, cstart, csn, w, corr);
    coupling_phase<T, 1, CG>(cstart[1] + off, cstart[2], stride, m, N, cstart, csn, w, corr);
    coupling_phase<T, 2, CG>(cstart[2] + off, cstart[3], stride, m, N, cstart, csn, w, corr);
    coupling_phase<T, 3, CG>(cstart[3] + off, cstart[4], stride, m, N, cstart, csn, w, corr);
  }
}

// All eight phases of one column in one CTA, the column in shared memory (meshes whose column
// fits): CTA b solves column a0 + b.  The solution goes to column a of Z and, contiguous, back
// over column a of Rt (as the cluster kernel leaves it), where the coupling scatter reads it.
// A single-column launch first prefetches the column's factors (and coupling stencil) into L2, so
// only the first phase waits for HBM.
template <typename T>
__global__ void __launch_bounds__(1024) color_cta_kernel(int m, int N, int ldN, int P, int a0,
                                                        int fac_per_col, const int* __restrict__ cstart_g,
                                                        const T* __restrict__ cfs,
                                                        T* __restrict__ Rt, T* __restrict__ Z,
                                                        const int* __restrict__ done,
                                                        const T* __restrict__ cs, T* __restrict__ corr,
                                                        int stage) {
  if (done != nullptr && *done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* w = reinterpret_cast<T*>(smem_raw);
  __shared__ int cstart[5];
  const int a = a0 + blockIdx.x;
  const T* cf = cfs + (size_t)(fac_per_col ? a : 0) * 9 * N;
  T* rhs = Rt + (size_t)a * ldN;
  const T* corr_in = (cs != nullptr && a > 0) ? corr : nullptr;
  const T* csn = (cs != nullptr && a + 1 < P) ? cs + (size_t)a * 9 * N : nullptr;
  // stage >= 1: the factors (stage 2: also the coupling stencil) are copied into shared memory
  // after the column by one bulk copy each, issued before the column load so the two overlap; a
  // copy takes the 16-byte-aligned range around its array (the arrays are padded for that) and
  // the phases index from the offset.  Should the bounded wait give up, the phases read the
  // arrays in global memory instead (same values).
  __shared__ unsigned long long bar;
  unsigned char* buf = smem_raw + sizeof(T) * (size_t)ldN;
  const T* cf_s = nullptr;
  const T* cs_s = nullptr;
  if (stage >= 1) {
    if (threadIdx.x == 0) {
      mbar_init(&bar, 1);
      asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      const unsigned long long slot_bytes = sizeof(T) * 9ull * (unsigned long long)N;
      auto span = [&](const T* p, unsigned long long& lo) {
        const unsigned long long b0 = reinterpret_cast<unsigned long long>(p);
        lo = b0 & ~15ull;
        return (unsigned)(((b0 + slot_bytes + 15ull) & ~15ull) - lo);
      };
      unsigned long long lo_cf = 0, lo_cs = 0;
      const unsigned n_cf = span(cf, lo_cf);
      const unsigned n_cs = (stage >= 2 && csn != nullptr) ? span(csn, lo_cs) : 0u;
      mbar_expect_tx(&bar, n_cf + n_cs);
      bulk_g2s(buf, reinterpret_cast<const void*>(lo_cf), n_cf, &bar);
      if (n_cs) bulk_g2s(buf + kColorSlotBuf(N, sizeof(T)), reinterpret_cast<const void*>(lo_cs), n_cs, &bar);
    }
  } else if (gridDim.x == 1) {
    l2_prefetch(cf, sizeof(T) * 9 * (size_t)N, 0, 1);
    if (csn != nullptr) l2_prefetch(csn, sizeof(T) * 9 * (size_t)N, 0, 1);
  }
  if (threadIdx.x < 5) cstart[threadIdx.x] = cstart_g[threadIdx.x];
  for (int i = threadIdx.x; i < N; i += blockDim.x) w[i] = rhs[i];
  __syncthreads();
  bool staged = false;
  if (stage >= 1) {
    staged = mbar_wait_bounded(&bar, 0);
    if (staged) {
      cf_s = reinterpret_cast<const T*>(buf + (reinterpret_cast<unsigned long long>(cf) & 15ull));
      cf = cf_s;
      if (stage >= 2 && csn != nullptr) {
        cs_s = reinterpret_cast<const T*>(buf + kColorSlotBuf(N, sizeof(T)) +
                                          (reinterpret_cast<unsigned long long>(csn) & 15ull));
        csn = cs_s;
      }
    }
  }
  color_sweeps<T, false>(threadIdx.x, blockDim.x, m, N, P, a, cstart, cf, w, corr_in, csn, corr,
                         (T*)nullptr, []() { __syncthreads(); });
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    if (Z != nullptr) Z[(size_t)i * P + a] = w[i];
    rhs[i] = w[i];
  }
  if (stage >= 1 && !staged) mbar_wait_bounded(&bar, 0);  // no copy may land after the exit
}

// All eight phases of one column on a thread-block cluster of CL CTAs (grid = columns x CL): the
// column stays in global memory (L2), every CTA takes a share of each colour's nodes, and a
// cluster barrier (release / acquire at cluster scope) separates the phases.  Neighbour values
// are read at L2 (ld.global.cg) so no SM reads a stale L1 line written by another.  Each CTA of a
// single-column launch first prefetches its share of the column's factors (and coupling stencil)
// into L2.  The coupling of column a - 1, left in ``corr`` by the previous solve, is subtracted
// from each node's right-hand side in the lower phase of its colour, before the node's own
// update; after the last phase the cluster computes the coupling of column a + 1 into ``corr``.
template <typename T, int CL>
__global__ void __launch_bounds__(1024) color_cluster_kernel(
    int m, int N, int ldN, int P, int a0, int fac_per_col, const int* __restrict__ cstart_g,
    const T* __restrict__ cfs, T* __restrict__ Rt, T* __restrict__ Z, const int* __restrict__ done,
    const T* __restrict__ cs, T* __restrict__ corr) {
  if (done != nullptr && *done) return;  // uniform over the cluster: no barrier is skipped by some
  __shared__ int cstart[5];
  const int a = a0 + blockIdx.x / CL;
  const int rank = blockIdx.x % CL;
  const T* cf = cfs + (size_t)(fac_per_col ? a : 0) * 9 * N;
  T* w = Rt + (size_t)a * ldN;
  const T* corr_in = (cs != nullptr && a > 0) ? corr : nullptr;
  const T* csn = (cs != nullptr && a + 1 < P) ? cs + (size_t)a * 9 * N : nullptr;
  if (gridDim.x == CL) {
    l2_prefetch(cf, sizeof(T) * 9 * (size_t)N, rank, CL);
    if (csn != nullptr) l2_prefetch(csn, sizeof(T) * 9 * (size_t)N, rank, CL);
  }
  if (threadIdx.x < 5) cstart[threadIdx.x] = cstart_g[threadIdx.x];
  __syncthreads();
  const int stride = CL * blockDim.x;
  const int off = rank * blockDim.x + threadIdx.x;
  color_sweeps<T, true>(off, stride, m, N, P, a, cstart, cf, w, corr_in, csn, corr, Z, []() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n"
                 "barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
  });
}



// Whether clusters of 16 CTAs of 1024 threads (a non-portable size) can be scheduled on this
// device: asked once per process and kernel; on any failure the answer is no.
template <typename T>
bool cluster16_ok() {
  static int ok = -1;
  if (ok < 0) {
    ok = 0;
    auto kern = color_cluster_kernel<T, 16>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(16, 1, 1);
      cfg.blockDim = dim3(1024, 1, 1);
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = 16;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      int nclusters = 0;
      if (cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg) == cudaSuccess && nclusters >= 2)
        ok = 1;
    }
    cudaGetLastError();
  }
  return ok == 1;
}

template <typename T, int CL>
int launch_cluster(System& s, int a0, int ncols, int fac_per_col, const T* lu, T* Rt, T* Z,
                   cudaStream_t st, const int* done, const T* cs, T* corr) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(ncols * CL), 1, 1);
  cfg.blockDim = dim3(1024, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributePriority;
  attr[1].val.priority = s.prio_hi;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  TimeScope ts(s.timer, K_ILU_SOLVE, st);
  SG_CUDA(cudaLaunchKernelEx(&cfg, color_cluster_kernel<T, CL>, s.pat.m, s.N, s.ldN, s.P, a0,
                             fac_per_col, (const int*)s.cstart.p, lu, Rt, Z, done, cs, corr));
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
  SG_TRY(s.lu9.alloc((size_t)s.nfac * 9 * s.N + kColorPad));
  const long long total = (long long)s.N * s.nfac;
  const int grid = (int)std::max(1LL, std::min((total + 255) / 256, 152LL * 32));
  color_slots_kernel<<<grid, 256, 0, st>>>(m, s.N, s.pat.nnz, s.nfac, s.rowptr.p, s.col.p,
                                           s.cstart.p, s.fac.p, s.lu9.p);
  return check_launch("color_slots");
}

// Block solves of columns a0 .. a0 + ncols - 1 from Rt into Z (colour-ordered factors).
template <typename T>
int launch_color_solve(System& s, int a0, int ncols, int fac_per_col, const T* lu, T* Rt, T* Z,
                       cudaStream_t st, const int* done, const T* cs, T* corr) {
  if (cs != nullptr && (ncols != 1 || corr == nullptr))
    return fail(SG_ERR_ARG, "four-colour solve: the coupled form takes one column and a buffer");
  const int m = s.pat.m;
  // a cluster of CTAs once one CTA would hold more than ~2048 nodes per colour (two per thread);
  // one CTA with the column in shared memory below that.  A single-column solve with more than
  // 16384 nodes per colour takes a cluster of 16 where the device schedules one.
  const int per_colour = (s.N + 3) / 4;
  if (per_colour > 2048) {
    if (per_colour > 8 * 2048 && ncols == 1 && cluster16_ok<T>())
      return launch_cluster<T, 16>(s, a0, ncols, fac_per_col, lu, Rt, Z, st, done, cs, corr);
    if (per_colour > 4 * 2048)
      return launch_cluster<T, 8>(s, a0, ncols, fac_per_col, lu, Rt, Z, st, done, cs, corr);
    if (per_colour > 2 * 2048)
      return launch_cluster<T, 4>(s, a0, ncols, fac_per_col, lu, Rt, Z, st, done, cs, corr);
    return launch_cluster<T, 2>(s, a0, ncols, fac_per_col, lu, Rt, Z, st, done, cs, corr);
  }
  {
    // shared memory: the column, then the factors and the coupling stencil where they fit
    int stage = 0;
    size_t smem = sizeof(T) * (size_t)s.ldN;
    const size_t slots = kColorSlotBuf(s.N, sizeof(T));
    if (smem + slots <= kColorSmemMax) {
      stage = 1;
      smem += slots;
      if (cs != nullptr && smem + slots <= kColorSmemMax) {
        stage = 2;
        smem += slots;
      }
    }
    auto kern = color_cta_kernel<T>;
    SG_TRY(ensure_smem((const void*)kern, smem));
    TimeScope ts(s.timer, K_ILU_SOLVE, st);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)ncols, 1, 1);
    cfg.blockDim = dim3(1024, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributePriority;
    attr[0].val.priority = s.prio_hi;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    SG_CUDA(cudaLaunchKernelEx(&cfg, kern, m, s.N, s.ldN, s.P, a0, fac_per_col,
                               (const int*)s.cstart.p, lu, Rt, Z, done, cs, corr, stage));
    return check_launch("color_cta");
  }
  return fail(SG_ERR_ARG, "four-colour block solve: column larger than shared memory");
}

template int launch_color_solve<double>(System&, int, int, int, const double*, double*, double*,
                                        cudaStream_t, const int*, const double*, double*);
template int launch_color_solve<float>(System&, int, int, int, const float*, float*, float*,
                                       cudaStream_t, const int*, const float*, float*);

int launch_color_coupling(System& s, cudaStream_t st) {
  if (s.P < 2) return SG_OK;
  if (s.stack_km.p == nullptr) return fail(SG_ERR_ARG, "coupling stencils: no FP64 k-major stack");
  const size_t n = (size_t)(s.P - 1) * 9 * s.N;
  const long long total = (long long)(s.P - 1) * s.N;
  const int grid = (int)std::max(1LL, std::min((total + 255) / 256, 152LL * 32));
  const bool lowp = s.prm.precision != SG_FP64;
  const int round_bf16 = lowp && (s.prm.precision == SG_MIXED_BF16 || s.prm.coupling_bf16) ? 1 : 0;
  if (lowp) {
    SG_TRY(s.gsn_corr32.alloc((size_t)s.N));
    SG_TRY(s.gsn_cs32.alloc(n + kColorPad));
    color_coupling_kernel<float><<<grid, 256, 0, st>>>(
        s.pat.m, s.N, s.pat.nnz, s.P, round_bf16, s.rowptr.p, s.col.p, s.cstart.p, s.stack_km.p,
        s.gsn_kptr.p, s.gsn_k.p, s.gsn_eptr.p, s.gsn_ea.p, s.gsn_eg.p, s.gsn_cs32.p);
  } else {
    SG_TRY(s.gsn_corr.alloc((size_t)s.N));
    SG_TRY(s.gsn_cs.alloc(n + kColorPad));
    color_coupling_kernel<double><<<grid, 256, 0, st>>>(
        s.pat.m, s.N, s.pat.nnz, s.P, 0, s.rowptr.p, s.col.p, s.cstart.p, s.stack_km.p,
        s.gsn_kptr.p, s.gsn_k.p, s.gsn_eptr.p, s.gsn_ea.p, s.gsn_eg.p, s.gsn_cs.p);
  }
  return check_launch("color_coupling");
}

}  // namespace sg
