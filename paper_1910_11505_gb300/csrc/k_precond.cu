// Preconditioners of the SG system.
//
//  * mean-based: Z[:,a] = ILU0(A_0)^{-1} R[:,a] for every chaos column a (block diagonal
//    I (x) A_0, the mean-based preconditioner the paper cites in Sec. 1);
//  * field split (Sec. 3, Eq. P_preconditioner): the block lower triangle of K, swept block by
//    block (Gauss-Seidel over the chaos modes), or its block diagonal (Jacobi); each diagonal
//    block K_aa approximated by its ILU(0) factors with ``inner_iters`` Richardson steps;
//  * both wrapped in ``outer_sweeps`` steps of the level solver of Eq. level_solver.
//
// The block solves read their right-hand sides from contiguous columns (rhs_t, P columns of
// stride ldN, filled from the N x P residual by a tiled transpose).  The ILU(0) triangular solves
// run as wavefronts: rows of one level of the lower (upper) graph of the pattern depend only on
// rows of earlier levels; one CTA owns one chaos column and walks all levels with a CTA barrier
// in between, keeping only a window of level rows in shared memory, so any mesh takes the same
// path.  The off-diagonal coupling of the Gauss-Seidel sweep, sum_{b<a} K_ab z_b, is subtracted
// from the later columns of rhs_t after each block b by a grid-wide kernel:
// T[k] = sum_e A[e,k] z_b[j_e] once per (row, k), then rhs_t[a] -= G_k[a,b] T[k] for a > b.
#include "sg_internal.h"

namespace sg {

namespace {

// Wavefront schedule of the 9-point Q1 pattern in natural order: row (x, y) of the lower factor
// depends on (x-1, y-1), (x, y-1), (x+1, y-1), (x-1, y), so the rows with x + 2y = l form level l;
// the upper factor uses the same levels in reverse.  Factors are stored per factor set as 9 slot
// arrays in level-major row order (slot (dy+1)*3 + (dx+1), absent neighbours 0; slot 4 holds
// 1/u_ii and the upper slots u_ij/u_ii), so a level needs no index loads and its factors can be
// fetched ahead.
//
// Only interior rows (1 <= x, y <= m-2) take part.  Dirichlet rows and columns are eliminated at
// assembly, so every block has the rows d e_i on the boundary and no coupling from an interior
// row to a boundary node, and ILU(0) keeps both (L = I and U = d there, couplings exactly 0): a
// boundary row's solve is its scaling by 1/u_ii.
//
// Two thread groups share each level.  On level l the lower factor reads two rows of level l-1
// ((x+1, y-1), (x-1, y)), one of level l-2 ((x, y-1)) and one of level l-3 ((x-1, y-1)); the
// upper factor mirrors this with (x+1, y), (x-1, y+1) | (x, y+1) | (x+1, y+1).  The critical
// group applies the two level-(l-1) couplings on level l.  The lookahead group owns level l+1,
// next in sweep order: one step before it, it forms w_i - f * z for the level-(l-2) neighbour
// (w_i / u_ii - ... in the upper sweep) and keeps it in a register; in the step itself it applies
// the remaining coupling.  So the dependent chain after each barrier is two FMAs for the critical
// group and one for the lookahead group, where one thread per row would have four (an FP64
// instruction holds its SM sub-partition for many cycles, and the groups' warps issue on
// different sub-partitions).  No thread writes a row that another reads in the same step.
__device__ __forceinline__ void interior_level(int l, int m, const int* lev_off, int& y0, int& cnt,
                                               int& pos0) {
  const int ylo = max(0, (l - (m - 1) + 1) >> 1);  // first row of the full level
  y0 = max(1, (l - (m - 2) + 1) >> 1);
  const int y1 = min(m - 2, (l - 1) >> 1);
  cnt = y1 - y0 + 1;
  pos0 = lev_off[l] + (y0 - ylo);
}

// Factors of the next kAhead levels are copied into shared-memory rings with cp.async while the
// current level is computed.  Ordinary loads cannot run ahead like this: the level barrier waits
// for every load the thread has in flight, so each level would pay a full L2 round trip.  One
// warp issues all copies and waits for them (cp.async.wait_group) before a level barrier, which
// then publishes them to the compute threads.
constexpr int kAhead = kTriAhead;
constexpr int kTriMaxThreads = 1024;

template <typename T>
__device__ __forceinline__ void cp_async_elem(T* dst, const T* src) {
  unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(sa), "l"(src), "n"(sizeof(T))
               : "memory");
}
__device__ __forceinline__ void cp_async_16(void* dst, const void* src) {
  unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// ---------------------------------------------------------------- whole column in shared memory
// (meshes whose column fits: the staging warp streams only factors)

// Interior rows of level l for the compute threads, from l alone: row of thread t, or -1.
__device__ __forceinline__ int interior_row(int l, int m, int t) {
  const int y0 = max(1, (l - (m - 2) + 1) >> 1), y1 = min(m - 2, (l - 1) >> 1);
  return t <= y1 - y0 ? l + (m - 2) * (y0 + t) : -1;  // x + m y with x = l - 2y
}

// One sweep (lower or upper) over the nl interior levels; every thread of the CTA calls it and
// passes nl + 2 barriers.  List position j is level 3 + j (lower) or 3m - 6 - j (upper).  The
// critical group (role 0) takes position j at step j; the lookahead group (role 1) works on
// position j during steps j - 3 .. j - 1.  The staging warp (role 2) copies the factors of both
// groups into the rings (kAhead x 2 x wc critical, kAhead x 3 x wc lookahead), position
// s + kAhead - 1 at step s, and before the barrier that ends step s waits until position s + 4
// has landed; the barrier then makes it visible to the compute threads, which therefore neither
// issue copies nor wait for them.
template <typename T, bool UPPER>
__device__ __forceinline__ void column_sweep(T* w, T* ring, int wc, const T* __restrict__ lu, int m,
                                           int N, const int* lev_s, int nl, int role, int t) {
  auto level = [&](int j) { return UPPER ? 3 * m - 6 - j : 3 + j; };
  auto row = [&](int j) { return j < nl ? interior_row(level(j), m, t) : -1; };
  T* cring = ring;
  T* lring = ring + (size_t)kAhead * 2 * wc;
  if (role == 2) {
    // critical: lower slots 2, 3 / upper 5, 6; lookahead: early lower 0 / upper 8, late lower 1 /
    // upper 7, and upper 1/u_ii (slot 4)
    const T* fA = lu + (size_t)(UPPER ? 5 : 2) * N;
    const T* fE = lu + (size_t)(UPPER ? 8 : 0) * N;
    const T* fL = lu + (size_t)(UPPER ? 7 : 1) * N;
    const T* fD = lu + (size_t)4 * N;
    auto stage = [&](int j) {
      if (j < nl) {
        int y0, cnt, pos0;
        interior_level(level(j), m, lev_s, y0, cnt, pos0);
        T* c = cring + (size_t)(j % kAhead) * 2 * wc;
        T* d = lring + (size_t)(j % kAhead) * 3 * wc;
        for (int r = t; r < cnt; r += 32) {
          cp_async_elem(c + r, fA + pos0 + r);
          cp_async_elem(c + wc + r, fA + N + pos0 + r);
          cp_async_elem(d + r, fE + pos0 + r);
          cp_async_elem(d + wc + r, fL + pos0 + r);
          if (UPPER) cp_async_elem(d + 2 * wc + r, fD + pos0 + r);
        }
      }
      cp_async_commit();
    };
#pragma unroll
    for (int d = 0; d < kAhead - 2; ++d) stage(d);
    cp_async_wait<kAhead - 5>();  // positions 0 .. 2 landed
    __syncthreads();
    for (int step = -1; step < nl; ++step) {
      stage(step + kAhead - 1);
      cp_async_wait<kAhead - 5>();  // positions up to step + 4 landed
      __syncthreads();
    }
    cp_async_wait<0>();
  } else if (role == 0) {
    // lower: slots 2, 3 at i - m + 1, i - 1; upper: slots 5, 6 at i + 1, i + m - 1
    const int oA = UPPER ? 1 : -m + 1, oB = UPPER ? m - 1 : -1;
    __syncthreads();
    int ci = row(0);
    for (int step = -1; step < nl; ++step) {
      if (step >= 0) {
        const int cur = ci;
        if (cur >= 0) {
          const T* f = cring + (size_t)(step % kAhead) * 2 * wc + t;
          const T fa = f[0], fb = f[wc];
          T v = w[cur];
          const T zA = w[cur + oA], zB = w[cur + oB];
          ci = row(step + 1);
          v -= fa * zA;
          v -= fb * zB;
          w[cur] = v;
        } else {
          ci = row(step + 1);
        }
      }
      __syncthreads();
    }
  } else {
    // position j in three steps, so that no step holds a dependent FP64 pair:
    //   A (step j - 3): w_i, times 1/u_ii (slot 4) in the upper sweep;
    //   B (step j - 2): minus the early coupling, slot 0 at i - m - 1 / slot 8 at i + m + 1;
    //   C (step j - 1): minus the late coupling, slot 1 at i - m / slot 7 at i + m, stored.
    const int oE = UPPER ? m + 1 : -m - 1, oL = UPPER ? m : -m;
    auto stage_a = [&](int j, int& r, T& v) {
      r = row(j);
      if (r >= 0) {
        v = w[r];
        if (UPPER) v *= lring[(size_t)(j % kAhead) * 3 * wc + 2 * wc + t];
      }
    };
    auto stage_b = [&](int j, int r, T v, int& ro, T& po, T& fo) {
      ro = r;
      if (r >= 0) {
        const T* f = lring + (size_t)(j % kAhead) * 3 * wc + t;
        po = v - f[0] * w[r + oE];
        fo = f[wc];
      }
    };
    int rb = -1, rc = -1;
    T vb = T(0), pc = T(0), fc = T(0);
    __syncthreads();
    {
      int r0;
      T v0 = T(0);
      stage_a(0, r0, v0);
      stage_b(0, r0, v0, rc, pc, fc);
      if (1 < nl) stage_a(1, rb, vb);
    }
    for (int step = -1; step < nl; ++step) {
      const int j = step + 1;
      const int cur = j < nl ? rc : -1;
      const T cpc = pc, cfc = fc;
      T zl = T(0);
      if (cur >= 0) zl = w[cur + oL];
      rc = -1;
      if (j + 1 < nl) stage_b(j + 1, rb, vb, rc, pc, fc);
      rb = -1;
      if (j + 2 < nl) stage_a(j + 2, rb, vb);
      if (cur >= 0) w[cur] = cpc - cfc * zl;
      __syncthreads();
    }
  }
}

// w <- U^{-1} L^{-1} w for one column: boundary rows by their scaling, interior rows by the two
// sweeps.  Threads [0, wc) form the critical group, [wc, 2wc) the lookahead group, the last warp
// stages the factors.
template <typename T>
__device__ __forceinline__ void column_solve(T* w, T* ring, int wc, const T* __restrict__ lu, int m,
                                           int N, const int* lev_s) {
  const int nb = 4 * (m - 1);
  for (int k = threadIdx.x; k < nb; k += blockDim.x) {
    const int side = k / (m - 1), s = k - side * (m - 1);
    const int x = side == 0 ? s : side == 1 ? m - 1 : side == 2 ? m - 1 - s : 0;
    const int y = side == 0 ? 0 : side == 1 ? s : side == 2 ? m - 1 : m - 1 - s;
    const int l = x + 2 * y, ylo = max(0, (l - (m - 1) + 1) >> 1);
    w[x + m * y] *= lu[(size_t)4 * N + lev_s[l] + (y - ylo)];
  }
  __syncthreads();
  const int nl = 3 * m - 8;
  const int tid = threadIdx.x;
  const int role = tid < wc ? 0 : tid < 2 * wc ? 1 : 2;
  const int t = tid - role * wc;
  column_sweep<T, false>(w, ring, wc, lu, m, N, lev_s, nl, role, t);
  column_sweep<T, true>(w, ring, wc, lu, m, N, lev_s, nl, role, t);
}

// CTA c solves column a = a0 + c with factor set (fac_per_col ? a : 0) and right-hand side
// rhs = Rt[a * ldN ...], holding the whole column in shared memory:  z = ILU^{-1}(rhs), then
// inner-1 times z += ILU^{-1}(rhs - K_blk z).
template <typename T>
__global__ void __launch_bounds__(kTriMaxThreads) ilu_column_kernel(
    int m, int N, int ldN, int P, int nnz, int a0, int fac_per_col, const int* __restrict__ lev_off,
    int nlev, int wc, const T* __restrict__ lu9s, const int* __restrict__ rowptr,
    const int* __restrict__ col, const T* __restrict__ blks, const T* __restrict__ Rt,
    T* __restrict__ Z, int inner, const int* __restrict__ done) {
  if (done != nullptr && *done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int a = a0 + blockIdx.x;
  const int fsel = fac_per_col ? a : 0;
  const T* lu = lu9s + (size_t)fsel * 9 * N;
  const T* blk = blks + (size_t)fsel * nnz;
  const T* rhs = Rt + (size_t)a * ldN;
  T* w = reinterpret_cast<T*>(smem_raw);
  T* ring = reinterpret_cast<T*>(smem_raw + sizeof(T) * (size_t)ldN);
  int* lev_s = reinterpret_cast<int*>(ring + (size_t)kAhead * 5 * wc);
  for (int l = threadIdx.x; l <= nlev; l += blockDim.x) lev_s[l] = lev_off[l];
  {  // the column (ldN * sizeof(T) bytes, 16-byte aligned) in one burst of copies
    const int nchunk = (int)((size_t)ldN * sizeof(T) / 16);
    for (int c = threadIdx.x; c < nchunk; c += blockDim.x)
      cp_async_16(reinterpret_cast<unsigned char*>(w) + 16 * (size_t)c,
                  reinterpret_cast<const unsigned char*>(rhs) + 16 * (size_t)c);
    cp_async_commit();
    cp_async_wait<0>();
  }
  __syncthreads();
  column_solve<T>(w, ring, wc, lu, m, N, lev_s);
#pragma unroll 4
  for (int i = threadIdx.x; i < N; i += blockDim.x) Z[(size_t)i * P + a] = w[i];
  for (int it = 1; it < inner; ++it) {
    __syncthreads();
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
      T v = rhs[i];
      for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) v -= blk[e] * Z[(size_t)col[e] * P + a];
      w[i] = v;
    }
    __syncthreads();
    column_solve<T>(w, ring, wc, lu, m, N, lev_s);
    for (int i = threadIdx.x; i < N; i += blockDim.x) Z[(size_t)i * P + a] += w[i];
  }
}

// ---------------------------------------------------------------- level window
// (larger meshes: the column stays in global memory, a window of level rows on chip)

// Row y of thread t on level l (interior rows only), or -1; the row's node is x + m y, x = l - 2y.
__device__ __forceinline__ int interior_y(int l, int m, int t) {
  const int y0 = max(1, (l - (m - 2) + 1) >> 1), y1 = min(m - 2, (l - 1) >> 1);
  return t <= y1 - y0 ? y0 + t : -1;
}

// Level window: the sweep at step s touches only list positions s-1 .. s+3 (neighbours one to
// three levels back and the lookahead's rows), so the working values live in a shared-memory
// ring of kWin level rows indexed by y (window row p & (kWin-1) holds list position p).  The
// staging threads gather the values of position s + kWin - 2 into the window at step s (ten
// steps before their first reader, which hides the strided reads' L2 latency) and write
// position s-2, whose last reader was step s-1, back to global memory; the compute threads read
// and write only the window.  Entries outside a level's interior rows hold 0 or an earlier
// level's value (their factors are exactly 0).
constexpr int kWin = kTriWin;

// One sweep (lower or upper) over the nl interior levels; every thread of the CTA calls it and
// passes nl + 4 barriers.  List position j is level 3 + j (lower) or 3m - 6 - j (upper).  The
// critical group (role 0) takes position j at step j; the lookahead group (role 1) works on
// position j during steps j - 3 .. j - 1.  The staging threads (role 2) copy, at step s, the
// factors of position s + kAhead - 1 into the rings (kAhead x 2 x wc critical, kAhead x 3 x wc
// lookahead) and the values of position s + kWin - 2 from ``src`` into the window, then wait
// until everything for positions up to s + 4 has landed (copy groups of step s - 3 and before);
// the barrier that ends step s publishes it.
// Values are read from src[i * ss]; final values of each position go to dst[i * ds] (added to it
// when ``acc``).
template <typename T, bool UPPER>
__device__ __forceinline__ void window_sweep(T* win, T* ring, int wc, const T* __restrict__ lu,
                                           int m, int N, const int* lev_s, int nl, int role, int t,
                                           const T* src, int ss, T* dst, int ds, bool acc) {
  auto level = [&](int j) { return UPPER ? 3 * m - 6 - j : 3 + j; };
  auto wrow = [&](int p) { return win + (size_t)(p & (kWin - 1)) * m; };
  const int nst = (int)blockDim.x - 2 * wc;  // staging threads
  auto ypos = [&](int j) { return j < nl ? interior_y(level(j), m, t) : -1; };
  T* cring = ring;
  T* lring = ring + (size_t)kAhead * 2 * wc;
  for (int k = threadIdx.x; k < kWin * m; k += blockDim.x) win[k] = T(0);
  __syncthreads();
  if (role == 2) {
    // critical: lower slots 2, 3 / upper 5, 6; lookahead: early lower 0 / upper 8, late lower 1 /
    // upper 7, and upper 1/u_ii (slot 4)
    const T* fA = lu + (size_t)(UPPER ? 5 : 2) * N;
    const T* fE = lu + (size_t)(UPPER ? 8 : 0) * N;
    const T* fL = lu + (size_t)(UPPER ? 7 : 1) * N;
    const T* fD = lu + (size_t)4 * N;
    auto factors = [&](int j) {
      if (j < nl) {
        int y0, cnt, pos0;
        interior_level(level(j), m, lev_s, y0, cnt, pos0);
        T* c = cring + (size_t)(j % kAhead) * 2 * wc;
        T* d = lring + (size_t)(j % kAhead) * 3 * wc;
        for (int r = t; r < cnt; r += nst) {
          cp_async_elem(c + r, fA + pos0 + r);
          cp_async_elem(c + wc + r, fA + N + pos0 + r);
          cp_async_elem(d + r, fE + pos0 + r);
          cp_async_elem(d + wc + r, fL + pos0 + r);
          if (UPPER) cp_async_elem(d + 2 * wc + r, fD + pos0 + r);
        }
      }
    };
    auto gather = [&](int j) {
      if (j < nl) {
        const int l = level(j);
        const int y0 = max(1, (l - (m - 2) + 1) >> 1), y1 = min(m - 2, (l - 1) >> 1);
        T* wr = wrow(j);
        for (int y = y0 + t; y <= y1; y += nst)
          cp_async_elem(wr + y, src + ((size_t)l + (size_t)(m - 2) * y) * ss);
      }
    };
    auto writeout = [&](int j) {
      if (j >= 0 && j < nl) {
        const int l = level(j);
        const int y0 = max(1, (l - (m - 2) + 1) >> 1), y1 = min(m - 2, (l - 1) >> 1);
        const T* wr = wrow(j);
        for (int y = y0 + t; y <= y1; y += nst) {
          T* d = dst + ((size_t)l + (size_t)(m - 2) * y) * ds;
          const T v = wr[y];
          *d = acc ? *d + v : v;
        }
      }
    };
    factors(0);
    for (int j = 0; j < kWin - 3; ++j) gather(j);
    cp_async_commit();
#pragma unroll 1
    for (int j = 1; j < kAhead - 2; ++j) {
      factors(j);
      cp_async_commit();
    }
    cp_async_wait<3>();  // positions 0 .. 2 landed
    __syncthreads();
    for (int step = -1; step < nl; ++step) {
      writeout(step - 2);
      factors(step + kAhead - 1);
      gather(step + kWin - 2);
      cp_async_commit();
      cp_async_wait<3>();  // positions up to step + 4 landed
      __syncthreads();
    }
    cp_async_wait<0>();
    writeout(nl - 2);
    writeout(nl - 1);
  } else if (role == 0) {
    // lower: slot 2 at (x+1, y-1), slot 3 at (x-1, y); upper: slot 5 at (x+1, y), slot 6 at
    // (x-1, y+1); both neighbours on the previous position
    const int dA = UPPER ? 0 : -1, dB = UPPER ? 1 : 0;
    __syncthreads();
    for (int step = -1; step < nl; ++step) {
      if (step >= 0) {
        const int y = ypos(step);
        if (y >= 0) {
          const T* f = cring + (size_t)(step % kAhead) * 2 * wc + t;
          T* cur = wrow(step);
          const T* prev = wrow(step - 1);
          const T fa = f[0], fb = f[wc];
          T v = cur[y];
          const T zA = prev[y + dA], zB = prev[y + dB];
          v -= fa * zA;
          v -= fb * zB;
          cur[y] = v;
        }
      }
      __syncthreads();
    }
  } else {
    // position j in three steps, so that no step holds a dependent FP64 pair:
    //   A (step j - 3): the row's value, times 1/u_ii (slot 4) in the upper sweep;
    //   B (step j - 2): minus the early coupling, slot 0 at (x-1, y-1) / slot 8 at (x+1, y+1),
    //                   three positions back;
    //   C (step j - 1): minus the late coupling, slot 1 at (x, y-1) / slot 7 at (x, y+1), two
    //                   positions back, stored.
    const int dE = UPPER ? 1 : -1;
    auto stage_a = [&](int j, int& y, T& v) {
      y = ypos(j);
      if (y >= 0) {
        v = wrow(j)[y];
        if (UPPER) v *= lring[(size_t)(j % kAhead) * 3 * wc + 2 * wc + t];
      }
    };
    auto stage_b = [&](int j, int y, T v, int& yo, T& po, T& fo) {
      yo = y;
      if (y >= 0) {
        const T* f = lring + (size_t)(j % kAhead) * 3 * wc + t;
        po = v - f[0] * wrow(j - 3)[y + dE];
        fo = f[wc];
      }
    };
    int yb = -1, yc = -1;
    T vb = T(0), pc = T(0), fc = T(0);
    __syncthreads();
    {
      int y0;
      T v0 = T(0);
      stage_a(0, y0, v0);
      stage_b(0, y0, v0, yc, pc, fc);
      if (1 < nl) stage_a(1, yb, vb);
    }
    for (int step = -1; step < nl; ++step) {
      const int j = step + 1;
      const int ycur = j < nl ? yc : -1;
      const T cpc = pc, cfc = fc;
      T zl = T(0);
      if (ycur >= 0) zl = wrow(j - 2)[ycur + dE];
      yc = -1;
      if (j + 1 < nl) stage_b(j + 1, yb, vb, yc, pc, fc);
      yb = -1;
      if (j + 2 < nl) stage_a(j + 2, yb, vb);
      if (ycur >= 0) wrow(j)[ycur] = cpc - cfc * zl;
      __syncthreads();
    }
  }
  __syncthreads();  // the staging warp's last write-outs before the window is reused
}

// One column: z = U^{-1} L^{-1} src, written to out[i * P] (added to it when ``acc``).  Boundary
// rows are solved by their scaling; the forward values of interior rows pass through fwd[i * fs]
// on their way to the upper sweep.  Threads [0, wc) form the critical group, [wc, 2wc) the
// lookahead group, the remaining threads stage factors and values.
template <typename T>
__device__ __forceinline__ void window_solve(T* win, T* ring, int wc, const T* __restrict__ lu,
                                           int m, int N, const int* lev_s, const T* src, T* fwd,
                                           int fs, T* out, int P, bool acc) {
  const int nb = 4 * (m - 1);
  for (int k = threadIdx.x; k < nb; k += blockDim.x) {
    const int side = k / (m - 1), s = k - side * (m - 1);
    const int x = side == 0 ? s : side == 1 ? m - 1 : side == 2 ? m - 1 - s : 0;
    const int y = side == 0 ? 0 : side == 1 ? s : side == 2 ? m - 1 : m - 1 - s;
    const int l = x + 2 * y, ylo = max(0, (l - (m - 1) + 1) >> 1), i = x + m * y;
    const T v = src[i] * lu[(size_t)4 * N + lev_s[l] + (y - ylo)];
    T* d = out + (size_t)i * P;
    *d = acc ? *d + v : v;
  }
  const int nl = 3 * m - 8;
  const int tid = threadIdx.x;
  const int role = tid < wc ? 0 : tid < 2 * wc ? 1 : 2;
  const int t = tid - role * wc;
  window_sweep<T, false>(win, ring, wc, lu, m, N, lev_s, nl, role, t, src, 1, fwd, fs, false);
  window_sweep<T, true>(win, ring, wc, lu, m, N, lev_s, nl, role, t, fwd, fs, out, P, acc);
}

// CTA c solves column a = a0 + c with factor set (fac_per_col ? a : 0) and right-hand side
// rhs = Rt[a * ldN ...]:  z = ILU^{-1}(rhs), then inner-1 times z += ILU^{-1}(rhs - K_blk z)
// (the residual and the forward values of those passes in wglob[a * ldN ...]).  The first pass
// keeps its forward values in the output column itself.
template <typename T>
__global__ void __launch_bounds__(kTriMaxThreads) ilu_window_kernel(
    int m, int N, int ldN, int P, int nnz, int a0, int fac_per_col, const int* __restrict__ lev_off,
    int nlev, int wc, const T* __restrict__ lu9s, const int* __restrict__ rowptr,
    const int* __restrict__ col, const T* __restrict__ blks, const T* __restrict__ Rt,
    T* __restrict__ Z, T* __restrict__ wglob, int inner, const int* __restrict__ done) {
  if (done != nullptr && *done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int a = a0 + blockIdx.x;
  const int fsel = fac_per_col ? a : 0;
  const T* lu = lu9s + (size_t)fsel * 9 * N;
  const T* blk = blks + (size_t)fsel * nnz;
  const T* rhs = Rt + (size_t)a * ldN;
  T* zc = Z + a;
  T* win = reinterpret_cast<T*>(smem_raw);
  T* ring = win + (size_t)kWin * m;
  int* lev_s = reinterpret_cast<int*>(ring + (size_t)kAhead * 5 * wc);
  for (int l = threadIdx.x; l <= nlev; l += blockDim.x) lev_s[l] = lev_off[l];
  __syncthreads();
  window_solve<T>(win, ring, wc, lu, m, N, lev_s, rhs, zc, P, zc, P, false);
  for (int it = 1; it < inner; ++it) {
    T* wg = wglob + (size_t)a * ldN;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
      T v = rhs[i];
      for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) v -= blk[e] * zc[(size_t)col[e] * P];
      wg[i] = v;
    }
    __syncthreads();
    window_solve<T>(win, ring, wc, lu, m, N, lev_s, wg, wg, 1, zc, P, true);
    __syncthreads();
  }
}

// Rt[c * ld + r] = R[r * P + c] for the N x P residual: 32 x 32 tiles through shared memory.
template <typename T>
__global__ void columns_kernel(const T* __restrict__ R, T* __restrict__ Rt, int N, int P, int ld,
                               const int* __restrict__ done) {
  if (done != nullptr && *done) return;
  __shared__ T tile[32][33];
  const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
  for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
    const int r = r0 + dy, c = c0 + threadIdx.x;
    tile[dy][threadIdx.x] = (r < N && c < P) ? R[(size_t)r * P + c] : T(0);
  }
  __syncthreads();
  for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
    const int c = c0 + dy, r = r0 + threadIdx.x;
    if (r < N && c < P) Rt[(size_t)c * ld + r] = tile[threadIdx.x][dy];
  }
}

// Z[r * P + c] = Rt[c * ld + r]: the P columns back into the N x P row-major layout.
template <typename T>
__global__ void rows_kernel(const T* __restrict__ Rt, T* __restrict__ Z, int N, int P, int ld,
                            const int* __restrict__ done) {
  if (done != nullptr && *done) return;
  __shared__ T tile[32][33];
  const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
  for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
    const int c = c0 + dy, r = r0 + threadIdx.x;
    tile[dy][threadIdx.x] = (r < N && c < P) ? Rt[(size_t)c * ld + r] : T(0);
  }
  __syncthreads();
  for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
    const int r = r0 + dy, c = c0 + threadIdx.x;
    if (r < N && c < P) Z[(size_t)r * P + c] = tile[threadIdx.x][dy];
  }
}

constexpr int kScatterRows = 32;   // rows per tile of the later-column scatter (one per lane)
constexpr int kScatterWarps = 8;
// k of one warp whose stiffness loads are in flight together (fewer for 8-byte values, so the
// kernel stays within 85 registers a thread)
template <typename TV>
__host__ __device__ constexpr int scatter_ku() { return sizeof(TV) >= 8 ? 2 : 4; }
constexpr int kScatterTW = 12;     // target columns of one warp whose Rt values are prefetched
constexpr int kScatterDirectTiles = 256;  // meshes with fewer 32-row tiles scatter per entry

// After block b of the Gauss-Seidel sweep, for the target columns a_lo <= a <= a_hi (all > b):
// Rt[a, i] -= sum_k G_k[a,b] (A_k z_b)[i] for every row i.  kptr / klist / eptr / ek / eg are the
// tables of those targets.  A tile of 32 rows per step, one row per lane: each warp forms
// T[k, row] = sum_e A_k[e] z_b[col_e] for its share of the k list (the stiffness values from the
// k-major copy, stack_km[k * nnz + e], consecutive rows reading consecutive entries; z_b read
// once per lane from the column zc with stride zs), then each warp subtracts the G-weighted sums
// of its share of the target columns.  The loads are issued in batches (kScatterKU k at a time,
// the Rt values of a warp's targets before the stiffness loads) so that a warp waits for memory
// once per batch rather than once per k or target.  A CTA holds at most a third of an SM's
// registers.
template <typename T, typename TV>
__global__ void __launch_bounds__(kScatterWarps * 32, 3) fs_scatter_kernel(
    int N, int P, int ldN, int nnz, int b, int a_lo, int a_hi, const int* __restrict__ rowptr,
    const int* __restrict__ col, const TV* __restrict__ stack_km, const int* __restrict__ kptr,
    const int* __restrict__ klist, const int* __restrict__ eptr, const int* __restrict__ ek,
    const T* __restrict__ eg, const T* __restrict__ zc, int zs, T* __restrict__ Rt,
    const int* __restrict__ done) {
  if (done != nullptr && *done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Ts = reinterpret_cast<T*>(smem_raw);  // klen x 32
  const int k0 = kptr[b], klen = kptr[b + 1] - k0;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int* ep = eptr + (size_t)b * (P + 1);
  const int ntiles = (N + kScatterRows - 1) / kScatterRows;
  constexpr int kChunk = kScatterWarps * kScatterTW;  // target columns per prefetch round
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int i = tile * kScatterRows + lane;
    const bool live = i < N;
    T r[kScatterTW];
    auto prefetch = [&](int cb) {
#pragma unroll
      for (int j = 0; j < kScatterTW; ++j) {
        const int a = cb + w + kScatterWarps * j;
        r[j] = (live && a <= a_hi && ep[a] < ep[a + 1]) ? Rt[(size_t)a * ldN + i] : T(0);
      }
    };
    prefetch(a_lo);
    const int e0 = live ? rowptr[i] : 0;
    const int ne = live ? rowptr[i + 1] - e0 : 0;
    T z[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) z[e] = e < ne ? zc[(size_t)col[e0 + e] * zs] : T(0);
    constexpr int kScatterKU = scatter_ku<TV>();
    for (int kb = w * kScatterKU; kb < klen; kb += kScatterWarps * kScatterKU) {
      TV av[kScatterKU][9];
#pragma unroll
      for (int u = 0; u < kScatterKU; ++u) {
        const TV* ak = stack_km + (size_t)klist[k0 + min(kb + u, klen - 1)] * nnz + e0;
#pragma unroll
        for (int e = 0; e < 9; ++e) av[u][e] = e < ne ? ak[e] : TV(0);
      }
#pragma unroll
      for (int u = 0; u < kScatterKU; ++u) {
        T t = T(0);
#pragma unroll
        for (int e = 0; e < 9; ++e)
          if (e < ne) t += (T)av[u][e] * z[e];
        if (kb + u < klen) Ts[(size_t)(kb + u) * kScatterRows + lane] = t;
      }
    }
    __syncthreads();
    for (int cb = a_lo; cb <= a_hi; cb += kChunk) {
      if (cb != a_lo) prefetch(cb);
#pragma unroll
      for (int j = 0; j < kScatterTW; ++j) {
        const int a = cb + w + kScatterWarps * j;
        if (a > a_hi) break;
        const int q0 = ep[a], q1 = ep[a + 1];
        if (q0 == q1) continue;  // no coupling into this column: nothing read or written
        T s = T(0);
        for (int q = q0; q < q1; ++q) s += eg[q] * Ts[(size_t)ek[q] * kScatterRows + lane];
        if (live) Rt[(size_t)a * ldN + i] = r[j] - s;
      }
    }
    __syncthreads();
  }
}

// The same update for small meshes, one warp per (32-row tile, target column) with the rows on
// the lanes: the warp forms sum_q G_q[a,b] (A_{k_q} z_b)[i] over the target's entries directly
// (the product A_k z_b once per entry rather than once per k: the entries of a source block name
// each k about once), so the many short work items spread over the whole GPU and no item waits
// on a long chain of dependent loads.  Same arithmetic, in the same order, as fs_scatter_kernel.
template <typename T, typename TV>
__global__ void __launch_bounds__(256) fs_scatter_direct_kernel(
    int N, int P, int ldN, int nnz, int b, int a_lo, int a_hi, const int* __restrict__ rowptr,
    const int* __restrict__ col, const TV* __restrict__ stack_km, const int* __restrict__ kptr,
    const int* __restrict__ klist, const int* __restrict__ eptr, const int* __restrict__ ek,
    const T* __restrict__ eg, const T* __restrict__ zc, int zs, T* __restrict__ Rt,
    const int* __restrict__ done) {
  if (done != nullptr && *done) return;
  const int lane = threadIdx.x & 31;
  const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nw = (int)((gridDim.x * blockDim.x) >> 5);
  const int ntiles = (N + 31) / 32, na = a_hi - a_lo + 1;
  const int k0 = kptr[b];
  const int* ep = eptr + (size_t)b * (P + 1);
  for (int item = gw; item < ntiles * na; item += nw) {
    const int tile = item / na, a = a_lo + item % na;
    const int q0 = ep[a], q1 = ep[a + 1];
    if (q0 == q1) continue;
    const int i = tile * 32 + lane;
    const bool live = i < N;
    const T r = live ? Rt[(size_t)a * ldN + i] : T(0);
    const int e0 = live ? rowptr[i] : 0;
    const int ne = live ? rowptr[i + 1] - e0 : 0;
    T z[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) z[e] = e < ne ? zc[(size_t)col[e0 + e] * zs] : T(0);
    T s = T(0);
    for (int q = q0; q < q1; ++q) {
      const TV* ak = stack_km + (size_t)klist[k0 + ek[q]] * nnz + e0;
      T t = T(0);
#pragma unroll
      for (int e = 0; e < 9; ++e)
        if (e < ne) t += (T)ak[e] * z[e];
      s += eg[q] * t;
    }
    if (live) Rt[(size_t)a * ldN + i] = r - s;
  }
}

// After block b, for the next column only: Rt[b+1, i] -= sum_k G_k[b+1,b] (A_k z_b)[i], one
// thread per row (the row's stencil values of z_b loaded once, then the short k list of the
// next-column tables).  Same arithmetic order as fs_scatter_kernel: per k the stencil sum in
// entry order, then the G-weighted sum in table order.  z_b comes from the column zcol with
// stride zs (the contiguous column the four-colour solve leaves, or column b of Z).
template <typename T, typename TV>
__global__ void __launch_bounds__(256) fs_next_kernel(
    int N, int P, int ldN, int nnz, int b, const int* __restrict__ rowptr,
    const int* __restrict__ col, const TV* __restrict__ stack_km, const int* __restrict__ kptr,
    const int* __restrict__ klist, const int* __restrict__ eptr, const int* __restrict__ ek,
    const T* __restrict__ eg, const T* __restrict__ zcol, int zs, T* __restrict__ Rt,
    const int* __restrict__ done) {
  if (done != nullptr && *done) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int a = b + 1;
  const int e0 = rowptr[i], ne = rowptr[i + 1] - e0;  // at most 9
  T zc[9];
#pragma unroll
  for (int e = 0; e < 9; ++e) zc[e] = e < ne ? zcol[(size_t)col[e0 + e] * zs] : T(0);
  const int k0 = kptr[b];
  const int* ep = eptr + (size_t)b * (P + 1);
  T s = T(0);
  for (int q = ep[a]; q < ep[a + 1]; ++q) {
    const TV* ak = stack_km + (size_t)klist[k0 + ek[q]] * nnz + e0;
    T t = T(0);
#pragma unroll
    for (int e = 0; e < 9; ++e)
      if (e < ne) t += (T)ak[e] * zc[e];
    s += eg[q] * t;
  }
  Rt[(size_t)a * ldN + i] -= s;
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
  static double* rhs_t(System& s) { return s.rhs_t.p; }
  static double* tmp(System& s) { return s.tmp.p; }
  static double* tmp2(System& s) { return s.tmp2.p; }
  static double* triw(System& s) { return s.tri_w.p; }
  static bool full(const System& s) { return s.tri_full; }
  static const double* eg(const System& s) { return s.gs_eg.p; }
  static const double* cs(const System& s) { return s.gsn_cs.p; }
  static double* corr(System& s) { return s.gsn_corr.p; }
};
template <>
struct PcBufs<float> {
  static const float* lu9(const System& s) { return s.lu9_f32.p; }
  static const float* blk(const System& s) { return s.blk_f32.p; }
  static float* rhs_t(System& s) { return s.rhs_t32.p; }
  static float* tmp(System& s) { return s.tmp32.p; }
  static float* tmp2(System& s) { return s.tmp232.p; }
  static float* triw(System& s) { return s.tri_w32.p; }
  static bool full(const System& s) { return s.tri_full32; }
  static const float* eg(const System& s) { return s.gs_eg_f32.p; }
  static const float* cs(const System& s) { return s.gsn_cs32.p; }
  static float* corr(System& s) { return s.gsn_corr32.p; }
};

template <typename T>
int launch_columns(System& s, const T* R, T* Rt, cudaStream_t st, const int* done) {
  dim3 block(32, 8), grid((unsigned)((s.N + 31) / 32), (unsigned)((s.P + 31) / 32));
  TimeScope ts(s.timer, K_OTHER, st);
  columns_kernel<T><<<grid, block, 0, st>>>(R, Rt, s.N, s.P, s.ldN, done);
  return check_launch("columns");
}

template <typename T>
int launch_rows(System& s, const T* Rt, T* Z, cudaStream_t st, const int* done) {
  dim3 block(32, 8), grid((unsigned)((s.N + 31) / 32), (unsigned)((s.P + 31) / 32));
  TimeScope ts(s.timer, K_OTHER, st);
  rows_kernel<T><<<grid, block, 0, st>>>(Rt, Z, s.N, s.P, s.ldN, done);
  return check_launch("rows");
}

template <typename T>
int launch_block_solve(System& s, int a0, int ncols, int fac_per_col, const T* Rt, T* Z,
                       cudaStream_t st, const int* done) {
  using B = PcBufs<T>;
  if (s.prm.ilu_order == SG_ILU_COLOR4)
    return launch_color_solve<T>(s, a0, ncols, fac_per_col, B::lu9(s), const_cast<T*>(Rt), Z, st, done);
  const int wc = s.tri_wc;
  const bool full = B::full(s);
  const int nthreads = 2 * wc + (full ? 32 : tri_staging_threads(wc));
  if (wc < 32 || nthreads > kTriMaxThreads || s.ldN % 4 != 0)
    return fail(SG_ERR_ARG, "wavefront solve: unsupported mesh width");
  if (!full && s.prm.inner_iters > 1 && B::triw(s) == nullptr)
    return fail(SG_ERR_ARG, "wavefront solve: no work column for inner iterations");
  size_t smem = full ? sizeof(T) * ((size_t)s.ldN + tri_ring_entries(wc)) +
                           sizeof(int) * (size_t)(s.nlev9 + 1)
                     : tri_smem_bytes(s.pat.m, wc, sizeof(T));
  // a single-column (Gauss-Seidel) solve takes a whole SM: other kernels' CTAs that shared it
  // would take issue slots from its dependency chain
  if (ncols == 1) smem = std::max(smem, smem_optin_max());
  const int inner = std::max(1, s.prm.inner_iters);
  if (full) {
    auto kern = ilu_column_kernel<T>;
    SG_TRY(ensure_smem((const void*)kern, smem));
    TimeScope ts(s.timer, K_ILU_SOLVE, st);
    kern<<<ncols, nthreads, smem, st>>>(s.pat.m, s.N, s.ldN, s.P, s.pat.nnz, a0, fac_per_col,
                                        s.lev9_off.p, s.nlev9, wc, B::lu9(s), s.rowptr.p, s.col.p,
                                        B::blk(s), Rt, Z, inner, done);
  } else {
    auto kern = ilu_window_kernel<T>;
    SG_TRY(ensure_smem((const void*)kern, smem));
    TimeScope ts(s.timer, K_ILU_SOLVE, st);
    kern<<<ncols, nthreads, smem, st>>>(s.pat.m, s.N, s.ldN, s.P, s.pat.nnz, a0, fac_per_col,
                                        s.lev9_off.p, s.nlev9, wc, B::lu9(s), s.rowptr.p, s.col.p,
                                        B::blk(s), Rt, Z, B::triw(s), inner, done);
  }
  return check_launch("ilu_block_solve");
}

// Scatter of block b into column b + 1 (next = true) or into columns b + 2 .. P - 1.
template <typename T, typename TV>
int launch_scatter_t(System& s, int b, bool next, const TV* stack_km, const T* eg_next,
                     const T* eg_later, const T* Z, T* Rt, cudaStream_t st, const int* done) {
  // z_b: the four-colour solve leaves it contiguous in column b of Rt; else column b of Z
  const bool col_z = s.prm.ilu_order == SG_ILU_COLOR4;
  const T* zc = col_z ? Rt + (size_t)b * s.ldN : Z + b;
  const int zs = col_z ? 1 : s.P;
  TimeScope ts(s.timer, K_GS_SCATTER, st);
  if (next) {
    fs_next_kernel<T, TV><<<(s.N + 255) / 256, 256, 0, st>>>(
        s.N, s.P, s.ldN, s.pat.nnz, b, s.rowptr.p, s.col.p, stack_km, s.gsn_kptr.p, s.gsn_k.p,
        s.gsn_eptr.p, s.gsn_ea.p, eg_next, zc, zs, Rt, done);
  } else {
    // at the lowest launch priority: SMs that its CTAs free go to a pending block solve first
    const int ntiles = (s.N + kScatterRows - 1) / kScatterRows;
    const bool direct = ntiles < kScatterDirectTiles;
    const size_t smem = direct ? 0 : sizeof(T) * kScatterRows * std::max(1, s.gs_max_klen);
    auto kern = direct ? fs_scatter_direct_kernel<T, TV> : fs_scatter_kernel<T, TV>;
    if (!direct) SG_TRY(ensure_smem((const void*)kern, smem));
    const long long items = (long long)ntiles * std::max(1, s.P - 1 - (b + 2) + 1);
    cudaLaunchConfig_t cfg = {};
    // the tiled kernel: one CTA per 32-row tile; the direct one: one warp per (tile, target)
    cfg.gridDim = dim3((unsigned)(direct ? std::max(1LL, (items + 7) / 8) : std::max(1, ntiles)), 1, 1);
    cfg.blockDim = dim3(kScatterWarps * 32, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributePriority;
    attr[0].val.priority = s.prio_lo;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    SG_CUDA(cudaLaunchKernelEx(&cfg, kern, s.N, s.P, s.ldN, s.pat.nnz, b, b + 2, s.P - 1,
                               (const int*)s.rowptr.p, (const int*)s.col.p, stack_km,
                               (const int*)s.gs_kptr.p, (const int*)s.gs_k.p,
                               (const int*)s.gs_eptr.p, (const int*)s.gs_ea.p, eg_later, zc, zs,
                               Rt, done));
  }
  return check_launch("fs_scatter");
}

template <typename T>
int launch_scatter(System& s, int b, bool next, const T* Z, T* Rt, cudaStream_t st,
                   const int* done);
template <>
int launch_scatter<double>(System& s, int b, bool next, const double* Z, double* Rt,
                           cudaStream_t st, const int* done) {
  if (s.stack_km.p == nullptr)
    return fail(SG_ERR_ARG, "the FP64 field-split Gauss-Seidel sweep is not kept for a "
                            "mixed-precision system (its sweeps run in FP32)");
  return launch_scatter_t<double, double>(s, b, next, s.stack_km.p, s.gsn_eg.p, s.gs_eg.p, Z, Rt,
                                          st, done);
}
template <>
int launch_scatter<float>(System& s, int b, bool next, const float* Z, float* Rt, cudaStream_t st,
                          const int* done) {
  if (s.prm.precision == SG_MIXED_BF16 || s.prm.coupling_bf16)
    return launch_scatter_t<float, __nv_bfloat16>(s, b, next, s.stack_km16.p, s.gsn_eg_f32.p,
                                                  s.gs_eg_f32.p, Z, Rt, st, done);
  return launch_scatter_t<float, float>(s, b, next, s.stack_km32.p, s.gsn_eg_f32.p,
                                        s.gs_eg_f32.p, Z, Rt, st, done);
}

// Field-split Gauss-Seidel: block a solved from column a of Rt, then its coupling subtracted from
// the later columns.  Only column a + 1 must be complete before block a + 1 starts; with ``fork``
// the scatter into columns a + 2 .. runs on the system's second stream, overlapping the solve of
// block a + 1.  Ordering: that scatter waits for z_a; the next-column scatter of block a waits for
// the later-column scatter of block a - 1, which also subtracts into column a + 1; the sweep ends
// by joining the second stream.  In the four-colour ordering the next-column coupling is part of
// the block solves (its stencil K_{a+1,a} assembled at setup): the solve of block a leaves
// K_{a+1,a} z_a in a buffer that the solve of block a + 1 subtracts, and the solve of block a + 1
// waits for the later-column scatter of block a - 1 instead; the solves leave z_a in column a of
// Rt, and one transpose at the end writes D.
template <typename T>
int fs_gs_sweep(System& s, const T* R, T* D, T* Rt, cudaStream_t st, const int* done, bool fork) {
  SG_TRY(launch_columns<T>(s, R, Rt, st, done));
  cudaStream_t s2 = fork ? s.stream2 : st;
  const T* cs = PcBufs<T>::cs(s);
  if (s.prm.ilu_order == SG_ILU_COLOR4 && cs != nullptr) {
    for (int a = 0; a < s.P; ++a) {
      if (fork && a >= 2) SG_CUDA(cudaStreamWaitEvent(st, s.ev_r[(a - 2) & 1], 0));
      SG_TRY(launch_color_solve<T>(s, a, 1, 1, PcBufs<T>::lu9(s), Rt, (T*)nullptr, st, done, cs,
                                   PcBufs<T>::corr(s)));
      if (a + 2 < s.P) {
        if (fork) {
          SG_CUDA(cudaEventRecord(s.ev_z, st));
          SG_CUDA(cudaStreamWaitEvent(s2, s.ev_z, 0));
        }
        SG_TRY(launch_scatter<T>(s, a, false, D, Rt, s2, done));
        if (fork) SG_CUDA(cudaEventRecord(s.ev_r[a & 1], s2));
      }
    }
    if (fork && s.P >= 3) SG_CUDA(cudaStreamWaitEvent(st, s.ev_r[(s.P - 3) & 1], 0));
    // every column of Rt now holds its block's solution
    return launch_rows<T>(s, Rt, D, st, done);
  }
  for (int a = 0; a < s.P; ++a) {
    SG_TRY(launch_block_solve<T>(s, a, 1, 1, Rt, D, st, done));
    if (a + 1 >= s.P) break;
    if (a + 2 < s.P) {
      if (fork) {
        SG_CUDA(cudaEventRecord(s.ev_z, st));
        SG_CUDA(cudaStreamWaitEvent(s2, s.ev_z, 0));
      }
      SG_TRY(launch_scatter<T>(s, a, false, D, Rt, s2, done));
      if (fork) SG_CUDA(cudaEventRecord(s.ev_r[a & 1], s2));
    }
    if (fork && a >= 1) SG_CUDA(cudaStreamWaitEvent(st, s.ev_r[(a - 1) & 1], 0));
    SG_TRY(launch_scatter<T>(s, a, true, D, Rt, st, done));
  }
  if (fork && s.P >= 3) SG_CUDA(cudaStreamWaitEvent(st, s.ev_r[(s.P - 3) & 1], 0));
  return SG_OK;
}

// One application of the block preconditioner whose factors the system holds: D = P^{-1} R.
template <typename T>
int apply_block(System& s, const T* R, T* D, cudaStream_t st, const int* done) {
  using B = PcBufs<T>;
  switch (s.pc_fac) {
    case SG_PC_MEAN:
    case SG_PC_FS_JACOBI:
      SG_TRY(launch_columns<T>(s, R, B::rhs_t(s), st, done));
      return launch_block_solve<T>(s, 0, s.P, s.pc_fac == SG_PC_FS_JACOBI ? 1 : 0,
                                   B::rhs_t(s), D, st, done);
    case SG_PC_FS_GS:
      return fs_gs_sweep<T>(s, R, D, B::rhs_t(s), st, done, true);
    case SG_PC_FG:
      return fg_apply<T>(s, R, D, st, done);
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

template <typename T>
int launch_axpy(System& s, size_t n, const T* x, T* y, cudaStream_t st, const int* done) {
  TimeScope ts(s.timer, K_OTHER, st);
  axpy_kernel<T><<<1216, 256, 0, st>>>(n, x, y, done);
  return check_launch("axpy");
}

// Multigrid vectors of one level in the working precision.
template <typename T>
struct MgBufs;
template <>
struct MgBufs<double> {
  static double* b(System& s) { return s.mg_b.p; }
  static double* u(System& s) { return s.mg_u.p; }
  static double* r(System& s) { return s.mg_r.p; }
  static double* d(System& s) { return s.mg_d.p; }
};
template <>
struct MgBufs<float> {
  static float* b(System& s) { return s.mg_b32.p; }
  static float* u(System& s) { return s.mg_u32.p; }
  static float* r(System& s) { return s.mg_r32.p; }
  static float* d(System& s) { return s.mg_d32.p; }
};

// One V-cycle (Sec. 3) for K u = b on level li of the hierarchy top.mg[0 .. ] + top, from u = 0:
// one pre-smoothing step of Eq. level_solver (from zero: u = S^{-1} b), restriction of the
// residual, the V-cycle of the level below, prolongation of its correction, one post-smoothing
// step; the coarsest level is solved directly.
template <typename T>
int vcycle(System& top, int li, const T* b, T* u, cudaStream_t st, const int* done) {
  using G = MgBufs<T>;
  System& s = li == (int)top.mg.size() ? top : *top.mg[li];
  if (li == 0) return launch_coarse_solve<T>(s, b, u, st, done);
  System& c = *top.mg[li - 1];
  T* r = G::r(s);
  T* d = G::d(s);
  const size_t n = (size_t)s.N * s.P;
  SG_TRY(apply_block<T>(s, b, u, st, done));
  SG_TRY(matvec_t<T>(s, u, r, T(-1), b, T(1), st, done));
  SG_TRY(launch_restrict<T>(r, G::b(c), c.n, s.P, st, done, s.timer));
  SG_TRY(vcycle<T>(top, li - 1, G::b(c), G::u(c), st, done));
  SG_TRY(launch_prolong_add<T>(G::u(c), u, c.n, s.P, st, done, s.timer));
  SG_TRY(matvec_t<T>(s, u, r, T(-1), b, T(1), st, done));
  SG_TRY(apply_block<T>(s, r, d, st, done));
  return launch_axpy<T>(s, n, d, u, st, done);
}

// One application of the system's preconditioner (no outer sweeps).
template <typename T>
int apply_once(System& s, const T* R, T* D, cudaStream_t st, const int* done) {
  if (s.prm.precond == SG_PC_MG) return vcycle<T>(s, (int)s.mg.size(), R, D, st, done);
  return apply_block<T>(s, R, D, st, done);
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
    SG_TRY(launch_axpy<T>(s, n, B::tmp2(s), Z, st, done));
  }
  return SG_OK;
}

}  // namespace

int fs_gs_apply_f64_with(System& s, const double* R, double* Z, double* rhs_t, cudaStream_t st) {
  return fs_gs_sweep<double>(s, R, Z, rhs_t, st, nullptr, false);
}

int precond_apply_f64(System& s, const double* R, double* Z, cudaStream_t st, const int* done) {
  return precond_apply_t<double>(s, R, Z, st, done);
}
int precond_apply_f32(System& s, const float* R, float* Z, cudaStream_t st, const int* done) {
  return precond_apply_t<float>(s, R, Z, st, done);
}

}  // namespace sg
