// Grouped field split (Sec. 3, Eq. P_group) and the ILU(0) of multi-field blocks of K (G-I,
// G-M-I, G-M-Fg-I).
//
// The fields form splits (fg_split_ranges); the diagonal block K_ss of a split s with fields
// [f0, f1) (Q of them) is taken node-major — a node's Q fields together — on the block pattern
// where every field of a node couples to every field of each 9-point neighbour, and factored by
// ILU(0) with the nodes in the four-colour order.  On that pattern scalar ILU(0) equals block
// ILU(0) with exact dense factorisations of the diagonal blocks:
//
//   for each node i in order, for each lower neighbour k in order:
//     A_ij -= A_ik D_k^-1 A_kj   for every neighbour j of i that follows k and neighbours k
//   D_i = A_ii (so updated)
//
// stored as lower blocks L_ik D_k^-1, the inverse D_i^-1 and upper blocks D_i^-1 U_ij, so that
// one application is y_i = r_i - sum_lower (L D^-1)_ik y_k over the colours in turn, then
// z_i = D_i^-1 y_i - sum_upper (D^-1 U)_ij z_j over the colours in reverse.  No two nodes of a
// colour are neighbours, so every node of a colour is factored and solved at the same time.
//
// Block storage: per colour-major node position, 9 slots ((dy+1)*3 + (dx+1)) of a Q x Q block,
// column-major (entry (r, c) at c*Q + r); absent neighbours hold zero blocks.
#include <algorithm>

#include "sg_internal.h"

namespace sg {

std::vector<std::pair<int, int>> fg_split_ranges(int M, int p, int rule) {
  std::vector<int> J = total_degree_set(M, p);
  const int P = (int)J.size() / M;
  std::vector<std::pair<int, int>> groups, out;
  if (rule == SG_FG_WHOLE) return {{0, P}};
  for (int a = 0; a < P; ++a) {
    if (groups.empty() || J[(size_t)a * M] != J[(size_t)groups.back().first * M])
      groups.push_back({a, a + 1});
    else
      groups.back().second = a + 1;
  }
  if (rule == SG_FG_GROUPS) return groups;
  for (auto& g : groups) {
    bool all_equal = false;
    for (int a = g.first; a < g.second && !all_equal; ++a) {
      bool eq = true;
      for (int d = 1; d < M; ++d) eq = eq && J[(size_t)a * M + d] == J[(size_t)a * M];
      all_equal = eq;
    }
    if (all_equal || out.empty())
      out.push_back(g);
    else
      out.back().second = g.second;
  }
  return out;
}

namespace {

__device__ __forceinline__ int fg_colour(int x, int y) { return (x & 1) + 2 * (y & 1); }

__device__ __forceinline__ int fg_pos(int x, int y, int m, const int* __restrict__ cstart) {
  const int cx = x & 1, cy = y & 1;
  const int nx = (m - cx + 1) >> 1;
  return cstart[cx + 2 * cy] + ((y - cy) >> 1) * nx + ((x - cx) >> 1);
}

__device__ __forceinline__ void fg_xy(int c, int pos, int m, const int* __restrict__ cstart,
                                      int& x, int& y) {
  const int cx = c & 1, cy = c >> 1;
  const int nx = (m - cx + 1) >> 1;
  const int q = pos - cstart[c];
  y = cy + 2 * (q / nx);
  x = cx + 2 * (q % nx);
}

// Diagonal block of a split, assembled: thread (position, slot, row r) forms row r of the block
// of slot sl, K_ss[(i, f0 + r), (j, f0 + c)] = sum over the triples (k, f0 + r, f0 + c) of
// G_k[a, b] A_k[i, j] (in FP64, triples of a row in (c, k) order), j the slot's neighbour of node
// i.  Blocks of absent neighbours stay zero (the buffer is cleared first).
template <typename D>
__global__ void fg_assemble_kernel(int m, int N, int L, int Q, const int* __restrict__ rowptr,
                                   const int* __restrict__ col, const int* __restrict__ cstart,
                                   const double* __restrict__ stack,
                                   const int* __restrict__ tptr, const int* __restrict__ tkc,
                                   const double* __restrict__ tg, D* __restrict__ out) {
  const long long total = (long long)N * 9 * Q;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(t % Q);
    const int sl = (int)((t / Q) % 9);
    const int i = (int)(t / ((long long)Q * 9));  // node (natural numbering)
    const int x = i % m, y = i / m;
    const int jx = x + sl % 3 - 1, jy = y + sl / 3 - 1;
    if (jx < 0 || jy < 0 || jx >= m || jy >= m) continue;
    const int j = jx + m * jy;
    int e = -1;
    for (int q = rowptr[i]; q < rowptr[i + 1]; ++q)
      if (col[q] == j) e = q;
    if (e < 0) continue;
    const int pos = fg_pos(x, y, m, cstart);
    D* blk = out + ((size_t)pos * 9 + sl) * Q * Q;
    const double* a = stack + (size_t)e * L;
    int c_cur = -1;
    double acc = 0.0;
    for (int q = tptr[r]; q < tptr[r + 1]; ++q) {
      const int c = tkc[2 * q + 1];
      if (c != c_cur) {
        if (c_cur >= 0) blk[(size_t)c_cur * Q + r] = (D)acc;
        c_cur = c;
        acc = 0.0;
      }
      acc += tg[q] * a[tkc[2 * q]];
    }
    if (c_cur >= 0) blk[(size_t)c_cur * Q + r] = (D)acc;
  }
}

constexpr int kFgMaxQ = 96;   // fields per split: the 16 x 16 threads' 6 x 6 tiles of a block
constexpr int kFgTile = 6;

// C = A B (SUB: C -= A B) for Q x Q column-major blocks, A and B in shared memory, C in global
// memory; 256 threads as 16 x 16, each a 6 x 6 tile of rows tx + 16 i and columns ty + 16 j,
// the sum over t in increasing order.
template <typename T, bool SUB>
__device__ __forceinline__ void fg_gemm(int Q, const T* A, const T* B, T* C) {
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  T acc[kFgTile][kFgTile];
#pragma unroll
  for (int i = 0; i < kFgTile; ++i)
#pragma unroll
    for (int j = 0; j < kFgTile; ++j) acc[i][j] = T(0);
  for (int t = 0; t < Q; ++t) {
    T a[kFgTile], b[kFgTile];
#pragma unroll
    for (int i = 0; i < kFgTile; ++i) {
      const int r = tx + 16 * i;
      a[i] = r < Q ? A[t * Q + r] : T(0);
    }
#pragma unroll
    for (int j = 0; j < kFgTile; ++j) {
      const int c = ty + 16 * j;
      b[j] = c < Q ? B[c * Q + t] : T(0);
    }
#pragma unroll
    for (int i = 0; i < kFgTile; ++i)
#pragma unroll
      for (int j = 0; j < kFgTile; ++j) acc[i][j] += a[i] * b[j];
  }
#pragma unroll
  for (int i = 0; i < kFgTile; ++i)
#pragma unroll
    for (int j = 0; j < kFgTile; ++j) {
      const int r = tx + 16 * i, c = ty + 16 * j;
      if (r < Q && c < Q) {
        const size_t idx = (size_t)c * Q + r;
        C[idx] = SUB ? C[idx] - acc[i][j] : acc[i][j];
      }
    }
}

template <typename T>
__device__ __forceinline__ void fg_load_block(int Q, const T* __restrict__ src, T* dst) {
  for (int t = threadIdx.x; t < Q * Q; t += blockDim.x) dst[t] = src[t];
}

// Block ILU(0) of one colour: CTA b factors the b-th node of colour c (see the file comment).
// Shared memory: two Q x Q blocks, reused as the Q x 2Q matrix [D | I] of the Gauss-Jordan
// inversion (partial pivoting) of the diagonal block.  A zero pivot sets *err and leaves NaN.
template <typename T>
__global__ void __launch_bounds__(256) fg_factor_kernel(int m, int Q, int c,
                                                        const int* __restrict__ cstart_g,
                                                        T* __restrict__ fac, int* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* S0 = reinterpret_cast<T*>(smem_raw);
  T* S1 = S0 + Q * Q;
  __shared__ int cstart[5];
  __shared__ int nlow, low_slot[8], low_pos[8];
  __shared__ int ntgt[8], tgt_slot[8][9], tgt_kslot[8][9];
  __shared__ int piv_row;
  __shared__ T colk[kFgMaxQ];
  if (threadIdx.x < 5) cstart[threadIdx.x] = cstart_g[threadIdx.x];
  __syncthreads();
  const int pos = cstart[c] + blockIdx.x;
  int x, y;
  fg_xy(c, pos, m, cstart, x, y);
  const size_t QQ = (size_t)Q * Q;
  T* row = fac + (size_t)pos * 9 * QQ;
  if (threadIdx.x == 0) {
    // lower neighbours in increasing colour-major position; for each, the neighbours j of this
    // node that follow it and neighbour it (this node included)
    int n = 0;
    for (int sl = 0; sl < 9; ++sl) {
      if (sl == 4) continue;
      const int kx = x + sl % 3 - 1, ky = y + sl / 3 - 1;
      if (kx < 0 || ky < 0 || kx >= m || ky >= m || fg_colour(kx, ky) >= c) continue;
      const int pk = fg_pos(kx, ky, m, cstart);
      int at = n++;
      while (at > 0 && low_pos[at - 1] > pk) {
        low_pos[at] = low_pos[at - 1];
        low_slot[at] = low_slot[at - 1];
        --at;
      }
      low_pos[at] = pk;
      low_slot[at] = sl;
    }
    nlow = n;
    for (int t = 0; t < n; ++t) {
      const int kx = x + low_slot[t] % 3 - 1, ky = y + low_slot[t] / 3 - 1;
      int nt = 0;
      for (int sj = 0; sj < 9; ++sj) {
        const int jx = x + sj % 3 - 1, jy = y + sj / 3 - 1;
        if (jx < 0 || jy < 0 || jx >= m || jy >= m) continue;
        if (abs(jx - kx) > 1 || abs(jy - ky) > 1) continue;
        if (fg_pos(jx, jy, m, cstart) <= low_pos[t]) continue;
        tgt_slot[t][nt] = sj;
        tgt_kslot[t][nt] = (jy - ky + 1) * 3 + (jx - kx + 1);
        ++nt;
      }
      ntgt[t] = nt;
    }
  }
  __syncthreads();
  for (int t = 0; t < nlow; ++t) {
    const T* krow = fac + (size_t)low_pos[t] * 9 * QQ;
    fg_load_block(Q, row + low_slot[t] * QQ, S0);  // A_ik, final: every earlier k is applied
    for (int u = 0; u < ntgt[t]; ++u) {
      __syncthreads();
      fg_load_block(Q, krow + tgt_kslot[t][u] * QQ, S1);  // D_k^-1 A_kj
      __syncthreads();
      fg_gemm<T, true>(Q, S0, S1, row + tgt_slot[t][u] * QQ);
    }
    __syncthreads();
    fg_load_block(Q, krow + 4 * QQ, S1);  // D_k^-1
    __syncthreads();
    fg_gemm<T, false>(Q, S0, S1, row + low_slot[t] * QQ);  // L_ik D_k^-1
    __syncthreads();
  }
  // D_i^-1 by Gauss-Jordan on [D_i | I] (row-major, Q x 2Q, in S0 and S1)
  T* Aug = S0;
  const int W = 2 * Q;
  for (int t = threadIdx.x; t < Q * W; t += blockDim.x) {
    const int r = t / W, cc = t % W;
    Aug[t] = cc < Q ? row[4 * QQ + (size_t)cc * Q + r] : (cc - Q == r ? T(1) : T(0));
  }
  __syncthreads();
  for (int k = 0; k < Q; ++k) {
    if (threadIdx.x < 32) {
      T best = T(-1);
      int bi = k;
      for (int r = k + threadIdx.x; r < Q; r += 32) {
        const T v = fabs(Aug[r * W + k]);
        if (v > best) {
          best = v;
          bi = r;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const T ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) {
          best = ob;
          bi = oi;
        }
      }
      if (threadIdx.x == 0) {
        piv_row = bi;
        if (!(best > T(0))) atomicExch(err, 1);
      }
    }
    __syncthreads();
    const int pr = piv_row;
    if (pr != k)
      for (int cc = threadIdx.x; cc < W; cc += blockDim.x) {
        const T tmp = Aug[k * W + cc];
        Aug[k * W + cc] = Aug[pr * W + cc];
        Aug[pr * W + cc] = tmp;
      }
    __syncthreads();
    const T inv = T(1) / Aug[k * W + k];
    for (int r = threadIdx.x; r < Q; r += blockDim.x) colk[r] = Aug[r * W + k];
    __syncthreads();
    for (int cc = threadIdx.x; cc < W; cc += blockDim.x) Aug[k * W + cc] *= inv;
    __syncthreads();
    for (int t = threadIdx.x; t < Q * W; t += blockDim.x) {
      const int r = t / W, cc = t % W;
      if (r != k) Aug[t] -= colk[r] * Aug[k * W + cc];
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < (int)QQ; t += blockDim.x) {
    const int cc = t / Q, r = t % Q;
    row[4 * QQ + t] = Aug[r * W + Q + cc];
  }
  __syncthreads();
  // D_i^-1 A_ij for the higher-colour neighbours
  fg_load_block(Q, row + 4 * QQ, S0);
  for (int sj = 0; sj < 9; ++sj) {
    if (sj == 4) continue;
    const int jx = x + sj % 3 - 1, jy = y + sj / 3 - 1;
    if (jx < 0 || jy < 0 || jx >= m || jy >= m || fg_colour(jx, jy) <= c) continue;
    __syncthreads();
    fg_load_block(Q, row + sj * QQ, S1);
    __syncthreads();
    fg_gemm<T, false>(Q, S0, S1, row + sj * QQ);
  }
}

// Lanes per node in the solve kernels (the rows of a block, in whole warps) and threads per CTA:
// one node of 3 or 4 warps, else 128 threads holding 2 or 4 nodes.
__host__ __device__ constexpr int fg_lanes(int Q) {
  return Q > 96 ? 128 : Q > 64 ? 96 : Q > 32 ? 64 : 32;
}
__host__ __device__ constexpr int fg_cta_threads(int Q) { return fg_lanes(Q) == 96 ? 96 : 128; }

// Block storage of the solve kernels.  FP32 / FP64 factors: each Q x Q block column-major.
// BF16 factors: columns in fours, (r, c) at ((c / 4) * Q + r) * 4 + (c & 3), the column count
// rounded up to a multiple of four (Qc) with zero columns, so a lane reads four values of its
// row in one 8-byte load and a warp's load covers 256 contiguous bytes.
template <typename TV>
__host__ __device__ constexpr bool fg_quads() { return sizeof(TV) == 2; }
__host__ __device__ inline int fg_qc(int Q) { return (Q + 3) & ~3; }

// Row r of block blk times the vector v (Qc values, zero-padded): four partial sums.
template <typename T, typename TV>
__device__ __forceinline__ T fg_block_row_dot(const TV* __restrict__ blk, int Q, int r,
                                              const T* v) {
  T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
  if constexpr (fg_quads<TV>()) {
    const uint2* b4 = reinterpret_cast<const uint2*>(blk) + r;
    const int nq = fg_qc(Q) >> 2;
#pragma unroll 21  // all of a row's loads in flight at once for up to 84 fields
    for (int cq = 0; cq < nq; ++cq) {
      const uint2 w = b4[(size_t)cq * Q];
      const float2 u0 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w.x));
      const float2 u1 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w.y));
      s0 += (T)u0.x * v[4 * cq];
      s1 += (T)u0.y * v[4 * cq + 1];
      s2 += (T)u1.x * v[4 * cq + 2];
      s3 += (T)u1.y * v[4 * cq + 3];
    }
  } else {
    const TV* b = blk + r;
    int cc = 0;
#pragma unroll 2
    for (; cc + 4 <= Q; cc += 4) {
      s0 += (T)b[(size_t)cc * Q] * v[cc];
      s1 += (T)b[(size_t)(cc + 1) * Q] * v[cc + 1];
      s2 += (T)b[(size_t)(cc + 2) * Q] * v[cc + 2];
      s3 += (T)b[(size_t)(cc + 3) * Q] * v[cc + 3];
    }
    for (; cc < Q; ++cc) s0 += (T)b[(size_t)cc * Q] * v[cc];
  }
  return (s0 + s1) + (s2 + s3);
}

// Whether neighbour slot sl (0..8, 4 = the node itself) takes part in a phase of colour c: the
// forward sweep uses the slots of lower colours, the backward sweep the diagonal and the slots
// of higher colours.  A neighbour's colour follows from the node's parities, so the set is the
// same for every node of the launch.
__device__ __forceinline__ bool fg_slot_used(int c, int sl, bool upper) {
  if (sl == 4) return upper;
  const int nc = fg_colour((c & 1) + sl % 3 - 1 + 2, (c >> 1) + sl / 3 - 1 + 2);
  return upper ? nc > c : nc < c;
}

// One colour of a sweep of a split (fields [f0, f0 + Q) of the N x P arrays).
//   forward (UPPER = false): y_i = r_i - sub_i - sum over the lower-colour slots of
//     (L D^-1)_{i,slot} y_nb;
//   backward (UPPER = true, in place): z_i = D_i^-1 y_i - sum over the higher-colour slots of
//     (D^-1 U)_{i,slot} z_nb.
// Each node is a group of lanes (lane r: row r of every block).  The Q values of every slot the
// phase uses (the node's own y_i included in the backward sweep) are staged in shared memory
// first, behind one barrier; then each lane streams its rows of those blocks.  Neighbours
// outside the mesh have zero blocks and are staged as zero vectors.  No other node of the
// colour reads node i, so writing it in place is safe.
template <typename T, typename TV, bool UPPER>
__global__ void __launch_bounds__(128) fg_phase_kernel(int m, int P, int Q, int f0, int c,
                                                       const int* __restrict__ cstart_g,
                                                       const TV* __restrict__ fac,
                                                       const T* __restrict__ R,
                                                       const T* __restrict__ sub, T* Y,
                                                       const int* __restrict__ done) {
  if (done != nullptr && *done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int G = fg_lanes(Q), npc = fg_cta_threads(Q) / G;
  const int g = threadIdx.x / G, r = threadIdx.x % G;
  const int c0 = cstart_g[c], cnt = cstart_g[c + 1] - c0;
  const int idx = blockIdx.x * npc + g;
  const bool live = idx < cnt;
  const int pos = c0 + (live ? idx : cnt - 1);
  int x, y;
  {
    const int cx = c & 1, cy = c >> 1, nx = (m - cx + 1) >> 1, q = pos - c0;
    y = cy + 2 * (q / nx);
    x = cx + 2 * (q % nx);
  }
  const int i = x + m * y;
  const int Qc = fg_qc(Q);
  const size_t QQ = (size_t)Q * (fg_quads<TV>() ? Qc : Q);
  const TV* blocks = fac + (size_t)pos * 9 * QQ;
  T* v = reinterpret_cast<T*>(smem_raw) + (size_t)g * 9 * Qc;  // one vector per used slot
  int k = 0;
#pragma unroll
  for (int sl = 0; sl < 9; ++sl) {
    if (!fg_slot_used(c, sl, UPPER)) continue;
    // a neighbour outside the mesh has a zero block and a zero vector: its clamped stand-in may
    // be a node this sweep has not written yet (the node itself at an even-sized mesh's edge)
    const int nx = x + sl % 3 - 1, ny = y + sl / 3 - 1;
    const bool inside = nx >= 0 && ny >= 0 && nx < m && ny < m;
    const int jx = min(max(nx, 0), m - 1), jy = min(max(ny, 0), m - 1);
    const T* src = Y + ((size_t)jx + (size_t)m * jy) * P + f0;
    for (int t = r; t < Qc; t += G) v[k * Qc + t] = t < Q && inside ? src[t] : T(0);
    ++k;
  }
  T acc = T(0);
  if (!UPPER && r < Q)
    acc = R[(size_t)i * P + f0 + r] - (sub != nullptr ? sub[(size_t)i * P + f0 + r] : T(0));
  __syncthreads();
  if (r < Q) {
    unsigned used = 0;
#pragma unroll
    for (int sl = 0; sl < 9; ++sl) used |= fg_slot_used(c, sl, UPPER) ? 1u << sl : 0u;
    // slot sl's vector is the k-th staged one, k = the used slots before it
    if (UPPER)  // the diagonal first
      acc = fg_block_row_dot<T, TV>(blocks + 4 * QQ, Q, r, v + (size_t)__popc(used & 15u) * Qc);
#pragma unroll 1
    for (int sl = 0; sl < 9; ++sl) {
      if (sl == 4 || !(used >> sl & 1u)) continue;
      acc -= fg_block_row_dot<T, TV>(blocks + sl * QQ, Q, r,
                                     v + (size_t)__popc(used & ((1u << sl) - 1u)) * Qc);
    }
  }
  if (live && r < Q) Y[(size_t)i * P + f0 + r] = acc;
}

// tmp = D with the fields >= f0 set to zero (the earlier splits' solution).
template <typename T>
__global__ void fg_mask_kernel(size_t N, int P, int f0, const T* __restrict__ D, T* __restrict__ tmp,
                               const int* __restrict__ done) {
  if (done != nullptr && *done) return;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < N * P;
       t += (size_t)gridDim.x * blockDim.x)
    tmp[t] = (int)(t % P) < f0 ? D[t] : T(0);
}

// FP32 blocks (column-major, Q x Q) -> BF16 blocks in the layout of fours (Q x Qc, zero columns
// up to a multiple of four); one thread per destination element.
__global__ void fg_round_bf16_kernel(size_t nblocks, int Q, const float* __restrict__ src,
                                     __nv_bfloat16* __restrict__ dst) {
  const int Qc = fg_qc(Q);
  const size_t per = (size_t)Q * Qc, total = nblocks * per;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const size_t blk = t / per;
    const int o = (int)(t - blk * per);
    const int cc = 4 * (o / (4 * Q)) + (o & 3), r = (o >> 2) % Q;
    dst[t] = cc < Q ? __float2bfloat16_rn(src[blk * Q * Q + (size_t)cc * Q + r])
                    : __float2bfloat16_rn(0.0f);
  }
}

template <typename T>
struct FgBufs;
template <>
struct FgBufs<double> {
  static double* fac(System::FgSplit& sp) { return sp.fac.p; }
  static double* tmp(System& s) { return s.fg_tmp.p; }
  static double* tmp2(System& s) { return s.fg_tmp2.p; }
};
template <>
struct FgBufs<float> {
  static float* fac(System::FgSplit& sp) { return sp.fac32.p; }
  static float* tmp(System& s) { return s.fg_tmp32.p; }
  static float* tmp2(System& s) { return s.fg_tmp232.p; }
};

template <typename T>
int fg_factor(System& s, System::FgSplit& sp, T* fac, cudaStream_t st) {
  const int Q = sp.f1 - sp.f0;
  const size_t smem = 2 * sizeof(T) * (size_t)Q * Q;
  auto kern = fg_factor_kernel<T>;
  SG_TRY(ensure_smem((const void*)kern, smem));
  DBuf<int> err;
  SG_TRY(err.alloc(1));
  SG_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), st));
  for (int c = 0; c < 4; ++c) {
    const int cnt = s.cstart_h[c + 1] - s.cstart_h[c];
    if (cnt <= 0) continue;
    kern<<<cnt, 256, smem, st>>>(s.pat.m, Q, c, s.cstart.p, fac, err.p);
    SG_TRY(check_launch("fg_factor"));
  }
  int herr = 0;
  SG_CUDA(cudaMemcpyAsync(&herr, err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  SG_CUDA(cudaStreamSynchronize(st));
  err.release();
  if (herr) return fail(SG_ERR_ARG, "grouped field split: a diagonal block of ILU(0) is singular");
  return SG_OK;
}

}  // namespace

int fg_setup(System& s, cudaStream_t st) {
  const sg_params& p = s.prm;
  const bool lowp = p.precision != SG_FP64;
  const int m = s.pat.m;
  // colour offsets of the four-colour order (shared with the scalar colour ILU)
  s.cstart_h.assign(5, 0);
  for (int c = 0; c < 4; ++c) {
    const int cx = c & 1, cy = c >> 1;
    s.cstart_h[c + 1] = s.cstart_h[c] + ((m - cx + 1) / 2) * ((m - cy + 1) / 2);
  }
  if (s.cstart.p == nullptr) {
    SG_TRY(s.cstart.alloc(5));
    SG_TRY(s.cstart.upload(s.cstart_h, st));
  }
  auto ranges = fg_split_ranges(p.M, p.p, p.fg_rule);
  s.fg.clear();
  s.fg.resize(ranges.size());
  for (size_t si = 0; si < ranges.size(); ++si) {
    System::FgSplit& sp = s.fg[si];
    sp.f0 = ranges[si].first;
    sp.f1 = ranges[si].second;
    const int Q = sp.f1 - sp.f0;
    if (Q > kFgMaxQ)
      return fail(SG_ERR_ARG, "grouped field split: a split of " + std::to_string(Q) +
                                  " fields (at most " + std::to_string(kFgMaxQ) + ")");
    // the split's triples per row r = a - f0, in (c, k) order
    std::vector<std::vector<std::pair<std::pair<int, int>, double>>> rows(Q);
    for (auto& t : s.triples)
      if (t.a >= sp.f0 && t.a < sp.f1 && t.b >= sp.f0 && t.b < sp.f1)
        rows[t.a - sp.f0].push_back({{t.b - sp.f0, t.k}, t.g});
    std::vector<int> tptr(Q + 1, 0), tkc;
    std::vector<double> tg;
    for (int r = 0; r < Q; ++r) {
      std::sort(rows[r].begin(), rows[r].end(),
                [](const auto& u, const auto& v) { return u.first < v.first; });
      for (auto& e : rows[r]) {
        tkc.push_back(e.first.second);
        tkc.push_back(e.first.first);
        tg.push_back(e.second);
      }
      tptr[r + 1] = (int)tg.size();
    }
    DBuf<int> dptr, dkc;
    DBuf<double> dg;
    SG_TRY(dptr.alloc(tptr.size()));
    SG_TRY(dptr.upload(tptr, st));
    SG_TRY(dkc.alloc(std::max<size_t>(1, tkc.size())));
    if (!tkc.empty()) SG_TRY(dkc.upload(tkc, st));
    SG_TRY(dg.alloc(std::max<size_t>(1, tg.size())));
    if (!tg.empty()) SG_TRY(dg.upload(tg, st));
    const size_t nblk = (size_t)s.N * 9 * Q * Q;
    const long long total = (long long)s.N * 9 * Q;
    const int grid = (int)std::max(1LL, std::min((total + 255) / 256, 152LL * 64));
    if (lowp) {
      SG_TRY(sp.fac32.alloc(nblk));
      SG_CUDA(cudaMemsetAsync(sp.fac32.p, 0, sizeof(float) * nblk, st));
      fg_assemble_kernel<float><<<grid, 256, 0, st>>>(m, s.N, s.L, Q, s.rowptr.p, s.col.p,
                                                      s.cstart.p, s.stack.p, dptr.p, dkc.p, dg.p,
                                                      sp.fac32.p);
      SG_TRY(check_launch("fg_assemble"));
      SG_TRY(fg_factor<float>(s, sp, sp.fac32.p, st));
      if (p.fg_bf16) {  // the factors in BF16 for the applications, the FP32 copy dropped
        const size_t nb = (size_t)s.N * 9;
        SG_TRY(sp.fac16.alloc(nb * Q * fg_qc(Q)));
        fg_round_bf16_kernel<<<1216, 256, 0, st>>>(nb, Q, sp.fac32.p, sp.fac16.p);
        SG_TRY(check_launch("fg_round_bf16"));
        SG_CUDA(cudaStreamSynchronize(st));
        sp.fac32.release();
      }
    } else {
      SG_TRY(sp.fac.alloc(nblk));
      SG_CUDA(cudaMemsetAsync(sp.fac.p, 0, sizeof(double) * nblk, st));
      fg_assemble_kernel<double><<<grid, 256, 0, st>>>(m, s.N, s.L, Q, s.rowptr.p, s.col.p,
                                                       s.cstart.p, s.stack.p, dptr.p, dkc.p,
                                                       dg.p, sp.fac.p);
      SG_TRY(check_launch("fg_assemble"));
      SG_TRY(fg_factor<double>(s, sp, sp.fac.p, st));
    }
  }
  if (s.fg.size() > 1) {
    const size_t NP = (size_t)s.N * s.P;
    if (lowp) {
      SG_TRY(s.fg_tmp32.alloc(NP));
      SG_TRY(s.fg_tmp232.alloc(NP));
    } else {
      SG_TRY(s.fg_tmp.alloc(NP));
      SG_TRY(s.fg_tmp2.alloc(NP));
    }
  }
  return SG_OK;
}

template <typename T>
int fg_apply(System& s, const T* R, T* D, cudaStream_t st, const int* done) {
  using B = FgBufs<T>;
  for (size_t si = 0; si < s.fg.size(); ++si) {
    System::FgSplit& sp = s.fg[si];
    const T* fac = B::fac(sp);
    const __nv_bfloat16* fac16 = sizeof(T) == 4 ? sp.fac16.p : nullptr;
    if (fac == nullptr && fac16 == nullptr)
      return fail(SG_ERR_ARG, "grouped field split: no factors in this precision");
    const int Q = sp.f1 - sp.f0;
    const T* sub = nullptr;
    if (si > 0) {  // Eq. P_group: subtract sum_{t < s} K_st z_t, from K applied to z masked
      TimeScope ts(s.timer, K_OTHER, st);
      fg_mask_kernel<T><<<1216, 256, 0, st>>>((size_t)s.N, s.P, sp.f0, D, B::tmp(s), done);
      SG_TRY(check_launch("fg_mask"));
      if (sizeof(T) == 8)
        SG_TRY(launch_matvec_f64(s, (const double*)B::tmp(s), (double*)B::tmp2(s), 1.0, nullptr,
                                 0.0, st, done));
      else
        SG_TRY(launch_matvec_f32(s, (const float*)B::tmp(s), (float*)B::tmp2(s), 1.0f, nullptr,
                                 0.0f, st, done));
      sub = B::tmp2(s);
    }
    const int G = fg_lanes(Q), nthr = fg_cta_threads(Q), npc = nthr / G;
    const size_t smem = sizeof(T) * (size_t)npc * 9 * fg_qc(Q);
    for (int c = 0; c < 4; ++c) {
      const int cnt = s.cstart_h[c + 1] - s.cstart_h[c];
      if (cnt <= 0) continue;
      TimeScope ts(s.timer, K_ILU_SOLVE, st);
      const int grid = (cnt + npc - 1) / npc;
      if (fac16 != nullptr)
        fg_phase_kernel<T, __nv_bfloat16, false><<<grid, nthr, smem, st>>>(
            s.pat.m, s.P, Q, sp.f0, c, s.cstart.p, fac16, R, sub, D, done);
      else
        fg_phase_kernel<T, T, false><<<grid, nthr, smem, st>>>(s.pat.m, s.P, Q, sp.f0, c,
                                                              s.cstart.p, fac, R, sub, D, done);
      SG_TRY(check_launch("fg_phase (forward)"));
    }
    for (int c = 3; c >= 0; --c) {
      const int cnt = s.cstart_h[c + 1] - s.cstart_h[c];
      if (cnt <= 0) continue;
      TimeScope ts(s.timer, K_ILU_SOLVE, st);
      const int grid = (cnt + npc - 1) / npc;
      if (fac16 != nullptr)
        fg_phase_kernel<T, __nv_bfloat16, true><<<grid, nthr, smem, st>>>(
            s.pat.m, s.P, Q, sp.f0, c, s.cstart.p, fac16, nullptr, nullptr, D, done);
      else
        fg_phase_kernel<T, T, true><<<grid, nthr, smem, st>>>(s.pat.m, s.P, Q, sp.f0, c,
                                                             s.cstart.p, fac, nullptr, nullptr, D,
                                                             done);
      SG_TRY(check_launch("fg_phase (backward)"));
    }
  }
  return SG_OK;
}

template int fg_apply<double>(System&, const double*, double*, cudaStream_t, const int*);
template int fg_apply<float>(System&, const float*, float*, cudaStream_t, const int*);

}  // namespace sg
