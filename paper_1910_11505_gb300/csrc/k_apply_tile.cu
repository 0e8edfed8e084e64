// The SG operator Y = sum_k A_k X G_k^T (Eqs. stochastic_matrix and K_matrix), row-tiled form.
//
// Per interior node row i with its 9 stencil entries e = (dy + 1) * 3 + (dx + 1) (neighbour
// j_e = i + dx + m dy):
//   T[k,b] = sum_e A[e,k] X[j_e, b]     for the (k, b) pairs that meet a nonzero G_k[a,b]
//   Y[i,a] = sum_{(k,b)} G_k[a,b] T[k,b]
// (9 U + nnz_G multiply-adds per row; U = number of such pairs).
//
// Layout of the work.  A CTA owns a tile of 32 consecutive interior nodes of one grid line, one
// node per lane, so every warp instruction works on 32 rows with the same (k, b, a) and all
// control is uniform.  The stiffness values of a tile are stored contiguously as
// [k in a permuted order][e][row] ("tiled stack"), and streamed in chunks of consecutive k into a
// two-slot shared-memory ring by 1-D TMA bulk copies (cp.async.bulk) completing on mbarriers.  The
// three grid lines of X the tile touches (34 nodes each, all P chaos values) sit in shared memory.
//
// Stage 1: each warp takes one group of kappa k (their 9 kappa stencil values in registers) and
// walks the union of their b lists; for each b it loads the 9 neighbour values of X once and forms
// T for every k of the group that needs this b (a uniform bit mask), writing T[slot][row] to shared
// memory.  Grouping k with similar b lists (chosen at setup) is what cuts the X loads per pair.
// Stage 2: each warp owns the outputs a = warp + 8 j and adds G_k[a,b] T[slot] over the chunk's
// entries of those a, in registers across chunks.  The tile's Y rows are written at the end
// through shared memory, coalesced.  Boundary rows (identity rows of K) are Y = alpha X + beta B.
//
// Every wait on an mbarrier is bounded: after kWaitLimit polls the kernel raises the error word,
// waits (bounded again) for its own copies in flight and returns with NaN in the rows it owns.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "sg_internal.h"

namespace sg {

namespace {

constexpr int kTW = 32;       // rows per tile
constexpr int kWarps = 8;     // warps per CTA: groups per chunk and a-strides of stage 2
constexpr int kSlab = kTW + 2;
constexpr long long kWaitLimit = 1LL << 22;

struct TileDims {
  int m, tiles_per_line, ntiles, P, Pp, nchunks;
  int abuf_elems, tbuf_elems, xslab_elems;
};

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the given phase parity of an mbarrier.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity) {
  for (long long it = 0; it < kWaitLimit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes,
                                         unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

template <typename T>
__device__ __forceinline__ T nan_of();
template <>
__device__ __forceinline__ double nan_of<double>() { return __longlong_as_double(0x7ff8000000000000LL); }
template <>
__device__ __forceinline__ float nan_of<float>() { return __int_as_float(0x7fc00000); }

template <typename T, int KAPPA, int APW>
__global__ void __launch_bounds__(kWarps * 32, 1) sg_apply_tile_kernel(
    TileDims d, const int4* __restrict__ chunk, const int4* __restrict__ group,
    const int2* __restrict__ ulist, const int* __restrict__ ent_ptr,
    const int* __restrict__ ent_slot, const T* __restrict__ ent_g, const T* __restrict__ stack,
    const T* __restrict__ X, T* __restrict__ Y, T alpha, const T* __restrict__ B, T beta,
    const int* __restrict__ done, int* __restrict__ err) {
  if (done != nullptr && *done) return;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem_raw);  // 2 barriers
  int* s_fail = reinterpret_cast<int*>(smem_raw + 16);
  T* Abuf0 = reinterpret_cast<T*>(smem_raw + 128);
  T* Abuf1 = Abuf0 + d.abuf_elems;
  T* Ts = Abuf1 + d.abuf_elems;
  T* Xs = Ts + d.tbuf_elems;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int P = d.P, Pp = d.Pp, m = d.m;

  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    *s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  }
  __syncthreads();

  // the stack of tile t starts at t * kstride elements; chunk c at chunk[c].x * 9 * 32 within it
  const size_t kstride = (size_t)chunk[d.nchunks - 1].x * 9 * kTW + (size_t)chunk[d.nchunks - 1].y * 9 * kTW;
  auto issue = [&](int t, int c, int slot) {
    const int4 cd = chunk[c];
    const unsigned bytes = (unsigned)((size_t)cd.y * 9 * kTW * sizeof(T));
    T* dst = slot ? Abuf1 : Abuf0;
    const T* src = stack + (size_t)t * kstride + (size_t)cd.x * 9 * kTW;
    mbar_expect_tx(&bar[slot], bytes);
    bulk_g2s(dst, src, bytes, &bar[slot]);
  };

  T acc[APW];
  long long it = 0;  // work items (tile, chunk) of this CTA so far
  bool next_issued = false;  // whether the copy of item it + 1 is in flight
  if (blockIdx.x < d.ntiles && tid == 0) issue(blockIdx.x, 0, 0);
  bool failed = false;

  for (int t = blockIdx.x; t < d.ntiles && !failed; t += gridDim.x) {
    const int y = 1 + t / d.tiles_per_line;
    const int x0 = 1 + (t % d.tiles_per_line) * kTW;
    const int nrows = min(kTW, m - 1 - x0);
    // X on lines y-1, y, y+1 for nodes x0-1 .. x0+32 (zero beyond the mesh)
    for (int idx = tid; idx < 3 * kSlab * P; idx += blockDim.x) {
      const int dy = idx / (kSlab * P);
      const int rem = idx - dy * kSlab * P;
      const int xi = rem / P, b = rem - xi * P;
      const int x = x0 - 1 + xi;
      T v = T(0);
      if (x < m) v = X[((size_t)(y - 1 + dy) * m + x) * P + b];
      Xs[(dy * kSlab + xi) * Pp + b] = v;
    }
#pragma unroll
    for (int j = 0; j < APW; ++j) acc[j] = T(0);

    for (int c = 0; c < d.nchunks; ++c, ++it) {
      // prefetch the next work item into the other slot (its last reader finished before the
      // barrier that closed the previous item)
      if (tid == 0) {
        int tn = t, cn = c + 1;
        if (cn == d.nchunks) {
          tn = t + gridDim.x;
          cn = 0;
        }
        if (tn < d.ntiles) {
          issue(tn, cn, (int)((it + 1) & 1));
          next_issued = true;
        } else {
          next_issued = false;
        }
      }
      const int slot = (int)(it & 1);
      if (!mbar_wait_bounded(&bar[slot], (unsigned)((it >> 1) & 1))) *s_fail = 1;
      __syncthreads();
      if (*s_fail) {
        failed = true;
        break;
      }
      const T* Ab = slot ? Abuf1 : Abuf0;
      const int4 cd = chunk[c];
      // ---- stage 1: T for the pairs of this warp's group
      if (w < cd.w) {
        const int4 gd = group[cd.z + w];  // ulist start, length, first k position, k count
        T a[KAPPA][9];
#pragma unroll
        for (int j = 0; j < KAPPA; ++j) {
          if (j < gd.w) {
#pragma unroll
            for (int e = 0; e < 9; ++e) a[j][e] = Ab[((size_t)(gd.z + j) * 9 + e) * kTW + lane];
          } else {
#pragma unroll
            for (int e = 0; e < 9; ++e) a[j][e] = T(0);
          }
        }
        const int2* ul = ulist + gd.x;
        for (int u = 0; u < gd.y; ++u) {
          const int2 ue = ul[u];
          const int b = ue.x & 0xffff, mask = ue.x >> 16;
          int sl = ue.y;
          T xv[9];
#pragma unroll
          for (int dy = 0; dy < 3; ++dy)
#pragma unroll
            for (int dx = 0; dx < 3; ++dx) xv[dy * 3 + dx] = Xs[(dy * kSlab + lane + dx) * Pp + b];
#pragma unroll
          for (int j = 0; j < KAPPA; ++j) {
            if (mask & (1 << j)) {
              T s = a[j][0] * xv[0];
#pragma unroll
              for (int e = 1; e < 9; ++e) s = fma(a[j][e], xv[e], s);
              Ts[(size_t)sl * kTW + lane] = s;
              ++sl;
            }
          }
        }
      }
      __syncthreads();
      // ---- stage 2: Y[row, a] += sum G T over this chunk's entries of the warp's outputs
      const int* ep = ent_ptr + (size_t)c * (P + 1);
#pragma unroll
      for (int j = 0; j < APW; ++j) {
        const int a = w + kWarps * j;
        if (a < P) {
          T s = T(0);
          const int q1 = ep[a + 1];
          for (int q = ep[a]; q < q1; ++q) s = fma(ent_g[q], Ts[(size_t)ent_slot[q] * kTW + lane], s);
          acc[j] += s;
        }
      }
      __syncthreads();
    }
    if (failed) break;
    // ---- epilogue: Y rows of the tile through shared memory (coalesced)
#pragma unroll
    for (int j = 0; j < APW; ++j) {
      const int a = w + kWarps * j;
      if (a < P) Ts[(size_t)a * kTW + lane] = acc[j];
    }
    __syncthreads();
    const size_t row0 = (size_t)y * m + x0;
    for (int idx = tid; idx < nrows * P; idx += blockDim.x) {
      const int r = idx / P, a = idx - r * P;
      const size_t o = row0 * P + idx;
      T v = alpha * Ts[(size_t)a * kTW + r];
      if (B != nullptr) v = fma(beta, B[o], v);
      Y[o] = v;
    }
    __syncthreads();
  }
  if (failed) {
    // a bulk copy did not complete in time: record it, let the copies this CTA issued land
    // (bounded), and leave NaN in every row of the CTA's tiles so no caller takes them as results
    if (tid == 0) {
      atomicExch(err, 1);
      mbar_wait_bounded(&bar[it & 1], (unsigned)((it >> 1) & 1));
      if (next_issued) mbar_wait_bounded(&bar[(it + 1) & 1], (unsigned)(((it + 1) >> 1) & 1));
    }
    __syncthreads();
    for (int t = blockIdx.x; t < d.ntiles; t += gridDim.x) {
      const int y = 1 + t / d.tiles_per_line;
      const int x0 = 1 + (t % d.tiles_per_line) * kTW;
      const int nrows = min(kTW, m - 1 - x0);
      for (int idx = tid; idx < nrows * P; idx += blockDim.x)
        Y[((size_t)y * m + x0) * P + idx] = nan_of<T>();
    }
    return;
  }
  // ---- boundary rows: identity rows of K
  const int nb = 4 * (m - 1);
  for (long long idx = (long long)blockIdx.x * blockDim.x + tid; idx < (long long)nb * P;
       idx += (long long)gridDim.x * blockDim.x) {
    const int q = (int)(idx / P), a = (int)(idx - (long long)q * P);
    int x, y;
    if (q < m) { x = q; y = 0; }
    else if (q < 2 * m) { x = q - m; y = m - 1; }
    else if (q < 3 * m - 2) { x = 0; y = q - 2 * m + 1; }
    else { x = m - 1; y = q - (3 * m - 2) + 1; }
    const size_t o = ((size_t)y * m + x) * P + a;
    T v = alpha * X[o];
    if (B != nullptr) v = fma(beta, B[o], v);
    Y[o] = v;
  }
}

// Tiled stack from the nnz x L stack: for tile t, permuted k position kp, entry e, row r:
// value of A_{kperm[kp]} at entry e of node (x0 + r, y), 0 for rows beyond the line.
template <typename TS>
__global__ void tile_stack_kernel(int m, int tiles_per_line, int ntiles, int Lu, int L,
                                  const int* __restrict__ rowptr, const int* __restrict__ kperm,
                                  const double* __restrict__ stack, TS* __restrict__ out) {
  const long long total = (long long)ntiles * Lu * 9 * kTW;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(idx % kTW);
    long long rest = idx / kTW;
    const int e = (int)(rest % 9);
    rest /= 9;
    const int kp = (int)(rest % Lu);
    const int t = (int)(rest / Lu);
    const int y = 1 + t / tiles_per_line;
    const int x = 1 + (t % tiles_per_line) * kTW + r;
    double v = 0.0;
    if (x <= m - 2) {
      const int node = y * m + x;
      v = stack[((size_t)rowptr[node] + e) * L + kperm[kp]];
    }
    out[idx] = (TS)v;
  }
}

}  // namespace

// ------------------------------------------------------------------ host: tables and launch

int plan_tile_op(const System& s, int kappa, int elem, size_t smem_max, TilePlan& op) {
  const int P = s.P, L = s.L, m = s.pat.m;
  op = TilePlan();
  op.kappa = kappa;
  op.elem = elem;
  if (m < 3 || kappa < 1 || kappa > 4 || P > 256) return fail(SG_ERR_ARG, "tile operator: unsupported sizes");
  op.tiles_per_line = (m - 2 + kTW - 1) / kTW;
  op.ntiles = op.tiles_per_line * (m - 2);
  op.Pp = P | 1;
  // b lists per k as bit sets
  const int words = (P + 63) / 64;
  std::vector<unsigned long long> bset((size_t)L * words, 0ULL);
  std::vector<int> bcount(L, 0);
  for (const Triple& t : s.triples) {
    unsigned long long& wd = bset[(size_t)t.k * words + t.b / 64];
    const unsigned long long bit = 1ULL << (t.b % 64);
    if (!(wd & bit)) {
      wd |= bit;
      bcount[t.k]++;
    }
  }
  // greedy groups of kappa k with similar b lists, seeds in order of total degree
  std::vector<int> Jq = total_degree_set(s.M, s.prm.q);
  std::vector<int> deg(L, 0), order;
  for (int k = 0; k < L; ++k)
    for (int n = 0; n < s.M; ++n) deg[k] += Jq[(size_t)k * s.M + n];
  for (int k = 0; k < L; ++k)
    if (bcount[k] > 0) order.push_back(k);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return deg[a] < deg[b]; });
  std::vector<char> used(L, 0);
  std::vector<std::vector<int>> groups;
  for (int seed : order) {
    if (used[seed]) continue;
    std::vector<int> g{seed};
    used[seed] = 1;
    std::vector<unsigned long long> S(bset.begin() + (size_t)seed * words,
                                      bset.begin() + (size_t)(seed + 1) * words);
    while ((int)g.size() < kappa) {
      int best = -1;
      double bj = -1.0;
      for (int k : order) {
        if (used[k]) continue;
        int inter = 0, uni = 0;
        for (int q = 0; q < words; ++q) {
          inter += __builtin_popcountll(S[q] & bset[(size_t)k * words + q]);
          uni += __builtin_popcountll(S[q] | bset[(size_t)k * words + q]);
        }
        const double j = uni ? (double)inter / uni : 0.0;
        if (j > bj) {
          bj = j;
          best = k;
        }
      }
      if (best < 0) break;
      used[best] = 1;
      g.push_back(best);
      for (int q = 0; q < words; ++q) S[q] |= bset[(size_t)best * words + q];
    }
    groups.push_back(g);
  }
  // group union lists and pair slots; chunks of at most kWarps groups and slot capacity
  const size_t xslab = (size_t)3 * kSlab * op.Pp;
  const size_t fixed = 128 + elem * (xslab + 2 * (size_t)kWarps * kappa * 9 * kTW);
  if (fixed + (size_t)elem * P * kTW > smem_max) return fail(SG_ERR_ARG, "tile operator: P too large for shared memory");
  const int slot_cap = (int)std::min<size_t>(16384, (smem_max - fixed) / ((size_t)elem * kTW));
  std::vector<int4> gdesc, cdesc;
  std::vector<int2> ul;
  std::vector<int> kperm;
  std::vector<int> pair_slot((size_t)L * P, -1), pair_chunk((size_t)L * P, -1);
  int cur_groups = 0, cur_slots = 0, cur_k0 = 0;
  auto close_chunk = [&]() {
    if (cur_groups == 0) return;
    const int k1 = (int)kperm.size();
    cdesc.push_back(make_int4(cur_k0, k1 - cur_k0, (int)gdesc.size() - cur_groups, cur_groups));
    op.max_chunk_k = std::max(op.max_chunk_k, k1 - cur_k0);
    op.max_slots = std::max(op.max_slots, cur_slots);
    cur_groups = 0;
    cur_slots = 0;
    cur_k0 = k1;
  };
  for (auto& g : groups) {
    int gslots = 0;
    for (int k : g) gslots += bcount[k];
    if (gslots > slot_cap) return fail(SG_ERR_ARG, "tile operator: a k group exceeds the slot capacity");
    if (cur_groups == kWarps || cur_slots + gslots > slot_cap) close_chunk();
    const int kloc = (int)kperm.size() - cur_k0;
    const int ul0 = (int)ul.size();
    int sl = cur_slots;
    const int c = (int)cdesc.size();
    for (int b = 0; b < P; ++b) {
      unsigned mask = 0;
      for (int j = 0; j < (int)g.size(); ++j)
        if (bset[(size_t)g[j] * words + b / 64] >> (b % 64) & 1ULL) mask |= 1u << j;
      if (!mask) continue;
      ul.push_back(make_int2(b | (int)(mask << 16), sl));
      for (int j = 0; j < (int)g.size(); ++j)
        if (mask >> j & 1u) {
          pair_slot[(size_t)g[j] * P + b] = sl++;
          pair_chunk[(size_t)g[j] * P + b] = c;
        }
    }
    gdesc.push_back(make_int4(ul0, (int)ul.size() - ul0, kloc, (int)g.size()));
    for (int k : g) kperm.push_back(k);
    cur_slots = sl;
    ++cur_groups;
  }
  close_chunk();
  op.nchunks = (int)cdesc.size();
  op.Lu = (int)kperm.size();
  op.ngroups = (int)gdesc.size();
  // stage 2 entries per (chunk, a), sorted by slot
  std::vector<std::vector<std::pair<int, double>>> per((size_t)op.nchunks * P);
  for (const Triple& t : s.triples) {
    const size_t pk = (size_t)t.k * P + t.b;
    per[(size_t)pair_chunk[pk] * P + t.a].push_back({pair_slot[pk], t.g});
  }
  std::vector<int> eptr((size_t)op.nchunks * (P + 1)), eslot;
  std::vector<double> eg;
  for (int c = 0; c < op.nchunks; ++c) {
    for (int a = 0; a < P; ++a) {
      auto& v = per[(size_t)c * P + a];
      std::sort(v.begin(), v.end());
      eptr[(size_t)c * (P + 1) + a] = (int)eslot.size();
      for (auto& pr : v) {
        eslot.push_back(pr.first);
        eg.push_back(pr.second);
      }
    }
    eptr[(size_t)c * (P + 1) + P] = (int)eslot.size();
  }
  op.abuf_elems = op.max_chunk_k * 9 * kTW;
  op.tbuf_elems = std::max(op.max_slots, P) * kTW;
  op.xslab_elems = (int)xslab;
  op.smem = 128 + (size_t)elem * (2 * (size_t)op.abuf_elems + op.tbuf_elems + op.xslab_elems);
  if (op.smem > smem_max) return fail(SG_ERR_ARG, "tile operator: shared memory budget exceeded");
  op.apw = (P + kWarps - 1) / kWarps;
  op.pairs = (long long)std::count_if(pair_slot.begin(), pair_slot.end(), [](int v) { return v >= 0; });
  op.entries = (long long)eslot.size();
  op.cdesc.swap(cdesc);
  op.gdesc.swap(gdesc);
  op.ul.swap(ul);
  op.kperm.swap(kperm);
  op.eptr.swap(eptr);
  op.eslot.swap(eslot);
  op.eg.swap(eg);
  return SG_OK;
}

int build_tile_op(System& s, TileOp& op, int kappa, int elem, size_t smem_max, cudaStream_t st) {
  TilePlan pl;
  op = TileOp();
  SG_TRY(plan_tile_op(s, kappa, elem, smem_max, pl));
  const int m = s.pat.m, L = s.L;
  op.kappa = pl.kappa;
  op.elem = pl.elem;
  op.tiles_per_line = pl.tiles_per_line;
  op.ntiles = pl.ntiles;
  op.Pp = pl.Pp;
  op.Lu = pl.Lu;
  op.nchunks = pl.nchunks;
  op.ngroups = pl.ngroups;
  op.max_chunk_k = pl.max_chunk_k;
  op.max_slots = pl.max_slots;
  op.apw = pl.apw;
  op.abuf_elems = pl.abuf_elems;
  op.tbuf_elems = pl.tbuf_elems;
  op.xslab_elems = pl.xslab_elems;
  op.smem = pl.smem;
  SG_TRY(op.chunk.alloc(pl.cdesc.size()));
  SG_TRY(op.chunk.upload(pl.cdesc, st));
  SG_TRY(op.group.alloc(pl.gdesc.size()));
  SG_TRY(op.group.upload(pl.gdesc, st));
  SG_TRY(op.ulist.alloc(pl.ul.size()));
  SG_TRY(op.ulist.upload(pl.ul, st));
  SG_TRY(op.ent_ptr.alloc(pl.eptr.size()));
  SG_TRY(op.ent_ptr.upload(pl.eptr, st));
  SG_TRY(op.ent_slot.alloc(pl.eslot.size()));
  SG_TRY(op.ent_slot.upload(pl.eslot, st));
  if (elem == 8) {
    SG_TRY(op.ent_g.alloc(pl.eg.size()));
    SG_TRY(op.ent_g.upload(pl.eg, st));
  } else {
    std::vector<float> ef(pl.eg.begin(), pl.eg.end());
    SG_TRY(op.ent_g32.alloc(ef.size()));
    SG_TRY(op.ent_g32.upload(ef, st));
  }
  // the tiled stack
  DBuf<int> dperm;
  SG_TRY(dperm.alloc(pl.kperm.size()));
  SG_TRY(dperm.upload(pl.kperm, st));
  const size_t total = (size_t)op.ntiles * op.Lu * 9 * kTW;
  const int grid = (int)std::min<size_t>((total + 255) / 256, 152 * 64);
  if (elem == 8) {
    SG_TRY(op.stack.alloc(total));
    tile_stack_kernel<double><<<grid, 256, 0, st>>>(m, op.tiles_per_line, op.ntiles, op.Lu, L,
                                                    s.rowptr.p, dperm.p, s.stack.p, op.stack.p);
  } else {
    SG_TRY(op.stack32.alloc(total));
    tile_stack_kernel<float><<<grid, 256, 0, st>>>(m, op.tiles_per_line, op.ntiles, op.Lu, L,
                                                   s.rowptr.p, dperm.p, s.stack.p, op.stack32.p);
  }
  SG_TRY(check_launch("tile_stack"));
  SG_CUDA(cudaStreamSynchronize(st));
  dperm.release();
  SG_TRY(op.err.alloc(1));
  SG_CUDA(cudaMemsetAsync(op.err.p, 0, sizeof(int), st));
  SG_CUDA(cudaStreamSynchronize(st));
  op.ready = true;
  return SG_OK;
}

void free_tile_op(TileOp& op) {
  op.chunk.release();
  op.group.release();
  op.ulist.release();
  op.ent_ptr.release();
  op.ent_slot.release();
  op.ent_g.release();
  op.ent_g32.release();
  op.stack.release();
  op.stack32.release();
  op.err.release();
  op.ready = false;
}

template <typename T, int KAPPA, int APW>
static int launch_tile_k(const System& s, const TileOp& op, const T* X, T* Y, T alpha, const T* B,
                         T beta, cudaStream_t st, const int* done) {
  auto kern = sg_apply_tile_kernel<T, KAPPA, APW>;
  SG_TRY(ensure_smem((const void*)kern, op.smem));
  TileDims d{s.pat.m, op.tiles_per_line, op.ntiles, s.P, op.Pp, op.nchunks,
             op.abuf_elems, op.tbuf_elems, op.xslab_elems};
  int sms = 152;
  {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  }
  const int grid = std::max(1, std::min(op.ntiles, sms));
  const T* eg;
  const T* stack;
  if constexpr (sizeof(T) == 8) {
    eg = op.ent_g.p;
    stack = op.stack.p;
  } else {
    eg = op.ent_g32.p;
    stack = op.stack32.p;
  }
  TimeScope ts(s.timer, sizeof(T) == 8 ? K_APPLY_F64 : K_APPLY_LOWP, st);
  kern<<<grid, kWarps * 32, op.smem, st>>>(d, op.chunk.p, op.group.p, op.ulist.p, op.ent_ptr.p,
                                           op.ent_slot.p, eg, stack, X, Y, alpha, B, beta, done,
                                           op.err.p);
  return check_launch("sg_apply_tile");
}

template <typename T, int KAPPA>
static int launch_tile_apw(const System& s, const TileOp& op, const T* X, T* Y, T alpha,
                           const T* B, T beta, cudaStream_t st, const int* done) {
  if (op.apw <= 4) return launch_tile_k<T, KAPPA, 4>(s, op, X, Y, alpha, B, beta, st, done);
  if (op.apw <= 8) return launch_tile_k<T, KAPPA, 8>(s, op, X, Y, alpha, B, beta, st, done);
  if (op.apw <= 16) return launch_tile_k<T, KAPPA, 16>(s, op, X, Y, alpha, B, beta, st, done);
  return launch_tile_k<T, KAPPA, 32>(s, op, X, Y, alpha, B, beta, st, done);
}

template <typename T>
int launch_tile_op(const System& s, const TileOp& op, const T* X, T* Y, T alpha, const T* B,
                   T beta, cudaStream_t st, const int* done) {
  if (!op.ready) return fail(SG_ERR_ARG, "tile operator not built");
  switch (op.kappa) {
    case 1: return launch_tile_apw<T, 1>(s, op, X, Y, alpha, B, beta, st, done);
    case 2: return launch_tile_apw<T, 2>(s, op, X, Y, alpha, B, beta, st, done);
    case 3: return launch_tile_apw<T, 3>(s, op, X, Y, alpha, B, beta, st, done);
    default: return launch_tile_apw<T, 4>(s, op, X, Y, alpha, B, beta, st, done);
  }
}

template int launch_tile_op<double>(const System&, const TileOp&, const double*, double*, double,
                                    const double*, double, cudaStream_t, const int*);
template int launch_tile_op<float>(const System&, const TileOp&, const float*, float*, float,
                                   const float*, float, cudaStream_t, const int*);

}  // namespace sg
