// The SG operator Y = sum_k A_k X G_k^T (Eqs. stochastic_matrix and K_matrix), row-tiled form:
// the kernel template, shared by the FP64 and FP32 translation units.
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
#pragma once

#include <algorithm>

#include "sg_internal.h"

namespace sg {

namespace {

constexpr int kTW = 32;       // rows per tile
constexpr int kWarps = 8;     // warps per CTA: groups per chunk and a-strides of stage 2
constexpr int kSlab = kTW + 2;
constexpr long long kWaitLimit = 1LL << 22;

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

// Stage-2 entry of the side table: T slot and G_k[a,b].
template <typename T>
struct TEnt;
template <>
struct TEnt<float> {
  int slot;
  float g;
};
template <>
struct TEnt<double> {
  int slot, pad;
  double g;
};

struct TileArgs {
  int m, tiles_per_line, ntiles, P, Pp, nchunks;
  long long kstride;                      // elements of one tile's stack
  int abytes_slot, sbytes_slot, tbuf_elems;
};

template <typename T, int KAPPA, int APW, int MINB>
__global__ void __launch_bounds__(kWarps * 32, MINB) sg_apply_tile_kernel(
    TileArgs d, const int4* __restrict__ chunk, const int4* __restrict__ chunkx,
    const int4* __restrict__ group, const unsigned char* __restrict__ side,
    const T* __restrict__ stack, const T* __restrict__ X, T* __restrict__ Y, T alpha,
    const T* __restrict__ B, T beta, const int* __restrict__ done, int* __restrict__ err) {
  if (done != nullptr && *done) return;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem_raw);  // 2 barriers
  int* s_fail = reinterpret_cast<int*>(smem_raw + 16);
  unsigned char* Aslot[2] = {smem_raw + 128, smem_raw + 128 + d.abytes_slot};
  unsigned char* Sslot[2] = {smem_raw + 128 + 2 * (size_t)d.abytes_slot,
                             smem_raw + 128 + 2 * (size_t)d.abytes_slot + d.sbytes_slot};
  T* Ts = reinterpret_cast<T*>(smem_raw + 128 + 2 * (size_t)d.abytes_slot + 2 * (size_t)d.sbytes_slot);
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

  // one work item = (tile, chunk): the chunk's stack values of the tile and its side table (union
  // lists and stage-2 entries), two bulk copies completing on the slot's barrier
  auto issue = [&](int t, int c, int slot) {
    const int4 cd = chunk[c], cx = chunkx[c];
    const unsigned abytes = (unsigned)((size_t)cd.y * 9 * kTW * sizeof(T));
    mbar_expect_tx(&bar[slot], abytes + (unsigned)cx.y);
    bulk_g2s(Aslot[slot], stack + (size_t)t * d.kstride + (size_t)cd.x * 9 * kTW, abytes, &bar[slot]);
    bulk_g2s(Sslot[slot], side + (size_t)cx.x * 16, (unsigned)cx.y, &bar[slot]);
  };

  T acc[APW];
  long long it = 0;          // work items of this CTA so far
  bool next_issued = false;  // whether the copies of item it + 1 are in flight
  if (blockIdx.x < d.ntiles && tid == 0) issue(blockIdx.x, 0, 0);
  bool failed = false;

  for (int t = blockIdx.x; t < d.ntiles && !failed; t += gridDim.x) {
    const int y = 1 + t / d.tiles_per_line;
    const int x0 = 1 + (t % d.tiles_per_line) * kTW;
    const int nrows = min(kTW, m - 1 - x0);
    // X on lines y-1, y, y+1 for nodes x0-1 .. x0+32 (zero beyond the mesh): one warp per node
    for (int nd = w; nd < 3 * kSlab; nd += kWarps) {
      const int dy = nd / kSlab, xi = nd - dy * kSlab;
      const int x = x0 - 1 + xi;
      const T* src = X + ((size_t)(y - 1 + dy) * m + x) * P;
      T* dst = Xs + (size_t)nd * Pp;
      for (int b = lane; b < P; b += 32) dst[b] = x < m ? src[b] : T(0);
    }
#pragma unroll
    for (int j = 0; j < APW; ++j) acc[j] = T(0);

    for (int c = 0; c < d.nchunks; ++c, ++it) {
      // prefetch the next work item into the other slot (its last readers finished before the
      // barrier that closed the previous item)
      if (tid == 0) {
        int tn = t, cn = c + 1;
        if (cn == d.nchunks) {
          tn = t + gridDim.x;
          cn = 0;
        }
        next_issued = tn < d.ntiles;
        if (next_issued) issue(tn, cn, (int)((it + 1) & 1));
      }
      const int slot = (int)(it & 1);
      if (!mbar_wait_bounded(&bar[slot], (unsigned)((it >> 1) & 1))) *s_fail = 1;
      __syncthreads();
      if (*s_fail) {
        failed = true;
        break;
      }
      const T* Ab = reinterpret_cast<const T*>(Aslot[slot]);
      const unsigned char* Sb = Sslot[slot];
      const int4 cd = chunk[c];
      // ---- stage 1: T for the pairs of this warp's group, two b per step
      if (w < cd.w) {
        const int4 gd = group[cd.z + w];  // union list start (in the chunk), length, k position, k count
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
        const int2* ul = reinterpret_cast<const int2*>(Sb) + gd.x;
        auto pairs_of = [&](int bm, int sl, const T* xv) {
          const int mask = bm >> 16;
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
        };
        int u = 0;
        for (; u + 1 < gd.y; u += 2) {
          const int2 e0 = ul[u], e1 = ul[u + 1];
          const int b0 = e0.x & 0xffff, b1 = e1.x & 0xffff;
          T x0v[9], x1v[9];
#pragma unroll
          for (int dy = 0; dy < 3; ++dy)
#pragma unroll
            for (int dx = 0; dx < 3; ++dx) {
              const int base = (dy * kSlab + lane + dx) * Pp;
              x0v[dy * 3 + dx] = Xs[base + b0];
              x1v[dy * 3 + dx] = Xs[base + b1];
            }
          pairs_of(e0.x, e0.y, x0v);
          pairs_of(e1.x, e1.y, x1v);
        }
        if (u < gd.y) {
          const int2 e0 = ul[u];
          const int b0 = e0.x & 0xffff;
          T x0v[9];
#pragma unroll
          for (int dy = 0; dy < 3; ++dy)
#pragma unroll
            for (int dx = 0; dx < 3; ++dx) x0v[dy * 3 + dx] = Xs[(dy * kSlab + lane + dx) * Pp + b0];
          pairs_of(e0.x, e0.y, x0v);
        }
      }
      __syncthreads();
      // ---- stage 2: Y[row, a] += sum G T over this chunk's entries of the warp's outputs
      {
        const int4 cx = chunkx[c];
        const int* ep = reinterpret_cast<const int*>(Sb + cx.z);
        const TEnt<T>* ent = reinterpret_cast<const TEnt<T>*>(Sb + cx.w);
#pragma unroll
        for (int j = 0; j < APW; ++j) {
          const int a = w + kWarps * j;
          if (a < P) {
            T s0 = T(0), s1 = T(0);
            int q = ep[a];
            const int q1 = ep[a + 1];
            for (; q + 1 < q1; q += 2) {
              const TEnt<T> f0 = ent[q], f1 = ent[q + 1];
              s0 = fma(f0.g, Ts[(size_t)f0.slot * kTW + lane], s0);
              s1 = fma(f1.g, Ts[(size_t)f1.slot * kTW + lane], s1);
            }
            if (q < q1) {
              const TEnt<T> f0 = ent[q];
              s0 = fma(f0.g, Ts[(size_t)f0.slot * kTW + lane], s0);
            }
            acc[j] += s0 + s1;
          }
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
    for (int r = w; r < nrows; r += kWarps) {
      const size_t o = (row0 + r) * P;
      for (int a = lane; a < P; a += 32) {
        T v = alpha * Ts[(size_t)a * kTW + r];
        if (B != nullptr) v = fma(beta, B[o + a], v);
        Y[o + a] = v;
      }
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

// Kernel variants that are instantiated (the others would spill registers or are not needed):
// FP64 with kappa 1 or 2, two CTAs per SM only without spills; FP32 with kappa 1, 2 or 4.
inline int tile_apw_bucket(int apw) { return apw <= 8 ? 8 : apw <= 16 ? 16 : 32; }
inline bool tile_variant_ok(int elem, int kappa, int apw, int ctas) {
  const int b = tile_apw_bucket(apw);
  if (elem == 8) {
    if (kappa != 1 && kappa != 2) return false;
    if (ctas == 2) return (kappa == 1 && b <= 16) || (kappa == 2 && b == 8);
    return true;
  }
  if (kappa != 1 && kappa != 2 && kappa != 4) return false;
  return ctas == 1 || b <= 16;
}

template <typename T, int KAPPA, int APW, int MINB>
int launch_tile_k(const System& s, const TileOp& op, const T* X, T* Y, T alpha, const T* B,
                  T beta, cudaStream_t st, const int* done) {
  auto kern = sg_apply_tile_kernel<T, KAPPA, APW, MINB>;
  SG_TRY(ensure_smem((const void*)kern, op.smem));
  TileArgs d{s.pat.m, op.tiles_per_line, op.ntiles, s.P, op.Pp, op.nchunks,
             (long long)op.Lu * 9 * kTW, op.abytes_slot, op.sbytes_slot, op.tbuf_elems};
  int sms = 152;
  {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  }
  const int grid = std::max(1, std::min(op.ntiles, sms * MINB));
  const T* stack;
  if constexpr (sizeof(T) == 8) stack = op.stack.p;
  else stack = op.stack32.p;
  TimeScope ts(s.timer, sizeof(T) == 8 ? K_APPLY_F64 : K_APPLY_LOWP, st);
  kern<<<grid, kWarps * 32, op.smem, st>>>(d, op.chunk.p, op.chunkx.p, op.group.p, op.side.p,
                                           stack, X, Y, alpha, B, beta, done, op.err.p);
  return check_launch("sg_apply_tile");
}

}  // namespace

}  // namespace sg
