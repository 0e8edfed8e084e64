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
// FP32 runs both stages in packed FP32x2 arithmetic: a lane owns two adjacent rows and the two
// half-warps take different union entries (stage 1) or entry ranges (stage 2), which halves the
// load and multiply-add instructions per row; the stencil product is taken in difference form
// (the row sum in the centre slot, see stencil_diffs_f32).  Its work is split at setup into equal
// contiguous shares (eight per chunk in stage 1, sixteen in stage 2).  FP64 keeps one row per lane.
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

// ---- FP32 stages in packed FP32x2 arithmetic (fma.rn.f32x2: one instruction for two rows)
//
// In FP32 a lane owns the row pair (2 lp, 2 lp + 1) of the tile, lp = lane mod 16, and the two
// half-warps work on different items (union entries in stage 1, runs in stage 2), so one warp
// instruction still serves 32 row-items but the loads of a row pair are single 8-byte accesses
// and the multiply-adds are packed.  Row 2 lp reads its stencil columns at slab offsets 2 lp ..
// 2 lp + 2 and row 2 lp + 1 at 2 lp + 1 .. 2 lp + 3, so two aligned 8-byte loads per grid line
// give both rows' three values.

__device__ __forceinline__ float2 ld2(const float* p) { return *reinterpret_cast<const float2*>(p); }
__device__ __forceinline__ void st2(float* p, float2 v) { *reinterpret_cast<float2*>(p) = v; }

// The stencil values of both rows for chaos index b (xp = the b slab + 2 lp) in difference form:
// d[4] = x_c, d[e] = x_e - x_c otherwise (each difference rounded once), so that
// sum_e A_e x_e = (sum_e A_e) x_c + sum_{e != c} A_e (x_e - x_c) with the row sum stored in the
// centre slot.  A stiffness row sums to about zero, so the direct form cancels ~1/h^2-sized
// terms in FP32, while the differences of a smooth x are small and their products carry no such
// cancellation (the mixed solver's refinement then gains more digits per cycle).
__device__ __forceinline__ void stencil_diffs_f32(const float* xp, float2 (&d)[9]) {
  float2 p0[3], p1[3];
#pragma unroll
  for (int dy = 0; dy < 3; ++dy) {
    p0[dy] = ld2(xp + dy * kSlab);
    p1[dy] = ld2(xp + dy * kSlab + 2);
  }
  const float2 xc = make_float2(p0[1].y, p1[1].x);
  const float2 m1 = make_float2(-1.0f, -1.0f);
#pragma unroll
  for (int dy = 0; dy < 3; ++dy) {
    d[dy * 3 + 0] = __ffma2_rn(xc, m1, p0[dy]);
    d[dy * 3 + 2] = __ffma2_rn(xc, m1, p1[dy]);
    if (dy != 1) d[dy * 3 + 1] = make_float2(p0[dy].y - xc.x, p1[dy].x - xc.y);
  }
  d[4] = xc;
}

// T for the k of a group that need this b (mask bit j for the group's j-th k): the row sum times
// x_c plus the eight stiffness values times the differences, one dependent chain per k (the
// chains of the group's k and of the two half-warps' entries overlap).
template <int KAPPA>
__device__ __forceinline__ void pair_products_f32(const float2 (&a)[KAPPA][9],
                                                  const float2 (&d)[9], int mask, int sl,
                                                  float* Tp) {
#pragma unroll
  for (int j = 0; j < KAPPA; ++j) {
    float2 t0 = __fmul2_rn(a[j][4], d[4]);
#pragma unroll
    for (int e = 0; e < 9; ++e)
      if (e != 4) t0 = __ffma2_rn(a[j][e], d[e], t0);
    if (mask >> j & 1) st2(Tp + (size_t)(sl + __popc(mask & ((1 << j) - 1))) * kTW, t0);
  }
}

// Stage 1 of one piece (count entries of the union list gl of group gd): half-warp h takes the
// entries u + h, u = 0, 2, 4, ...  An idle half (odd count) reads entry 0 and stores nothing.
template <int KAPPA>
__device__ __forceinline__ void stage1_piece_f32(int count, int4 gd, const float* Ab,
                                                 const int2* gl, const float* Xs, float* Ts,
                                                 int lane) {
  const int half = lane >> 4, lp = lane & 15;
  float2 a[KAPPA][9];
#pragma unroll
  for (int j = 0; j < KAPPA; ++j)
#pragma unroll
    for (int e = 0; e < 9; ++e)
      a[j][e] = j < gd.w ? ld2(Ab + ((size_t)(gd.z + j) * 9 + e) * kTW + 2 * lp)
                         : make_float2(0.0f, 0.0f);
  const float* xl = Xs + 2 * lp;
  float* Tp = Ts + 2 * lp;
#pragma unroll 2
  for (int u = 0; u < count; u += 2) {
    const int q = u + half;
    const int2 e = gl[q < count ? q : 0];
    float2 d[9];
    stencil_diffs_f32(xl + (e.x & 0xffff) * (3 * kSlab), d);
    pair_products_f32<KAPPA>(a, d, q < count ? (e.x >> 16) : 0, e.y, Tp);
  }
}

// Stage 2 of one half-warp: its entries [q0, q1) (whole runs, in order of a; packed slot | a << 16
// | last << 24) accumulated per row pair and added to Y[a] at the last entry of each run.  The
// two halves of a warp step side by side for as many steps as the longer range.
__device__ __forceinline__ void stage2_range_f32(int q0, int q1, const TEnt<float>* ent,
                                                 const float* Ts, float* Ys, int lane) {
  const int lp = lane & 15;
  const float* Tp = Ts + 2 * lp;
  float* Yp = Ys + 2 * lp;
  const int n = q1 - q0;
  const int steps = max(n, __shfl_xor_sync(0xffffffffu, n, 16));
  float2 acc = make_float2(0.0f, 0.0f);
  for (int t = 0; t < steps; t += 2) {
    // two entries per step: their loads go before either product
    const bool ok0 = t < n, ok1 = t + 1 < n;
    // (an idle half reads entry 0 of the chunk and T slot 0, both in range, and uses neither)
    const TEnt<float> f0 = ent[ok0 ? q0 + t : 0];
    const TEnt<float> f1 = ent[ok1 ? q0 + t + 1 : 0];
    const float2 t0 = ld2(Tp + (size_t)(ok0 ? f0.slot & 0xffff : 0) * kTW);
    const float2 t1 = ld2(Tp + (size_t)(ok1 ? f1.slot & 0xffff : 0) * kTW);
    if (ok0) {
      acc = __ffma2_rn(make_float2(f0.g, f0.g), t0, acc);
      if (f0.slot >> 24) {
        float* yp = Yp + (size_t)(f0.slot >> 16 & 0xff) * kTW;
        st2(yp, __fadd2_rn(ld2(yp), acc));
        acc = make_float2(0.0f, 0.0f);
      }
    }
    if (ok1) {
      acc = __ffma2_rn(make_float2(f1.g, f1.g), t1, acc);
      if (f1.slot >> 24) {
        float* yp = Yp + (size_t)(f1.slot >> 16 & 0xff) * kTW;
        st2(yp, __fadd2_rn(ld2(yp), acc));
        acc = make_float2(0.0f, 0.0f);
      }
    }
  }
}

// Side table of one chunk (16-byte aligned sections, offsets in the header, bytes):
//   int hdr[8]   = {off_ul, off_s1ptr, off_s1, off_s2ptr, off_s2, off_ent, off_gd, 0}
//   int2 ul[]    union lists of the chunk's groups: (b | mask << 16, first T slot)
//   int s1ptr[9] per-warp ranges of stage-1 pieces; int4 s1[] = {group, first entry, count, 0}
//   int s2ptr[9] per-warp ranges of stage-2 runs;   int4 s2[] = {a, first entry, end entry, 0}
//   TEnt ent[]   stage-2 entries (T slot, G_k[a,b]) sorted by a
//   int4 gd[]    the chunk's groups: {union list start, length, first k position, k count}
// The pieces and runs are split over the warps at setup so every warp gets about the same work,
// and each output a of a chunk belongs to one warp's run, so Y accumulates without conflicts.
template <typename T, int KAPPA, int MINB>
__global__ void __launch_bounds__(kWarps * 32, MINB) sg_apply_tile_kernel(
    TileArgs d, const int4* __restrict__ chunk, const int4* __restrict__ chunkx,
    const unsigned char* __restrict__ side,
    const T* __restrict__ stack, const T* __restrict__ X, T* __restrict__ Y, T alpha,
    const T* __restrict__ B, T beta, const int* __restrict__ done, int* __restrict__ err) {
  if (done != nullptr && *done) return;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem_raw);  // 2 barriers
  int* s_fail = reinterpret_cast<int*>(smem_raw + 16);
  // the ring slots are addressed as smem_raw + offset (not through an array of pointers), so
  // that every access to them compiles to a shared-memory access
  const unsigned a_base = 128, s_base = 128 + 2 * (unsigned)d.abytes_slot;
  T* Ts = reinterpret_cast<T*>(smem_raw + 128 + 2 * (size_t)d.abytes_slot + 2 * (size_t)d.sbytes_slot);
  T* Ys = Ts + d.tbuf_elems;              // P x 32 accumulators of the tile
  T* Xs = Ys + (size_t)d.P * kTW;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int P = d.P, m = d.m;

  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    *s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  }
  __syncthreads();

  // one work item = (tile, chunk): the chunk's stack values of the tile and its side table,
  // two bulk copies completing on the slot's barrier
  auto issue = [&](int t, int c, int slot) {
    const int4 cd = chunk[c], cx = chunkx[c];
    const unsigned abytes = (unsigned)((size_t)cd.y * 9 * kTW * sizeof(T));
    mbar_expect_tx(&bar[slot], abytes + (unsigned)cx.y);
    bulk_g2s(smem_raw + a_base + slot * d.abytes_slot,
             stack + (size_t)t * d.kstride + (size_t)cd.x * 9 * kTW, abytes, &bar[slot]);
    bulk_g2s(smem_raw + s_base + slot * d.sbytes_slot, side + (size_t)cx.x * 16, (unsigned)cx.y,
             &bar[slot]);
  };

  long long it = 0;          // work items of this CTA so far
  bool next_issued = false;  // whether the copies of item it + 1 are in flight
  if (blockIdx.x < d.ntiles && tid == 0) issue(blockIdx.x, 0, 0);
  bool failed = false;

  for (int t = blockIdx.x; t < d.ntiles && !failed; t += gridDim.x) {
    const int y = 1 + t / d.tiles_per_line;
    const int x0 = 1 + (t % d.tiles_per_line) * kTW;
    const int nrows = min(kTW, m - 1 - x0);
    // X on lines y-1, y, y+1 for nodes x0-1 .. x0+32 (zero beyond the mesh), chaos-major:
    // Xs[(b * 3 + dy) * kSlab + xi], so a lane's 9 stencil neighbours of one b sit at fixed
    // offsets from one address; one warp per node reads the node's P values (coalesced)
    for (int nd = w; nd < 3 * kSlab; nd += kWarps) {
      const int dy = nd / kSlab, xi = nd - dy * kSlab;
      const int x = x0 - 1 + xi;
      const T* src = X + ((size_t)(y - 1 + dy) * m + x) * P;
      for (int b = lane; b < P; b += 32) Xs[(b * 3 + dy) * kSlab + xi] = x < m ? src[b] : T(0);
    }
    for (int i = tid; i < P * kTW; i += blockDim.x) Ys[i] = T(0);

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
      const T* Ab = reinterpret_cast<const T*>(smem_raw + a_base + slot * d.abytes_slot);
      const unsigned char* Sb = smem_raw + s_base + slot * d.sbytes_slot;
      const int* hdr = reinterpret_cast<const int*>(Sb);
      const int4* gdl = reinterpret_cast<const int4*>(Sb + hdr[6]);
      const int4 cd = chunk[c];
      // ---- stage 1: this warp's pieces of the groups' union lists
      if constexpr (sizeof(T) == 4) {
        const int2* ul = reinterpret_cast<const int2*>(Sb + hdr[0]);
        const int* s1ptr = reinterpret_cast<const int*>(Sb + hdr[1]);
        const int4* s1 = reinterpret_cast<const int4*>(Sb + hdr[2]);
        for (int pc = s1ptr[w]; pc < s1ptr[w + 1]; ++pc) {
          const int4 piece = s1[pc];
          const int4 gd = gdl[piece.x];
          stage1_piece_f32<KAPPA>(piece.z, gd, Ab, ul + gd.x + piece.y, Xs, Ts, lane);
        }
      } else {
        // FP64: one row per lane, two b per step
        const int2* ul = reinterpret_cast<const int2*>(Sb + hdr[0]);
        const int* s1ptr = reinterpret_cast<const int*>(Sb + hdr[1]);
        const int4* s1 = reinterpret_cast<const int4*>(Sb + hdr[2]);
        for (int pc = s1ptr[w]; pc < s1ptr[w + 1]; ++pc) {
          const int4 piece = s1[pc];
          const int4 gd = gdl[piece.x];  // union start, length, first k position, k count
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
          const int2* gl = ul + gd.x + piece.y;
          // T for the k of the group that need this b, each 9-term sum as three partial sums
          // over the stencil lines (a short dependency chain); only the needed k are computed
          // (the FP64 pipe, not latency, bounds this form on this GPU)
          auto pairs_of = [&](int bm, int sl, const T* xv) {
            const int mask = bm >> 16;
#pragma unroll
            for (int j = 0; j < KAPPA; ++j) {
              const bool need = mask & (1 << j);
              if (!need) continue;
              T s0 = a[j][0] * xv[0], s1 = a[j][3] * xv[3], s2 = a[j][6] * xv[6];
              s0 = fma(a[j][1], xv[1], s0);
              s1 = fma(a[j][4], xv[4], s1);
              s2 = fma(a[j][7], xv[7], s2);
              s0 = fma(a[j][2], xv[2], s0);
              s1 = fma(a[j][5], xv[5], s1);
              s2 = fma(a[j][8], xv[8], s2);
              if (need) Ts[(size_t)(sl + __popc(mask & ((1 << j) - 1))) * kTW + lane] = (s0 + s1) + s2;
            }
          };
          int u = 0;
          for (; u + 1 < piece.z; u += 2) {
            const int2 e0 = gl[u], e1 = gl[u + 1];
            const int b0 = e0.x & 0xffff, b1 = e1.x & 0xffff;
            T x0v[9], x1v[9];
            const T* xp0 = Xs + b0 * (3 * kSlab) + lane;
            const T* xp1 = Xs + b1 * (3 * kSlab) + lane;
#pragma unroll
            for (int dy = 0; dy < 3; ++dy)
#pragma unroll
              for (int dx = 0; dx < 3; ++dx) {
                x0v[dy * 3 + dx] = xp0[dy * kSlab + dx];
                x1v[dy * 3 + dx] = xp1[dy * kSlab + dx];
              }
            pairs_of(e0.x, e0.y, x0v);
            pairs_of(e1.x, e1.y, x1v);
          }
          if (u < piece.z) {
            const int2 e0 = gl[u];
            const int b0 = e0.x & 0xffff;
            T x0v[9];
            const T* xp0 = Xs + b0 * (3 * kSlab) + lane;
#pragma unroll
            for (int dy = 0; dy < 3; ++dy)
#pragma unroll
              for (int dx = 0; dx < 3; ++dx) x0v[dy * 3 + dx] = xp0[dy * kSlab + dx];
            pairs_of(e0.x, e0.y, x0v);
          }
        }
      }
      __syncthreads();
      // ---- stage 2: this warp's runs: Y[a, row] += sum over the run's entries of G T[slot]
      if constexpr (sizeof(T) == 4) {
        const int* s2ptr = reinterpret_cast<const int*>(Sb + hdr[3]);
        const int wk = 2 * w + (lane >> 4);
        stage2_range_f32(s2ptr[wk], s2ptr[wk + 1],
                         reinterpret_cast<const TEnt<float>*>(Sb + hdr[5]), Ts, Ys, lane);
      } else {
        const int* s2ptr = reinterpret_cast<const int*>(Sb + hdr[3]);
        const int4* s2 = reinterpret_cast<const int4*>(Sb + hdr[4]);
        const TEnt<T>* ent = reinterpret_cast<const TEnt<T>*>(Sb + hdr[5]);
        // runs are short (about two entries), so four of them go at a time: their chains of
        // dependent shared-memory loads overlap; the runs of a warp have distinct outputs a
        const int r_end = s2ptr[w + 1];
        int rn = s2ptr[w];
        for (; rn + 4 <= r_end; rn += 4) {
          int4 run[4];
          T acc[4];
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            run[v] = s2[rn + v];
            acc[v] = T(0);
          }
          int len = 0;
#pragma unroll
          for (int v = 0; v < 4; ++v) len = max(len, run[v].z - run[v].y);
          for (int t = 0; t < len; ++t) {
#pragma unroll
            for (int v = 0; v < 4; ++v) {
              const int q = run[v].y + t;
              if (q < run[v].z) {
                const TEnt<T> f = ent[q];
                acc[v] = fma(f.g, Ts[(size_t)f.slot * kTW + lane], acc[v]);
              }
            }
          }
#pragma unroll
          for (int v = 0; v < 4; ++v) Ys[(size_t)run[v].x * kTW + lane] += acc[v];
        }
        for (; rn < r_end; ++rn) {
          const int4 run = s2[rn];
          T s0 = T(0);
          for (int q = run.y; q < run.z; ++q) {
            const TEnt<T> f0 = ent[q];
            s0 = fma(f0.g, Ts[(size_t)f0.slot * kTW + lane], s0);
          }
          Ys[(size_t)run.x * kTW + lane] += s0;
        }
      }
      __syncthreads();
    }
    if (failed) break;
    // ---- epilogue: Y rows of the tile (coalesced)
    const size_t row0 = (size_t)y * m + x0;
    for (int r = w; r < nrows; r += kWarps) {
      const size_t o = (row0 + r) * P;
      for (int a = lane; a < P; a += 32) {
        T v = alpha * Ys[(size_t)a * kTW + r];
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

// Kernel variants that are instantiated: FP64 with kappa 1 or 2, FP32 with kappa 1, 2 or 4,
// each for one or two CTAs per SM.
inline bool tile_variant_ok(int elem, int kappa, int ctas) {
  if (ctas != 1 && ctas != 2) return false;
  if (elem == 8) return kappa == 1 || kappa == 2;
  return kappa == 1 || kappa == 2 || kappa == 4;
}

template <typename T, int KAPPA, int MINB>
int launch_tile_k(const System& s, const TileOp& op, const T* X, T* Y, T alpha, const T* B,
                  T beta, cudaStream_t st, const int* done) {
  auto kern = sg_apply_tile_kernel<T, KAPPA, MINB>;
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
  kern<<<grid, kWarps * 32, op.smem, st>>>(d, op.chunk.p, op.chunkx.p, op.side.p,
                                           stack, X, Y, alpha, B, beta, done, op.err.p);
  return check_launch("sg_apply_tile");
}

}  // namespace

}  // namespace sg
