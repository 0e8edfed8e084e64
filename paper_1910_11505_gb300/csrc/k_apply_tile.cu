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
#include <array>
#include <cmath>
#include <cstring>
#include <map>
#include <numeric>

#include "k_apply_tile.cuh"

namespace sg {

namespace {

// Tiled stack from the nnz x L stack: for tile t, permuted k position kp, entry e, row r:
// value of A_{kperm[kp]} at entry e of node (x0 + r, y), 0 for rows beyond the line.  In FP32 the
// centre entry (e = 4) holds the row sum of the nine instead (summed in FP64), for the difference
// form of the stencil product (see k_apply_tile.cuh).
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
      if (sizeof(TS) == 4 && e == 4)
        for (int q = 0; q < 9; ++q) v += stack[((size_t)rowptr[node] + q) * L + kperm[kp]];
      else
        v = stack[((size_t)rowptr[node] + e) * L + kperm[kp]];
    }
    out[idx] = (TS)v;
  }
}

}  // namespace

// ------------------------------------------------------------------ host: tables and launch

static size_t round16(size_t v) { return (v + 15) / 16 * 16; }
static size_t round128(size_t v) { return (v + 127) / 128 * 128; }

// Plan of the row-tiled operator for kappa k per group and ``ctas`` CTAs per SM, whose shared
// memory must fit smem_max bytes per CTA.  Groups: seeds in order of total degree, each grown by
// the k whose b list overlaps the group's union most (Jaccard).  Chunks: consecutive groups, at
// most one per warp, cut so that T slots, stack values and side table fit the budget.
int plan_tile_op(const System& s, int kappa, int elem, size_t smem_max, TilePlan& op, int ctas) {
  const int P = s.P, L = s.L, m = s.pat.m;
  op = TilePlan();
  op.kappa = kappa;
  op.elem = elem;
  op.ctas = ctas;
  if (m < 3 || kappa < 1 || kappa > 4 || P > 256 || ctas < 1 || ctas > 2)
    return fail(SG_ERR_ARG, "tile operator: unsupported sizes");
  if (!tile_variant_ok(elem, kappa, ctas))
    return fail(SG_ERR_ARG, "tile operator: no kernel variant for these sizes");
  op.tiles_per_line = (m - 2 + kTW - 1) / kTW;
  op.ntiles = op.tiles_per_line * (m - 2);
  op.Pp = P | 1;
  const int words = (P + 63) / 64;
  std::vector<unsigned long long> bset((size_t)L * words, 0ULL);
  std::vector<int> bcount(L, 0);
  std::vector<std::vector<int>> nA((size_t)L * P);  // a of each (k, b)
  for (const Triple& t : s.triples) {
    unsigned long long& wd = bset[(size_t)t.k * words + t.b / 64];
    const unsigned long long bit = 1ULL << (t.b % 64);
    if (!(wd & bit)) {
      wd |= bit;
      bcount[t.k]++;
    }
  }
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
  // entries (a, G) per (k, b), a ascending
  std::vector<std::vector<std::pair<int, double>>> pe((size_t)L * P);
  for (const Triple& t : s.triples) pe[(size_t)t.k * P + t.b].push_back({t.a, t.g});
  const size_t esize = elem == 8 ? 16 : 8;
  const size_t xslab = (size_t)3 * kSlab * op.Pp;
  const size_t abytes_max = round128((size_t)kWarps * kappa * 9 * kTW * elem);
  const size_t fixed = 128 + 2 * abytes_max + round128(elem * xslab) + (size_t)elem * P * kTW;
  if (fixed + (size_t)elem * kTW > smem_max)
    return fail(SG_ERR_ARG, "tile operator: P too large for shared memory");
  int slot_cap = (int)std::min<size_t>(16384, (smem_max - fixed) / ((size_t)elem * kTW));
  for (int attempt = 0; attempt < 40; ++attempt) {
    // cut the chunks for this slot capacity
    op.cdesc.clear();
    op.cxdesc.clear();
    op.gdesc.clear();
    op.kperm.clear();
    op.side.clear();
    op.max_chunk_k = op.max_slots = 0;
    op.max_side = 0;
    op.pairs = op.entries = 0;
    op.visits = op.s1_steps = op.s2_steps = 0;
    bool ok = true;
    size_t gi = 0;
    while (gi < groups.size() && ok) {
      const int k0 = (int)op.kperm.size();
      const int g0 = (int)op.gdesc.size();
      int slots = 0;
      std::vector<int2> ul;
      std::vector<std::vector<std::pair<int, double>>> perA(P);  // (slot, G) per a
      while (gi < groups.size() && (int)op.gdesc.size() - g0 < kWarps) {
        const auto& g = groups[gi];
        int gslots = 0;
        for (int k : g) gslots += bcount[k];
        if (gslots > slot_cap) {
          ok = false;
          break;
        }
        if (slots + gslots > slot_cap) break;
        const int kloc = (int)op.kperm.size() - k0;
        const int ul0 = (int)ul.size();
        for (int b = 0; b < P; ++b) {
          unsigned mask = 0;
          for (int j = 0; j < (int)g.size(); ++j)
            if (bset[(size_t)g[j] * words + b / 64] >> (b % 64) & 1ULL) mask |= 1u << j;
          if (!mask) continue;
          ul.push_back(make_int2(b | (int)(mask << 16), slots));
          for (int j = 0; j < (int)g.size(); ++j)
            if (mask >> j & 1u) {
              for (auto& ae : pe[(size_t)g[j] * P + b]) perA[ae.first].push_back({slots, ae.second});
              ++slots;
              ++op.pairs;
            }
        }
        op.gdesc.push_back(make_int4(ul0, (int)ul.size() - ul0, kloc, (int)g.size()));
        for (int k : g) op.kperm.push_back(k);
        ++gi;
      }
      if (!ok) break;
      // side table of the chunk (layout in k_apply_tile.cuh): union lists, the stage-1 pieces
      // and stage-2 runs of each warp, the entries sorted by a
      const int ng = (int)op.gdesc.size() - g0;
      // stage 1: split the groups' union lists into pieces of about equal cost per warp
      std::vector<std::vector<int4>> pw(kWarps);
      if (elem == 4) {
        // FP32 forms every k of a group for each union entry, so every entry costs the same: the
        // union entries in group order, cut into eight contiguous ranges of at most
        // ceil(entries / 8) each (a range that spans groups is one piece per group)
        const int total = (int)ul.size();
        const int per = std::max(1, (total + kWarps - 1) / kWarps);
        int wk = 0, filled = 0;
        for (int g = 0; g < ng; ++g) {
          const int4 gd = op.gdesc[g0 + g];
          int u = 0;
          while (u < gd.y) {
            if (filled >= per && wk < kWarps - 1) {
              ++wk;
              filled = 0;
            }
            const int take = wk == kWarps - 1 ? gd.y - u : std::min(gd.y - u, per - filled);
            pw[wk].push_back(make_int4(g, u, take, 0));
            u += take;
            filled += take;
          }
        }
      } else {
        // FP64 forms only the needed pairs: cost of a union entry = its 9 X loads plus 10 per pair
        double total = 0.0;
        std::vector<double> cost(ul.size());
        for (size_t u = 0; u < ul.size(); ++u) {
          cost[u] = 9.0 + 10.0 * __builtin_popcount((unsigned)ul[u].x >> 16);
          total += cost[u];
        }
        const double per = total / kWarps;
        int wk = 0;
        double acc = 0.0;
        for (int g = 0; g < ng; ++g) {
          const int4 gd = op.gdesc[g0 + g];
          int u0 = 0;
          for (int u = 0; u < gd.y; ++u) {
            acc += cost[gd.x + u];
            if (acc >= per * (wk + 1) && wk < kWarps - 1 && u + 1 < gd.y) {
              pw[wk].push_back(make_int4(g, u0, u + 1 - u0, 0));
              u0 = u + 1;
              ++wk;
            }
          }
          if (gd.y > u0) pw[wk].push_back(make_int4(g, u0, gd.y - u0, 0));
          while (wk < kWarps - 1 && acc >= per * (wk + 1)) ++wk;
        }
      }
      // stage 2: runs (one per a with entries), entries sorted by a, split over the warps at run
      // boundaries with about equal entry counts
      std::vector<int4> runs;
      size_t nent = 0;
      for (int a = 0; a < P; ++a) {
        std::sort(perA[a].begin(), perA[a].end());
        if (!perA[a].empty()) {
          runs.push_back(make_int4(a, (int)nent, (int)(nent + perA[a].size()), 0));
          nent += perA[a].size();
        }
      }
      // FP32: sixteen workers (the half-warps) take contiguous ranges of whole runs with about
      // equal entry counts; s2ptr holds their entry offsets.  FP64: the warps take ranges of runs
      // with about equal cost; s2ptr holds their run offsets.
      const int nworkers = elem == 4 ? 2 * kWarps : kWarps;
      std::vector<int> s2ptr(nworkers + 1, elem == 4 ? (int)nent : (int)runs.size());
      if (elem == 4) {
        const double per = (double)nent / nworkers;
        int wk = 0;
        s2ptr[0] = 0;
        // cut at the run boundary nearest to each target
        for (size_t r = 0; r < runs.size(); ++r) {
          while (wk < nworkers - 1 && runs[r].z > per * (wk + 1)) {
            const double before = per * (wk + 1) - runs[r].y, after = runs[r].z - per * (wk + 1);
            if (before <= after) {
              s2ptr[++wk] = runs[r].y;
            } else {
              s2ptr[++wk] = runs[r].z;
              break;
            }
          }
        }
        while (wk < nworkers - 1) s2ptr[++wk] = (int)nent;
        s2ptr[nworkers] = (int)nent;
      } else {
        const double per = (double)(nent + runs.size()) / kWarps;
        double acc = 0.0;
        int wk = 0;
        s2ptr[0] = 0;
        for (size_t r = 0; r < runs.size(); ++r) {
          while (wk < kWarps - 1 && acc >= per * (wk + 1)) s2ptr[++wk] = (int)r;
          acc += 1.0 + (runs[r].z - runs[r].y);
        }
        while (wk < kWarps - 1) s2ptr[++wk] = (int)runs.size();
        s2ptr[kWarps] = (int)runs.size();
        // a warp takes its runs four at a time for as many steps as the longest of the four:
        // runs of equal length side by side waste no steps
        for (int wk2 = 0; wk2 < kWarps; ++wk2)
          std::stable_sort(runs.begin() + s2ptr[wk2], runs.begin() + s2ptr[wk2 + 1],
                           [](const int4& a, const int4& b) { return a.z - a.y > b.z - b.y; });
      }
      std::vector<int> s1ptr(kWarps + 1, 0);
      std::vector<int4> s1;
      for (int wk = 0; wk < kWarps; ++wk) {
        s1ptr[wk] = (int)s1.size();
        s1.insert(s1.end(), pw[wk].begin(), pw[wk].end());
      }
      s1ptr[kWarps] = (int)s1.size();
      const size_t off_ul = 32;
      const size_t off_s1ptr = round16(off_ul + 8 * ul.size());
      const size_t off_s1 = round16(off_s1ptr + 4 * (kWarps + 1));
      const size_t off_s2ptr = round16(off_s1 + 16 * s1.size());
      const size_t off_s2 = round16(off_s2ptr + 4 * (size_t)(nworkers + 1));
      const size_t off_ent = round16(off_s2 + 16 * runs.size());
      const size_t off_gd = round16(off_ent + esize * nent);
      const size_t bytes = round16(off_gd + 16 * (size_t)ng);
      const size_t base = op.side.size();
      op.side.resize(base + bytes, 0);
      unsigned char* sb = op.side.data() + base;
      const int hdr[8] = {(int)off_ul, (int)off_s1ptr, (int)off_s1, (int)off_s2ptr, (int)off_s2,
                          (int)off_ent, (int)off_gd, 0};
      std::memcpy(sb, hdr, sizeof(hdr));
      std::memcpy(sb + off_ul, ul.data(), 8 * ul.size());
      std::memcpy(sb + off_s1ptr, s1ptr.data(), 4 * s1ptr.size());
      std::memcpy(sb + off_s1, s1.data(), 16 * s1.size());
      std::memcpy(sb + off_s2ptr, s2ptr.data(), 4 * s2ptr.size());
      std::memcpy(sb + off_s2, runs.data(), 16 * runs.size());
      std::memcpy(sb + off_gd, op.gdesc.data() + g0, 16 * (size_t)ng);
      size_t q = 0;
      for (int a = 0; a < P; ++a)
        for (auto& e : perA[a]) {
          unsigned char* dst = sb + off_ent + esize * q;
          if (elem == 8) {
            std::memcpy(dst, &e.first, 4);
            std::memcpy(dst + 8, &e.second, 8);
          } else {
            // slot | a << 16 | (last entry of the run) << 24
            const float gf = (float)e.second;
            const int packed = e.first | a << 16 | (&e == &perA[a].back() ? 1 << 24 : 0);
            std::memcpy(dst, &packed, 4);
            std::memcpy(dst + 4, &gf, 4);
          }
          ++q;
        }
      op.entries += (long long)nent;
      op.visits += (long long)ul.size();
      {
        const int st1 = 2;
        long long w1 = 0, w2 = 0;
        for (int wk2 = 0; wk2 < kWarps; ++wk2) {
          long long a1 = 0, a2 = 0;
          for (const int4& pc : pw[wk2]) a1 += (pc.z + st1 - 1) / st1 + 1;
          if (elem == 4) {
            // the half-warps step through their entries side by side
            a2 = std::max(s2ptr[2 * wk2 + 1] - s2ptr[2 * wk2], s2ptr[2 * wk2 + 2] - s2ptr[2 * wk2 + 1]);
          } else {
            auto blk = [&](int b0, int b1) {  // longest run of runs [b0, b1)
              int l = 0;
              for (int r = b0; r < b1 && r < s2ptr[wk2 + 1]; ++r) l = std::max(l, runs[r].z - runs[r].y);
              return l;
            };
            const int r0 = s2ptr[wk2], r1 = s2ptr[wk2 + 1];
            int rb = r0;
            for (; rb + 4 <= r1; rb += 4) a2 += blk(rb, rb + 4) + 1;
            for (; rb < r1; ++rb) a2 += blk(rb, rb + 1) + 1;
          }
          w1 = std::max(w1, a1);
          w2 = std::max(w2, a2);
        }
        op.s1_steps += w1;
        op.s2_steps += w2;
      }
      const int nk = (int)op.kperm.size() - k0;
      op.cdesc.push_back(make_int4(k0, nk, g0, (int)op.gdesc.size() - g0));
      op.cxdesc.push_back(make_int4((int)(base / 16), (int)bytes, (int)off_s2, (int)off_ent));
      op.max_chunk_k = std::max(op.max_chunk_k, nk);
      op.max_slots = std::max(op.max_slots, slots);
      op.max_side = std::max(op.max_side, bytes);
    }
    if (!ok) return fail(SG_ERR_ARG, "tile operator: a k group exceeds the slot capacity");
    op.abytes_slot = (int)round128((size_t)op.max_chunk_k * 9 * kTW * elem);
    op.sbytes_slot = (int)round128(op.max_side);
    op.tbuf_elems = std::max(op.max_slots, 1) * kTW;
    op.xslab_elems = (int)xslab;
    op.smem = 128 + 2 * (size_t)op.abytes_slot + 2 * (size_t)op.sbytes_slot +
              (size_t)elem * (op.tbuf_elems + (size_t)P * kTW + op.xslab_elems);
    if (op.smem <= smem_max) break;
    slot_cap = std::max(1, (int)(slot_cap * 0.85));
  }
  if (op.smem > smem_max) return fail(SG_ERR_ARG, "tile operator: shared memory budget exceeded");
  op.nchunks = (int)op.cdesc.size();
  op.ngroups = (int)op.gdesc.size();
  op.Lu = (int)op.kperm.size();
  op.apw = (P + kWarps - 1) / kWarps;
  return SG_OK;
}

// Decode a plan's tables the way the kernel reads them and check them against the triple
// products: every (k, b) pair of a nonzero G_k[a, b] gets exactly one T slot, every nonzero
// G_k[a, b] exactly one stage-2 entry with its value, and every read stays inside its chunk's
// side table, stack slot and T buffer.  Host only.
int verify_tile_plan(const System& s, const TilePlan& pl) {
  const int P = s.P;
  const size_t esize = pl.elem == 8 ? 16 : 8;
  std::map<std::array<int, 3>, double> want;
  for (const Triple& t : s.triples) want[{t.k, t.a, t.b}] = t.g;
  std::map<std::array<int, 3>, double> got;
  std::vector<char> seen((size_t)s.L * P, 0);
  auto rd = [](const unsigned char* p, size_t off, void* dst, size_t n) { std::memcpy(dst, p + off, n); };
  for (int c = 0; c < pl.nchunks; ++c) {
    const int4 cd = pl.cdesc[c], cx = pl.cxdesc[c];
    if ((size_t)cx.x * 16 + cx.y > pl.side.size() || cx.y % 16 || cx.y > pl.sbytes_slot)
      return fail(SG_ERR_ARG, "plan: side table out of range");
    if ((size_t)cd.y * 9 * 32 * pl.elem > (size_t)pl.abytes_slot) return fail(SG_ERR_ARG, "plan: stack slot");
    const unsigned char* sb = pl.side.data() + (size_t)cx.x * 16;
    int hdr[8];
    rd(sb, 0, hdr, sizeof(hdr));
    for (int i = 0; i < 7; ++i)
      if (hdr[i] % 16 || hdr[i] > cx.y) return fail(SG_ERR_ARG, "plan: header");
    if ((size_t)hdr[6] + 16 * (size_t)cd.w > (size_t)cx.y) return fail(SG_ERR_ARG, "plan: groups");
    for (int g = 0; g < cd.w; ++g) {
      int4 gd;
      rd(sb, hdr[6] + 16 * (size_t)g, &gd, 16);
      const int4 want_gd = pl.gdesc[cd.z + g];
      if (gd.x != want_gd.x || gd.y != want_gd.y || gd.z != want_gd.z || gd.w != want_gd.w)
        return fail(SG_ERR_ARG, "plan: group descriptor");
    }
    // union lists: every entry of every group exactly once in the warps' pieces
    std::vector<std::vector<char>> covered(cd.w);
    for (int g = 0; g < cd.w; ++g) covered[g].assign(pl.gdesc[cd.z + g].y, 0);
    int s1ptr[9];
    rd(sb, hdr[1], s1ptr, sizeof(s1ptr));
    if (s1ptr[0] != 0) return fail(SG_ERR_ARG, "plan: stage-1 lists");
    for (int w = 0; w < 8; ++w) {
      if (s1ptr[w + 1] < s1ptr[w]) return fail(SG_ERR_ARG, "plan: stage-1 lists");
      for (int pc = s1ptr[w]; pc < s1ptr[w + 1]; ++pc) {
        int4 piece;
        rd(sb, hdr[2] + 16 * (size_t)pc, &piece, 16);
        if (hdr[2] + 16 * (size_t)(pc + 1) > (size_t)hdr[3]) return fail(SG_ERR_ARG, "plan: piece range");
        if (piece.x < 0 || piece.x >= cd.w) return fail(SG_ERR_ARG, "plan: piece group");
        const int4 gd = pl.gdesc[cd.z + piece.x];
        if (piece.y < 0 || piece.z < 1 || piece.y + piece.z > gd.y) return fail(SG_ERR_ARG, "plan: piece");
        for (int u = piece.y; u < piece.y + piece.z; ++u) {
          if (covered[piece.x][u]++) return fail(SG_ERR_ARG, "plan: union entry twice");
        }
      }
    }
    std::vector<std::array<int, 2>> slot_kb;  // (k, b) of each slot
    for (int g = 0; g < cd.w; ++g) {
      const int4 gd = pl.gdesc[cd.z + g];
      if (gd.z + gd.w > cd.y || hdr[0] + 8 * (size_t)(gd.x + gd.y) > (size_t)hdr[1])
        return fail(SG_ERR_ARG, "plan: group out of range");
      for (int u = 0; u < gd.y; ++u) {
        if (!covered[g][u]) return fail(SG_ERR_ARG, "plan: union entry not covered");
        int2 e;
        rd(sb, hdr[0] + 8 * (size_t)(gd.x + u), &e, 8);
        const int b = e.x & 0xffff, mask = e.x >> 16;
        int sl = e.y;
        for (int j = 0; j < gd.w; ++j)
          if (mask >> j & 1) {
            const int k = pl.kperm[cd.x + gd.z + j];
            if (sl != (int)slot_kb.size()) return fail(SG_ERR_ARG, "plan: slots not consecutive");
            if (seen[(size_t)k * P + b]++) return fail(SG_ERR_ARG, "plan: pair placed twice");
            slot_kb.push_back({k, b});
            ++sl;
          }
        if (mask >> gd.w) return fail(SG_ERR_ARG, "plan: mask beyond the group");
      }
    }
    if ((int)slot_kb.size() > pl.max_slots || (size_t)pl.max_slots * 32 > (size_t)pl.tbuf_elems)
      return fail(SG_ERR_ARG, "plan: T buffer");
    std::vector<char> a_seen(P, 0);
    if (pl.elem == 4) {
      // FP32 stage 2: sixteen entry ranges of whole runs; a run is the consecutive entries of one
      // a (one run per a at most), the last flagged
      int s2p[17];
      rd(sb, hdr[3], s2p, sizeof(s2p));
      if (s2p[0] != 0) return fail(SG_ERR_ARG, "plan: stage-2 ranges");
      for (int w = 0; w < 16; ++w)
        if (s2p[w + 1] < s2p[w]) return fail(SG_ERR_ARG, "plan: stage-2 ranges");
      const int nent = s2p[16];
      if ((size_t)hdr[5] + 8 * (size_t)nent > (size_t)cx.y) return fail(SG_ERR_ARG, "plan: entry out of range");
      std::vector<char> starts(nent + 1, 0);
      for (int w = 0; w <= 16; ++w) starts[s2p[w]] = 1;
      bool open = false;
      int cur_a = -1;
      for (int q = 0; q < nent; ++q) {
        int packed;
        float gf;
        rd(sb, hdr[5] + 8 * (size_t)q, &packed, 4);
        rd(sb, hdr[5] + 8 * (size_t)q + 4, &gf, 4);
        const int slot = packed & 0xffff, a = packed >> 16 & 0xff, last = packed >> 24;
        if (last > 1 || a >= P) return fail(SG_ERR_ARG, "plan: entry fields");
        if (starts[q] && open) return fail(SG_ERR_ARG, "plan: range cuts a run");
        if (!open) {
          if (a_seen[a]++) return fail(SG_ERR_ARG, "plan: run output");
          open = true;
          cur_a = a;
        } else if (a != cur_a) {
          return fail(SG_ERR_ARG, "plan: run not flagged");
        }
        if (last) open = false;
        if (slot >= (int)slot_kb.size()) return fail(SG_ERR_ARG, "plan: entry slot");
        auto key = std::array<int, 3>{slot_kb[slot][0], a, slot_kb[slot][1]};
        if (got.count(key)) return fail(SG_ERR_ARG, "plan: entry placed twice");
        got[key] = gf;
      }
      if (open) return fail(SG_ERR_ARG, "plan: last run not flagged");
      continue;
    }
    // FP64 stage-2 runs: one per a at most, covering the entries once
    int s2ptr[9];
    rd(sb, hdr[3], s2ptr, sizeof(s2ptr));
    if (s2ptr[0] != 0) return fail(SG_ERR_ARG, "plan: stage-2 lists");
    for (int w = 0; w < 8; ++w) {
      if (s2ptr[w + 1] < s2ptr[w]) return fail(SG_ERR_ARG, "plan: stage-2 lists");
      for (int rn = s2ptr[w]; rn < s2ptr[w + 1]; ++rn) {
        int4 run;
        rd(sb, hdr[4] + 16 * (size_t)rn, &run, 16);
        if (hdr[4] + 16 * (size_t)(rn + 1) > (size_t)hdr[5]) return fail(SG_ERR_ARG, "plan: run range");
        if (run.x < 0 || run.x >= P || a_seen[run.x]++) return fail(SG_ERR_ARG, "plan: run output");
        for (int q = run.y; q < run.z; ++q) {
          if ((size_t)hdr[5] + esize * (q + 1) > (size_t)cx.y) return fail(SG_ERR_ARG, "plan: entry out of range");
          int slot;
          double g;
          rd(sb, hdr[5] + esize * q, &slot, 4);
          if (pl.elem == 8) {
            rd(sb, hdr[5] + esize * q + 8, &g, 8);
          } else {
            float gf;
            rd(sb, hdr[5] + esize * q + 4, &gf, 4);
            g = gf;
          }
          if (slot < 0 || slot >= (int)slot_kb.size()) return fail(SG_ERR_ARG, "plan: entry slot");
          auto key = std::array<int, 3>{slot_kb[slot][0], run.x, slot_kb[slot][1]};
          if (got.count(key)) return fail(SG_ERR_ARG, "plan: entry placed twice");
          got[key] = g;
        }
      }
    }
  }
  if (got.size() != want.size()) return fail(SG_ERR_ARG, "plan: entries missing");
  for (auto& kv : want) {
    auto it = got.find(kv.first);
    if (it == got.end()) return fail(SG_ERR_ARG, "plan: entry missing");
    const double tol = pl.elem == 8 ? 0.0 : 1e-7 * std::fabs(kv.second);
    if (std::fabs(it->second - kv.second) > tol) return fail(SG_ERR_ARG, "plan: entry value");
  }
  const size_t smem = 128 + 2 * (size_t)pl.abytes_slot + 2 * (size_t)pl.sbytes_slot +
                      (size_t)pl.elem * (pl.tbuf_elems + (size_t)P * 32 + pl.xslab_elems);
  if (smem != pl.smem || pl.abytes_slot % 128 || pl.sbytes_slot % 128) return fail(SG_ERR_ARG, "plan: layout");
  return SG_OK;
}

int build_tile_op(System& s, TileOp& op, int kappa, int elem, size_t smem_max, cudaStream_t st,
                  int ctas) {
  TilePlan pl;
  op = TileOp();
  SG_TRY(plan_tile_op(s, kappa, elem, smem_max, pl, ctas));
  const int m = s.pat.m, L = s.L;
  op.kappa = pl.kappa;
  op.elem = pl.elem;
  op.ctas = pl.ctas;
  op.tiles_per_line = pl.tiles_per_line;
  op.ntiles = pl.ntiles;
  op.Pp = pl.Pp;
  op.Lu = pl.Lu;
  op.nchunks = pl.nchunks;
  op.ngroups = pl.ngroups;
  op.max_chunk_k = pl.max_chunk_k;
  op.max_slots = pl.max_slots;
  op.apw = pl.apw;
  op.abytes_slot = pl.abytes_slot;
  op.sbytes_slot = pl.sbytes_slot;
  op.tbuf_elems = pl.tbuf_elems;
  op.xslab_elems = pl.xslab_elems;
  op.smem = pl.smem;
  SG_TRY(op.chunk.alloc(pl.cdesc.size()));
  SG_TRY(op.chunk.upload(pl.cdesc, st));
  SG_TRY(op.chunkx.alloc(pl.cxdesc.size()));
  SG_TRY(op.chunkx.upload(pl.cxdesc, st));
  SG_TRY(op.side.alloc(pl.side.size()));
  SG_TRY(op.side.upload(pl.side, st));
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
  op.chunkx.release();
  op.side.release();
  op.stack.release();
  op.stack32.release();
  op.err.release();
  op.ready = false;
}

int launch_tile_op_f64(const System& s, const TileOp& op, const double* X, double* Y, double alpha,
                      const double* B, double beta, cudaStream_t st, const int* done);
int launch_tile_op_f32(const System& s, const TileOp& op, const float* X, float* Y, float alpha,
                      const float* B, float beta, cudaStream_t st, const int* done);

template <typename T>
int launch_tile_op(const System& s, const TileOp& op, const T* X, T* Y, T alpha, const T* B,
                   T beta, cudaStream_t st, const int* done) {
  if (!op.ready) return fail(SG_ERR_ARG, "tile operator not built");
  if constexpr (sizeof(T) == 8) return launch_tile_op_f64(s, op, X, Y, alpha, B, beta, st, done);
  else return launch_tile_op_f32(s, op, X, Y, alpha, B, beta, st, done);
}

template int launch_tile_op<double>(const System&, const TileOp&, const double*, double*, double,
                                    const double*, double, cudaStream_t, const int*);
template int launch_tile_op<float>(const System&, const TileOp&, const float*, float*, float,
                                   const float*, float, cudaStream_t, const int*);

}  // namespace sg
