// C ABI of the SG solver (include/sg.h): setup of the systems, the operator, preconditioner and
// right-hand-side entry points, and the restarted GMRES driver (Sec. 3) that queues whole Arnoldi
// cycles per system on the system's own stream and synchronises once per cycle.
#include <algorithm>
#include <array>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <thread>

#include "sg_internal.h"

namespace sg {

// ------------------------------------------------------------------ errors and launch counting

static thread_local std::string g_last_error;
static std::atomic<long long> g_launches{0};

void set_error(const std::string& msg) { g_last_error = msg; }
int fail(int code, const std::string& msg) {
  set_error(msg);
  return code;
}
void count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
int check_launch(const char* what) {
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(SG_ERR_CUDA, std::string("launch of ") + what + ": " + cudaGetErrorString(e));
  return SG_OK;
}

int ensure_smem(const void* kernel, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, size_t> done;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(mu);
  auto key = std::make_pair(kernel, dev);
  auto it = done.find(key);
  if (it != done.end() && it->second >= bytes) return SG_OK;
  SG_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  done[key] = bytes;
  return SG_OK;
}

size_t smem_optin_max() {
  static std::mutex mu;
  static std::map<int, size_t> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(dev);
  if (it != cache.end()) return it->second;
  int v = 0;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) v = 0;
  cache[dev] = (size_t)v;
  return (size_t)v;
}

TimeScope::TimeScope(Timer* t_, int cls_, cudaStream_t st_) : t(t_), cls(cls_), st(st_) {
  if (!t || !t->on) return;
  long long c = t->count[cls]++;
  if (c % t->stride != 0 || t->used + 2 > t->ev.size()) return;
  idx = (long long)t->used;
  t->used += 2;
  cudaEventRecord(t->ev[idx], st);
}
TimeScope::~TimeScope() {
  if (idx < 0) return;
  cudaEventRecord(t->ev[idx + 1], st);
  t->recs.push_back({cls, (size_t)idx});
}

template <typename T>
int DBuf<T>::alloc(size_t count) {
  release();
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)&p, sizeof(T) * count);
  if (e != cudaSuccess) {
    p = nullptr;
    cudaGetLastError();
    return fail(SG_ERR_OOM, "cudaMalloc of " + std::to_string(sizeof(T) * count) + " bytes: " + cudaGetErrorString(e));
  }
  n = count;
  return SG_OK;
}
template <typename T>
int DBuf<T>::upload(const std::vector<T>& h, cudaStream_t s) {
  if (h.empty()) return SG_OK;
  if (h.size() > n) return fail(SG_ERR_ARG, "upload larger than buffer");
  SG_CUDA(cudaMemcpyAsync(p, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice, s));
  SG_CUDA(cudaStreamSynchronize(s));
  return SG_OK;
}
template <typename T>
void DBuf<T>::release() {
  if (p) cudaFree(p);
  p = nullptr;
  n = 0;
}
template struct DBuf<double>;
template struct DBuf<float>;
template struct DBuf<int>;
template struct DBuf<int2>;
template struct DBuf<int4>;
template struct DBuf<unsigned char>;
template struct DBuf<unsigned int>;
template struct DBuf<__nv_bfloat16>;

// ------------------------------------------------------------------ host tables

static int validate(const sg_params& p) {
  if (p.n < 2 || p.n > 1024) return fail(SG_ERR_ARG, "n must be in [2, 1024]");
  if (p.M < 1 || p.M > 8) return fail(SG_ERR_ARG, "M must be in [1, 8]");
  if (p.p < 0 || p.p > 6) return fail(SG_ERR_ARG, "p must be in [0, 6]");
  if (p.q > 12) return fail(SG_ERR_ARG, "q must be <= 12");
  if (!(p.sigma >= 0.0) || !(p.ell > 0.0) || !(p.a_min >= 0.0))
    return fail(SG_ERR_ARG, "need sigma >= 0, ell > 0, a_min >= 0");
  if (!std::isfinite(p.mu) || !std::isfinite(p.f)) return fail(SG_ERR_ARG, "mu and f must be finite");
  if (p.precond < SG_PC_NONE || p.precond > SG_PC_FG) return fail(SG_ERR_ARG, "unknown preconditioner");
  if (p.precond == SG_PC_MG) {
    if (p.mg_smoother != SG_PC_MEAN && p.mg_smoother != SG_PC_FS_GS &&
        p.mg_smoother != SG_PC_FS_JACOBI && p.mg_smoother != SG_PC_FG)
      return fail(SG_ERR_ARG, "mg_smoother must be SG_PC_MEAN, SG_PC_FS_GS, SG_PC_FS_JACOBI or SG_PC_FG");
    if (p.mg_coarse < 2) return fail(SG_ERR_ARG, "mg_coarse must be >= 2");
    int nn = p.n;
    while (nn > p.mg_coarse && nn % 2 == 0) nn /= 2;
    if (nn != p.mg_coarse || p.n == p.mg_coarse)
      return fail(SG_ERR_ARG, "multigrid needs n = mg_coarse * 2^k with k >= 1");
  }
  if (p.inner_iters < 1 || p.outer_sweeps < 1) return fail(SG_ERR_ARG, "inner_iters and outer_sweeps must be >= 1");
  if (p.restart < 1 || p.restart > 1024) return fail(SG_ERR_ARG, "restart must be in [1, 1024]");
  if (p.max_iters < 1) return fail(SG_ERR_ARG, "max_iters must be >= 1");
  if (!(p.rtol >= 0.0) || !(p.atol >= 0.0)) return fail(SG_ERR_ARG, "rtol, atol must be >= 0");
  if (p.precision < SG_FP64 || p.precision > SG_MIXED_BF16) return fail(SG_ERR_ARG, "unknown precision");
  if (p.precision != SG_FP64 && !(p.inner_rtol > 0.0 && p.inner_rtol < 1.0))
    return fail(SG_ERR_ARG, "inner_rtol must be in (0, 1)");
  if (p.graphs != 0 && p.graphs != 1) return fail(SG_ERR_ARG, "graphs must be 0 or 1");
  if (p.op_kernel < SG_OP_AUTO || p.op_kernel > SG_OP_TILE) return fail(SG_ERR_ARG, "unknown op_kernel");
  if (p.op_kappa != 0 && p.op_kappa != 1 && p.op_kappa != 2 && p.op_kappa != 4)
    return fail(SG_ERR_ARG, "op_kappa must be 0, 1, 2 or 4");
  if (p.op_ctas < 0 || p.op_ctas > 2) return fail(SG_ERR_ARG, "op_ctas must be 0, 1 or 2");
  if (p.ilu_order != SG_ILU_NATURAL && p.ilu_order != SG_ILU_COLOR4)
    return fail(SG_ERR_ARG, "unknown ilu_order");
  if (p.ilu_order == SG_ILU_COLOR4 && p.inner_iters != 1)
    return fail(SG_ERR_ARG, "the four-colour ILU(0) ordering takes inner_iters = 1");
  if (p.coupling_bf16 != 0 && p.coupling_bf16 != 1) return fail(SG_ERR_ARG, "coupling_bf16 must be 0 or 1");
  if (p.precond == SG_PC_FG || (p.precond == SG_PC_MG && p.mg_smoother == SG_PC_FG)) {
    if (p.fg_rule < SG_FG_PAPER || p.fg_rule > SG_FG_WHOLE) return fail(SG_ERR_ARG, "unknown fg_rule");
    if (p.ilu_order != SG_ILU_COLOR4)
      return fail(SG_ERR_ARG, "the grouped field split runs in the four-colour ILU(0) ordering");
  }
  if (p.fg_bf16 != 0 && p.fg_bf16 != 1) return fail(SG_ERR_ARG, "fg_bf16 must be 0 or 1");
  if (p.fg_bf16 && p.precision != SG_MIXED_FP32)
    return fail(SG_ERR_ARG, "fg_bf16 applies to SG_MIXED_FP32 systems");
  if (p.coupling_bf16 && p.precision != SG_MIXED_FP32)
    return fail(SG_ERR_ARG, "coupling_bf16 applies to SG_MIXED_FP32 systems");
  if (p.precond == SG_PC_MEAN || p.precond == SG_PC_FS_GS || p.precond == SG_PC_FS_JACOBI ||
      p.precond == SG_PC_MG) {
    // the wavefront solve: 2 wc compute and some staging threads; shared memory for its level
    // window, factor rings and level offsets
    const int wc = (interior_level_width(p.n + 1) + 31) / 32 * 32;
    if (2 * wc + tri_staging_threads(wc) > 1024 || tri_smem_bytes(p.n + 1, wc, 8) > 227 * 1024)
      return fail(SG_ERR_ARG, "n must be at most 769 for the ILU(0) preconditioners");
  }
  return SG_OK;
}

static int build_tables(System& s) {
  const sg_params& p = s.prm;
  std::vector<int> Jp = total_degree_set(p.M, p.p), Jq = total_degree_set(p.M, p.q);
  s.P = (int)Jp.size() / p.M;
  s.L = (int)Jq.size() / p.M;
  if (s.P > 4096 || s.L > 32767) return fail(SG_ERR_ARG, "chaos basis too large");
  // 1-D triple products e(i, j, k) for i <= q, j, k <= p
  const int Q1 = p.q + 1, P1 = p.p + 1;
  std::vector<double> e1((size_t)Q1 * P1 * P1);
  for (int i = 0; i < Q1; ++i)
    for (int j = 0; j < P1; ++j)
      for (int k = 0; k < P1; ++k) e1[((size_t)i * P1 + j) * P1 + k] = hermite_triple(i, j, k);
  s.triples.clear();
  for (int k = 0; k < s.L; ++k)
    for (int a = 0; a < s.P; ++a)
      for (int b = 0; b < s.P; ++b) {
        double g = 1.0;
        for (int d = 0; d < p.M && g != 0.0; ++d)
          g *= e1[((size_t)Jq[k * p.M + d] * P1 + Jp[a * p.M + d]) * P1 + Jp[b * p.M + d]];
        if (g != 0.0) s.triples.push_back({k, a, b, g});
      }
  s.nnzG = (long long)s.triples.size();
  // (k, b) pairs in (k, b) order and their chunks
  std::map<std::pair<int, int>, int> pid;
  for (auto& t : s.triples) pid[{t.k, t.b}] = 0;
  OpTables& op = s.op;
  op.pair_kb.clear();
  op.chunks.clear();
  int u = 0;
  for (auto& kv : pid) {
    kv.second = u++;
    op.pair_kb.push_back((kv.first.first << 16) | kv.first.second);
  }
  op.npairs = u;
  std::vector<int> chunk_of(u);
  for (int v = 0; v < u; ++v) {
    int k = op.pair_kb[v] >> 16;
    if (op.chunks.empty() || op.chunks.back().u1 - op.chunks.back().u0 >= kChunkPairs ||
        k - op.chunks.back().k0 >= kChunkK) {
      op.chunks.push_back({v, v, k, k});
    }
    op.chunks.back().u1 = v + 1;
    op.chunks.back().k1 = k + 1;
    chunk_of[v] = (int)op.chunks.size() - 1;
  }
  op.nchunks = (int)op.chunks.size();
  // entries per (chunk, a), sorted by pair
  std::vector<std::vector<std::pair<int, double>>> bucket((size_t)op.nchunks * s.P);
  for (auto& t : s.triples) {
    int v = pid[{t.k, t.b}];
    int c = chunk_of[v];
    bucket[(size_t)c * s.P + t.a].push_back({v - op.chunks[c].u0, t.g});
  }
  op.ent_ptr.assign((size_t)op.nchunks * (s.P + 1), 0);
  op.ent_u.clear();
  op.ent_g.clear();
  for (int c = 0; c < op.nchunks; ++c) {
    for (int a = 0; a < s.P; ++a) {
      auto& bk = bucket[(size_t)c * s.P + a];
      std::sort(bk.begin(), bk.end());
      op.ent_ptr[(size_t)c * (s.P + 1) + a] = (int)op.ent_u.size();
      for (auto& pr : bk) {
        op.ent_u.push_back(pr.first);
        op.ent_g.push_back(pr.second);
      }
    }
    op.ent_ptr[(size_t)c * (s.P + 1) + s.P] = (int)op.ent_u.size();
  }
  op.nent = (int)op.ent_u.size();
  return SG_OK;
}

int host_tables(System& s) {
  sg_params& p = s.prm;
  if (p.q <= 0) p.q = 2 * p.p;
  s.n = p.n;
  s.M = p.M;
  s.pat = make_pattern(p.n);
  s.N = s.pat.N;
  return build_tables(s);
}

// ------------------------------------------------------------------ operator kernel tuner

// The choice for one system shape and operator precision: the pair kernel, or the row-tiled kernel
// with kappa k per register group and shared memory planned for ``ctas`` CTAs per SM.
struct TuneChoice {
  int kernel = SG_OP_PAIRS, kappa = 0, ctas = 1;
  double ms = 0.0;
};
static std::mutex g_tune_mu;
static std::map<std::array<long long, 5>, TuneChoice> g_tune;

static std::string describe(const TuneChoice& c) {
  if (c.kernel == SG_OP_PAIRS) return "pairs";
  return "tile k" + std::to_string(c.kappa) + " x" + std::to_string(c.ctas);
}

// Shared memory one CTA may plan for when ``ctas`` CTAs share an SM.
static size_t smem_budget(int ctas) {
  const size_t opt = smem_optin_max();
  if (ctas <= 1) return opt;
  int dev = 0, per_sm = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess)
    per_sm = 0;
  const size_t each = per_sm > 0 ? (size_t)per_sm / ctas : opt / ctas;
  return std::min(opt, each > 1024 ? each - 1024 : each);
}

template <typename T>
static int time_operator(const System& s, const T* X, T* Y, cudaStream_t st, double* ms) {
  auto run = [&]() {
    if constexpr (sizeof(T) == 8) return launch_matvec_f64(s, X, Y, 1.0, nullptr, 0.0, st);
    else return launch_matvec_f32(s, X, Y, 1.0f, nullptr, 0.0f, st);
  };
  cudaEvent_t a, b;
  SG_CUDA(cudaEventCreate(&a));
  SG_CUDA(cudaEventCreate(&b));
  int rc = run();
  if (rc == SG_OK) rc = cudaEventRecord(a, st) == cudaSuccess ? SG_OK : SG_ERR_CUDA;
  for (int r = 0; r < 3 && rc == SG_OK; ++r) rc = run();
  if (rc == SG_OK) rc = cudaEventRecord(b, st) == cudaSuccess ? SG_OK : SG_ERR_CUDA;
  float t = 0.f;
  if (rc == SG_OK && cudaEventSynchronize(b) == cudaSuccess && cudaEventElapsedTime(&t, a, b) == cudaSuccess)
    *ms = t / 3.0;
  else if (rc == SG_OK)
    rc = fail(SG_ERR_CUDA, "timing the operator failed");
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return rc;
}

// Build the operator kernel of precision ``elem`` (8: FP64, 4: FP32) that op_kernel asks for.
// SG_OP_AUTO times the pair kernel and every row-tiled variant that fits (kappa 1, 2, 4; one or
// two CTAs per SM) on this system, keeps the fastest and caches the choice for the system's
// (N, P, L, q, element size).
static int choose_operator(System& s, int elem, cudaStream_t st) {
  TileOp& op = elem == 8 ? s.tile64 : s.tile32;
  const sg_params& p = s.prm;
  std::string& note = s.tile_msg;
  if (p.op_kernel == SG_OP_PAIRS) return SG_OK;
  if (p.op_kernel == SG_OP_TILE) {
    const int kappa = p.op_kappa ? p.op_kappa : (elem == 8 ? 2 : 4);
    const int ctas = p.op_ctas ? p.op_ctas : 1;
    if (build_tile_op(s, op, kappa, elem, smem_budget(ctas), st, ctas) != SG_OK) {
      note += (elem == 8 ? "fp64: " : "fp32: ") + g_last_error + "; ";
      free_tile_op(op);
      set_error("");
    }
    return SG_OK;
  }
  const std::array<long long, 5> key{s.N, s.P, s.L, p.q, elem};
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto itc = g_tune.find(key);
    if (itc != g_tune.end()) {
      const TuneChoice c = itc->second;
      note += std::string(elem == 8 ? "fp64: " : "fp32: ") + describe(c) + " (cached); ";
      if (c.kernel == SG_OP_PAIRS) return SG_OK;
      if (build_tile_op(s, op, c.kappa, elem, smem_budget(c.ctas), st, c.ctas) != SG_OK) {
        free_tile_op(op);
        set_error("");
      }
      return SG_OK;
    }
  }
  const size_t NP = (size_t)s.N * s.P;
  DBuf<unsigned char> xb, yb;
  SG_TRY(xb.alloc(NP * elem));
  SG_TRY(yb.alloc(NP * elem));
  SG_CUDA(cudaMemsetAsync(xb.p, 0, NP * elem, st));
  auto timed = [&](double* ms) {
    if (elem == 8)
      return time_operator<double>(s, (const double*)xb.p, (double*)yb.p, st, ms);
    return time_operator<float>(s, (const float*)xb.p, (float*)yb.p, st, ms);
  };
  TuneChoice best;
  std::string log = std::string(elem == 8 ? "fp64:" : "fp32:");
  SG_TRY(timed(&best.ms));  // the pair kernel (no row-tiled operator built yet)
  log += " pairs " + std::to_string(best.ms) + " ms";
  for (int ctas : {1, 2})
    for (int kappa : {1, 2, 4}) {
      TileOp cand;
      if (build_tile_op(s, cand, kappa, elem, smem_budget(ctas), st, ctas) != SG_OK) {
        free_tile_op(cand);
        set_error("");
        continue;
      }
      std::swap(op, cand);
      double ms = 0.0;
      const int rc = timed(&ms);
      std::swap(op, cand);
      TuneChoice c{SG_OP_TILE, kappa, ctas, ms};
      if (rc == SG_OK) log += ", " + describe(c) + " " + std::to_string(ms) + " ms";
      if (rc == SG_OK && ms < best.ms) {
        best = c;
        free_tile_op(op);
        op = std::move(cand);
        cand = TileOp();
      }
      free_tile_op(cand);
      set_error("");
    }
  xb.release();
  yb.release();
  note += log + "; chose " + describe(best) + "; ";
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune[key] = best;
  return SG_OK;
}

static int upload_i(DBuf<int>& d, const std::vector<int>& h, cudaStream_t st) {
  SG_TRY(d.alloc(h.size()));
  return d.upload(h, st);
}
static int upload_d(DBuf<double>& d, const std::vector<double>& h, cudaStream_t st) {
  SG_TRY(d.alloc(h.size()));
  return d.upload(h, st);
}
static int upload_f(DBuf<float>& d, const std::vector<double>& h, cudaStream_t st) {
  std::vector<float> f(h.begin(), h.end());
  SG_TRY(d.alloc(f.size()));
  return d.upload(f, st);
}

// Field-split Gauss-Seidel tables: for source block b, the k that couple b to some a > b and,
// per a > b, the (k index, G_k[a,b]) entries.
// Scatter tables of the Gauss-Seidel sweep for the target columns a = b + 1 (next) or
// a >= b + 2 (later): per source block b the k with a nonzero G_k[a,b] and per a the
// (local k index, G_k[a,b]) entries.
static int build_scatter_tables(System& s, bool next, DBuf<int>& dkptr, DBuf<int>& dk,
                                DBuf<int>& deptr, DBuf<int>& dea, DBuf<double>& deg,
                                DBuf<float>& deg32, cudaStream_t st) {
  std::vector<int> kptr(s.P + 1, 0), klist, eptr((size_t)s.P * (s.P + 1), 0), ea;
  std::vector<double> eg;
  auto target = [&](int a, int b) { return next ? a == b + 1 : a > b + 1; };
  for (int b = 0; b < s.P; ++b) {
    std::vector<int> ks;
    for (auto& t : s.triples)
      if (t.b == b && target(t.a, b)) ks.push_back(t.k);
    std::sort(ks.begin(), ks.end());
    ks.erase(std::unique(ks.begin(), ks.end()), ks.end());
    kptr[b] = (int)klist.size();
    klist.insert(klist.end(), ks.begin(), ks.end());
    s.gs_max_klen = std::max(s.gs_max_klen, (int)ks.size());
    std::vector<std::vector<std::pair<int, double>>> per_a(s.P);
    for (auto& t : s.triples)
      if (t.b == b && target(t.a, b)) {
        int kl = (int)(std::lower_bound(ks.begin(), ks.end(), t.k) - ks.begin());
        per_a[t.a].push_back({kl, t.g});
      }
    for (int a = 0; a < s.P; ++a) {
      eptr[(size_t)b * (s.P + 1) + a] = (int)ea.size();
      std::sort(per_a[a].begin(), per_a[a].end());
      for (auto& pr : per_a[a]) {
        ea.push_back(pr.first);
        eg.push_back(pr.second);
      }
    }
    eptr[(size_t)b * (s.P + 1) + s.P] = (int)ea.size();
  }
  kptr[s.P] = (int)klist.size();
  SG_TRY(upload_i(dkptr, kptr, st));
  SG_TRY(upload_i(dk, klist, st));
  SG_TRY(upload_i(deptr, eptr, st));
  SG_TRY(upload_i(dea, ea, st));
  SG_TRY(upload_d(deg, eg, st));
  if (s.prm.precision != SG_FP64) SG_TRY(upload_f(deg32, eg, st));
  return SG_OK;
}

static int build_gs_tables(System& s, cudaStream_t st) {
  s.gs_max_klen = 0;
  SG_TRY(build_scatter_tables(s, false, s.gs_kptr, s.gs_k, s.gs_eptr, s.gs_ea, s.gs_eg,
                              s.gs_eg_f32, st));
  SG_TRY(build_scatter_tables(s, true, s.gsn_kptr, s.gsn_k, s.gsn_eptr, s.gsn_ea, s.gsn_eg,
                              s.gsn_eg_f32, st));
  int prio_low = 0, prio_high = 0;
  SG_CUDA(cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high));
  s.prio_lo = prio_low;
  s.prio_hi = prio_high;
  SG_CUDA(cudaStreamCreateWithPriority(&s.stream2, cudaStreamNonBlocking, prio_low));
  SG_CUDA(cudaEventCreateWithFlags(&s.ev_z, cudaEventDisableTiming));
  SG_CUDA(cudaEventCreateWithFlags(&s.ev_r[0], cudaEventDisableTiming));
  SG_CUDA(cudaEventCreateWithFlags(&s.ev_r[1], cudaEventDisableTiming));
  return SG_OK;
}

static void free_system(System* s) {
  if (!s) return;
  free_tile_op(s->tile64);
  free_tile_op(s->tile32);
  for (System* c : s->mg) free_system(c);
  s->mg.clear();
  for (auto* b : {&s->mg_b, &s->mg_u, &s->mg_r, &s->mg_d, &s->mg_inv}) b->release();
  for (auto* b : {&s->mg_b32, &s->mg_u32, &s->mg_r32, &s->mg_d32, &s->mg_inv32}) b->release();
  s->mg_nodes.release();
  if (s->stream) cudaStreamSynchronize(s->stream);
  if (s->stream2) cudaStreamSynchronize(s->stream2);
  DBuf<int>* ib[] = {&s->rowptr, &s->col, &s->diag, &s->lev_f_ptr, &s->lev_f_rows, &s->lev_b_ptr,
                     &s->lev_b_rows, &s->pair_kb, &s->ent_ptr, &s->ent_u, &s->gs_kptr, &s->gs_k,
                     &s->gs_eptr, &s->gs_ea, &s->gsn_kptr, &s->gsn_k, &s->gsn_eptr,
                     &s->gsn_ea, &s->flags, &s->xzero};
  for (auto* b : ib) b->release();
  s->lev9_off.release();
  s->cstart.release();
  s->stack_km16.release();
  for (auto& sp : s->fg) {
    sp.fac.release();
    sp.fac32.release();
    sp.fac16.release();
  }
  s->fg.clear();
  for (auto* b : {&s->fg_tmp, &s->fg_tmp2}) b->release();
  for (auto* b : {&s->fg_tmp32, &s->fg_tmp232}) b->release();
  DBuf<double>* db[] = {&s->stack, &s->stack_km, &s->ent_g, &s->blk, &s->fac, &s->lu9, &s->gs_eg, &s->gsn_eg, &s->gsn_cs, &s->gsn_corr, &s->rhs_t, &s->tmp,
                        &s->tmp2, &s->tri_w, &s->V, &s->Z, &s->Hs, &s->cs, &s->sn, &s->g, &s->y,
                        &s->scal, &s->red, &s->rvec};
  for (auto* b : db) b->release();
  DBuf<float>* fb[] = {&s->stack_f32, &s->stack_km32, &s->ent_g_f32, &s->lu9_f32, &s->blk_f32, &s->gs_eg_f32, &s->gsn_eg_f32, &s->gsn_cs32, &s->gsn_corr32,
                       &s->rhs_t32, &s->tmp32, &s->tmp232, &s->tri_w32, &s->V32, &s->Z32,
                       &s->mv32a, &s->mv32b};
  for (auto* b : fb) b->release();
  s->stack_bf16.release();
  s->chunks.release();
  s->chunks_k.release();
  s->ticket.release();
  for (auto& g : s->graphs) cudaGraphExecDestroy(g.exec);
  s->graphs.clear();
  if (s->hpin) cudaFreeHost(s->hpin);
  if (s->ev) cudaEventDestroy(s->ev);
  for (cudaEvent_t e : {s->seg_ev[0], s->seg_ev[1]})
    if (e) cudaEventDestroy(e);
  if (s->stream2) cudaStreamDestroy(s->stream2);
  for (cudaEvent_t e : {s->ev_z, s->ev_r[0], s->ev_r[1]})
    if (e) cudaEventDestroy(e);
  if (s->stream) cudaStreamDestroy(s->stream);
  delete s;
}

static int setup_system(System& s, cudaStream_t st, bool krylov = true) {
  sg_params& p = s.prm;
  if (p.q <= 0) p.q = 2 * p.p;
  s.pc_fac = p.precond == SG_PC_MG ? p.mg_smoother : p.precond;
  s.n = p.n;
  s.M = p.M;
  s.pat = make_pattern(p.n);
  s.N = s.pat.N;
  s.kl = kl_terms_2d(p.sigma, p.ell, p.M);
  SG_TRY(build_tables(s));
  const bool lowp = p.precision != SG_FP64;
  // smem budgets of the kernels
  size_t apply_smem = sizeof(double) * 4 * (9 * kChunkK + 9 * (size_t)s.P + kChunkPairs + s.P);
  if (apply_smem > 220 * 1024) return fail(SG_ERR_ARG, "P too large for the operator kernel");
  {  // wavefront solve: group width, and whether a whole column fits on chip (mesh size limits
     // are checked in validate)
    s.ldN = (s.N + 3) / 4 * 4;
    s.tri_wc = (interior_level_width(p.n + 1) + 31) / 32 * 32;
    auto column_fits = [&](size_t elem) {
      return 2 * s.tri_wc + 32 <= 1024 &&
             elem * ((size_t)s.ldN + tri_ring_entries(s.tri_wc)) + sizeof(int) * 3 * (size_t)(p.n + 1) <=
                 227 * 1024;
    };
    s.tri_full = column_fits(8);
    s.tri_full32 = column_fits(4);
  }

  // the system's own stream carries the critical path (GMRES, block solves); the second stream of
  // the Gauss-Seidel sweep (later-column scatters) fills idle SMs at the lowest priority
  int prio_low = 0, prio_high = 0;
  SG_CUDA(cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high));
  s.prio_lo = prio_low;
  s.prio_hi = prio_high;
  SG_CUDA(cudaStreamCreateWithPriority(&s.stream, cudaStreamNonBlocking, prio_high));
  SG_CUDA(cudaEventCreateWithFlags(&s.ev, cudaEventDisableTiming));
  SG_CUDA(cudaEventCreateWithFlags(&s.seg_ev[0], cudaEventDisableTiming));
  SG_CUDA(cudaEventCreateWithFlags(&s.seg_ev[1], cudaEventDisableTiming));
  SG_CUDA(cudaMallocHost((void**)&s.hpin, 16 * sizeof(double)));

  SG_TRY(upload_i(s.rowptr, s.pat.rowptr, st));
  SG_TRY(upload_i(s.col, s.pat.col, st));
  SG_TRY(upload_i(s.diag, s.pat.diag, st));
  SG_TRY(upload_i(s.lev_f_ptr, s.pat.lev_f_ptr, st));
  SG_TRY(upload_i(s.lev_f_rows, s.pat.lev_f_rows, st));
  SG_TRY(upload_i(s.lev_b_ptr, s.pat.lev_b_ptr, st));
  SG_TRY(upload_i(s.lev_b_rows, s.pat.lev_b_rows, st));

  // operator tables
  SG_TRY(upload_i(s.pair_kb, s.op.pair_kb, st));
  SG_TRY(upload_i(s.ent_ptr, s.op.ent_ptr, st));
  SG_TRY(upload_i(s.ent_u, s.op.ent_u, st));
  SG_TRY(upload_d(s.ent_g, s.op.ent_g, st));
  if (lowp) SG_TRY(upload_f(s.ent_g_f32, s.op.ent_g, st));
  {
    std::vector<int2> cu(s.op.nchunks), ck(s.op.nchunks);
    for (int c = 0; c < s.op.nchunks; ++c) {
      cu[c] = make_int2(s.op.chunks[c].u0, s.op.chunks[c].u1);
      ck[c] = make_int2(s.op.chunks[c].k0, s.op.chunks[c].k1);
    }
    SG_TRY(s.chunks.alloc(cu.size()));
    SG_TRY(s.chunks.upload(cu, st));
    SG_TRY(s.chunks_k.alloc(ck.size()));
    SG_TRY(s.chunks_k.upload(ck, st));
  }

  // stiffness stack
  const size_t nnzL = (size_t)s.pat.nnz * s.L;
  SG_TRY(s.stack.alloc(nnzL));
  {
    DBuf<double> qp;
    SG_TRY(qp.alloc((size_t)p.n * p.n * 9 * (p.M + 1)));
    SG_TRY(launch_qp_table(s, qp.p, st));
    SG_TRY(launch_assemble(s, qp.p, st));
    SG_CUDA(cudaStreamSynchronize(st));
    qp.release();
  }
  if (p.precision == SG_MIXED_FP32) {
    SG_TRY(s.stack_f32.alloc(nnzL));
    SG_TRY(launch_cast_f32(s.stack.p, s.stack_f32.p, nnzL, st));
  } else if (p.precision == SG_MIXED_BF16) {
    SG_TRY(s.stack_bf16.alloc(nnzL));
    SG_TRY(launch_cast_bf16(s.stack.p, s.stack_bf16.p, nnzL, st));
  }
  // the SG operator kernels, chosen by op_kernel (timed per system shape when automatic)
  // In the mixed forms the FP64 operator serves only the outer residual (once per refinement):
  // the multigrid levels below the top keep the pair kernel on the FP64 stack unless the
  // row-tiled one is asked for, and the FP32 stack copy of the pair kernel is dropped once the
  // row-tiled FP32 operator serves.
  if (p.precision == SG_FP64 || p.op_kernel == SG_OP_TILE || krylov) SG_TRY(choose_operator(s, 8, st));
  if (p.precision == SG_MIXED_FP32) {
    SG_TRY(choose_operator(s, 4, st));
    if (s.tile32.ready) s.stack_f32.release();
  }

  // preconditioner blocks and factors
  const size_t NP = (size_t)s.N * s.P;
  if (s.pc_fac == SG_PC_FG) SG_TRY(fg_setup(s, st));
  if (s.pc_fac == SG_PC_MEAN || s.pc_fac == SG_PC_FS_GS || s.pc_fac == SG_PC_FS_JACOBI) {
    s.nfac = s.pc_fac == SG_PC_MEAN ? 1 : s.P;
    SG_TRY(s.blk.alloc((size_t)s.nfac * s.pat.nnz));
    SG_TRY(s.fac.alloc((size_t)s.nfac * s.pat.nnz));
    SG_TRY(launch_block_values(s, st));
    if (p.ilu_order == SG_ILU_COLOR4) {
      SG_TRY(launch_color_ilu(s, st));
    } else {
      SG_TRY(launch_ilu0(s, st));
      SG_TRY(launch_lu9(s, st));
    }
    if (lowp) {
      SG_TRY(s.lu9_f32.alloc(s.lu9.n));
      SG_TRY(s.blk_f32.alloc(s.blk.n));
      SG_TRY(launch_cast_f32(s.lu9.p, s.lu9_f32.p, s.lu9.n, st));
      SG_TRY(launch_cast_f32(s.blk.p, s.blk_f32.p, s.blk.n, st));
    }
    if (s.pc_fac == SG_PC_FS_GS) {
      SG_TRY(build_gs_tables(s, st));
      SG_TRY(s.stack_km.alloc(nnzL));
      SG_TRY(launch_transpose(s.stack.p, s.stack_km.p, (size_t)s.pat.nnz, s.L, st));
      if (p.precision == SG_MIXED_FP32 && !p.coupling_bf16) {
        SG_TRY(s.stack_km32.alloc(nnzL));
        SG_TRY(launch_cast_f32(s.stack_km.p, s.stack_km32.p, nnzL, st));
      } else if (p.precision == SG_MIXED_BF16 || p.coupling_bf16) {
        SG_TRY(s.stack_km16.alloc(nnzL));
        SG_TRY(launch_cast_bf16(s.stack_km.p, s.stack_km16.p, nnzL, st));
      }
      if (p.ilu_order == SG_ILU_COLOR4) SG_TRY(launch_color_coupling(s, st));
      // the mixed forms sweep in FP32 only: their FP64 k-major copy is not kept
      if (lowp) {
        SG_CUDA(cudaStreamSynchronize(st));
        s.stack_km.release();
      }
    }
    const size_t PL = (size_t)s.P * s.ldN;
    SG_TRY(s.rhs_t.alloc(PL));
    if (lowp) SG_TRY(s.rhs_t32.alloc(PL));
    if (p.inner_iters > 1) {
      SG_TRY(s.tri_w.alloc(PL));
      if (lowp) SG_TRY(s.tri_w32.alloc(PL));
    }
  }
  if (p.outer_sweeps > 1) {
    SG_TRY(s.tmp.alloc(NP));
    SG_TRY(s.tmp2.alloc(NP));
    if (lowp) {
      SG_TRY(s.tmp32.alloc(NP));
      SG_TRY(s.tmp232.alloc(NP));
    }
  }

  if (p.precond == SG_PC_MG) SG_TRY(mg_setup_levels(s, st));
  if (!krylov) {
    SG_CUDA(cudaStreamSynchronize(st));
    return SG_OK;
  }

  // GMRES workspace
  s.m = p.restart;
  const int mb = krylov_max_basis();
  SG_TRY(s.V.alloc((size_t)(s.m + 1) * NP));
  if (lowp) {
    SG_TRY(s.Z32.alloc((size_t)s.m * NP));
    SG_TRY(s.mv32a.alloc(NP));
    SG_TRY(s.mv32b.alloc(NP));
  } else {
    SG_TRY(s.Z.alloc((size_t)s.m * NP));
  }
  SG_TRY(s.rvec.alloc(NP));
  SG_TRY(s.Hs.alloc((size_t)(s.m + 1) * (s.m + 1)));
  SG_TRY(s.cs.alloc(mb));
  SG_TRY(s.sn.alloc(mb));
  SG_TRY(s.g.alloc(mb + 1));
  SG_TRY(s.y.alloc(3 * mb));
  SG_TRY(s.scal.alloc(8));
  SG_TRY(s.red.alloc((size_t)krylov_red_blocks() * mb));
  SG_TRY(s.flags.alloc(4));
  SG_TRY(s.xzero.alloc(1));
  SG_TRY(s.ticket.alloc(4));
  SG_CUDA(cudaMemsetAsync(s.ticket.p, 0, 4 * sizeof(unsigned int), st));
  SG_CUDA(cudaMemsetAsync(s.flags.p, 0, 4 * sizeof(int), st));
  SG_CUDA(cudaMemsetAsync(s.scal.p, 0, 8 * sizeof(double), st));
  SG_CUDA(cudaStreamSynchronize(st));
  return SG_OK;
}

int setup_system_public(System& s, cudaStream_t st, bool krylov) { return setup_system(s, st, krylov); }
void free_system_public(System* s) { free_system(s); }

static System* get_sys(const sg_handle* h, int sys) {
  if (!h || sys < 0 || sys >= (int)h->sys.size()) return nullptr;
  return h->sys[sys];
}

// ------------------------------------------------------------------ GMRES driver

struct SolveState {
  System* s;
  const double* F;
  double* X;
  double target = 0, bnorm = 0, beta = 0, prev_beta = 0;
  int iters = 0, restarts = 0, status = SG_OK;
  bool active = true, graphed = false;
  int jmax = 0;
  int seg_next = 0;     // first step of the next segment to queue
  int seg_queued = 0;   // segments queued in this cycle
  int seg_seen = 0;     // segments whose flags the host has read
  bool seg_more = false;  // more segments may be needed
};

static int iteration(System& s, int j, int last_col) {
  const size_t n = (size_t)s.N * s.P;
  cudaStream_t st = s.stream;
  const int* done = s.flags.p;
  double* vj = s.V.p + (size_t)j * n;
  double* w = s.V.p + (size_t)(j + 1) * n;
  if (s.prm.precision == SG_FP64) {
    double* zj = s.Z.p + (size_t)j * n;
    SG_TRY(precond_apply_f64(s, vj, zj, st, done));
    SG_TRY(launch_matvec_f64(s, zj, w, 1.0, nullptr, 0.0, st, done));
  } else {
    float* z32 = s.Z32.p + (size_t)j * n;
    SG_TRY(k_to_f32(n, vj, s.mv32a.p, done, st));
    SG_TRY(precond_apply_f32(s, s.mv32a.p, z32, st, done));
    SG_TRY(launch_matvec_f32(s, z32, s.mv32b.p, 1.0f, nullptr, 0.0f, st, done));
    SG_TRY(k_to_f64(n, s.mv32b.p, w, done, st));
  }
  return k_arnoldi(s, n, j, last_col, st);
}

// r = F - K x, beta = ||r||, mirrored to host with the cycle flags.  For the initial iterate
// (``first``) r starts as a copy of F and the operator product is skipped on the device when x
// is all zero (the common cold start).
static int residual(SolveState& ss, bool first = false) {
  System& s = *ss.s;
  const size_t n = (size_t)s.N * s.P;
  if (first) {
    SG_TRY(k_zero_flag(s, n, ss.X, s.xzero.p, s.stream));
    SG_CUDA(cudaMemcpyAsync(s.rvec.p, ss.F, sizeof(double) * n, cudaMemcpyDeviceToDevice, s.stream));
    SG_TRY(launch_matvec_f64(s, ss.X, s.rvec.p, -1.0, ss.F, 1.0, s.stream, s.xzero.p));
  } else {
    SG_TRY(launch_matvec_f64(s, ss.X, s.rvec.p, -1.0, ss.F, 1.0, s.stream));
  }
  SG_TRY(k_norm(s, n, s.rvec.p, s.scal.p + 1, s.stream));
  SG_CUDA(cudaMemcpyAsync(s.hpin, s.scal.p, 4 * sizeof(double), cudaMemcpyDeviceToHost, s.stream));
  SG_CUDA(cudaMemcpyAsync(s.hpin + 4, s.flags.p, 4 * sizeof(int), cudaMemcpyDeviceToHost, s.stream));
  return SG_OK;
}

// A cycle is queued in segments of Arnoldi steps.  After each segment the cycle's flags are copied
// to pinned host memory behind an event; the host queues the next segment only while the segment
// before the last one queued has not reported convergence, so at most two segments of steps that
// return at once (the device's done flag) follow the converged step, instead of the rest of the
// cycle.  A step of a large system takes milliseconds, ample time for the host to read a
// segment's flags and queue the next, so large systems queue two steps per segment (each step
// that runs empty still launches every kernel of a V-cycle); small ones six.
constexpr int kSegSteps = 6;
constexpr int kSegStepsLarge = 2;
constexpr long long kSegLargeUnknowns = 1LL << 18;

static int seg_steps(const System& s) {
  return (long long)s.N * s.P >= kSegLargeUnknowns ? kSegStepsLarge : kSegSteps;
}

// Steps [j0, j1) of the current cycle, as plain launches or as a graph captured on first use
// (keyed by the cycle length and j0).  Kernel timing is suspended during capture (events
// recorded there would become graph nodes).
static int launch_segment(SolveState& q, int j0, int j1) {
  System& s = *q.s;
  if (!q.graphed) {
    for (int j = j0; j < j1; ++j) SG_TRY(iteration(s, j, q.jmax - 1));
    return SG_OK;
  }
  for (auto& g : s.graphs)
    if (g.jmax == q.jmax && g.j0 == j0) {
      SG_CUDA(cudaGraphLaunch(g.exec, s.stream));
      count_launch((int)g.kernels);
      return SG_OK;
    }
  const bool timing = s.timer && s.timer->on;
  if (timing) s.timer->on = false;
  // launches queued during capture run only as the graph's kernel nodes: counted per replay
  const long long counted = sg_launch_count();
  SG_CUDA(cudaStreamBeginCapture(s.stream, cudaStreamCaptureModeThreadLocal));
  int rc = SG_OK;
  for (int j = j0; j < j1 && rc == SG_OK; ++j) rc = iteration(s, j, q.jmax - 1);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(s.stream, &graph);
  if (timing) s.timer->on = true;
  if (rc != SG_OK || e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return rc != SG_OK ? rc : fail(SG_ERR_CUDA, std::string("stream capture: ") + cudaGetErrorString(e));
  }
  count_launch((int)(counted - sg_launch_count()));
  size_t nnodes = 0;
  long long kernels = 0;
  if (cudaGraphGetNodes(graph, nullptr, &nnodes) == cudaSuccess && nnodes > 0) {
    std::vector<cudaGraphNode_t> nodes(nnodes);
    if (cudaGraphGetNodes(graph, nodes.data(), &nnodes) == cudaSuccess)
      for (auto nd : nodes) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++kernels;
      }
  }
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, cudaGraphInstantiateFlagUseNodePriority);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return fail(SG_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  s.graphs.push_back({q.jmax, j0, exec, kernels});
  SG_CUDA(cudaGraphLaunch(exec, s.stream));
  count_launch((int)kernels);
  return SG_OK;
}

// Queue the next segment of q's cycle and the read-back of its flags (slot = segment parity).
static int queue_segment(SolveState& q) {
  System& s = *q.s;
  const int j0 = q.seg_next, j1 = std::min(q.jmax, j0 + seg_steps(s));
  SG_TRY(launch_segment(q, j0, j1));
  const int slot = q.seg_queued & 1;
  SG_CUDA(cudaMemcpyAsync(s.hpin + 8 + 2 * slot, s.flags.p, 4 * sizeof(int), cudaMemcpyDeviceToHost,
                          s.stream));
  SG_CUDA(cudaEventRecord(s.seg_ev[slot], s.stream));
  q.seg_next = j1;
  q.seg_queued += 1;
  return SG_OK;
}

int gmres_solve_all(sg_handle* h, const double* const* F, double* const* X, sg_solve_info* info,
                    cudaStream_t user) {
  auto t0 = std::chrono::steady_clock::now();
  const int ns = (int)h->sys.size();
  std::vector<SolveState> st(ns);
  cudaEvent_t start;
  SG_CUDA(cudaEventCreateWithFlags(&start, cudaEventDisableTiming));
  SG_CUDA(cudaEventRecord(start, user));
  for (int i = 0; i < ns; ++i) {
    System& s = *h->sys[i];
    st[i].s = &s;
    st[i].F = F[i];
    st[i].X = X[i];
    SG_CUDA(cudaStreamWaitEvent(s.stream, start, 0));
    SG_TRY(k_norm(s, (size_t)s.N * s.P, F[i], s.scal.p + 2, s.stream));
    SG_TRY(residual(st[i], true));
  }
  cudaEventDestroy(start);
  for (int i = 0; i < ns; ++i) {
    System& s = *st[i].s;
    SG_CUDA(cudaStreamSynchronize(s.stream));
    st[i].bnorm = s.hpin[2];
    st[i].beta = s.hpin[1];
    st[i].target = std::max(s.prm.rtol * st[i].bnorm, s.prm.atol);
    st[i].prev_beta = st[i].beta;
    if (!std::isfinite(st[i].beta) || !std::isfinite(st[i].bnorm)) st[i].status = SG_ERR_NAN;
    if (st[i].bnorm == 0.0 && st[i].status == SG_OK) {  // K x = 0 has the solution x = 0
      SG_CUDA(cudaMemsetAsync(st[i].X, 0, sizeof(double) * (size_t)s.N * s.P, s.stream));
      st[i].beta = 0.0;
    }
  }
  while (true) {
    bool any = false;
    for (auto& q : st) {
      System& s = *q.s;
      q.active = q.status == SG_OK && q.beta > q.target && q.iters < s.prm.max_iters;
      if (!q.active) continue;
      any = true;
      double cyc = q.target;
      if (s.prm.precision != SG_FP64) cyc = std::max(q.target, s.prm.inner_rtol * q.beta);
      s.hpin[0] = cyc;
      q.jmax = std::min(s.m, s.prm.max_iters - q.iters);
      q.graphed = s.prm.graphs != 0;
      q.seg_next = q.seg_queued = q.seg_seen = 0;
      SG_CUDA(cudaMemcpyAsync(s.scal.p, s.hpin, sizeof(double), cudaMemcpyHostToDevice, s.stream));
      SG_TRY(k_init_cycle(s, (size_t)s.N * s.P, s.rvec.p, s.stream));
      // two segments in flight per system
      SG_TRY(queue_segment(q));
      if (q.seg_next < q.jmax) SG_TRY(queue_segment(q));
      q.seg_more = q.seg_next < q.jmax;
    }
    if (!any) break;
    // keep queuing segments while the device has not reported convergence
    bool pending = true;
    while (pending) {
      pending = false;
      for (auto& q : st) {
        if (!q.active || !q.seg_more) continue;
        System& s = *q.s;
        const int slot = q.seg_seen & 1;
        cudaError_t e = cudaEventQuery(s.seg_ev[slot]);
        if (e == cudaErrorNotReady) {
          pending = true;
          continue;
        }
        if (e != cudaSuccess) return fail(SG_ERR_CUDA, std::string("segment event: ") + cudaGetErrorString(e));
        const int* fl = reinterpret_cast<const int*>(s.hpin + 8 + 2 * slot);
        q.seg_seen += 1;
        if (fl[0] || q.seg_next >= q.jmax) {
          q.seg_more = false;
          continue;
        }
        SG_TRY(queue_segment(q));
        q.seg_more = q.seg_next < q.jmax;
        pending = pending || q.seg_more;
      }
      if (pending) std::this_thread::yield();
    }
    for (auto& q : st) {
      if (!q.active) continue;
      System& s = *q.s;
      SG_TRY(k_finish_cycle(s, (size_t)s.N * s.P, q.X, s.prm.precision != SG_FP64, s.stream));
      SG_TRY(residual(q));
    }
    for (auto& q : st) {
      if (!q.active) continue;
      System& s = *q.s;
      SG_CUDA(cudaStreamSynchronize(s.stream));
      const int* fl = reinterpret_cast<const int*>(s.hpin + 4);
      q.iters += fl[1];
      q.restarts += 1;
      q.prev_beta = q.beta;
      q.beta = s.hpin[1];
      if (fl[2] != SG_OK || !std::isfinite(q.beta)) q.status = SG_ERR_NAN;
      // a refinement step that does not reduce the true residual cannot make progress
      if (s.prm.precision != SG_FP64 && q.beta > q.target && q.beta >= q.prev_beta)
        q.status = SG_ERR_NOT_CONVERGED;
      if (fl[1] == 0 && q.beta > q.target && q.status == SG_OK) q.status = SG_ERR_NOT_CONVERGED;
    }
  }
  int rc = SG_OK;
  double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  for (int i = 0; i < ns; ++i) {
    auto& q = st[i];
    if (q.status == SG_OK && q.beta > q.target) q.status = SG_ERR_NOT_CONVERGED;
    info[i].iters = q.iters;
    info[i].restarts = q.restarts;
    info[i].status = q.status;
    info[i].rel_resid = q.bnorm > 0 ? q.beta / q.bnorm : 0.0;
    info[i].seconds = secs;
    if (q.status != SG_OK && rc == SG_OK) rc = q.status;
    SG_CUDA(cudaEventRecord(q.s->ev, q.s->stream));
    SG_CUDA(cudaStreamWaitEvent(user, q.s->ev, 0));
  }
  SG_CUDA(cudaStreamSynchronize(user));
  if (rc != SG_OK) set_error(rc == SG_ERR_NAN ? "NaN or Inf in a residual" : "GMRES did not reach the tolerance");
  return rc;
}

}  // namespace sg

using namespace sg;

// ------------------------------------------------------------------ C ABI

extern "C" {

void sg_default_params(sg_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->n = 16;
  p->M = 2;
  p->p = 2;
  p->q = 0;
  p->sigma = 0.5;
  p->ell = 1.0;
  p->a_min = 0.0;
  p->mu = 0.0;
  p->f = 1.0;
  p->precond = SG_PC_MEAN;
  p->inner_iters = 1;
  p->outer_sweeps = 1;
  p->restart = 30;
  p->max_iters = 2000;
  p->rtol = 1e-10;
  p->atol = 0.0;
  p->precision = SG_FP64;
  p->inner_rtol = 1e-4;
  p->graphs = 0;
  p->mg_smoother = SG_PC_FS_GS;
  p->fg_rule = SG_FG_PAPER;
  p->fg_bf16 = 0;
  p->mg_coarse = 2;
  p->op_kernel = SG_OP_AUTO;
  p->op_kappa = 0;
  p->op_ctas = 0;
  p->ilu_order = SG_ILU_NATURAL;
  p->coupling_bf16 = 0;
}

int sg_setup(const sg_params* prm, int nsys, void* stream, sg_handle** out) {
  if (!out) return fail(SG_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!prm || nsys < 1) return fail(SG_ERR_ARG, "need nsys >= 1 parameter sets");
  for (int i = 0; i < nsys; ++i) SG_TRY(validate(prm[i]));
  cudaStream_t st = (cudaStream_t)stream;
  sg_handle* h = new sg_handle();
  cudaGetDevice(&h->device);
  for (int i = 0; i < nsys; ++i) {
    System* s = new System();
    s->prm = prm[i];
    s->timer = &h->timer;
    h->sys.push_back(s);
    int rc = setup_system(*s, st);
    if (rc != SG_OK) {
      std::string msg = g_last_error;
      sg_free(h);
      return fail(rc, "system " + std::to_string(i) + ": " + msg);
    }
  }
  *out = h;
  return SG_OK;
}

int sg_dims(const sg_handle* h, int sys, int* N, int* P, int* L) {
  System* s = get_sys(h, sys);
  if (!s) return fail(SG_ERR_ARG, "bad handle or system index");
  if (N) *N = s->N;
  if (P) *P = s->P;
  if (L) *L = s->L;
  return SG_OK;
}

int sg_nnz(const sg_handle* h, int sys, long long* nnz_A, long long* nnz_G) {
  System* s = get_sys(h, sys);
  if (!s) return fail(SG_ERR_ARG, "bad handle or system index");
  if (nnz_A) *nnz_A = s->pat.nnz;
  if (nnz_G) *nnz_G = s->nnzG;
  return SG_OK;
}

int sg_matvec(sg_handle* h, int sys, const double* X, double* Y, void* stream) {
  System* s = get_sys(h, sys);
  if (!s || !X || !Y) return fail(SG_ERR_ARG, "bad handle, system index or pointer");
  return launch_matvec_f64(*s, X, Y, 1.0, nullptr, 0.0, (cudaStream_t)stream);
}

int sg_matvec_lowp(sg_handle* h, int sys, const float* X, float* Y, void* stream) {
  System* s = get_sys(h, sys);
  if (!s || !X || !Y) return fail(SG_ERR_ARG, "bad handle, system index or pointer");
  if (s->prm.precision == SG_FP64) return fail(SG_ERR_ARG, "system has no low-precision stack");
  return launch_matvec_f32(*s, X, Y, 1.0f, nullptr, 0.0f, (cudaStream_t)stream);
}

int sg_precond_apply(sg_handle* h, int sys, const double* R, double* Z, void* stream) {
  System* s = get_sys(h, sys);
  if (!s || !R || !Z) return fail(SG_ERR_ARG, "bad handle, system index or pointer");
  return precond_apply_f64(*s, R, Z, (cudaStream_t)stream);
}

int sg_precond_apply_lowp(sg_handle* h, int sys, const float* R, float* Z, void* stream) {
  System* s = get_sys(h, sys);
  if (!s || !R || !Z) return fail(SG_ERR_ARG, "bad handle, system index or pointer");
  if (s->prm.precision == SG_FP64) return fail(SG_ERR_ARG, "system has no low-precision factors");
  return precond_apply_f32(*s, R, Z, (cudaStream_t)stream);
}

int sg_rhs(sg_handle* h, int sys, double* F, void* stream) {
  System* s = get_sys(h, sys);
  if (!s || !F) return fail(SG_ERR_ARG, "bad handle, system index or pointer");
  return launch_rhs(*s, F, (cudaStream_t)stream);
}

int sg_gmres_solve(sg_handle* h, const double* const* F, double* const* X, sg_solve_info* info,
                   void* stream) {
  if (!h || !F || !X || !info) return fail(SG_ERR_ARG, "NULL argument");
  for (size_t i = 0; i < h->sys.size(); ++i)
    if (!F[i] || !X[i]) return fail(SG_ERR_ARG, "NULL F or X for system " + std::to_string(i));
  return gmres_solve_all(h, F, X, info, (cudaStream_t)stream);
}

int sg_export(const sg_handle* h, int sys, int what, void* dst, size_t bytes) {
  System* s = get_sys(h, sys);
  if (!s || !dst) return fail(SG_ERR_ARG, "bad handle, system index or pointer");
  const void* src = nullptr;
  size_t need = 0;
  std::vector<double> tmp;
  switch (what) {
    case 0: src = s->stack.p; need = sizeof(double) * (size_t)s->pat.nnz * s->L; break;
    case 1: src = s->pat.rowptr.data(); need = sizeof(int) * (s->N + 1); break;
    case 2: src = s->pat.col.data(); need = sizeof(int) * s->pat.nnz; break;
    case 3:
      for (auto& t : s->kl) tmp.push_back(t.lam);
      src = tmp.data();
      need = sizeof(double) * tmp.size();
      break;
    case 4:
      if (!s->fac.p || s->prm.precond != SG_PC_MEAN) return fail(SG_ERR_ARG, "no mean-block ILU factors");
      src = s->fac.p;
      need = sizeof(double) * s->pat.nnz;
      break;
    case 5:
      for (auto& t : s->triples) {
        tmp.push_back(t.k);
        tmp.push_back(t.a);
        tmp.push_back(t.b);
        tmp.push_back(t.g);
      }
      src = tmp.data();
      need = sizeof(double) * tmp.size();
      break;
    default: return fail(SG_ERR_ARG, "unknown export selector");
  }
  if (bytes < need) return fail(SG_ERR_ARG, "destination too small: need " + std::to_string(need));
  if (what == 0 || what == 4) {
    SG_CUDA(cudaDeviceSynchronize());
    SG_CUDA(cudaMemcpy(dst, src, need, cudaMemcpyDeviceToHost));
  } else {
    std::memcpy(dst, src, need);
  }
  return SG_OK;
}

long long sg_launch_count(void) { return g_launches.load(); }

int sg_op_info(const sg_handle* h, int sys, long long* info, char* msg, int msg_len) {
  System* s = get_sys(h, sys);
  if (!s || !info) return fail(SG_ERR_ARG, "bad handle, system index or pointer");
  const TileOp* ops[2] = {&s->tile64, &s->tile32};
  for (int i = 0; i < 2; ++i) {
    info[4 * i + 0] = ops[i]->ready ? 2 : 1;
    info[4 * i + 1] = ops[i]->ready ? ops[i]->kappa : 0;
    info[4 * i + 2] = ops[i]->ready ? (long long)ops[i]->smem : 0;
    info[4 * i + 3] = ops[i]->ready ? ops[i]->nchunks : 0;
  }
  if (s->prm.precision == SG_FP64) info[4] = 0;
  if (msg && msg_len > 0) {
    std::strncpy(msg, s->tile_msg.c_str(), (size_t)msg_len - 1);
    msg[msg_len - 1] = 0;
  }
  return SG_OK;
}

int sg_fg_splits(int M, int p, int rule, int* out, int* count) {
  if (M < 1 || M > 8 || p < 0 || p > 6 || rule < SG_FG_PAPER || rule > SG_FG_WHOLE ||
      out == nullptr || count == nullptr)
    return fail(SG_ERR_ARG, "sg_fg_splits: M, p or rule out of range");
  auto r = fg_split_ranges(M, p, rule);
  for (size_t i = 0; i < r.size(); ++i) {
    out[2 * i] = r[i].first;
    out[2 * i + 1] = r[i].second;
  }
  *count = (int)r.size();
  return SG_OK;
}

int sg_tune_plan(int n, int M, int p, int q, int precision, long long smem_max, long long* out) {
  if (!out) return fail(SG_ERR_ARG, "out is NULL");
  sg_params prm;
  sg_default_params(&prm);
  prm.n = n;
  prm.M = M;
  prm.p = p;
  prm.q = q;
  SG_TRY(validate(prm));
  System s;
  s.prm = prm;
  SG_TRY(host_tables(s));
  const int elem = precision == SG_FP64 ? 8 : 4;
  int row = 0;
  for (int ctas = 1; ctas <= 2; ++ctas)
    for (int kappa : {1, 2, 4}) {
      long long* o = out + 16 * row++;
      for (int i = 0; i < 16; ++i) o[i] = 0;
      o[0] = kappa;
      o[1] = ctas;
      TilePlan pl;
      const size_t budget = ctas == 1 ? (size_t)smem_max : (size_t)smem_max / 2;
      const int rc = plan_tile_op(s, kappa, elem, budget, pl, ctas);
      set_error("");
      o[2] = rc == SG_OK;
      if (rc != SG_OK) continue;
      o[3] = (long long)pl.smem;
      o[4] = pl.nchunks;
      o[5] = pl.max_slots;
      o[6] = pl.pairs;
      o[7] = pl.entries;
      o[8] = pl.Lu;
      o[9] = pl.ngroups;
      o[10] = verify_tile_plan(s, pl) == SG_OK;
      o[11] = (long long)budget;
      o[12] = pl.visits;
      o[13] = pl.s1_steps;
      o[14] = pl.s2_steps;
      set_error("");
    }
  return SG_OK;
}

int sg_timing_start(sg_handle* h, int stride) {
  if (!h || stride < 1) return fail(SG_ERR_ARG, "bad handle or stride");
  Timer& t = h->timer;
  if (t.ev.empty()) {
    t.ev.resize(1 << 16);
    for (auto& e : t.ev) SG_CUDA(cudaEventCreate(&e));
  }
  t.used = 0;
  t.recs.clear();
  for (auto& c : t.count) c = 0;
  t.stride = stride;
  t.on = true;
  return SG_OK;
}

int sg_timing_stop(sg_handle* h, double* ms, long long* timed, long long* launches) {
  if (!h) return fail(SG_ERR_ARG, "bad handle");
  Timer& t = h->timer;
  t.on = false;
  double acc[K_NCLASS] = {};
  long long nt[K_NCLASS] = {};
  for (auto& r : t.recs) {
    SG_CUDA(cudaEventSynchronize(t.ev[r.second + 1]));
    float e = 0.f;
    SG_CUDA(cudaEventElapsedTime(&e, t.ev[r.second], t.ev[r.second + 1]));
    acc[r.first] += e;
    nt[r.first] += 1;
  }
  for (int c = 0; c < K_NCLASS; ++c) {
    if (ms) ms[c] = acc[c];
    if (timed) timed[c] = nt[c];
    if (launches) launches[c] = t.count[c];
  }
  t.recs.clear();
  t.used = 0;
  return SG_OK;
}

void sg_free(sg_handle* h) {
  if (!h) return;
  for (auto* s : h->sys) free_system(s);
  for (auto& e : h->timer.ev) cudaEventDestroy(e);
  delete h;
}

const char* sg_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
