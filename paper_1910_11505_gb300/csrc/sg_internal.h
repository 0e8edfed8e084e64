// Internal declarations shared by the translation units of the SG solver library.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/sg.h"

namespace sg {

// ------------------------------------------------------------------ errors

void set_error(const std::string& msg);
int fail(int code, const std::string& msg);

struct Status {
  int code = SG_OK;
  std::string msg;
};

#define SG_CUDA(call)                                                                  \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return ::sg::fail(SG_ERR_CUDA, std::string(#call " failed: ") + cudaGetErrorString(e_) + \
                                         " at " __FILE__ ":" + std::to_string(__LINE__)); \
  } while (0)

#define SG_TRY(call)            \
  do {                          \
    int rc_ = (call);           \
    if (rc_ != SG_OK) return rc_; \
  } while (0)

void count_launch(int n = 1);
int check_launch(const char* what);
// Raise a kernel's dynamic shared-memory limit on the current device to ``bytes`` unless an
// earlier call already set at least that much (the attribute call is not repeated per launch).
int ensure_smem(const void* kernel, size_t bytes);
// Largest dynamic shared memory one CTA may opt into on the current device.
size_t smem_optin_max();
// Output layer of the learned warm start on the tensor cores (k_net_tc.cu): mode 0 writes
// Y = H2 W3^T + b3 (Yf or Yd), mode 1 the residual gradient dY and per-CTA loss partials.
int launch_out_tc(int mode, int B, int h2, int out, const float* H2, const __nv_bfloat16* W3h,
                  const float* b3, float* Yf, double* Yd, const float* T, __nv_bfloat16* dYh,
                  int outp, float* lpart, int* err, cudaStream_t st, int* nparts);
// dH2 = dY W3 split over the output units on the tensor cores (k_net_tc.cu), and the transposed
// BF16 copy of W3 it reads.
int launch_dh2_tc(int B, int outp, const __nv_bfloat16* dYh, const __nv_bfloat16* W3hT,
                  float* part, size_t part_stride, int ldp, int max_split, int* err,
                  cudaStream_t st, int* nsplit);
int launch_w3t_bf16(int out, int outp, int h2, const float* W3, __nv_bfloat16* W3hT,
                    cudaStream_t st);

// ------------------------------------------------------------------ live kernel timing

// Kernel classes timed by sg_timing_start / sg_timing_stop (values match SG_K_* in sg.h).
enum KClass { K_APPLY_F64 = 0, K_APPLY_LOWP = 1, K_ILU_SOLVE = 2, K_GS_SCATTER = 3,
              K_ARNOLDI = 4, K_OTHER = 5, K_NCLASS = 6 };

struct Timer {
  bool on = false;
  int stride = 1;
  std::vector<cudaEvent_t> ev;          // start / end pairs
  size_t used = 0;
  long long count[K_NCLASS] = {};
  std::vector<std::pair<int, size_t>> recs;
};

// Brackets one launch with events on its stream when the handle's timer is on and the launch
// falls on the sampling stride.
struct TimeScope {
  Timer* t;
  int cls;
  cudaStream_t st;
  long long idx = -1;
  TimeScope(Timer* t_, int cls_, cudaStream_t st_);
  ~TimeScope();
};

// ------------------------------------------------------------------ device helpers

#ifdef __CUDACC__
// Bulk prefetch of [base, base + bytes) into L2 (cp.async.bulk.prefetch.L2), in 16 KB pieces
// spread over the threads of ``nparts`` CTAs of which this is CTA ``part``.  The range is trimmed
// inward to 16-byte boundaries (the instruction's alignment rule), so nothing outside it is touched.
__device__ __forceinline__ void l2_prefetch(const void* base, size_t bytes, int part, int nparts) {
  const unsigned long long b0 = reinterpret_cast<unsigned long long>(base);
  const unsigned long long lo = (b0 + 15ull) & ~15ull, hi = (b0 + bytes) & ~15ull;
  constexpr unsigned long long kPiece = 16384ull;
  for (unsigned long long off = lo + (unsigned long long)(part * blockDim.x + threadIdx.x) * kPiece;
       off < hi; off += (unsigned long long)nparts * blockDim.x * kPiece) {
    const unsigned sz = (unsigned)(hi - off < kPiece ? hi - off : kPiece);
    unsigned long long g;
    asm volatile("cvta.to.global.u64 %0, %1;" : "=l"(g) : "l"(off));
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(g), "r"(sz) : "memory");
  }
}

// mbarrier and 1-D bulk-copy (cp.async.bulk) helpers.  Every wait is bounded: after kWaitLimit
// polls it gives up and the caller takes its error path.
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
#endif

// ------------------------------------------------------------------ device buffers

template <typename T>
struct DBuf {
  T* p = nullptr;
  size_t n = 0;
  int alloc(size_t count);
  int upload(const std::vector<T>& h, cudaStream_t s);
  void release();
};

// ------------------------------------------------------------------ host-side setup math

// One 1-D Karhunen-Loeve mode of the kernel exp(-|s-t|/ell) on [0,1], t = x - 1/2:
// even: cos(w t)/nrm, odd: sin(w t)/nrm, eigenvalue mu = 2c/(w^2+c^2), c = 1/ell.
struct KL1 {
  double w, nrm, mu;
  int odd;
};

struct KLTerm {  // one 2-D term: sqrt(lambda) f_i(x1) f_j(x2)
  KL1 fx, fy;
  double sqrt_lam;
  double lam;
  int i, j;
};

std::vector<KL1> kl_modes_1d(double ell, int count);
std::vector<KLTerm> kl_terms_2d(double sigma, double ell, int M);
std::vector<int> total_degree_set(int M, int p);  // |J| x M, lexicographic, last index fastest
double hermite_triple(int i, int j, int k);

struct Pattern {  // 9-point Q1 pattern, CSR with sorted columns
  int n = 0, m = 0, N = 0, nnz = 0;
  std::vector<int> rowptr, col, diag;
  std::vector<int> lev_f_ptr, lev_f_rows, lev_b_ptr, lev_b_rows;  // wavefront levels
  int max_width = 0;
};
Pattern make_pattern(int n);
// Largest number of interior nodes (1 <= x, y <= m - 2) on one wavefront level x + 2y = l.
int interior_level_width(int m);
// Factor-ring depth (levels fetched ahead) of the wavefront solve and its ring size in elements
// for wc threads per thread group (2 slots per level for one group, 3 for the other).
constexpr int kTriAhead = 8;
inline size_t tri_ring_entries(int wc) { return (size_t)kTriAhead * 5 * wc; }
// Level rows held in shared memory by the wavefront solve, and its shared memory in bytes for a
// mesh of m x m nodes: level window, factor rings, level offsets.
constexpr int kTriWin = 16;
// Staging threads of the wavefront solve: one warp per 64 rows of group width.
inline int tri_staging_threads(int wc) { return 32 * (wc > 64 ? wc / 64 : 1); }
inline size_t tri_smem_bytes(int m, int wc, size_t elem) {
  return elem * ((size_t)kTriWin * m + tri_ring_entries(wc)) + sizeof(int) * (size_t)(3 * m - 1);
}

// ------------------------------------------------------------------ matvec work tables

// The SG operator per node row i: T[k,b] = sum_e A[e,k] X[col_e, b] for every (k,b) pair that
// meets a nonzero G_k[a,b]; then Y[i,a] = sum G_k[a,b] T[k,b].  Pairs are sorted by (k, b) and cut
// into chunks of at most kChunkPairs pairs spanning at most kChunkK consecutive k.
constexpr int kChunkPairs = 512;
constexpr int kChunkK = 64;

struct ChunkDesc {
  int u0, u1;  // pair range
  int k0, k1;  // k range (inclusive k0, exclusive k1)
};

struct OpTables {
  int npairs = 0, nent = 0, nchunks = 0;
  std::vector<int> pair_kb;    // k << 16 | b
  std::vector<ChunkDesc> chunks;
  std::vector<int> ent_ptr;    // nchunks x (P + 1), offsets into ent_u / ent_g
  std::vector<int> ent_u;      // pair index local to the chunk
  std::vector<double> ent_g;   // G_k[a,b]
};

struct Triple {
  int k, a, b;
  double g;
};

// Row-tiled operator (k_apply_tile.cu): k permuted into groups of kappa with similar b lists,
// chunks of at most 8 groups, per group the union b list (b | mask << 16, first slot), per
// (chunk, a) the stage-2 entries (slot, G), the group descriptors in each chunk's side table, and
// the stack stored per tile of 32 interior rows of one grid line as [k position][entry][row].
struct TileOp {
  bool ready = false;
  int kappa = 0, elem = 0, ctas = 1, tiles_per_line = 0, ntiles = 0, Pp = 0, Lu = 0;
  int nchunks = 0, ngroups = 0, max_chunk_k = 0, max_slots = 0, apw = 0;
  int abytes_slot = 0, sbytes_slot = 0, tbuf_elems = 0, xslab_elems = 0;
  size_t smem = 0;
  DBuf<int4> chunk, chunkx;
  DBuf<unsigned char> side;
  DBuf<int> err;
  DBuf<double> stack;
  DBuf<float> stack32;
};

// Host-side plan of the row-tiled operator (tables before upload).  Per chunk: {first k position,
// k count, first group, groups} and {side table offset in 16-byte units, bytes, offset of the
// per-a entry offsets, offset of the entries}; per group {union list start within the chunk,
// length, first k position within the chunk, k count}; the side tables of all chunks.
struct TilePlan {
  int kappa = 0, elem = 0, ctas = 1, tiles_per_line = 0, ntiles = 0, Pp = 0, Lu = 0;
  int nchunks = 0, ngroups = 0, max_chunk_k = 0, max_slots = 0, apw = 0;
  int abytes_slot = 0, sbytes_slot = 0, tbuf_elems = 0, xslab_elems = 0;
  size_t smem = 0, max_side = 0;
  long long pairs = 0, entries = 0;
  // union entries, and the steps of the slowest warp summed over the chunks (stage 1: steps of
  // four union entries in FP32, two in FP64, plus one per piece; stage 2: steps of one entry of
  // four runs side by side, plus one per block of runs)
  long long visits = 0, s1_steps = 0, s2_steps = 0;
  std::vector<int4> cdesc, cxdesc, gdesc;
  std::vector<int> kperm;
  std::vector<unsigned char> side;
};

// ------------------------------------------------------------------ per-system state

struct System {
  sg_params prm;
  int pc_fac = SG_PC_NONE;     // block preconditioner whose factors this system holds: prm.precond,
                               // or the smoother of a multigrid system (prm.mg_smoother)
  int N = 0, P = 0, L = 0, M = 0, n = 0;
  long long nnzG = 0;
  Pattern pat;
  std::vector<KLTerm> kl;
  std::vector<Triple> triples;  // sorted by k, a, b
  OpTables op;

  // device: pattern
  DBuf<int> rowptr, col, diag, lev_f_ptr, lev_f_rows, lev_b_ptr, lev_b_rows;
  // device: operator
  DBuf<double> stack;          // nnz x L
  DBuf<float> stack_f32;       // nnz x L (SG_MIXED_FP32)
  DBuf<__nv_bfloat16> stack_bf16;  // nnz x L (SG_MIXED_BF16)
  DBuf<double> stack_km;       // L x nnz k-major copy for the Gauss-Seidel scatter
  DBuf<float> stack_km32;
  DBuf<__nv_bfloat16> stack_km16;
  DBuf<int> pair_kb, ent_ptr, ent_u;
  DBuf<int2> chunks;           // (u0 | u1 packed as two ints), k range in chunks_k
  DBuf<int2> chunks_k;
  DBuf<double> ent_g;
  DBuf<float> ent_g_f32;
  TileOp tile64, tile32;       // row-tiled operator in FP64 / FP32 (when built)
  std::string tile_msg;        // why a row-tiled operator was not built (empty if it was)
  // device: preconditioner
  int nfac = 0;                // number of factor sets (1 for mean, P for field split)
  DBuf<double> blk;            // nfac x nnz block matrices (A_0 or K_aa) before factorisation
  DBuf<double> fac;            // nfac x nnz ILU(0) factors
  DBuf<float> blk_f32;         // FP32 copy for the mixed inner solver
  DBuf<double> lu9;            // nfac x 9 x N level-major slot layout of the factors
  DBuf<float> lu9_f32;
  DBuf<int> lev9_off;          // start of each wavefront level in level-major order
  DBuf<int> cstart;            // four-colour ordering: start of each colour (5 offsets)
  int nlev9 = 0;
  int tri_wc = 0;              // threads per group of the wavefront solve (multiple of 32)
  int ldN = 0;                 // column stride of rhs_t / tri_w: N rounded up to a multiple of 4
  bool tri_full = false;       // the FP64 (FP32) block solve holds the whole column on chip
  bool tri_full32 = false;
  // field-split Gauss-Seidel scatter tables, per source block b: k list and (a, g) entries, for
  // the later columns a >= b + 2 (gs_*) and for the next column a = b + 1 (gsn_*)
  DBuf<int> gs_kptr, gs_k, gs_eptr, gs_ea;
  DBuf<double> gs_eg;
  DBuf<float> gs_eg_f32;
  DBuf<int> gsn_kptr, gsn_k, gsn_eptr, gsn_ea;
  DBuf<double> gsn_eg;
  DBuf<float> gsn_eg_f32;
  // four-colour sweeps: the next-column coupling K_{a,a-1} = sum_k G_k[a,a-1] A_k of every column
  // a >= 1 as a 9-slot stencil in the colour-major layout of the factors, (P - 1) x 9 x N; the
  // block solve of column a subtracts K_{a,a-1} z_{a-1} from its right-hand side itself
  DBuf<double> gsn_cs;
  DBuf<float> gsn_cs32;
  // the coupling term K_{a,a-1} z_{a-1} per colour-major position, left by the solve of column
  // a - 1 for the solve of column a
  DBuf<double> gsn_corr;
  DBuf<float> gsn_corr32;
  // grouped field split (SG_PC_FG): per split its fields [f0, f1) and the ILU(0) of its diagonal
  // block, N x 9 blocks of Q x Q (Q = f1 - f0) in the colour-major node order, block slot
  // (dy+1)*3 + (dx+1); lower-colour slots hold L_ij D_j^-1, slot 4 D_i^-1, higher-colour slots
  // D_i^-1 U_ij; each block column-major.  FP64 systems keep fac, mixed ones fac32 (or fac16).
  struct FgSplit {
    int f0 = 0, f1 = 0;
    DBuf<double> fac;
    DBuf<float> fac32;
    DBuf<__nv_bfloat16> fac16;  // fg_bf16: the FP32 factors rounded to BF16 (fac32 released)
  };
  std::vector<FgSplit> fg;
  std::vector<int> cstart_h;     // host copy of the four-colour offsets (grouped field split)
  DBuf<double> fg_tmp, fg_tmp2;  // splits after the first: the earlier splits' solution (other
  DBuf<float> fg_tmp32, fg_tmp232;  // fields zero) and K times it
  int gs_max_klen = 0;
  // device scratch
  DBuf<double> rhs_t;          // P columns of stride ldN: right-hand sides of the block solves
                               // (the Gauss-Seidel sweep subtracts sum_{b<a} K_ab z_b in place)
  DBuf<double> tmp, tmp2;      // N x P
  DBuf<double> tri_w;          // P x ldN work columns of the inner ILU iterations
  DBuf<float> rhs_t32, tmp32, tmp232, tri_w32;
  // GMRES workspace
  int m = 0;
  DBuf<double> V, Z, Hs, cs, sn, g, y, scal, red;  // see krylov.cu
  DBuf<int> flags;
  DBuf<int> xzero;             // the initial iterate is all zero (its operator product is skipped)
  DBuf<unsigned int> ticket;
  DBuf<float> V32, Z32;        // inner FGMRES basis for mixed precision (FP32 vectors)
  DBuf<double> rvec;           // FP64 residual r = F - K x
  DBuf<float> mv32a, mv32b;    // FP32 operand / result of the inner operator
  double* hpin = nullptr;      // pinned host mirror of state[0..3] and flags[0..2]
  Timer* timer = nullptr;      // the handle's timer
  struct CycleGraph {
    int jmax, j0;
    cudaGraphExec_t exec;
    long long kernels;  // kernel nodes: the launches one replay makes
  };
  std::vector<CycleGraph> graphs;  // captured segments of GMRES cycles (sg_params.graphs = 1)
  cudaEvent_t seg_ev[2] = {nullptr, nullptr};  // flags of the last two queued cycle segments
  cudaStream_t stream = nullptr;
  cudaEvent_t ev = nullptr;
  // Gauss-Seidel sweep: second stream for the later-column scatters, which overlap the next
  // block solve, and the events ordering the two streams
  cudaStream_t stream2 = nullptr;
  cudaEvent_t ev_z = nullptr, ev_r[2] = {nullptr, nullptr};
  // launch priorities (cudaDeviceGetStreamPriorityRange): the block solves of the sweep launch at
  // the highest, the later-column scatters at the lowest, so that the block scheduler gives SMs
  // freed by scatter CTAs to a pending block solve first (graphs keep the per-node priorities)
  int prio_lo = 0, prio_hi = 0;
  // multigrid (SG_PC_MG): the coarser levels, coarsest first, each a System on its own mesh with
  // the same stochastic data; per level the V-cycle's right-hand side b, iterate u, residual r and
  // smoother correction d (the finest level uses the caller's R and Z as b and u)
  std::vector<System*> mg;
  DBuf<double> mg_b, mg_u, mg_r, mg_d;
  DBuf<float> mg_b32, mg_u32, mg_r32, mg_d32;
  // coarsest level only: dense inverse of its interior SG matrix (nint P x nint P, row-major,
  // unknown index t * P + a for interior node t) and the interior node ids
  int mg_nint = 0;
  DBuf<double> mg_inv;
  DBuf<float> mg_inv32;
  DBuf<int> mg_nodes;
};

}  // namespace sg

struct sg_handle {
  std::vector<sg::System*> sys;
  int device = 0;
  sg::Timer timer;
};

namespace sg {

// ------------------------------------------------------------------ kernels (launchers)

int launch_qp_table(System& s, double* qp, cudaStream_t st);
int launch_assemble(System& s, const double* qp, cudaStream_t st);
int launch_rhs(System& s, double* F, cudaStream_t st);
int launch_block_values(System& s, cudaStream_t st);
int launch_ilu0(System& s, cudaStream_t st);
// ILU(0) in the four-colour ordering (k_ilu_color.cu): factors into lu9 (colour-major slots)
int launch_color_ilu(System& s, cudaStream_t st);
// Block solves of columns a0 .. a0 + ncols - 1 from Rt into Z (Z may be null: the solutions stay
// in the columns of Rt).  With ``cs`` (a coupling stencil set laid out as gsn_cs; one column):
// the solve of column a first subtracts the coupling of column a - 1 left in ``corr`` (a > 0),
// and leaves the coupling of column a + 1 in ``corr`` (a + 1 < P).
template <typename T>
int launch_color_solve(System& s, int a0, int ncols, int fac_per_col, const T* lu, T* Rt, T* Z,
                       cudaStream_t st, const int* done, const T* cs = nullptr, T* corr = nullptr);
// The next-column coupling stencils gsn_cs (FP64 systems) or gsn_cs32 (mixed systems, from the
// BF16-rounded stiffness values when the sweep couples in BF16), from the FP64 k-major stack.
int launch_color_coupling(System& s, cudaStream_t st);
int launch_lu9(System& s, cudaStream_t st);
int launch_cast_f32(const double* src, float* dst, size_t n, cudaStream_t st);
int launch_cast_bf16(const double* src, __nv_bfloat16* dst, size_t n, cudaStream_t st);
int launch_cast_f64(const float* src, double* dst, size_t n, cudaStream_t st);
// dst[c * rows + r] = src[r * cols + c]  (rows x cols -> cols x rows)
int launch_transpose(const double* src, double* dst, size_t rows, int cols, cudaStream_t st);

// Y = alpha * K X + beta * B  (B may be null when beta == 0)
int launch_matvec_f64(const System& s, const double* X, double* Y, double alpha, const double* B,
                      double beta, cudaStream_t st, const int* done = nullptr);
int launch_matvec_f32(const System& s, const float* X, float* Y, float alpha, const float* B,
                      float beta, cudaStream_t st, const int* done = nullptr);

int precond_apply_f64(System& s, const double* R, double* Z, cudaStream_t st,
                      const int* done = nullptr);
int precond_apply_f32(System& s, const float* R, float* Z, cudaStream_t st,
                      const int* done = nullptr);
// One field-split Gauss-Seidel application (outer_sweeps = 1) whose right-hand-side columns live
// in the caller's array ``rhs_t`` of P x ldN doubles (filled here from R).
int fs_gs_apply_f64_with(System& s, const double* R, double* Z, double* rhs_t, cudaStream_t st);

// Multigrid (k_mg.cu): the level hierarchy and dense coarsest inverse (setup), and the grid
// transfers: restriction (transpose of bilinear interpolation, zero on coarse boundary nodes)
// and prolongation added into the fine iterate.
int mg_setup_levels(System& s, cudaStream_t st);
// Grouped field split (k_bilu.cu): the splits of fg_rule as field ranges; the assembly and ILU(0)
// of every split's diagonal block; one application D = P^{-1} R of Eq. P_group.
std::vector<std::pair<int, int>> fg_split_ranges(int M, int p, int rule);
int fg_setup(System& s, cudaStream_t st);
template <typename T>
int fg_apply(System& s, const T* R, T* D, cudaStream_t st, const int* done);
template <typename T>
int launch_restrict(const T* rf, T* bc, int nc, int P, cudaStream_t st, const int* done,
                    Timer* timer);
template <typename T>
int launch_prolong_add(const T* uc, T* uf, int nc, int P, cudaStream_t st, const int* done,
                       Timer* timer);
template <typename T>
int launch_coarse_solve(const System& c, const T* b, T* u, cudaStream_t st, const int* done);
void free_system_public(System* s);
int setup_system_public(System& s, cudaStream_t st, bool krylov);

// Row-tiled operator (k_apply_tile.cu)
int plan_tile_op(const System& s, int kappa, int elem, size_t smem_max, TilePlan& plan, int ctas);
int build_tile_op(System& s, TileOp& op, int kappa, int elem, size_t smem_max, cudaStream_t st,
                  int ctas);
int verify_tile_plan(const System& s, const TilePlan& plan);
// Host-only setup pieces used by the planner entry point: the mesh pattern, the chaos index sets
// and the triple products of a parameter set.
int host_tables(System& s);
void free_tile_op(TileOp& op);
template <typename T>
int launch_tile_op(const System& s, const TileOp& op, const T* X, T* Y, T alpha, const T* B,
                   T beta, cudaStream_t st, const int* done);

// Krylov launchers (k_krylov.cu)
int k_norm(System& s, size_t n, const double* r, double* out, cudaStream_t st);
// *flag != 0 afterwards iff x[0..n) is all zero (the flag then skips kernels given it as done).
int k_zero_flag(System& s, size_t n, const double* x, int* flag, cudaStream_t st);
int k_init_cycle(System& s, size_t n, const double* r, cudaStream_t st);
int k_arnoldi(System& s, size_t n, int j, int last_col, cudaStream_t st);
int k_finish_cycle(System& s, size_t n, double* x, bool z32, cudaStream_t st);
int k_to_f32(size_t n, const double* src, float* dst, const int* flags, cudaStream_t st);
int k_to_f64(size_t n, const float* src, double* dst, const int* flags, cudaStream_t st);
int krylov_red_blocks();
int krylov_max_basis();

}  // namespace sg
