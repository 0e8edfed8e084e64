// Output layer of the learned warm start, and the back-propagation through it into the hidden
// layer, on the 5th-generation tensor cores (tcgen05).
//
// Y = H2 W3^T + b3 for a batch: H2 is B x h2 (h2 <= 64, FP32, rounded to BF16 here), W3 is
// out x h2 (the network's BF16 copy), Y is B x out.  One CTA of 128 threads computes a 128 x 128
// tile of Y (128 batch rows x 128 output units) as one tcgen05.mma.kind::f16 chain over K = 64
// (four K = 16 steps), BF16 operands from shared memory, FP32 accumulator in tensor memory
// (TMEM, 128 lanes x 128 columns).  The epilogue reads the accumulator back with tcgen05.ld (warp w
// owns TMEM lanes 32w .. 32w + 31, i.e. batch rows), turns each 32 x 32 piece over in shared
// memory so global rows are accessed 128 bytes at a time, and either writes Y + b3 (forward) or forms
// the residual against the targets T: dY = 2 (Y + b3 - T) / (B out), stored in BF16 for the
// back-propagation below, and the CTA's share of the sum of squares (training with a fixed
// output layer).
//
// Operand layout in shared memory: the canonical K-major layout without swizzle.  A tile of R
// rows x 64 K (BF16) is cut into core matrices of 8 rows x 16 bytes (8 K values), each 128
// contiguous bytes; core matrix (row group g, K chunk c) sits at byte (8 g + c) * 128.  So the
// matrix descriptor's leading byte offset (next core matrix along K) is 128 and its stride byte
// offset (next 8-row group) is 1024; the K = 16 step kk starts 256 kk bytes in.
//
// Every wait is bounded: if the MMA completion does not arrive within kWaitLimit polls the CTA
// raises the error word, waits (bounded again) and still frees its TMEM columns.
#include <cuda_bf16.h>

#include <algorithm>

#include "sg_internal.h"

namespace sg {
namespace {

constexpr int kTcRows = 128;           // batch rows per CTA (MMA M)
constexpr int kTcUnits = 128;          // output units per CTA (MMA N)
constexpr int kTcK = 64;               // K (h2 padded with zeros)
constexpr int kTcTileBytes = kTcRows * kTcK * 2;  // 16 KB per operand tile
// Dynamic shared memory requested per CTA: the two tiles plus room that keeps at most four CTAs
// on an SM, so their TMEM columns (128 each) never exceed the SM's 512.
constexpr int kTcSmem = 56 * 1024;
constexpr unsigned kTcCols = 128;

__device__ __forceinline__ unsigned long long tc_smem_desc(unsigned saddr) {
  const unsigned long long start = (saddr & 0x3FFFFu) >> 4;  // bits 0-13
  const unsigned long long lbo = 128u >> 4;                   // bits 16-29
  const unsigned long long sbo = 1024u >> 4;                  // bits 32-45
  return start | (lbo << 16) | (sbo << 32) | (1ull << 46);    // version 1; no swizzle
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both K-major, M = 128,
// N = 128.
constexpr unsigned kTcIdesc = (1u << 4)            // D format: F32
                              | (1u << 7)          // A format: BF16
                              | (1u << 10)         // B format: BF16
                              | ((kTcUnits >> 3) << 17)   // N >> 3
                              | ((kTcRows >> 4) << 24);   // M >> 4

// Byte offset of element (row, k) in the canonical layout above.
__device__ __forceinline__ int tc_off(int row, int k) {
  return (((row >> 3) * 8 + (k >> 3)) << 7) + ((row & 7) << 4) + ((k & 7) << 1);
}

template <int MODE, typename TY>
__global__ void __launch_bounds__(128) tc_out_kernel(int B, int h2, int out,
                                                     const float* __restrict__ H2,
                                                     const __nv_bfloat16* __restrict__ W3h,
                                                     const float* __restrict__ b3,
                                                     TY* __restrict__ Y, const float* __restrict__ T,
                                                     __nv_bfloat16* __restrict__ dYh, int outp,
                                                     float* __restrict__ lpart,
                                                     int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* At = smem_raw;                     // H2 rows
  unsigned char* Bt = smem_raw + kTcTileBytes;      // W3 rows
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem_raw + 2 * kTcTileBytes);
  unsigned* tslot = reinterpret_cast<unsigned*>(smem_raw + 2 * kTcTileBytes + 16);
  float* red = reinterpret_cast<float*>(smem_raw + 2 * kTcTileBytes + 32);
  float* stage = reinterpret_cast<float*>(smem_raw + 2 * kTcTileBytes + 64);  // 4 x 32 x 33
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int j0 = blockIdx.x * kTcUnits, b0 = blockIdx.y * kTcRows;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_u32(tslot)),
                 "r"(kTcCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  // operand tiles: 8 K values (16 bytes) per item; rows and K beyond the data are zero.  With
  // h2 = 64 a row is 16-byte aligned in both arrays and is read by vector loads.
  const bool full = h2 == kTcK;
  for (int it = tid; it < kTcRows * (kTcK / 8); it += blockDim.x) {
    const int row = it >> 3, kc = (it & 7) * 8;
    __align__(16) __nv_bfloat16 a[8], w[8];
    const int b = b0 + row, j = j0 + row;
    if (full) {
      float4 h0 = make_float4(0.f, 0.f, 0.f, 0.f), h1 = h0;
      if (b < B) {
        h0 = *reinterpret_cast<const float4*>(H2 + (size_t)b * kTcK + kc);
        h1 = *reinterpret_cast<const float4*>(H2 + (size_t)b * kTcK + kc + 4);
      }
      a[0] = __float2bfloat16_rn(h0.x); a[1] = __float2bfloat16_rn(h0.y);
      a[2] = __float2bfloat16_rn(h0.z); a[3] = __float2bfloat16_rn(h0.w);
      a[4] = __float2bfloat16_rn(h1.x); a[5] = __float2bfloat16_rn(h1.y);
      a[6] = __float2bfloat16_rn(h1.z); a[7] = __float2bfloat16_rn(h1.w);
      const uint4 wv = j < out ? *reinterpret_cast<const uint4*>(W3h + (size_t)j * kTcK + kc)
                               : make_uint4(0u, 0u, 0u, 0u);
      *reinterpret_cast<uint4*>(w) = wv;
    } else {
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const int k = kc + t;
        a[t] = __float2bfloat16_rn(b < B && k < h2 ? H2[(size_t)b * h2 + k] : 0.0f);
        w[t] = j < out && k < h2 ? W3h[(size_t)j * h2 + k] : __float2bfloat16_rn(0.0f);
      }
    }
    *reinterpret_cast<uint4*>(At + tc_off(row, kc)) = *reinterpret_cast<const uint4*>(a);
    *reinterpret_cast<uint4*>(Bt + tc_off(row, kc)) = *reinterpret_cast<const uint4*>(w);
  }
  // the tiles were written by ordinary stores: make them visible to the tensor core's proxy
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const unsigned tmem = *tslot;

  if (tid == 0) {
    const unsigned a0 = smem_u32(At), bb0 = smem_u32(Bt);
#pragma unroll
    for (int kk = 0; kk < kTcK / 16; ++kk) {
      const unsigned long long da = tc_smem_desc(a0 + 256u * kk);
      const unsigned long long db = tc_smem_desc(bb0 + 256u * kk);
      asm volatile(
          "{\n\t.reg .pred p;\n\t"
          "setp.ne.b32 p, %4, 0;\n\t"
          "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
          "l"(da), "l"(db), "r"(kTcIdesc), "r"(kk)
          : "memory");
    }
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
            smem_u32(bar))
        : "memory");
  }
  // warp-uniform: tcgen05.ld below is a .sync.aligned warp instruction
  const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(bar, 0));
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");

  float lsum = 0.0f;
  if (ok) {
    // each warp reads its 32 rows x 32 columns at a time (thread = row), turns them over in its
    // own shared-memory stage (padded rows), and writes / reads the global arrays a row at a time
    // with the lanes along the units (128-byte accesses)
    float* S = stage + warp * 32 * 33;
    const float scale = 2.0f / ((float)B * (float)out);
#pragma unroll 1
    for (int c0 = 0; c0 < kTcUnits; c0 += 32) {
      unsigned v[32];
      const unsigned taddr = tmem + ((unsigned)(warp * 32) << 16) + (unsigned)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
          "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
            "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
            "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]),
            "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
            "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]),
            "=r"(v[31])
          : "r"(taddr)
          : "memory");
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
      for (int t = 0; t < 32; ++t) S[lane * 33 + t] = __uint_as_float(v[t]);
      __syncwarp();
      const int j = j0 + c0 + lane;
      const float bias = j < out ? b3[j] : 0.0f;
#pragma unroll 4
      for (int r = 0; r < 32; ++r) {
        const int b = b0 + warp * 32 + r;
        if (b >= B) continue;
        if (j >= out) {  // the K padding of the back-propagation's dY rows
          if (MODE == 1 && j < outp) dYh[(size_t)b * outp + j] = __float2bfloat16_rn(0.0f);
          continue;
        }
        const float y = S[r * 33 + lane] + bias;
        const size_t o = (size_t)b * out + j;
        if (MODE == 0) {
          Y[o] = (TY)y;
        } else {
          const float res = y - T[o];
          dYh[(size_t)b * outp + j] = __float2bfloat16_rn(scale * res);
          lsum = fmaf(res, res, lsum);
        }
      }
      __syncwarp();
    }
  } else if (lane == 0) {
    atomicExch(err, 1);
    mbar_wait_bounded(bar, 0);  // let the MMAs finish (bounded) before the columns are freed
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  if (MODE == 1) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if (lane == 0) red[warp] = lsum;
  }
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                 "r"(kTcCols)
                 : "memory");
  }
  if (MODE == 1 && tid == 0)
    lpart[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = (red[0] + red[1]) + (red[2] + red[3]);
}

// Back-propagation into the hidden layer, dH2 = dY W3, on the tensor cores: split-K over the
// output units.  CTA (s, y) takes batch rows 128 y .. 128 y + 127 and the K stages (64 units each)
// s, s + S, ...; per stage the BF16 tiles dYh[rows][64 units] (A, M = 128) and W3hT[64 k][64 units]
// (B, N = 64) are copied into one of two shared-memory buffers in the canonical K-major layout
// while the MMAs of the previous stage run; four K = 16 MMAs accumulate into 64 TMEM columns;
// a buffer is refilled only after the commit of the stage that last read it has arrived.  The
// CTA's partial sum goes to part[s][row][k] (FP32); a fixed-order kernel sums the splits.
constexpr int kTcKs = 64;                          // units per K stage
constexpr int kTcBTileBytes = 64 * kTcKs * 2;      // 8 KB: W3hT tile
constexpr int kTcStageBytes = kTcTileBytes + kTcBTileBytes;
constexpr int kTcDh2Smem = 2 * kTcStageBytes + 64;
constexpr unsigned kTcDh2Cols = 64;
constexpr unsigned kTcDh2Idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((64u >> 3) << 17) |
                                 ((128u >> 4) << 24);

__global__ void __launch_bounds__(128) tc_dh2_kernel(int B, int outp, int nstages,
                                                     const __nv_bfloat16* __restrict__ dYh,
                                                     const __nv_bfloat16* __restrict__ W3hT,
                                                     float* __restrict__ part, size_t part_stride,
                                                     int ldp, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem_raw + 2 * kTcStageBytes);
  unsigned* tslot = reinterpret_cast<unsigned*>(smem_raw + 2 * kTcStageBytes + 16);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int b0 = blockIdx.y * kTcRows, S = gridDim.x;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_u32(tslot)),
                 "r"(kTcDh2Cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const unsigned tmem = *tslot;
  bool failed = false;
  int n = 0;  // stages of this CTA
  for (int st = blockIdx.x; st < nstages; st += S, ++n) {
    const int buf = n & 1;
    if (n >= 2) {  // the MMAs of stage n - 2 read this buffer
      const bool ok = mbar_wait_bounded(&bar[buf], (unsigned)(((n - 2) >> 1) & 1));
      if (__syncthreads_or(!ok)) {
        failed = true;
        break;
      }
    }
    unsigned char* At = smem_raw + buf * kTcStageBytes;
    unsigned char* Bt = At + kTcTileBytes;
    const size_t j0 = (size_t)st * kTcKs;
    for (int it = tid; it < kTcRows * 8; it += blockDim.x) {  // A: 128 rows x 8 chunks
      const int row = it >> 3, kc = (it & 7) * 8;
      const int b = b0 + row;
      const uint4 v = b < B ? *reinterpret_cast<const uint4*>(dYh + (size_t)b * outp + j0 + kc)
                            : make_uint4(0u, 0u, 0u, 0u);
      *reinterpret_cast<uint4*>(At + tc_off(row, kc)) = v;
    }
    for (int it = tid; it < 64 * 8; it += blockDim.x) {  // B: 64 hidden units x 8 chunks
      const int row = it >> 3, kc = (it & 7) * 8;
      *reinterpret_cast<uint4*>(Bt + tc_off(row, kc)) =
          *reinterpret_cast<const uint4*>(W3hT + (size_t)row * outp + j0 + kc);
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const unsigned a0 = smem_u32(At), bb0 = smem_u32(Bt);
#pragma unroll
      for (int kk = 0; kk < kTcKs / 16; ++kk) {
        const unsigned long long da = tc_smem_desc(a0 + 256u * kk);
        const unsigned long long db = tc_smem_desc(bb0 + 256u * kk);
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
            "l"(da), "l"(db), "r"(kTcDh2Idesc), "r"(n > 0 || kk > 0 ? 1 : 0)
            : "memory");
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
              smem_u32(&bar[buf]))
          : "memory");
    }
  }
  // the last commit covers every MMA this CTA issued
  bool ok = true;
  if (n > 0) ok = mbar_wait_bounded(&bar[(n - 1) & 1], (unsigned)(((n - 1) >> 1) & 1));
  ok = __all_sync(0xffffffffu, ok) && !failed;
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const int b = b0 + warp * 32 + lane;
  float* o = part + (size_t)blockIdx.x * part_stride + (size_t)b * ldp;
  if (ok && n > 0) {
#pragma unroll 1
    for (int c0 = 0; c0 < 64; c0 += 32) {
      unsigned v[32];
      const unsigned taddr = tmem + ((unsigned)(warp * 32) << 16) + (unsigned)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
          "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
            "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
            "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]),
            "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
            "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]),
            "=r"(v[31])
          : "r"(taddr)
          : "memory");
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
      if (b < B) {
#pragma unroll
        for (int t = 0; t < 32; ++t) o[c0 + t] = __uint_as_float(v[t]);
      }
    }
  } else {
    if (b < B)
      for (int t = 0; t < 64; ++t) o[t] = 0.0f;
    if (!ok && lane == 0) {
      atomicExch(err, 1);
      if (n > 0) mbar_wait_bounded(&bar[(n - 1) & 1], (unsigned)(((n - 1) >> 1) & 1));
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                 "r"(kTcDh2Cols)
                 : "memory");
  }
}

// W3hT[k][j] = BF16(W3[j][k]) for k < h2 and j < out, zero elsewhere (64 x outp).
__global__ void w3t_bf16_kernel(int out, int outp, int h2, const float* __restrict__ W3,
                                __nv_bfloat16* __restrict__ W3hT) {
  const size_t total = (size_t)64 * outp;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(t / outp);
    const int j = (int)(t - (size_t)k * outp);
    W3hT[t] = __float2bfloat16_rn(k < h2 && j < out ? W3[(size_t)j * h2 + k] : 0.0f);
  }
}

}  // namespace

// Launch of the tensor-core output layer (see the file comment).  mode 0: Y (float Yf or double
// Yd) = H2 W3^T + b3; mode 1: dY in BF16 (dYh, row stride outp, zero beyond out) and one loss
// partial per CTA in lpart (*nparts of them).
int launch_out_tc(int mode, int B, int h2, int out, const float* H2, const __nv_bfloat16* W3h,
                  const float* b3, float* Yf, double* Yd, const float* T, __nv_bfloat16* dYh,
                  int outp, float* lpart, int* err, cudaStream_t st, int* nparts) {
  if (h2 < 1 || h2 > kTcK || B < 1 || out < 1) return fail(SG_ERR_ARG, "tensor-core output layer: sizes");
  const dim3 grid((out + kTcUnits - 1) / kTcUnits, (B + kTcRows - 1) / kTcRows);
  if (nparts) *nparts = (int)(grid.x * grid.y);
  if (mode == 0 && Yd != nullptr) {
    auto k = tc_out_kernel<0, double>;
    SG_TRY(ensure_smem((const void*)k, kTcSmem));
    k<<<grid, 128, kTcSmem, st>>>(B, h2, out, H2, W3h, b3, Yd, nullptr, nullptr, 0, nullptr, err);
  } else if (mode == 0) {
    auto k = tc_out_kernel<0, float>;
    SG_TRY(ensure_smem((const void*)k, kTcSmem));
    k<<<grid, 128, kTcSmem, st>>>(B, h2, out, H2, W3h, b3, Yf, nullptr, nullptr, 0, nullptr, err);
  } else {
    if (outp % kTcKs || outp < out || outp > (int)grid.x * kTcUnits)
      return fail(SG_ERR_ARG, "tensor-core output layer: padded width");
    auto k = tc_out_kernel<1, float>;
    SG_TRY(ensure_smem((const void*)k, kTcSmem));
    k<<<grid, 128, kTcSmem, st>>>(B, h2, out, H2, W3h, b3, nullptr, T, dYh, outp, lpart, err);
  }
  return check_launch("tc_out");
}

// dH2 partial sums on the tensor cores (see tc_dh2_kernel): part[s][row][k] for s < *nsplit,
// rows of stride ldp, splits of stride part_stride floats; at most max_split splits.
int launch_dh2_tc(int B, int outp, const __nv_bfloat16* dYh, const __nv_bfloat16* W3hT,
                  float* part, size_t part_stride, int ldp, int max_split, int* err,
                  cudaStream_t st, int* nsplit) {
  if (B < 1 || outp < kTcKs || outp % kTcKs || ldp < 64) return fail(SG_ERR_ARG, "tensor-core dH2: sizes");
  const int nstages = outp / kTcKs;
  const int S = std::max(1, std::min(max_split, nstages));
  *nsplit = S;
  SG_TRY(ensure_smem((const void*)tc_dh2_kernel, kTcDh2Smem));
  tc_dh2_kernel<<<dim3(S, (B + kTcRows - 1) / kTcRows), 128, kTcDh2Smem, st>>>(
      B, outp, nstages, dYh, W3hT, part, part_stride, ldp, err);
  return check_launch("tc_dh2");
}

int launch_w3t_bf16(int out, int outp, int h2, const float* W3, __nv_bfloat16* W3hT,
                    cudaStream_t st) {
  w3t_bf16_kernel<<<608, 256, 0, st>>>(out, outp, h2, W3, W3hT);
  return check_launch("w3t_bf16");
}

}  // namespace sg
