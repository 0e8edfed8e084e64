// The learned warm-start network (include/sgnet.h): forward, mean-squared-error gradient and
// Adam, all in hand-written kernels.  The output layer (h2 -> D = N*P, almost all parameters)
// runs one thread per output unit j: the unit's weight row stays in registers while the batch's
// hidden activations stream through shared memory; its weight gradient accumulates in registers
// over the batch.  The back-propagation into the hidden layer is a split-K product over D with a
// deterministic second-stage sum.  Small layers run one CTA per sample.  No atomics: results do
// not depend on scheduling.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "sg_internal.h"
#include "../../include/sgnet.h"

namespace sg {
namespace {

constexpr int kMaxIn = 16, kMaxH1 = 128, kMaxH2 = 64, kMaxBatch = 1024;
constexpr int kOutThreads = 128;   // output units per CTA
constexpr int kBChunk = 128;       // batch rows staged per pass (kBChunk * kMaxH2 floats)
constexpr int kSplit = 152;        // CTAs of the split-K hidden-layer back-propagation
constexpr int kJT = 32;            // output units per split-K step

__global__ void small_fwd_kernel(int in, int h1, int h2, const float* __restrict__ Z,
                                 const float* __restrict__ mu, const float* __restrict__ sd,
                                 const float* __restrict__ P, int oW1, int ob1, int oW2, int ob2,
                                 float* __restrict__ Zh, float* __restrict__ H1,
                                 float* __restrict__ H2) {
  __shared__ float zs[kMaxIn], a1[kMaxH1];
  const int b = blockIdx.x, t = threadIdx.x;
  if (t < in) {
    float v = (Z[(size_t)b * in + t] - mu[t]) / sd[t];
    zs[t] = v;
    Zh[(size_t)b * in + t] = v;
  }
  __syncthreads();
  if (t < h1) {
    float s = P[ob1 + t];
    for (int i = 0; i < in; ++i) s = fmaf(P[oW1 + t * in + i], zs[i], s);
    float v = tanhf(s);
    a1[t] = v;
    H1[(size_t)b * h1 + t] = v;
  }
  __syncthreads();
  if (t < h2) {
    float s = P[ob2 + t];
    for (int i = 0; i < h1; ++i) s = fmaf(P[oW2 + t * h1 + i], a1[i], s);
    H2[(size_t)b * h2 + t] = tanhf(s);
  }
}

__device__ __forceinline__ float w3_at(const float* W3f, const __nv_bfloat16* W3h, size_t i) {
  return W3h != nullptr ? __bfloat162float(W3h[i]) : W3f[i];
}

// MODE 0: Y = W3 h2 + b3 (FP32 or FP64 output).  MODE 1: residual against T, dY, loss partial,
// and the gradient of W3 and b3.
template <int MODE, typename TY>
__global__ void __launch_bounds__(kOutThreads) out_kernel(
    int B, int h2, int out, const float* __restrict__ H2, const float* __restrict__ W3f,
    const __nv_bfloat16* __restrict__ W3h, const float* __restrict__ b3, TY* __restrict__ Y,
    const float* __restrict__ T, float* __restrict__ dY, float* __restrict__ gW3,
    float* __restrict__ gb3, float* __restrict__ loss_part) {
  __shared__ float hs[kBChunk * kMaxH2];
  __shared__ float red[kOutThreads / 32];
  const int j = blockIdx.x * kOutThreads + threadIdx.x;
  const bool act = j < out;
  float w[kMaxH2], g[kMaxH2];
#pragma unroll
  for (int k = 0; k < kMaxH2; ++k) {
    w[k] = (act && k < h2) ? w3_at(W3f, W3h, (size_t)j * h2 + k) : 0.f;
    g[k] = 0.f;
  }
  const float bias = act ? b3[j] : 0.f;
  const float scale = 2.f / ((float)B * (float)out);
  float gb = 0.f, lsum = 0.f;
  for (int b0 = 0; b0 < B; b0 += kBChunk) {
    const int nb = min(kBChunk, B - b0);
    __syncthreads();
    for (int t = threadIdx.x; t < nb * kMaxH2; t += blockDim.x) {
      int bb = t / kMaxH2, k = t - bb * kMaxH2;
      hs[t] = k < h2 ? H2[(size_t)(b0 + bb) * h2 + k] : 0.f;
    }
    __syncthreads();
    if (!act) continue;
    for (int bb = 0; bb < nb; ++bb) {
      const float* hr = hs + bb * kMaxH2;
      float y = bias;
#pragma unroll
      for (int k = 0; k < kMaxH2; ++k) y = fmaf(w[k], hr[k], y);
      const size_t o = (size_t)(b0 + bb) * out + j;
      if (MODE == 0) {
        Y[o] = (TY)y;
      } else {
        float r = y - T[o];
        float d = scale * r;
        dY[o] = d;
        lsum = fmaf(r, r, lsum);
        gb += d;
#pragma unroll
        for (int k = 0; k < kMaxH2; ++k) g[k] = fmaf(d, hr[k], g[k]);
      }
    }
  }
  if (MODE == 1) {
    if (act) {
      for (int k = 0; k < h2; ++k) gW3[(size_t)j * h2 + k] = g[k];
      gb3[j] = gb;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = lsum;
    __syncthreads();
    if (threadIdx.x == 0) {
      float s = 0.f;
      for (int i = 0; i < kOutThreads / 32; ++i) s += red[i];
      loss_part[blockIdx.x] = s;
    }
  }
}

// Sum of the per-CTA loss partials, divided by B*out: one CTA of 256 threads, strided FP64 sums
// and a fixed tree (the order does not depend on scheduling).
__global__ void __launch_bounds__(256) loss_final_kernel(int n, const float* __restrict__ part,
                                                         float denom, float* __restrict__ loss) {
  __shared__ double red[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += part[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *loss = (float)(red[0] / denom);
}

// Split-K partial of dH2 = dY W3 over the output units of this CTA; part[cta][b][k] for the
// 64-row batch slice blockIdx.y.  Each thread owns a 4 x 4 tile of (b, k).
__global__ void __launch_bounds__(256) dh2_partial_kernel(
    int B, int h2, int out, const float* __restrict__ dY, const float* __restrict__ W3f,
    const __nv_bfloat16* __restrict__ W3h, float* __restrict__ part) {
  __shared__ float ds[64][kJT + 1];
  __shared__ float ws[kJT][kMaxH2 + 1];
  const int b0 = blockIdx.y * 64;
  const int tb = threadIdx.x / 16, tk = threadIdx.x % 16;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[i][q] = 0.f;
  const int ntiles = (out + kJT - 1) / kJT;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int j0 = tile * kJT;
    __syncthreads();
    for (int t = threadIdx.x; t < 64 * kJT; t += blockDim.x) {
      int bb = t / kJT, jj = t - bb * kJT;
      int b = b0 + bb, j = j0 + jj;
      ds[bb][jj] = (b < B && j < out) ? dY[(size_t)b * out + j] : 0.f;
    }
    for (int t = threadIdx.x; t < kJT * kMaxH2; t += blockDim.x) {
      int jj = t / kMaxH2, k = t - jj * kMaxH2;
      int j = j0 + jj;
      ws[jj][k] = (j < out && k < h2) ? w3_at(W3f, W3h, (size_t)j * h2 + k) : 0.f;
    }
    __syncthreads();
#pragma unroll 4
    for (int jj = 0; jj < kJT; ++jj) {
      float a[4], c[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = ds[tb * 4 + i][jj];
#pragma unroll
      for (int q = 0; q < 4; ++q) c[q] = ws[jj][tk * 4 + q];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[i][q] = fmaf(a[i], c[q], acc[i][q]);
    }
  }
  float* o = part + (size_t)blockIdx.x * kMaxBatch * kMaxH2;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int b = b0 + tb * 4 + i, k = tk * 4 + q;
      if (b < B) o[(size_t)b * kMaxH2 + k] = acc[i][q];
    }
}

__global__ void dh2_final_kernel(int B, int h2, int nsplit, const float* __restrict__ part,
                                 float* __restrict__ dH2) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= B * h2) return;
  int b = t / h2, k = t - b * h2;
  float s = 0.f;
  for (int c = 0; c < nsplit; ++c) s += part[(size_t)c * kMaxBatch * kMaxH2 + (size_t)b * kMaxH2 + k];
  dH2[t] = s;
}

// Per sample: dA2 = dH2 * (1 - h2^2), dH1 = W2^T dA2, dA1 = dH1 * (1 - h1^2).
__global__ void small_bwd_kernel(int h1, int h2, const float* __restrict__ P, int oW2,
                                 const float* __restrict__ dH2, const float* __restrict__ H1,
                                 const float* __restrict__ H2, float* __restrict__ dA2,
                                 float* __restrict__ dA1) {
  __shared__ float a2[kMaxH2];
  const int b = blockIdx.x, t = threadIdx.x;
  if (t < h2) {
    float hv = H2[(size_t)b * h2 + t];
    float v = dH2[(size_t)b * h2 + t] * (1.f - hv * hv);
    a2[t] = v;
    dA2[(size_t)b * h2 + t] = v;
  }
  __syncthreads();
  if (t < h1) {
    float s = 0.f;
    for (int q = 0; q < h2; ++q) s = fmaf(P[oW2 + q * h1 + t], a2[q], s);
    float hv = H1[(size_t)b * h1 + t];
    dA1[(size_t)b * h1 + t] = s * (1.f - hv * hv);
  }
}

// Gradients of the small layers: gW2 = dA2^T H1, gb2, gW1 = dA1^T Zh, gb1 (sums over the batch).
__global__ void small_wgrad_kernel(int B, int in, int h1, int h2, const float* __restrict__ Zh,
                                   const float* __restrict__ H1, const float* __restrict__ dA1,
                                   const float* __restrict__ dA2, float* __restrict__ G, int oW1,
                                   int ob1, int oW2, int ob2) {
  const int nW2 = h2 * h1, nW1 = h1 * in;
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  float s = 0.f;
  if (t < nW2) {
    int q = t / h1, i = t - q * h1;
    for (int b = 0; b < B; ++b) s = fmaf(dA2[(size_t)b * h2 + q], H1[(size_t)b * h1 + i], s);
    G[oW2 + t] = s;
  } else if ((t -= nW2) < h2) {
    for (int b = 0; b < B; ++b) s += dA2[(size_t)b * h2 + t];
    G[ob2 + t] = s;
  } else if ((t -= h2) < nW1) {
    int q = t / in, i = t - q * in;
    for (int b = 0; b < B; ++b) s = fmaf(dA1[(size_t)b * h1 + q], Zh[(size_t)b * in + i], s);
    G[oW1 + t] = s;
  } else if ((t -= nW1) < h1) {
    for (int b = 0; b < B; ++b) s += dA1[(size_t)b * h1 + t];
    G[ob1 + t] = s;
  }
}

// Adam with bias correction: c1 = 1 - beta1^t, c2 = 1 - beta2^t.
__global__ void adam_kernel(size_t n, float* __restrict__ p, const float* __restrict__ g,
                            float* __restrict__ m, float* __restrict__ v, float lr, float c1,
                            float c2) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    float gi = g[i];
    float mi = 0.9f * m[i] + 0.1f * gi;
    float vi = 0.999f * v[i] + 0.001f * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
  }
}

__global__ void to_bf16_kernel(size_t n, const float* __restrict__ s, __nv_bfloat16* __restrict__ d) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    d[i] = __float2bfloat16(s[i]);
}

// Feature mean / standard deviation (one CTA, one thread per feature) and the output mean.
__global__ void in_stats_kernel(int n, int in, const float* __restrict__ Z, float* __restrict__ mu,
                                float* __restrict__ sd) {
  int i = threadIdx.x;
  if (i >= in) return;
  double s = 0.0, s2 = 0.0;
  for (int r = 0; r < n; ++r) s += Z[(size_t)r * in + i];
  double m = s / n;
  for (int r = 0; r < n; ++r) {
    double d = Z[(size_t)r * in + i] - m;
    s2 += d * d;
  }
  mu[i] = (float)m;
  sd[i] = (float)fmax(sqrt(s2 / n), 1e-6);
}
__global__ void out_mean_kernel(int n, int out, const float* __restrict__ T, float* __restrict__ b3) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= out) return;
  float s = 0.f;
  for (int r = 0; r < n; ++r) s += T[(size_t)r * out + j];
  b3[j] = s / n;
}

// ---- output basis from the training targets (sgnet_set_basis)
// V[j] = T[j] - b3 for the first nb training rows (j-major, D entries each).
__global__ void center_rows_kernel(int nb, int out, const float* __restrict__ T,
                                   const float* __restrict__ b3, float* __restrict__ V) {
  const size_t total = (size_t)nb * out;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x)
    V[i] = T[i] - b3[i % out];
}

// d[i] = V[i] . V[j] for i < ni (one CTA per i, FP64 accumulation, fixed-order tree).
__global__ void basis_dots_kernel(int out, const float* __restrict__ V, int j, double* __restrict__ d) {
  __shared__ double red[256];
  const int i = blockIdx.x;
  const float* a = V + (size_t)i * out;
  const float* b = V + (size_t)j * out;
  double s = 0.0;
  for (int u = threadIdx.x; u < out; u += blockDim.x) s += (double)a[u] * (double)b[u];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) d[i] = red[0];
}

// V[j] -= sum_{i<j} d[i] V[i]   (one classical Gram-Schmidt pass)
__global__ void basis_update_kernel(int out, float* __restrict__ V, int j, const double* __restrict__ d) {
  for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < out; u += gridDim.x * blockDim.x) {
    double v = V[(size_t)j * out + u];
    for (int i = 0; i < j; ++i) v -= d[i] * (double)V[(size_t)i * out + u];
    V[(size_t)j * out + u] = (float)v;
  }
}

// V[j] /= ||V[j]|| (d[j] holds the squared norm); a vector that vanished becomes 0
__global__ void basis_scale_kernel(int out, float* __restrict__ V, int j, const double* __restrict__ d) {
  const double nrm = sqrt(d[j]);
  const float f = nrm > 1e-30 ? (float)(1.0 / nrm) : 0.f;
  for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < out; u += gridDim.x * blockDim.x)
    V[(size_t)j * out + u] *= f;
}

// c[r, j] = Q[j] . (T[r] - b3) for every training row r (one CTA per (r, j), FP64 accumulation)
__global__ void basis_coef_kernel(int rows, int nb, int out, const float* __restrict__ Q,
                                  const float* __restrict__ T, const float* __restrict__ b3,
                                  double* __restrict__ c) {
  __shared__ double red[256];
  const int r = blockIdx.x, j = blockIdx.y;
  const float* q = Q + (size_t)j * out;
  const float* t = T + (size_t)r * out;
  double s = 0.0;
  for (int u = threadIdx.x; u < out; u += blockDim.x) s += (double)q[u] * ((double)t[u] - (double)b3[u]);
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) c[(size_t)r * nb + j] = red[0];
}

// W3[u, j] = Q[j, u] * s_j with s_j = max_r |c[r, j]| / 0.9 (the hidden layer's tanh then reaches
// every training coefficient), columns beyond nb zero
__global__ void basis_w3_kernel(int rows, int nb, int h2, int out, const float* __restrict__ Q,
                                const double* __restrict__ c, float* __restrict__ W3) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < (size_t)out * h2;
       i += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(i % h2);
    const size_t u = i / h2;
    float v = 0.f;
    if (j < nb) {
      double mx = 0.0;
      for (int r = 0; r < rows; ++r) mx = fmax(mx, fabs(c[(size_t)r * nb + j]));
      v = Q[(size_t)j * out + u] * (float)(mx / 0.9);
    }
    W3[i] = v;
  }
}

}  // namespace
}  // namespace sg

struct sgnet {
  int in = 0, h1 = 0, h2 = 0, out = 0, maxb = 0, bf16 = 0;
  int oW1 = 0, ob1 = 0, oW2 = 0, ob2 = 0, oW3 = 0, ob3 = 0;
  long long np = 0, step = 0;
  int frozen_out = 0;        // 1: Adam leaves the output layer (W3, b3) as set_basis left it
  sg::DBuf<float> P, G, M, V, mu, sd, Zh, H1, H2, dY, dH2, dA2, dA1, part, lpart, loss, Ytmp;
  sg::DBuf<__nv_bfloat16> W3h;
  // tensor-core back-propagation: W3 transposed (64 x outp) and dY (max batch x outp) in BF16,
  // outp = out rounded up to a multiple of 64
  int outp = 0;
  sg::DBuf<__nv_bfloat16> W3hT, dYh;
  sg::DBuf<int> err;         // raised by a tensor-core kernel whose MMA completion timed out
};

using namespace sg;

static int net_release(sgnet* n) {
  DBuf<float>* bs[] = {&n->P, &n->G, &n->M, &n->V, &n->mu, &n->sd, &n->Zh, &n->H1, &n->H2,
                       &n->dY, &n->dH2, &n->dA2, &n->dA1, &n->part, &n->lpart, &n->loss, &n->Ytmp};
  for (auto* b : bs) b->release();
  n->W3h.release();
  n->W3hT.release();
  n->dYh.release();
  n->err.release();
  return SG_OK;
}

// The output layer runs on the tensor cores (k_net_tc.cu) when its weights have a BF16 copy.
static bool use_tc(const sgnet* n) { return n->bf16 && n->h2 <= kMaxH2; }

static int check_net_err(sgnet* n, cudaStream_t st) {
  int e = 0;
  SG_CUDA(cudaMemcpyAsync(&e, n->err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  SG_CUDA(cudaStreamSynchronize(st));
  if (e) return fail(SG_ERR_CUDA, "tensor-core output layer: MMA completion wait timed out");
  return SG_OK;
}

static int refresh_bf16(sgnet* n, cudaStream_t st) {
  if (!n->bf16) return SG_OK;
  to_bf16_kernel<<<608, 256, 0, st>>>((size_t)n->out * n->h2, n->P.p + n->oW3, n->W3h.p);
  SG_TRY(check_launch("to_bf16"));
  if (n->W3hT.p) SG_TRY(launch_w3t_bf16(n->out, n->outp, n->h2, n->P.p + n->oW3, n->W3hT.p, st));
  return SG_OK;
}

static const __nv_bfloat16* w3h(const sgnet* n) { return n->bf16 ? n->W3h.p : nullptr; }

static int forward_hidden(sgnet* n, const float* Z, int B, cudaStream_t st) {
  small_fwd_kernel<<<B, 128, 0, st>>>(n->in, n->h1, n->h2, Z, n->mu.p, n->sd.p, n->P.p, n->oW1,
                                      n->ob1, n->oW2, n->ob2, n->Zh.p, n->H1.p, n->H2.p);
  return check_launch("small_fwd");
}

static int check_batch(const sgnet* n, int B) {
  if (!n || B < 1 || B > n->maxb) return fail(SG_ERR_ARG, "batch size out of range");
  return SG_OK;
}

extern "C" {

int sgnet_create(int in_dim, int h1, int h2, int out_dim, int max_batch, int bf16,
                 unsigned long long seed, sgnet** out) {
  if (!out) return fail(SG_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (in_dim < 1 || in_dim > kMaxIn || h1 < 1 || h1 > kMaxH1 || h2 < 1 || h2 > kMaxH2 ||
      out_dim < 1 || max_batch < 1 || max_batch > kMaxBatch)
    return fail(SG_ERR_ARG, "sgnet_create: need in <= 16, h1 <= 128, h2 <= 64, batch <= 1024");
  sgnet* n = new sgnet();
  n->in = in_dim;
  n->h1 = h1;
  n->h2 = h2;
  n->out = out_dim;
  n->maxb = max_batch;
  n->bf16 = bf16 ? 1 : 0;
  n->oW1 = 0;
  n->ob1 = n->oW1 + h1 * in_dim;
  n->oW2 = n->ob1 + h1;
  n->ob2 = n->oW2 + h2 * h1;
  n->oW3 = n->ob2 + h2;
  n->ob3 = n->oW3 + out_dim * h2;
  n->np = (long long)n->ob3 + out_dim;
  // Glorot-uniform weights from splitmix64, zero biases
  std::vector<float> p((size_t)n->np, 0.f);
  unsigned long long s = seed;
  auto uni = [&]() {
    s += 0x9E3779B97F4A7C15ull;
    unsigned long long z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);
  };
  auto fill = [&](int off, int rows, int cols) {
    double lim = std::sqrt(6.0 / (rows + cols));
    for (long long i = 0; i < (long long)rows * cols; ++i) p[off + i] = (float)((2.0 * uni() - 1.0) * lim);
  };
  fill(n->oW1, h1, in_dim);
  fill(n->oW2, h2, h1);
  fill(n->oW3, out_dim, h2);
  const size_t B = (size_t)max_batch;
  int rc = SG_OK;
  auto A = [&](DBuf<float>& b, size_t c) {
    if (rc == SG_OK) rc = b.alloc(c);
  };
  A(n->P, n->np); A(n->G, n->np); A(n->M, n->np); A(n->V, n->np);
  A(n->mu, in_dim); A(n->sd, in_dim);
  A(n->Zh, B * in_dim); A(n->H1, B * h1); A(n->H2, B * h2); A(n->dY, B * out_dim);
  A(n->dH2, B * h2); A(n->dA2, B * h2); A(n->dA1, B * h1);
  A(n->part, (size_t)kSplit * kMaxBatch * kMaxH2);
  // loss partials: one per CTA of the SIMT output kernel, or per 128 x 128 tile of the
  // tensor-core one
  A(n->lpart, (size_t)(out_dim + kOutThreads - 1) / kOutThreads * ((B + 127) / 128));
  A(n->loss, 1);
  if (rc == SG_OK && n->bf16) rc = n->W3h.alloc((size_t)out_dim * h2);
  if (rc == SG_OK && n->bf16 && h2 <= kMaxH2) {
    n->outp = (out_dim + 63) / 64 * 64;
    rc = n->W3hT.alloc((size_t)64 * n->outp);
    if (rc == SG_OK) rc = n->dYh.alloc(B * n->outp);
  }
  if (rc == SG_OK) rc = n->err.alloc(1);
  if (rc == SG_OK && cudaMemset(n->err.p, 0, sizeof(int)) != cudaSuccess)
    rc = fail(SG_ERR_CUDA, "cudaMemset of the error word failed");
  if (rc != SG_OK) {
    net_release(n);
    delete n;
    return rc;
  }
  cudaStream_t st = nullptr;
  std::vector<float> one(in_dim, 1.f), zero(in_dim, 0.f);
  if ((rc = n->P.upload(p, st)) || (rc = n->mu.upload(zero, st)) || (rc = n->sd.upload(one, st))) {
    net_release(n);
    delete n;
    return rc;
  }
  cudaMemset(n->M.p, 0, sizeof(float) * n->np);
  cudaMemset(n->V.p, 0, sizeof(float) * n->np);
  cudaMemset(n->G.p, 0, sizeof(float) * n->np);
  if ((rc = refresh_bf16(n, st)) != SG_OK) {
    net_release(n);
    delete n;
    return rc;
  }
  if (cudaDeviceSynchronize() != cudaSuccess) {
    net_release(n);
    delete n;
    return fail(SG_ERR_CUDA, "sgnet_create: device error");
  }
  *out = n;
  return SG_OK;
}

int sgnet_set_stats(sgnet* n, const float* Z, const float* T, int rows, void* stream) {
  if (!n || !Z || !T || rows < 1) return fail(SG_ERR_ARG, "bad arguments");
  cudaStream_t st = (cudaStream_t)stream;
  in_stats_kernel<<<1, 32, 0, st>>>(rows, n->in, Z, n->mu.p, n->sd.p);
  SG_TRY(check_launch("in_stats"));
  out_mean_kernel<<<(n->out + 255) / 256, 256, 0, st>>>(rows, n->out, T, n->P.p + n->ob3);
  return check_launch("out_mean");
}

int sgnet_set_basis(sgnet* n, const float* T, int rows, void* stream) {
  if (!n || !T || rows < 1) return fail(SG_ERR_ARG, "bad arguments");
  cudaStream_t st = (cudaStream_t)stream;
  const int nb = std::min(rows, n->h2);
  DBuf<float> Q;
  DBuf<double> d, c;
  SG_TRY(Q.alloc((size_t)nb * n->out));
  SG_TRY(d.alloc(n->h2));
  SG_TRY(c.alloc((size_t)rows * nb));
  const int g = std::min(608, (n->out + 255) / 256);
  center_rows_kernel<<<608, 256, 0, st>>>(nb, n->out, T, n->P.p + n->ob3, Q.p);
  SG_TRY(check_launch("center_rows"));
  for (int j = 0; j < nb; ++j) {
    for (int pass = 0; pass < 2 && j > 0; ++pass) {  // CGS2
      basis_dots_kernel<<<j, 256, 0, st>>>(n->out, Q.p, j, d.p);
      SG_TRY(check_launch("basis_dots"));
      basis_update_kernel<<<g, 256, 0, st>>>(n->out, Q.p, j, d.p);
      SG_TRY(check_launch("basis_update"));
    }
    basis_dots_kernel<<<1, 256, 0, st>>>(n->out, Q.p + (size_t)j * n->out, 0, d.p + j);
    SG_TRY(check_launch("basis_norm"));
    basis_scale_kernel<<<g, 256, 0, st>>>(n->out, Q.p, j, d.p);
    SG_TRY(check_launch("basis_scale"));
  }
  basis_coef_kernel<<<dim3(rows, nb), 256, 0, st>>>(rows, nb, n->out, Q.p, T, n->P.p + n->ob3, c.p);
  SG_TRY(check_launch("basis_coef"));
  basis_w3_kernel<<<608, 256, 0, st>>>(rows, nb, n->h2, n->out, Q.p, c.p, n->P.p + n->oW3);
  SG_TRY(check_launch("basis_w3"));
  SG_TRY(refresh_bf16(n, st));
  SG_CUDA(cudaStreamSynchronize(st));
  Q.release();
  d.release();
  c.release();
  n->frozen_out = 1;
  return SG_OK;
}

int sgnet_forward(sgnet* n, const float* Z, int B, float* Y, void* stream) {
  SG_TRY(check_batch(n, B));
  if (!Z || !Y) return fail(SG_ERR_ARG, "NULL pointer");
  cudaStream_t st = (cudaStream_t)stream;
  SG_TRY(forward_hidden(n, Z, B, st));
  if (use_tc(n))
    return launch_out_tc(0, B, n->h2, n->out, n->H2.p, n->W3h.p, n->P.p + n->ob3, Y, nullptr,
                         nullptr, nullptr, 0, nullptr, n->err.p, st, nullptr);
  out_kernel<0, float><<<(n->out + kOutThreads - 1) / kOutThreads, kOutThreads, 0, st>>>(
      B, n->h2, n->out, n->H2.p, n->P.p + n->oW3, w3h(n), n->P.p + n->ob3, Y, nullptr, nullptr,
      nullptr, nullptr, nullptr);
  return check_launch("out_fwd");
}

int sgnet_predict(sgnet* n, const float* Z, int B, double* X, void* stream) {
  SG_TRY(check_batch(n, B));
  if (!Z || !X) return fail(SG_ERR_ARG, "NULL pointer");
  cudaStream_t st = (cudaStream_t)stream;
  SG_TRY(forward_hidden(n, Z, B, st));
  if (use_tc(n))
    return launch_out_tc(0, B, n->h2, n->out, n->H2.p, n->W3h.p, n->P.p + n->ob3, nullptr, X,
                         nullptr, nullptr, 0, nullptr, n->err.p, st, nullptr);
  out_kernel<0, double><<<(n->out + kOutThreads - 1) / kOutThreads, kOutThreads, 0, st>>>(
      B, n->h2, n->out, n->H2.p, n->P.p + n->oW3, w3h(n), n->P.p + n->ob3, X, nullptr, nullptr,
      nullptr, nullptr, nullptr);
  return check_launch("out_predict");
}

int sgnet_loss_grad(sgnet* n, const float* Z, const float* T, int B, float* loss, void* stream) {
  SG_TRY(check_batch(n, B));
  if (!Z || !T) return fail(SG_ERR_ARG, "NULL pointer");
  cudaStream_t st = (cudaStream_t)stream;
  SG_TRY(forward_hidden(n, Z, B, st));
  int nblk = (n->out + kOutThreads - 1) / kOutThreads;
  const bool tc = use_tc(n) && n->frozen_out;
  if (tc) {
    // the output layer is fixed: only the residual gradient dY (BF16) and the loss are needed
    SG_TRY(launch_out_tc(1, B, n->h2, n->out, n->H2.p, n->W3h.p, n->P.p + n->ob3, nullptr,
                         nullptr, T, n->dYh.p, n->outp, n->lpart.p, n->err.p, st, &nblk));
  } else {
    out_kernel<1, float><<<nblk, kOutThreads, 0, st>>>(B, n->h2, n->out, n->H2.p,
                                                        n->P.p + n->oW3, w3h(n), n->P.p + n->ob3,
                                                        nullptr, T, n->dY.p, n->G.p + n->oW3,
                                                        n->G.p + n->ob3, n->lpart.p);
    SG_TRY(check_launch("out_grad"));
  }
  loss_final_kernel<<<1, 256, 0, st>>>(nblk, n->lpart.p, (float)B * (float)n->out, n->loss.p);
  SG_TRY(check_launch("loss_final"));
  int nsplit = kSplit;
  if (tc) {
    SG_TRY(launch_dh2_tc(B, n->outp, n->dYh.p, n->W3hT.p, n->part.p, (size_t)kMaxBatch * kMaxH2,
                         kMaxH2, kSplit, n->err.p, st, &nsplit));
  } else {
    dim3 g(kSplit, (B + 63) / 64);
    dh2_partial_kernel<<<g, 256, 0, st>>>(B, n->h2, n->out, n->dY.p, n->P.p + n->oW3, w3h(n),
                                          n->part.p);
    SG_TRY(check_launch("dh2_partial"));
  }
  dh2_final_kernel<<<(B * n->h2 + 255) / 256, 256, 0, st>>>(B, n->h2, nsplit, n->part.p, n->dH2.p);
  SG_TRY(check_launch("dh2_final"));
  small_bwd_kernel<<<B, 128, 0, st>>>(n->h1, n->h2, n->P.p, n->oW2, n->dH2.p, n->H1.p, n->H2.p,
                                      n->dA2.p, n->dA1.p);
  SG_TRY(check_launch("small_bwd"));
  int nsmall = n->h2 * n->h1 + n->h2 + n->h1 * n->in + n->h1;
  small_wgrad_kernel<<<(nsmall + 127) / 128, 128, 0, st>>>(B, n->in, n->h1, n->h2, n->Zh.p, n->H1.p,
                                                           n->dA1.p, n->dA2.p, n->G.p, n->oW1,
                                                           n->ob1, n->oW2, n->ob2);
  SG_TRY(check_launch("small_wgrad"));
  if (loss) {
    SG_CUDA(cudaMemcpyAsync(loss, n->loss.p, sizeof(float), cudaMemcpyDeviceToHost, st));
    SG_TRY(check_net_err(n, st));
  }
  return SG_OK;
}

int sgnet_adam_step(sgnet* n, float lr, void* stream) {
  if (!n) return fail(SG_ERR_ARG, "NULL network");
  cudaStream_t st = (cudaStream_t)stream;
  n->step += 1;
  float c1 = (float)(1.0 - std::pow(0.9, (double)n->step));
  float c2 = (float)(1.0 - std::pow(0.999, (double)n->step));
  const size_t nupd = n->frozen_out ? (size_t)n->oW3 : (size_t)n->np;  // W3, b3 come last
  adam_kernel<<<608, 256, 0, st>>>(nupd, n->P.p, n->G.p, n->M.p, n->V.p, lr, c1, c2);
  SG_TRY(check_launch("adam"));
  return refresh_bf16(n, st);
}

int sgnet_train_step(sgnet* n, const float* Z, const float* T, int B, float lr, float* loss,
                     void* stream) {
  SG_TRY(sgnet_loss_grad(n, Z, T, B, loss, stream));
  return sgnet_adam_step(n, lr, stream);
}

long long sgnet_num_params(const sgnet* n) { return n ? n->np : 0; }

int sgnet_get(const sgnet* n, int what, float* host, size_t count) {
  if (!n || !host) return fail(SG_ERR_ARG, "NULL argument");
  SG_CUDA(cudaDeviceSynchronize());
  if (what == 0 || what == 1) {
    if (count < (size_t)n->np) return fail(SG_ERR_ARG, "host buffer too small");
    SG_CUDA(cudaMemcpy(host, what == 0 ? n->P.p : n->G.p, sizeof(float) * n->np, cudaMemcpyDeviceToHost));
    return SG_OK;
  }
  if (what == 2) {
    if (count < (size_t)2 * n->in) return fail(SG_ERR_ARG, "host buffer too small");
    SG_CUDA(cudaMemcpy(host, n->mu.p, sizeof(float) * n->in, cudaMemcpyDeviceToHost));
    SG_CUDA(cudaMemcpy(host + n->in, n->sd.p, sizeof(float) * n->in, cudaMemcpyDeviceToHost));
    return SG_OK;
  }
  return fail(SG_ERR_ARG, "unknown selector");
}

int sgnet_set(sgnet* n, int what, const float* host, size_t count) {
  if (!n || !host) return fail(SG_ERR_ARG, "NULL argument");
  if (what == 0) {
    if (count != (size_t)n->np) return fail(SG_ERR_ARG, "parameter count mismatch");
    SG_CUDA(cudaMemcpy(n->P.p, host, sizeof(float) * n->np, cudaMemcpyHostToDevice));
    SG_TRY(refresh_bf16(n, nullptr));
    SG_CUDA(cudaDeviceSynchronize());
    return SG_OK;
  }
  if (what == 2) {
    if (count != (size_t)2 * n->in) return fail(SG_ERR_ARG, "expected mu and sd");
    SG_CUDA(cudaMemcpy(n->mu.p, host, sizeof(float) * n->in, cudaMemcpyHostToDevice));
    SG_CUDA(cudaMemcpy(n->sd.p, host + n->in, sizeof(float) * n->in, cudaMemcpyHostToDevice));
    return SG_OK;
  }
  return fail(SG_ERR_ARG, "unknown selector");
}

void sgnet_free(sgnet* n) {
  if (!n) return;
  cudaDeviceSynchronize();
  net_release(n);
  delete n;
}

}  // extern "C"
