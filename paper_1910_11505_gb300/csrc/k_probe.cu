// Arithmetic peak probe: dependent-chain-free FMA throughput of the device in FP64 and FP32, the
// denominator of the ALU rooflines (the FP64 SG operator is bound by FP64 FMA issue on this GPU).
// Every thread runs kChains independent FMA chains for ``iters`` steps; the result is written so
// the work cannot be removed.
#include "sg_internal.h"

namespace sg {

namespace {

constexpr int kChains = 8;

template <typename T>
__global__ void __launch_bounds__(256) fma_probe_kernel(int iters, T seed, T* out) {
  T v[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) v[c] = seed + T(threadIdx.x + c);
  const T a = T(0.999999), b = T(1e-7);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = fma(v[c], a, b);
  }
  T s = T(0);
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += v[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
int run_probe(double* gflops) {
  int dev = 0, sms = 0;
  SG_CUDA(cudaGetDevice(&dev));
  SG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = sms * 8, threads = 256;
  const int iters = sizeof(T) == 8 ? 2048 : 65536;
  DBuf<T> out;
  SG_TRY(out.alloc((size_t)blocks * threads));
  cudaEvent_t a, b;
  SG_CUDA(cudaEventCreate(&a));
  SG_CUDA(cudaEventCreate(&b));
  fma_probe_kernel<T><<<blocks, threads>>>(iters, T(1), out.p);  // warm-up
  SG_TRY(check_launch("fma_probe"));
  SG_CUDA(cudaEventRecord(a));
  fma_probe_kernel<T><<<blocks, threads>>>(iters, T(1), out.p);
  SG_TRY(check_launch("fma_probe"));
  SG_CUDA(cudaEventRecord(b));
  SG_CUDA(cudaEventSynchronize(b));
  float ms = 0.f;
  SG_CUDA(cudaEventElapsedTime(&ms, a, b));
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  out.release();
  *gflops = 2.0 * kChains * (double)iters * blocks * threads / (ms * 1e-3) / 1e9;
  return SG_OK;
}

}  // namespace

}  // namespace sg

extern "C" int sg_probe_fma(int precision, double* gflops) {
  if (!gflops) return sg::fail(SG_ERR_ARG, "gflops is NULL");
  return precision == SG_FP64 ? sg::run_probe<double>(gflops) : sg::run_probe<float>(gflops);
}
