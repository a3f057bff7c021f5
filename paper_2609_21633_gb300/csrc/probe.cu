// tn_probe_fma_peak: the fused multiply-add throughput of the current GPU, measured.
//
// The FP64 element kernels of the A, B and B^T applies are bound by the FP64 pipe, not by HBM,
// so their roofline denominator is the DFMA rate; the FP32 kernels' issue limit is the FFMA
// rate.  This kernel runs independent FMA chains (eight per thread, enough in flight to cover
// the pipe latency) on every SM and times them with CUDA events.
#include <algorithm>
#include <string>

#include "internal.h"

namespace tn {
namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;
constexpr int kBlocksPerSM = 8;

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_chains(int iters, T a, T b, T* sink) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == (T)-1.2345) sink[blockIdx.x] = s;  // never true for these inputs; keeps the chains live
}

template <typename T>
cudaError_t probe_t(cudaStream_t st, double* tflops) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int blocks = sms * kBlocksPerSM;
  const int iters = sizeof(T) == 8 ? 4096 : 65536;
  T* sink = nullptr;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  e = cudaMalloc(&sink, sizeof(T) * blocks);
  if (e == cudaSuccess) e = cudaEventCreate(&t0);
  if (e == cudaSuccess) e = cudaEventCreate(&t1);
  double best = 0;
  // x -> x a + b with a slightly below 1 stays bounded; one warm-up launch, then the best of three
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
    e = cudaEventRecord(t0, st);
    if (e == cudaSuccess) {
      k_fma_chains<T><<<blocks, kThreads, 0, st>>>(iters, (T)0.999999, (T)1e-3, sink);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(t1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(t1);
    float ms = 0;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
    if (e == cudaSuccess && rep > 0 && ms > 0) {
      const double flops = 2.0 * (double)iters * kChains * (double)blocks * kThreads;
      best = std::max(best, flops / (ms * 1e-3) / 1e12);
    }
  }
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  if (sink) cudaFree(sink);
  *tflops = best;
  return e;
}

}  // namespace
}  // namespace tn

using namespace tn;

extern "C" tn_status tn_probe_fma_peak(tn_prec prec, double* tflops, void* stream) {
  if (!tflops || (prec != TN_F64 && prec != TN_F32)) {
    set_error("tn_probe_fma_peak: bad arguments");
    return TN_EINVAL;
  }
  *tflops = 0;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = prec == TN_F64 ? probe_t<double>(st, tflops) : probe_t<float>(st, tflops);
  if (e != cudaSuccess) {
    set_error(std::string("tn_probe_fma_peak: ") + cudaGetErrorString(e));
    return TN_ECUDA;
  }
  return TN_OK;
}
