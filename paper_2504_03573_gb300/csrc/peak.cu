// Arithmetic peak of this GPU's FP64 or FP32 units, measured: independent FMA
// chains in every thread of as many CTAs as fit on the device, timed with CUDA
// events.  The apply's roofline takes its FP64 denominator from here, so that
// the fraction it reports is of a rate this part actually reaches.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "handle.h"

namespace {

constexpr int kChains = 8;     // independent FMA chains per thread
constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_chains(T a, T b, int iters, T* sink) {
  T c[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) c[k] = (T)(threadIdx.x + k) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) c[k] = fma(c[k], a, b);
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += c[k];
  // a, b are chosen so that s stays finite; the store keeps the chains alive
  if (s == (T)-12345.0) sink[blockIdx.x] = s;
}

template <typename T>
int measure(int iters, cudaStream_t s, double* tflops) {
  int dev = 0, nsm = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_chains<T>, kThreads, 0);
  if (e != cudaSuccess) return sip::cuda_fail(e, "sip_fp_peak: device query");
  const int grid = nsm * std::max(1, per_sm);
  T* sink = nullptr;
  e = cudaMalloc((void**)&sink, sizeof(T) * grid);
  if (e != cudaSuccess) return sip::cuda_fail(e, "sip_fp_peak: buffer");
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  e = cudaEventCreate(&ev0);
  if (e == cudaSuccess) e = cudaEventCreate(&ev1);
  const T a = (T)0.999999, b = (T)1e-6;
  float best = 0.0f;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {  // the first launch warms up
    e = cudaEventRecord(ev0, s);
    k_fma_chains<T><<<grid, kThreads, 0, s>>>(a, b, iters, sink);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(ev1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev0, ev1);
    if (e == cudaSuccess && rep > 0 && (best == 0.0f || ms < best)) best = ms;
  }
  if (ev0) cudaEventDestroy(ev0);
  if (ev1) cudaEventDestroy(ev1);
  cudaFree(sink);
  if (e != cudaSuccess) return sip::cuda_fail(e, "sip_fp_peak");
  const double flops = 2.0 * kChains * (double)iters * kThreads * grid;
  *tflops = flops / (best * 1e-3) / 1e12;
  return SIP_OK;
}

}  // namespace

extern "C" int sip_fp_peak(int precision, int iters, void* stream, double* tflops_out) {
  if (!tflops_out) return sip::fail(SIP_ERR_ARG, "null output");
  if (iters < 1) return sip::fail(SIP_ERR_ARG, "iters must be >= 1");
  if (precision == SIP_FP64) return measure<double>(iters, (cudaStream_t)stream, tflops_out);
  if (precision == SIP_FP32) return measure<float>(iters, (cudaStream_t)stream, tflops_out);
  return sip::fail(SIP_ERR_ARG, "precision");
}
