// Stand-alone measurement program, not part of libsip: FP64 FMA throughput of
// the GPU against the number of active lanes per warp.  Every thread of a warp
// whose lane index is below `active` runs 8 independent FMA chains; the others
// return at once.  Build and run:
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o /tmp/fp64_lanes_probe \
//        paper_2504_03573_gb300/probes/fp64_lanes_probe.cu && /tmp/fp64_lanes_probe
#include <cstdio>

#include <cuda_runtime.h>

__global__ void chains(double* out, int iters, int active) {
  const int lane = threadIdx.x & 31;
  if (lane >= active) return;
  double a0 = threadIdx.x * 1e-3, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3, a4 = a0 + 4, a5 = a0 + 5, a6 = a0 + 6,
         a7 = a0 + 7;
  const double b = 0.9999999, c = 1e-9;
  for (int i = 0; i < iters; ++i) {
    a0 = fma(a0, b, c); a1 = fma(a1, b, c); a2 = fma(a2, b, c); a3 = fma(a3, b, c);
    a4 = fma(a4, b, c); a5 = fma(a5, b, c); a6 = fma(a6, b, c); a7 = fma(a7, b, c);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
}

int main() {
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, 0);
  const int blocks = nsm * 8, threads = 256, iters = 4096, reps = 5;
  double* out = nullptr;
  if (cudaMalloc(&out, sizeof(double) * blocks * threads) != cudaSuccess) return 1;
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  for (int active : {32, 24, 16, 8, 4, 1}) {
    chains<<<blocks, threads>>>(out, iters, active);
    cudaEventRecord(a);
    for (int r = 0; r < reps; ++r) chains<<<blocks, threads>>>(out, iters, active);
    cudaEventRecord(b);
    cudaEventSynchronize(b);
    float ms = 0;
    cudaEventElapsedTime(&ms, a, b);
    const double warp_fma = (double)blocks * threads / 32 * iters * 8 * reps;
    printf("active lanes %2d: warp DFMA/s %.3e, thread DFMA/s %.3e (%.3f TFLOP/s)\n", active, warp_fma / (ms / 1e3),
           warp_fma * active / (ms / 1e3), 2e-12 * warp_fma * active / (ms / 1e3));
  }
  const cudaError_t e = cudaGetLastError();
  printf("%s\n", cudaGetErrorString(e));
  cudaFree(out);
  return e == cudaSuccess ? 0 : 1;
}
