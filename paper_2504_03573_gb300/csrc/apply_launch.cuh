// Launch wrapper instantiated once per (point rule, dimension, precision)
// translation unit; the unit defines SIP_TU_RULE (default Gauss-Legendre) before
// including this header.
#pragma once
#include <cuda_runtime.h>

#include "apply_kernels.cuh"
#include "aux_kernels.cuh"


#define SIP_DEFINE_APPLY_TU(SUFFIX, TYPE, DIM)                                                     \
  namespace sip {                                                                                 \
  cudaError_t upload_tables_##SUFFIX(const double* tab_d, const float* tab_f, const int* ioff,     \
                                     const double* gw_d, const float* gw_f) {                     \
    cudaError_t e = cudaMemcpyToSymbol(c_tab_d, tab_d, sizeof(double) * kTabSize);                 \
    if (e != cudaSuccess) return e;                                                               \
    e = cudaMemcpyToSymbol(c_tab_f, tab_f, sizeof(float) * kTabSize);                             \
    if (e != cudaSuccess) return e;                                                               \
    e = cudaMemcpyToSymbol(c_gw_d, gw_d, sizeof(double) * (kQMax + 1) * kQMax);                   \
    if (e != cudaSuccess) return e;                                                               \
    e = cudaMemcpyToSymbol(c_gw_f, gw_f, sizeof(float) * (kQMax + 1) * kQMax);                    \
    if (e != cudaSuccess) return e;                                                               \
    return cudaMemcpyToSymbol(c_ioff, ioff, sizeof(int) * (kQMax + 1) * (kQMax + 1));             \
  }                                                                                               \
  cudaError_t prepare_##SUFFIX() {                                                                 \
    cudaError_t e = cudaSuccess;                                                                  \
    for (auto fn : {k_trace<TYPE, DIM, false, kTuRule>, k_trace<TYPE, DIM, true, kTuRule>,          \
                    k_main<TYPE, DIM, false, kTuRule>, k_main<TYPE, DIM, true, kTuRule>,            \
                    k_apply<TYPE, DIM, false, kTuRule>, k_apply<TYPE, DIM, true, kTuRule>})        \
      if (e == cudaSuccess)                                                                       \
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);    \
    return e;                                                                                     \
  }                                                                                               \
  cudaError_t occupancy_##SUFFIX(int threads, size_t smem_trace, size_t smem_main, int* blocks) { \
    int bt = 0, bm = 0;                                                                           \
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bt, k_trace<TYPE, DIM, false, kTuRule>,   \
                                                                  threads, smem_trace);           \
    if (e != cudaSuccess) return e;                                                               \
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bm, k_main<TYPE, DIM, false, kTuRule>, threads,      \
                                                      smem_main);                                 \
    *blocks = bt < bm ? bt : bm;                                                                  \
    return e;                                                                                     \
  }                                                                                               \
  /* resident CTAs per SM of the single-launch kernel (both phases' shared memory) */             \
  cudaError_t occupancy_fused_##SUFFIX(int threads, size_t smem, int* blocks) {                   \
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k_apply<TYPE, DIM, false, kTuRule>, \
                                                         threads, smem);                          \
  }                                                                                               \
  cudaError_t launch_apply_##SUFFIX(const ApplyArgs<TYPE>& a, int nctas, int nrhs, int threads,   \
                                    size_t smem_trace, size_t smem_main, cudaStream_t s,          \
                                    cudaEvent_t ev0, cudaEvent_t ev1, cudaEvent_t ev2, bool fused) { \
    if (nctas == 0) return cudaSuccess;                                                           \
    dim3 grid(nctas, nrhs);                                                                       \
    if (fused) {                                                                                  \
      /* one cooperative launch: every CTA resident, so the grid barrier completes */            \
      if (ev0) cudaEventRecord(ev0, s);                                                           \
      if (ev1) cudaEventRecord(ev1, s);                                                           \
      cudaLaunchConfig_t cfg = {};                                                                \
      cfg.gridDim = grid;                                                                         \
      cfg.blockDim = dim3(threads);                                                               \
      cfg.dynamicSmemBytes = smem_trace > smem_main ? smem_trace : smem_main;                     \
      cfg.stream = s;                                                                             \
      cudaLaunchAttribute attr[1];                                                                \
      attr[0].id = cudaLaunchAttributeCooperative;                                                \
      attr[0].val.cooperative = 1;                                                                \
      cfg.attrs = attr;                                                                           \
      cfg.numAttrs = 1;                                                                           \
      cudaError_t e = cudaLaunchKernelEx(&cfg, a.p2p_I ? k_apply<TYPE, DIM, true, kTuRule>        \
                                                       : k_apply<TYPE, DIM, false, kTuRule>, a);  \
      if (e == cudaErrorCooperativeLaunchTooLarge) {                                              \
        /* the device will not hold every CTA at once: run the two kernels */                     \
        cudaGetLastError();                                                                       \
        ++g_fused_fallbacks;                                                                      \
      } else {                                                                                    \
        if (e != cudaSuccess) return e;                                                           \
        if (ev2) cudaEventRecord(ev2, s);                                                         \
        return cudaGetLastError();                                                                \
      }                                                                                           \
    }                                                                                             \
    /* programmatic dependent launch, except when events time each kernel */                      \
    const bool pdl = ev0 == nullptr;                                                              \
    if (ev0) cudaEventRecord(ev0, s);                                                             \
    cudaError_t e = launch_dependent(a.p2p_I ? k_trace<TYPE, DIM, true, kTuRule> : k_trace<TYPE, DIM, false, kTuRule>, \
                                     grid, dim3(threads), smem_trace, s, pdl, a);                 \
    if (e != cudaSuccess) return e;                                                               \
    if (ev1) cudaEventRecord(ev1, s);                                                             \
    e = launch_dependent(a.p2p_I ? k_main<TYPE, DIM, true, kTuRule> : k_main<TYPE, DIM, false, kTuRule>, grid, \
                         dim3(threads), smem_main, s, pdl, a);                                    \
    if (e != cudaSuccess) return e;                                                               \
    if (ev2) cudaEventRecord(ev2, s);                                                             \
    return cudaGetLastError();                                                                    \
  }                                                                                               \
  }

#define SIP_DEFINE_AUX_TU(SUFFIX, DIM)                                                           \
  namespace sip {                                                                                \
  cudaError_t prepare_aux_##SUFFIX() {                                                           \
    return cudaFuncSetAttribute(k_aux<DIM, kTuRule>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                200 * 1024);                                                     \
  }                                                                                              \
  cudaError_t launch_aux_##SUFFIX(const AuxArgs& a, int ntiles, size_t smem, cudaStream_t s) {   \
    if (ntiles == 0) return cudaSuccess;                                                         \
    k_aux<DIM, kTuRule><<<ntiles, 256, smem, s>>>(a);                                            \
    return cudaGetLastError();                                                                   \
  }                                                                                              \
  }
