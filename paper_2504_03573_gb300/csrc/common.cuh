// Definitions shared by the apply and auxiliary kernels: kernel arguments,
// the 1D tables in __constant__ memory, line-per-thread contractions used by
// the auxiliary kernels, face geometry helpers.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>
#include <utility>

#include "sip_internal.h"

namespace sip {

template <typename T>
struct ApplyArgs {
  const int64_t* dof_off;
  const int64_t* vgoff;
  const T* vgeo;
  const int64_t* quad_off;
  const T* kappa;          // nullptr: kappa = 1
  const FaceSlot* slots;
  const int64_t* f_troff;
  const int64_t* f_goff;
  const T* f_tau;
  const T* fgeo;
  const int32_t* elist;
  const Tile* tiles;
  const int32_t* cta_off;  // CTA b runs tiles cta_off[b] .. cta_off[b+1]-1 (one order)
  const uint16_t* flists;  // face lists of the tiles (Tile::flist)
  const int8_t* eaff;      // per element: 1 if its volume geometry is stored as constants
  const ElemDesc* desc_e;  // per position of the order-sorted element list
  const SlotDesc* desc_s;  // [position][2 dim]
  const T* x;
  T* y;
  T* trace;
  T* ug;                   // FP64: Gauss-point values from the trace kernel, [nrhs][nquad]
  int64_t ndof;            // per-RHS stride of x and y
  int64_t nquad;           // per-RHS stride of ug
  int64_t trace_stride;    // per-RHS stride of the trace buffer
  T lambda;
  int transpose;
  // SIP_FACES_P2P: Lagrange interpolation between Gauss rules, the matrix from the
  // f-point to the t-point rule at p2p_I + (f (kQMax+1) + t) kQMax^2, entry
  // [z][r] = l^G_{f,r}(xi^G_{t,z}) at z kQMax + r; nullptr with a shared rule
  const T* p2p_I;
  // single-launch apply (k_apply): grid barrier words {arrived, generation,
  // status}; the status word is set when a wait gives up
  unsigned int* gbar;
  // the rule's 1D tables and weights in global memory (source of the per-CTA copy)
  const T* gtab;
  const T* ggw;
};

constexpr int ipow(int b, int e) { return e == 0 ? 1 : b * ipow(b, e - 1); }

// single-launch applies that the device refused as too large for one
// cooperative launch and that ran as the two kernels instead (this thread)
extern thread_local int g_fused_fallbacks;

// The point rule of this translation unit's tables and kernels (volume and face
// points, P + 2 per direction): Gauss-Legendre unless the unit defines
// SIP_TU_RULE before including this header.  With Gauss-Lobatto-Legendre points
// the boundary points of the volume rule are the face points: traces are
// gathered and fluxes scattered back (GathrInterp / ScatrInterp, Sec. 3.2).
#ifndef SIP_TU_RULE
#define SIP_TU_RULE SIP_RULE_GAUSS
#endif
constexpr int kTuRule = SIP_TU_RULE;
constexpr bool kGatherScatter = kTuRule == SIP_RULE_GLL;

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialisation (launch_dependent below) may start while the kernel before it
// in the stream is still running.  Everything a kernel does before
// grid_dep_wait() reads only data that no kernel writes (tables, the mesh's
// face slots and tile lists); the wait returns once the previous kernel has
// completed and its writes are visible.  Without the launch attribute it
// returns at once.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
// lets the next kernel in the stream (launched with the attribute) start its
// CTAs, which then wait in grid_dep_wait() for this kernel to complete
__device__ __forceinline__ void grid_dep_launch_next() { asm volatile("griddepcontrol.launch_dependents;" :::); }

// Launch with programmatic stream serialisation when pdl.
template <typename... P, typename... A>
inline cudaError_t launch_dependent(void (*kern)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, bool pdl,
                                    A&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, std::forward<A>(args)...);
}

// ---- constant tables; each translation unit that includes this header holds
// its own copy, uploaded by sip_upload_tables_<tu>() at handle creation.
static __constant__ double c_tab_d[kTabSize];
static __constant__ float c_tab_f[kTabSize];
static __constant__ int c_ioff[kQMax + 1][kQMax + 1];
static __constant__ double c_gw_d[kQMax + 1][kQMax];  // weights of the q-point rule
static __constant__ float c_gw_f[kQMax + 1][kQMax];

template <typename T>
__device__ __forceinline__ T cgw(int q, int z) {
  if constexpr (std::is_same<T, double>::value) return c_gw_d[q][z];
  else return c_gw_f[q][z];
}

template <typename T>
__device__ __forceinline__ T ctab(int i) {
  if constexpr (std::is_same<T, double>::value) return c_tab_d[i];
  else return c_tab_f[i];
}

// Contraction of a per-element 3-index array [E2][E1][E0] (E0 fastest) along
// axis AX with a 1D operator: out[.., k, ..] (+)= sum_j M[k][j] in[.., j, ..]
// (M = table at MOFF, [NOUT][NIN]; TR: M stored [NIN][NOUT], i.e. M^T applied).
template <typename T, int E0, int E1, int E2, int AX, int NOUT, int MOFF, bool TR, bool ACC>
__device__ __forceinline__ void contract(const T* __restrict__ in, T* __restrict__ out, int stride, int ne) {
  constexpr int NIN = AX == 0 ? E0 : (AX == 1 ? E1 : E2);
  constexpr int O0 = AX == 0 ? NOUT : E0;
  constexpr int O1 = AX == 1 ? NOUT : E1;
  constexpr int SI = AX == 0 ? 1 : (AX == 1 ? E0 : E0 * E1);
  constexpr int SO = AX == 0 ? 1 : (AX == 1 ? O0 : O0 * O1);
  constexpr int LA = AX == 0 ? E1 : E0;
  constexpr int LB = AX == 2 ? E1 : E2;
  constexpr int LINES = LA * LB;
  for (int w = threadIdx.x; w < ne * LINES; w += blockDim.x) {
    const int el = w / LINES;
    const int l = w - el * LINES;
    const int la = l % LA, lb = l / LA;
    int bi, bo;
    if (AX == 0) { bi = la * E0 + lb * E0 * E1; bo = la * O0 + lb * O0 * O1; }
    else if (AX == 1) { bi = la + lb * E0 * E1; bo = la + lb * O0 * O1; }
    else { bi = la + lb * E0; bo = la + lb * O0; }
    const T* src = in + el * stride + bi;
    T* dst = out + el * stride + bo;
    T v[NIN];
#pragma unroll
    for (int j = 0; j < NIN; ++j) v[j] = src[j * SI];
#pragma unroll
    for (int k = 0; k < NOUT; ++k) {
      T acc = ACC ? dst[k * SO] : T(0);
#pragma unroll
      for (int j = 0; j < NIN; ++j)
        acc = fma(ctab<T>(MOFF + (TR ? j * NOUT + k : k * NIN + j)), v[j], acc);
      dst[k * SO] = acc;
    }
  }
}

// GLL coefficients -> Gauss values.  in: buffers bA (holding N^DIM coefficients),
// scratch bB; returns pointer (bA or bB) holding Q^DIM values.
template <typename T, int DIM, int N, int Q>
__device__ __forceinline__ T* to_gauss(T* bA, T* bB, int stride, int ne) {
  if constexpr (DIM == 2) {
    contract<T, N, N, 1, 0, Q, tab_B(N, Q), false, false>(bA, bB, stride, ne);
    __syncthreads();
    contract<T, Q, N, 1, 1, Q, tab_B(N, Q), false, false>(bB, bA, stride, ne);
    __syncthreads();
    return bA;
  } else {
    contract<T, N, N, N, 0, Q, tab_B(N, Q), false, false>(bA, bB, stride, ne);
    __syncthreads();
    contract<T, Q, N, N, 1, Q, tab_B(N, Q), false, false>(bB, bA, stride, ne);
    __syncthreads();
    contract<T, Q, Q, N, 2, Q, tab_B(N, Q), false, false>(bA, bB, stride, ne);
    __syncthreads();
    return bB;
  }
}

template <int DIM, int A>
struct Tang {  // tangential axes of the faces normal to axis A
  static constexpr int t0 = DIM == 2 ? (A == 0 ? 1 : 0) : (A == 0 ? 1 : 0);
  static constexpr int t1 = DIM == 2 ? -1 : (A == 2 ? 1 : 2);
};

// plus side: own tangential index -> canonical face index
__device__ __forceinline__ int canon(int dim, int side, int code, int qf, int j0, int j1) {
  if (side == 0) return j0 + qf * j1;
  if (dim == 2) return (code & 1) ? qf - 1 - j0 : j0;
  const int a = (code & 1) ? qf - 1 - j0 : j0;
  const int b = (code & 2) ? qf - 1 - j1 : j1;
  return (code & 4) ? b + qf * a : a + qf * b;
}


}  // namespace sip
