// Auxiliary per-element FP64 kernels: kappa gradient, mass inner product, IProduct.
#pragma once

#include "apply_kernels.cuh"

namespace sip {

// ============================================================ auxiliary element kernels (FP64)
// kappa gradient w|J| grad a . grad b, mass inner product a^T M b, IProduct,
// at the volume points of the translation unit's rule.
struct AuxArgs {
  const int64_t* dof_off;
  const int64_t* quad_off;
  const int64_t* vgoff;
  const double* vgeo;
  const int32_t* elist;
  const Tile* tiles;
  const int8_t* eaff;
  const double* a;
  const double* b;
  double* out;
  int accumulate;
  int mode;  // 0: kappa gradient, 1: mass dot partials (one per tile), 2: IProduct
};

inline int aux_smem_per_element(int dim, int n, int q) {
  (void)n;
  const int qv = dim == 2 ? q * q : q * q * q;
  return 2 * (dim + 1) * qv;
}

// load N^DIM coefficients of vector v into U (via scratch S) and interpolate to
// the Gauss points: result in U.
template <int DIM, int N, int Q>
__device__ __forceinline__ void load_to_gauss(const AuxArgs& a, const Tile& t, const double* v,
                                              double* U, double* S, int per) {
  constexpr int NV = ipow(N, DIM);
  double* dst = DIM == 2 ? U : S;
  for (int w = threadIdx.x; w < t.count * NV; w += blockDim.x) {
    const int el = w / NV, i = w - el * NV;
    const int e = a.elist[t.start + el];
    dst[el * per + i] = v[a.dof_off[e] + i];
  }
  __syncthreads();
  if constexpr (DIM == 2) to_gauss<double, 2, N, Q>(U, S, per, t.count);
  else to_gauss<double, 3, N, Q>(S, U, per, t.count);
}

template <int DIM, int Q>
__device__ __forceinline__ void gauss_grad(const double* U, double* G0, double* G1, double* G2, int per, int ne) {
  if constexpr (DIM == 2) {
    contract<double, Q, Q, 1, 0, Q, tab_D(Q), false, false>(U, G0, per, ne);
    contract<double, Q, Q, 1, 1, Q, tab_D(Q), false, false>(U, G1, per, ne);
  } else {
    contract<double, Q, Q, Q, 0, Q, tab_D(Q), false, false>(U, G0, per, ne);
    contract<double, Q, Q, Q, 1, Q, tab_D(Q), false, false>(U, G1, per, ne);
    contract<double, Q, Q, Q, 2, Q, tab_D(Q), false, false>(U, G2, per, ne);
  }
  __syncthreads();
}

// volume factor comp (0..nG-1) of element e at Gauss point q (affine elements
// store constants without the Gauss weight)
template <int DIM, int Q>
__device__ __forceinline__ double vfac(const AuxArgs& a, int e, int q, int comp) {
  constexpr int QV = ipow(Q, DIM);
  const double* g = a.vgeo + a.vgoff[e];
  if (!a.eaff[e]) return g[comp * QV + q];
  double w = c_gw_d[Q][q % Q] * c_gw_d[Q][(q / Q) % Q];
  if (DIM == 3) w *= c_gw_d[Q][q / (Q * Q)];
  return w * g[comp];
}

template <int DIM, int N, int Q>
__device__ void aux_tile(const AuxArgs& a, const Tile& t, double* sm) {
  constexpr int QV = ipow(Q, DIM), NV = ipow(N, DIM);
  constexpr int PER = 2 * (DIM + 1) * QV;
  const int ne = t.count;
  double* Ua = sm;
  double* Ga = sm + QV;                 // DIM buffers
  double* Ub = sm + (DIM + 1) * QV;
  double* Gb = sm + (DIM + 2) * QV;     // DIM buffers
  if (a.mode == 0) {
    load_to_gauss<DIM, N, Q>(a, t, a.a, Ua, Ga, PER);
    gauss_grad<DIM, Q>(Ua, Ga, Ga + QV, Ga + 2 * QV, PER, ne);
    load_to_gauss<DIM, N, Q>(a, t, a.b, Ub, Gb, PER);
    gauss_grad<DIM, Q>(Ub, Gb, Gb + QV, Gb + 2 * QV, PER, ne);
    for (int w = threadIdx.x; w < ne * QV; w += blockDim.x) {
      const int el = w / QV, q = w - el * QV;
      const int e = a.elist[t.start + el];
      const double* ga = Ga + el * PER + q;
      const double* gb = Gb + el * PER + q;
      double v;
      if constexpr (DIM == 2) {
        v = vfac<DIM, Q>(a, e, q, 0) * ga[0] * gb[0] + vfac<DIM, Q>(a, e, q, 1) * (ga[0] * gb[QV] + ga[QV] * gb[0]) +
            vfac<DIM, Q>(a, e, q, 2) * ga[QV] * gb[QV];
      } else {
        v = vfac<DIM, Q>(a, e, q, 0) * ga[0] * gb[0] + vfac<DIM, Q>(a, e, q, 3) * ga[QV] * gb[QV] +
            vfac<DIM, Q>(a, e, q, 5) * ga[2 * QV] * gb[2 * QV] +
            vfac<DIM, Q>(a, e, q, 1) * (ga[0] * gb[QV] + ga[QV] * gb[0]) +
            vfac<DIM, Q>(a, e, q, 2) * (ga[0] * gb[2 * QV] + ga[2 * QV] * gb[0]) +
            vfac<DIM, Q>(a, e, q, 4) * (ga[QV] * gb[2 * QV] + ga[2 * QV] * gb[QV]);
      }
      double* o = a.out + a.quad_off[e] + q;
      *o = a.accumulate ? *o + v : v;
    }
  } else if (a.mode == 1) {
    load_to_gauss<DIM, N, Q>(a, t, a.a, Ua, Ga, PER);
    load_to_gauss<DIM, N, Q>(a, t, a.b, Ub, Gb, PER);
    double s = 0.0;
    constexpr int WJ = DIM == 2 ? 3 : 6;
    for (int w = threadIdx.x; w < ne * QV; w += blockDim.x) {
      const int el = w / QV, q = w - el * QV;
      const int e = a.elist[t.start + el];
      s += vfac<DIM, Q>(a, e, q, WJ) * Ua[el * PER + q] * Ub[el * PER + q];
    }
    // fixed-order block reduction (deterministic)
    __syncthreads();
    double* red = sm + ne * PER;
    red[threadIdx.x] = s;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
      if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
      __syncthreads();
    }
    if (threadIdx.x == 0) a.out[blockIdx.x] = red[0];
  } else {
    constexpr int WJ = DIM == 2 ? 3 : 6;
    for (int w = threadIdx.x; w < ne * QV; w += blockDim.x) {
      const int el = w / QV, q = w - el * QV;
      const int e = a.elist[t.start + el];
      Ua[el * PER + q] = vfac<DIM, Q>(a, e, q, WJ) * a.a[a.quad_off[e] + q];
    }
    __syncthreads();
    double* t1 = Ga;
    double* t2 = Ga + QV;
    double* res;
    if constexpr (DIM == 2) {
      contract<double, Q, Q, 1, 0, N, tab_B(N, Q), true, false>(Ua, t1, PER, ne);
      __syncthreads();
      contract<double, N, Q, 1, 1, N, tab_B(N, Q), true, false>(t1, t2, PER, ne);
      res = t2;
    } else {
      contract<double, Q, Q, Q, 0, N, tab_B(N, Q), true, false>(Ua, t1, PER, ne);
      __syncthreads();
      contract<double, N, Q, Q, 1, N, tab_B(N, Q), true, false>(t1, t2, PER, ne);
      __syncthreads();
      contract<double, N, N, Q, 2, N, tab_B(N, Q), true, false>(t2, t1, PER, ne);
      res = t1;
    }
    __syncthreads();
    for (int w = threadIdx.x; w < ne * NV; w += blockDim.x) {
      const int el = w / NV, i = w - el * NV;
      const int e = a.elist[t.start + el];
      a.out[a.dof_off[e] + i] = res[el * PER + i];
    }
  }
}

// RULE: the translation unit's point rule (kTuRule), part of the kernel's name.
template <int DIM, int RULE>
__global__ void __launch_bounds__(256) k_aux(AuxArgs a) {
  static_assert(RULE == kTuRule, "kernel instantiated in a unit of another rule");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* sm = reinterpret_cast<double*>(smem_raw);
  const Tile t = a.tiles[blockIdx.x];
#define SIP_AUX_CASE(NN, QQ) aux_tile<DIM, NN, QQ>(a, t, sm)
  SIP_ORDER_SWITCH(SIP_AUX_CASE)
#undef SIP_AUX_CASE
}

}  // namespace sip
