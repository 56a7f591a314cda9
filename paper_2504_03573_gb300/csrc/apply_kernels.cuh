// Matrix-free SIP Helmholtz apply, y = A x, on quad (DIM = 2) and hex
// (DIM = 3) elements with per-element order.  Two kernels per apply:
//
//  k_trace  (TracePhysEval, Sec. 3.2):  per element, interpolate the nodal
//           coefficients to the volume Gauss points (BwdTrans, sum
//           factorisation), evaluate u and the normal derivative
//           c . grad_ref u (c = J^-1 n) on every face at the face's shared Gauss
//           points (extrapolation along the normal with the Gauss-Lagrange
//           basis at +-1, collocation derivative along the face, interpolation
//           to the finer shared rule on p-non-conforming faces, Sec. 3.3) and
//           store them in the trace buffer in the face's canonical point order.
//  k_main   (HelmholtzDGwithAverJump + HelmholtzIPDGTraceFlux, Sec. 5.1):
//           per element, recompute u and its reference gradient at the Gauss
//           points (PhysDeriv by collocation), apply kappa G and lambda w|J|,
//           evaluate the SIP flux on each of its faces from the two sides'
//           traces (Eq. IP: jump, average and penalty), project the flux back
//           from the shared face rule (TraceIProduct) and extrude it into the
//           Gauss-point arrays, then one transposed gradient + IProduct
//           produces y.  Each element writes only its own y: no atomics.
//
// Elements are grouped in tiles of equal order (the paper's element groups);
// one CTA per tile and right-hand side, a switch on the order selects the
// compile-time specialisation (loop bounds and table offsets are constants,
// Sec. 5.1 "separate kernels for different orders").
#pragma once

#include <cstdint>
#include <type_traits>

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
  const T* x;
  T* y;
  T* trace;
  int64_t ndof;            // per-RHS stride of x and y
  int64_t trace_stride;    // per-RHS stride of the trace buffer
  T lambda;
  int transpose;
};

constexpr int ipow(int b, int e) { return e == 0 ? 1 : b * ipow(b, e - 1); }

// ---- per-element shared-memory footprint (in T units)
template <int DIM, int N>
struct Sizes {
  static constexpr int Q = N + 1;
  static constexpr int NV = ipow(N, DIM);
  static constexpr int QV = ipow(Q, DIM);
  static constexpr int QF1 = ipow(Q, DIM - 1);
  static constexpr int FMAX = ipow(kQMax, DIM - 1);
  static constexpr int FT = DIM == 3 ? kQMax * Q : 0;
  static constexpr int FACE = (DIM + 1) * (QF1 + FT + FMAX);
  static constexpr int PER_TRACE = 2 * QV + FACE;
  static constexpr int PER_MAIN = (DIM + 1) * QV + FACE;
};

inline int smem_per_element(int dim, int n, bool main_kernel) {
  const int q = n + 1;
  const int qv = dim == 2 ? q * q : q * q * q;
  const int qf1 = dim == 2 ? q : q * q;
  const int fmax = dim == 2 ? kQMax : kQMax * kQMax;
  const int ft = dim == 3 ? kQMax * q : 0;
  const int face = (dim + 1) * (qf1 + ft + fmax);
  return main_kernel ? (dim + 1) * qv + face : 2 * qv + face;
}

// ---- constant tables; each translation unit that includes this header holds
// its own copy, uploaded by sip_upload_tables_<tu>() at handle creation.
static __constant__ double c_tab_d[kTabSize];
static __constant__ float c_tab_f[kTabSize];
static __constant__ int c_ioff[kQMax + 1][kQMax + 1];

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
template <typename T, int DIM, int N>
__device__ __forceinline__ T* to_gauss(T* bA, T* bB, int stride, int ne) {
  constexpr int Q = N + 1;
  if constexpr (DIM == 2) {
    contract<T, N, N, 1, 0, Q, tab_B(N), false, false>(bA, bB, stride, ne);
    __syncthreads();
    contract<T, Q, N, 1, 1, Q, tab_B(N), false, false>(bB, bA, stride, ne);
    __syncthreads();
    return bA;
  } else {
    contract<T, N, N, N, 0, Q, tab_B(N), false, false>(bA, bB, stride, ne);
    __syncthreads();
    contract<T, Q, N, N, 1, Q, tab_B(N), false, false>(bB, bA, stride, ne);
    __syncthreads();
    contract<T, Q, Q, N, 2, Q, tab_B(N), false, false>(bA, bB, stride, ne);
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

// ============================================================ trace kernel
template <typename T, int DIM, int N, int K>
__device__ __forceinline__ void trace_face(const ApplyArgs<T>& a, const Tile& t, int rhs, T* sm,
                                           const T* U) {
  using S = Sizes<DIM, N>;
  constexpr int Q = S::Q, QF1 = S::QF1, FMAX = S::FMAX, PER = S::PER_TRACE;
  constexpr int AXN = K / 2, SIDE = K % 2;
  constexpr int T0 = Tang<DIM, AXN>::t0, T1 = Tang<DIM, AXN>::t1;
  constexpr int SA = ipow(Q, AXN), S0 = ipow(Q, T0), S1 = DIM == 3 ? ipow(Q, T1 < 0 ? 0 : T1) : 0;
  constexpr int LOFF = tab_L(Q);
  const int ne = t.count;
  // face buffers of element el: Fq at 2 QV, Ft after, Ff after
  auto Fq = [&](int el) { return sm + el * PER + 2 * S::QV; };
  auto Ft = [&](int el) { return sm + el * PER + 2 * S::QV + (DIM + 1) * QF1; };
  auto Ff = [&](int el) { return sm + el * PER + 2 * S::QV + (DIM + 1) * (QF1 + S::FT); };
  // 1. values and normal derivative at the element's own Q^(DIM-1) face points
  for (int w = threadIdx.x; w < ne * QF1; w += blockDim.x) {
    const int el = w / QF1, j = w - el * QF1;
    const int j0 = j % Q, j1 = j / Q;
    const T* u = U + el * PER + j0 * S0 + j1 * S1;
    T uf = 0, dn = 0;
#pragma unroll
    for (int r = 0; r < Q; ++r) {
      const T v = u[r * SA];
      uf = fma(ctab<T>(LOFF + SIDE * Q + r), v, uf);
      dn = fma(ctab<T>(LOFF + (2 + SIDE) * Q + r), v, dn);
    }
    Fq(el)[0 * QF1 + j] = uf;
    Fq(el)[1 * QF1 + j] = dn;
  }
  __syncthreads();
  // 2. tangential derivatives of the face values (collocation on the Gauss points)
  for (int w = threadIdx.x; w < ne * QF1 * (DIM - 1); w += blockDim.x) {
    const int el = w / (QF1 * (DIM - 1));
    const int rem = w - el * QF1 * (DIM - 1);
    const int m = rem / QF1, j = rem - m * QF1;
    const int j0 = j % Q, j1 = j / Q;
    const T* uf = Fq(el);
    T d = 0;
    if (m == 0) {
#pragma unroll
      for (int r = 0; r < Q; ++r) d = fma(ctab<T>(tab_D(Q) + j0 * Q + r), uf[r + Q * j1], d);
    } else {
#pragma unroll
      for (int r = 0; r < Q; ++r) d = fma(ctab<T>(tab_D(Q) + j1 * Q + r), uf[j0 + Q * r], d);
    }
    Fq(el)[(2 + m) * QF1 + j] = d;
  }
  __syncthreads();
  // 3. interpolation to the shared face rule where it is finer (p-non-conforming)
  if constexpr (DIM == 2) {
    for (int w = threadIdx.x; w < ne * (DIM + 1) * kQMax; w += blockDim.x) {
      const int el = w / ((DIM + 1) * kQMax);
      const int rem = w - el * (DIM + 1) * kQMax;
      const int f = rem / kQMax, z = rem - f * kQMax;
      const int e = a.elist[t.start + el];
      const int qf = a.slots[e * 2 * DIM + K].qf;
      if (qf == Q || z >= qf) continue;
      const int io = c_ioff[Q][qf];
      T s = 0;
      for (int r = 0; r < Q; ++r) s = fma(ctab<T>(io + z * Q + r), Fq(el)[f * QF1 + r], s);
      Ff(el)[f * FMAX + z] = s;
    }
    __syncthreads();
  } else {
    for (int w = threadIdx.x; w < ne * (DIM + 1) * Q * kQMax; w += blockDim.x) {
      const int el = w / ((DIM + 1) * Q * kQMax);
      const int rem = w - el * (DIM + 1) * Q * kQMax;
      const int f = rem / (Q * kQMax), r2 = rem - f * Q * kQMax;
      const int j1 = r2 / kQMax, z0 = r2 - j1 * kQMax;
      const int e = a.elist[t.start + el];
      const int qf = a.slots[e * 2 * DIM + K].qf;
      if (qf == Q || z0 >= qf) continue;
      const int io = c_ioff[Q][qf];
      T s = 0;
      for (int r = 0; r < Q; ++r) s = fma(ctab<T>(io + z0 * Q + r), Fq(el)[f * QF1 + j1 * Q + r], s);
      Ft(el)[f * S::FT + j1 * kQMax + z0] = s;
    }
    __syncthreads();
    for (int w = threadIdx.x; w < ne * (DIM + 1) * FMAX; w += blockDim.x) {
      const int el = w / ((DIM + 1) * FMAX);
      const int rem = w - el * (DIM + 1) * FMAX;
      const int f = rem / FMAX, zz = rem - f * FMAX;
      const int z1 = zz / kQMax, z0 = zz - z1 * kQMax;
      const int e = a.elist[t.start + el];
      const int qf = a.slots[e * 2 * DIM + K].qf;
      if (qf == Q || z0 >= qf || z1 >= qf) continue;
      const int io = c_ioff[Q][qf];
      T s = 0;
      for (int r = 0; r < Q; ++r) s = fma(ctab<T>(io + z1 * Q + r), Ft(el)[f * S::FT + r * kQMax + z0], s);
      Ff(el)[f * FMAX + z0 + qf * z1] = s;
    }
    __syncthreads();
  }
  // 4. normal derivative c . grad_ref u and store in canonical order
  constexpr int MAXP = DIM == 2 ? kQMax : kQMax * kQMax;
  for (int w = threadIdx.x; w < ne * MAXP; w += blockDim.x) {
    const int el = w / MAXP, z = w - el * MAXP;
    const int e = a.elist[t.start + el];
    const FaceSlot sl = a.slots[e * 2 * DIM + K];
    const int qf = sl.qf;
    const int npts = DIM == 2 ? qf : qf * qf;
    if (z >= npts) continue;
    const bool fine = qf != Q;
    const T* src = fine ? Ff(el) : Fq(el);
    const int fs = fine ? FMAX : QF1;
    const T uf = src[0 * fs + z];
    const T dn = src[1 * fs + z];
    const T d0 = src[2 * fs + z];
    const T d1 = DIM == 3 ? src[3 * fs + z] : T(0);
    const int j0 = z % qf, j1 = z / qf;
    const int zc = canon(DIM, sl.side, sl.orient, qf, j0, j1);
    const int64_t go = a.f_goff[sl.face];
    const T* c = a.fgeo + go + (int64_t)(1 + sl.side * DIM) * npts + zc;
    T g = c[(int64_t)AXN * npts] * dn + c[(int64_t)T0 * npts] * d0;
    if constexpr (DIM == 3) g += c[(int64_t)T1 * npts] * d1;
    T* tr = a.trace + rhs * a.trace_stride + 4 * a.f_troff[sl.face] + (int64_t)(2 * sl.side) * npts + zc;
    tr[0] = uf;
    tr[npts] = g;
  }
  __syncthreads();
}

template <typename T, int DIM, int N>
__device__ void trace_tile(const ApplyArgs<T>& a, const Tile& t, int rhs, T* sm) {
  using S = Sizes<DIM, N>;
  constexpr int PER = S::PER_TRACE;
  const int ne = t.count;
  for (int w = threadIdx.x; w < ne * S::NV; w += blockDim.x) {
    const int el = w / S::NV, i = w - el * S::NV;
    const int e = a.elist[t.start + el];
    sm[el * PER + i] = a.x[rhs * a.ndof + a.dof_off[e] + i];
  }
  __syncthreads();
  T* U = to_gauss<T, DIM, N>(sm, sm + S::QV, PER, ne);
  trace_face<T, DIM, N, 0>(a, t, rhs, sm, U);
  trace_face<T, DIM, N, 1>(a, t, rhs, sm, U);
  trace_face<T, DIM, N, 2>(a, t, rhs, sm, U);
  trace_face<T, DIM, N, 3>(a, t, rhs, sm, U);
  if constexpr (DIM == 3) {
    trace_face<T, DIM, N, 4>(a, t, rhs, sm, U);
    trace_face<T, DIM, N, 5>(a, t, rhs, sm, U);
  }
}

// ============================================================ main kernel
template <typename T, int DIM, int N, int K>
__device__ __forceinline__ void lift_face(const ApplyArgs<T>& a, const Tile& t, int rhs, T* sm) {
  using S = Sizes<DIM, N>;
  constexpr int Q = S::Q, QV = S::QV, QF1 = S::QF1, FMAX = S::FMAX, PER = S::PER_MAIN;
  constexpr int AXN = K / 2, SIDE = K % 2;
  constexpr int T0 = Tang<DIM, AXN>::t0, T1 = Tang<DIM, AXN>::t1;
  constexpr int LOFF = tab_L(Q);
  constexpr int MAXP = DIM == 2 ? kQMax : kQMax * kQMax;
  const int ne = t.count;
  auto Fq = [&](int el) { return sm + el * PER + (DIM + 1) * QV; };
  auto Ft = [&](int el) { return sm + el * PER + (DIM + 1) * QV + (DIM + 1) * QF1; };
  auto Ff = [&](int el) { return sm + el * PER + (DIM + 1) * QV + (DIM + 1) * (QF1 + S::FT); };
  // a. flux at the shared face points (own point order), fields s, c_m t
  for (int w = threadIdx.x; w < ne * MAXP; w += blockDim.x) {
    const int el = w / MAXP, z = w - el * MAXP;
    const int e = a.elist[t.start + el];
    const FaceSlot sl = a.slots[e * 2 * DIM + K];
    const int qf = sl.qf;
    const int npts = DIM == 2 ? qf : qf * qf;
    if (z >= npts) continue;
    const int zc = canon(DIM, sl.side, sl.orient, qf, z % qf, z / qf);
    const T* tr = a.trace + rhs * a.trace_stride + 4 * a.f_troff[sl.face] + zc;
    const int64_t go = a.f_goff[sl.face];
    const T W = a.fgeo[go + zc];
    const T tau = a.f_tau[sl.face];
    const T uo = tr[(int64_t)(2 * sl.side) * npts];
    const T go_ = tr[(int64_t)(2 * sl.side + 1) * npts];
    T s, tt;
    if (sl.bnd) {
      // Nitsche: -(grad v.n, u) - (v, grad u.n) + tau (v, u)
      if (!a.transpose) { s = W * (tau * uo - go_); tt = -W * uo; }
      else { s = W * tau * uo - W * go_; tt = -(W * uo); }
    } else {
      const int oth = 1 - sl.side;
      const T un = tr[(int64_t)(2 * oth) * npts];
      const T gn = tr[(int64_t)(2 * oth + 1) * npts];
      if (!a.transpose) {
        // rows of the per-point flux: s = W (tau [u] - {du/dn}), t = -W [u] / 2
        const T jmp = uo - un;
        const T avg = T(0.5) * (go_ - gn);
        s = W * (tau * jmp - avg);
        tt = T(-0.5) * W * jmp;
      } else {
        // columns of the same flux (trial and test roles exchanged)
        s = W * tau * uo - W * tau * un - T(0.5) * W * go_ + T(0.5) * W * gn;
        tt = T(0.5) * W * un - T(0.5) * W * uo;
      }
    }
    const bool fine = qf != Q;
    T* dst = fine ? Ff(el) : Fq(el);
    const int fs = fine ? FMAX : QF1;
    dst[z] = s;
    const T* c = a.fgeo + go + (int64_t)(1 + sl.side * DIM) * npts + zc;
#pragma unroll
    for (int m = 0; m < DIM; ++m) dst[(1 + m) * fs + z] = c[(int64_t)m * npts] * tt;
  }
  __syncthreads();
  // b. projection from the shared rule to the element's own Gauss points (transpose of the interpolation)
  if constexpr (DIM == 2) {
    for (int w = threadIdx.x; w < ne * (DIM + 1) * Q; w += blockDim.x) {
      const int el = w / ((DIM + 1) * Q);
      const int rem = w - el * (DIM + 1) * Q;
      const int f = rem / Q, r = rem - f * Q;
      const int e = a.elist[t.start + el];
      const int qf = a.slots[e * 2 * DIM + K].qf;
      if (qf == Q) continue;
      const int io = c_ioff[Q][qf];
      T s = 0;
      for (int z = 0; z < qf; ++z) s = fma(ctab<T>(io + z * Q + r), Ff(el)[f * FMAX + z], s);
      Fq(el)[f * QF1 + r] = s;
    }
    __syncthreads();
  } else {
    // Ft[f][z1][r0] = sum_z0 I[z0][r0] Ff[f][z1][z0]
    for (int w = threadIdx.x; w < ne * (DIM + 1) * kQMax * Q; w += blockDim.x) {
      const int el = w / ((DIM + 1) * kQMax * Q);
      const int rem = w - el * (DIM + 1) * kQMax * Q;
      const int f = rem / (kQMax * Q), r2 = rem - f * kQMax * Q;
      const int z1 = r2 / Q, r0 = r2 - z1 * Q;
      const int e = a.elist[t.start + el];
      const int qf = a.slots[e * 2 * DIM + K].qf;
      if (qf == Q || z1 >= qf) continue;
      const int io = c_ioff[Q][qf];
      T s = 0;
      for (int z0 = 0; z0 < qf; ++z0) s = fma(ctab<T>(io + z0 * Q + r0), Ff(el)[f * FMAX + z0 + qf * z1], s);
      Ft(el)[f * S::FT + z1 * Q + r0] = s;
    }
    __syncthreads();
    // Fq[f][r1][r0] = sum_z1 I[z1][r1] Ft[f][z1][r0]
    for (int w = threadIdx.x; w < ne * (DIM + 1) * QF1; w += blockDim.x) {
      const int el = w / ((DIM + 1) * QF1);
      const int rem = w - el * (DIM + 1) * QF1;
      const int f = rem / QF1, r = rem - f * QF1;
      const int r0 = r % Q, r1 = r / Q;
      const int e = a.elist[t.start + el];
      const int qf = a.slots[e * 2 * DIM + K].qf;
      if (qf == Q) continue;
      const int io = c_ioff[Q][qf];
      T s = 0;
      for (int z1 = 0; z1 < qf; ++z1) s = fma(ctab<T>(io + z1 * Q + r1), Ft(el)[f * S::FT + z1 * Q + r0], s);
      Fq(el)[f * QF1 + r] = s;
    }
    __syncthreads();
  }
  // c. extrude along the normal with l_r(+-1): r += l s~, q_m += l (c_m t)~
  constexpr int SA = ipow(Q, AXN), S0 = ipow(Q, T0), S1 = DIM == 3 ? ipow(Q, T1 < 0 ? 0 : T1) : 0;
  for (int w = threadIdx.x; w < ne * QV; w += blockDim.x) {
    const int el = w / QV, q = w - el * QV;
    const int qa = (q / SA) % Q;
    const int j0 = (q / S0) % Q;
    const int j1 = DIM == 3 ? (q / S1) % Q : 0;
    const int j = j0 + Q * j1;
    const T l = ctab<T>(LOFF + SIDE * Q + qa);
    T* base = sm + el * PER;
    const T* fq = Fq(el);
    base[q] = fma(l, fq[j], base[q]);
#pragma unroll
    for (int m = 0; m < DIM; ++m) base[(1 + m) * QV + q] = fma(l, fq[(1 + m) * QF1 + j], base[(1 + m) * QV + q]);
  }
  __syncthreads();
}

template <typename T, int DIM, int N>
__device__ void main_tile(const ApplyArgs<T>& a, const Tile& t, int rhs, T* sm) {
  using S = Sizes<DIM, N>;
  constexpr int Q = S::Q, QV = S::QV, PER = S::PER_MAIN;
  const int ne = t.count;
  // layout per element: U [QV], G_0..G_{DIM-1} [QV each], face buffers
  T* U = sm;
  T* G0 = sm + QV;
  T* G1 = sm + 2 * QV;
  T* G2 = sm + 3 * QV;
  // load coefficients into G0 and interpolate: 2D G0 -> G1 -> U ; 3D G0 -> G1 -> G2 -> U
  for (int w = threadIdx.x; w < ne * S::NV; w += blockDim.x) {
    const int el = w / S::NV, i = w - el * S::NV;
    const int e = a.elist[t.start + el];
    G0[el * PER + i] = a.x[rhs * a.ndof + a.dof_off[e] + i];
  }
  __syncthreads();
  if constexpr (DIM == 2) {
    contract<T, N, N, 1, 0, Q, tab_B(N), false, false>(G0, G1, PER, ne);
    __syncthreads();
    contract<T, Q, N, 1, 1, Q, tab_B(N), false, false>(G1, U, PER, ne);
    __syncthreads();
    // reference gradient by collocation
    contract<T, Q, Q, 1, 0, Q, tab_D(Q), false, false>(U, G0, PER, ne);
    contract<T, Q, Q, 1, 1, Q, tab_D(Q), false, false>(U, G1, PER, ne);
  } else {
    contract<T, N, N, N, 0, Q, tab_B(N), false, false>(G0, G1, PER, ne);
    __syncthreads();
    contract<T, Q, N, N, 1, Q, tab_B(N), false, false>(G1, G2, PER, ne);
    __syncthreads();
    contract<T, Q, Q, N, 2, Q, tab_B(N), false, false>(G2, U, PER, ne);
    __syncthreads();
    contract<T, Q, Q, Q, 0, Q, tab_D(Q), false, false>(U, G0, PER, ne);
    contract<T, Q, Q, Q, 1, Q, tab_D(Q), false, false>(U, G1, PER, ne);
    contract<T, Q, Q, Q, 2, Q, tab_D(Q), false, false>(U, G2, PER, ne);
  }
  __syncthreads();
  // pointwise: q = kappa G grad_ref u, r = lambda w|J| u
  constexpr int NG = DIM == 2 ? 4 : 7;
  for (int w = threadIdx.x; w < ne * QV; w += blockDim.x) {
    const int el = w / QV, q = w - el * QV;
    const int e = a.elist[t.start + el];
    const T* geo = a.vgeo + a.vgoff[e] + q;
    const T kap = a.kappa ? a.kappa[a.quad_off[e] + q] : T(1);
    T* b = sm + el * PER;
    if constexpr (DIM == 2) {
      const T g0 = b[QV + q], g1 = b[2 * QV + q];
      const T a00 = geo[0], a01 = geo[QV], a11 = geo[2 * QV], wj = geo[3 * QV];
      b[QV + q] = kap * (a00 * g0 + a01 * g1);
      b[2 * QV + q] = kap * (a01 * g0 + a11 * g1);
      b[q] = a.lambda * wj * b[q];
    } else {
      const T g0 = b[QV + q], g1 = b[2 * QV + q], g2 = b[3 * QV + q];
      const T a00 = geo[0], a01 = geo[QV], a02 = geo[2 * QV], a11 = geo[3 * QV], a12 = geo[4 * QV],
              a22 = geo[5 * QV], wj = geo[6 * QV];
      b[QV + q] = kap * (a00 * g0 + a01 * g1 + a02 * g2);
      b[2 * QV + q] = kap * (a01 * g0 + a11 * g1 + a12 * g2);
      b[3 * QV + q] = kap * (a02 * g0 + a12 * g1 + a22 * g2);
      b[q] = a.lambda * wj * b[q];
    }
    (void)NG;
  }
  __syncthreads();
  // faces: flux, projection, extrusion into U and G
  lift_face<T, DIM, N, 0>(a, t, rhs, sm);
  lift_face<T, DIM, N, 1>(a, t, rhs, sm);
  lift_face<T, DIM, N, 2>(a, t, rhs, sm);
  lift_face<T, DIM, N, 3>(a, t, rhs, sm);
  if constexpr (DIM == 3) {
    lift_face<T, DIM, N, 4>(a, t, rhs, sm);
    lift_face<T, DIM, N, 5>(a, t, rhs, sm);
  }
  // U += sum_m D_m^T G_m ; then y = (B^T x B^T (x B^T)) U
  if constexpr (DIM == 2) {
    contract<T, Q, Q, 1, 0, Q, tab_D(Q), true, true>(G0, U, PER, ne);
    __syncthreads();
    contract<T, Q, Q, 1, 1, Q, tab_D(Q), true, true>(G1, U, PER, ne);
    __syncthreads();
    contract<T, Q, Q, 1, 0, N, tab_B(N), true, false>(U, G0, PER, ne);
    __syncthreads();
    contract<T, N, Q, 1, 1, N, tab_B(N), true, false>(G0, G1, PER, ne);
    __syncthreads();
    for (int w = threadIdx.x; w < ne * S::NV; w += blockDim.x) {
      const int el = w / S::NV, i = w - el * S::NV;
      const int e = a.elist[t.start + el];
      a.y[rhs * a.ndof + a.dof_off[e] + i] = G1[el * PER + i];
    }
  } else {
    contract<T, Q, Q, Q, 0, Q, tab_D(Q), true, true>(G0, U, PER, ne);
    __syncthreads();
    contract<T, Q, Q, Q, 1, Q, tab_D(Q), true, true>(G1, U, PER, ne);
    __syncthreads();
    contract<T, Q, Q, Q, 2, Q, tab_D(Q), true, true>(G2, U, PER, ne);
    __syncthreads();
    contract<T, Q, Q, Q, 0, N, tab_B(N), true, false>(U, G0, PER, ne);
    __syncthreads();
    contract<T, N, Q, Q, 1, N, tab_B(N), true, false>(G0, G1, PER, ne);
    __syncthreads();
    contract<T, N, N, Q, 2, N, tab_B(N), true, false>(G1, G2, PER, ne);
    __syncthreads();
    for (int w = threadIdx.x; w < ne * S::NV; w += blockDim.x) {
      const int el = w / S::NV, i = w - el * S::NV;
      const int e = a.elist[t.start + el];
      a.y[rhs * a.ndof + a.dof_off[e] + i] = G2[el * PER + i];
    }
  }
}

// ============================================================ auxiliary element kernels (FP64)
// kappa gradient w|J| grad a . grad b, mass inner product a^T M b, IProduct.
struct AuxArgs {
  const int64_t* dof_off;
  const int64_t* quad_off;
  const int64_t* vgoff;
  const double* vgeo;
  const int32_t* elist;
  const Tile* tiles;
  const double* a;
  const double* b;
  double* out;
  int accumulate;
  int mode;  // 0: kappa gradient, 1: mass dot partials (one per tile), 2: IProduct
};

inline int aux_smem_per_element(int dim, int n) {
  const int q = n + 1;
  const int qv = dim == 2 ? q * q : q * q * q;
  return 2 * (dim + 1) * qv;
}

// load N^DIM coefficients of vector v into U (via scratch S) and interpolate to
// the Gauss points: result in U.
template <int DIM, int N>
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
  if constexpr (DIM == 2) to_gauss<double, 2, N>(U, S, per, t.count);
  else to_gauss<double, 3, N>(S, U, per, t.count);
}

template <int DIM, int N>
__device__ __forceinline__ void gauss_grad(const double* U, double* G0, double* G1, double* G2, int per, int ne) {
  constexpr int Q = N + 1;
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

template <int DIM, int N>
__device__ void aux_tile(const AuxArgs& a, const Tile& t, double* sm) {
  constexpr int Q = N + 1, QV = ipow(Q, DIM), NV = ipow(N, DIM);
  constexpr int PER = 2 * (DIM + 1) * QV;
  const int ne = t.count;
  double* Ua = sm;
  double* Ga = sm + QV;                 // DIM buffers
  double* Ub = sm + (DIM + 1) * QV;
  double* Gb = sm + (DIM + 2) * QV;     // DIM buffers
  if (a.mode == 0) {
    load_to_gauss<DIM, N>(a, t, a.a, Ua, Ga, PER);
    gauss_grad<DIM, N>(Ua, Ga, Ga + QV, Ga + 2 * QV, PER, ne);
    load_to_gauss<DIM, N>(a, t, a.b, Ub, Gb, PER);
    gauss_grad<DIM, N>(Ub, Gb, Gb + QV, Gb + 2 * QV, PER, ne);
    for (int w = threadIdx.x; w < ne * QV; w += blockDim.x) {
      const int el = w / QV, q = w - el * QV;
      const int e = a.elist[t.start + el];
      const double* g = a.vgeo + a.vgoff[e] + q;
      const double* ga = Ga + el * PER + q;
      const double* gb = Gb + el * PER + q;
      double v;
      if constexpr (DIM == 2) {
        v = g[0] * ga[0] * gb[0] + g[QV] * (ga[0] * gb[QV] + ga[QV] * gb[0]) + g[2 * QV] * ga[QV] * gb[QV];
      } else {
        v = g[0] * ga[0] * gb[0] + g[3 * QV] * ga[QV] * gb[QV] + g[5 * QV] * ga[2 * QV] * gb[2 * QV] +
            g[QV] * (ga[0] * gb[QV] + ga[QV] * gb[0]) + g[2 * QV] * (ga[0] * gb[2 * QV] + ga[2 * QV] * gb[0]) +
            g[4 * QV] * (ga[QV] * gb[2 * QV] + ga[2 * QV] * gb[QV]);
      }
      double* o = a.out + a.quad_off[e] + q;
      *o = a.accumulate ? *o + v : v;
    }
  } else if (a.mode == 1) {
    load_to_gauss<DIM, N>(a, t, a.a, Ua, Ga, PER);
    load_to_gauss<DIM, N>(a, t, a.b, Ub, Gb, PER);
    double s = 0.0;
    constexpr int WJ = DIM == 2 ? 3 : 6;
    for (int w = threadIdx.x; w < ne * QV; w += blockDim.x) {
      const int el = w / QV, q = w - el * QV;
      const int e = a.elist[t.start + el];
      s += a.vgeo[a.vgoff[e] + WJ * QV + q] * Ua[el * PER + q] * Ub[el * PER + q];
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
      Ua[el * PER + q] = a.vgeo[a.vgoff[e] + WJ * QV + q] * a.a[a.quad_off[e] + q];
    }
    __syncthreads();
    double* t1 = Ga;
    double* t2 = Ga + QV;
    double* res;
    if constexpr (DIM == 2) {
      contract<double, Q, Q, 1, 0, N, tab_B(N), true, false>(Ua, t1, PER, ne);
      __syncthreads();
      contract<double, N, Q, 1, 1, N, tab_B(N), true, false>(t1, t2, PER, ne);
      res = t2;
    } else {
      contract<double, Q, Q, Q, 0, N, tab_B(N), true, false>(Ua, t1, PER, ne);
      __syncthreads();
      contract<double, N, Q, Q, 1, N, tab_B(N), true, false>(t1, t2, PER, ne);
      __syncthreads();
      contract<double, N, N, Q, 2, N, tab_B(N), true, false>(t2, t1, PER, ne);
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

template <int DIM>
__global__ void __launch_bounds__(256) k_aux(AuxArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* sm = reinterpret_cast<double*>(smem_raw);
  const Tile t = a.tiles[blockIdx.x];
  switch (t.n) {
    case 2: aux_tile<DIM, 2>(a, t, sm); break;
    case 3: aux_tile<DIM, 3>(a, t, sm); break;
    case 4: aux_tile<DIM, 4>(a, t, sm); break;
    case 5: aux_tile<DIM, 5>(a, t, sm); break;
    case 6: aux_tile<DIM, 6>(a, t, sm); break;
    case 7: aux_tile<DIM, 7>(a, t, sm); break;
    case 8: aux_tile<DIM, 8>(a, t, sm); break;
    case 9: aux_tile<DIM, 9>(a, t, sm); break;
    default: break;
  }
}

template <typename T, int DIM>
__global__ void __launch_bounds__(256) k_trace(ApplyArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const Tile t = a.tiles[blockIdx.x];
  const int rhs = blockIdx.y;
  switch (t.n) {
    case 2: trace_tile<T, DIM, 2>(a, t, rhs, sm); break;
    case 3: trace_tile<T, DIM, 3>(a, t, rhs, sm); break;
    case 4: trace_tile<T, DIM, 4>(a, t, rhs, sm); break;
    case 5: trace_tile<T, DIM, 5>(a, t, rhs, sm); break;
    case 6: trace_tile<T, DIM, 6>(a, t, rhs, sm); break;
    case 7: trace_tile<T, DIM, 7>(a, t, rhs, sm); break;
    case 8: trace_tile<T, DIM, 8>(a, t, rhs, sm); break;
    case 9: trace_tile<T, DIM, 9>(a, t, rhs, sm); break;
    default: break;
  }
}

template <typename T, int DIM>
__global__ void __launch_bounds__(256) k_main(ApplyArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const Tile t = a.tiles[blockIdx.x];
  const int rhs = blockIdx.y;
  switch (t.n) {
    case 2: main_tile<T, DIM, 2>(a, t, rhs, sm); break;
    case 3: main_tile<T, DIM, 3>(a, t, rhs, sm); break;
    case 4: main_tile<T, DIM, 4>(a, t, rhs, sm); break;
    case 5: main_tile<T, DIM, 5>(a, t, rhs, sm); break;
    case 6: main_tile<T, DIM, 6>(a, t, rhs, sm); break;
    case 7: main_tile<T, DIM, 7>(a, t, rhs, sm); break;
    case 8: main_tile<T, DIM, 8>(a, t, rhs, sm); break;
    case 9: main_tile<T, DIM, 9>(a, t, rhs, sm); break;
    default: break;
  }
}

}  // namespace sip
