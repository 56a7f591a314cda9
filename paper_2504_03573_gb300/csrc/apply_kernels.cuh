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
//           In FP64 it also stores the Gauss-point values for k_main: moving 16
//           bytes through HBM costs less than recomputing them with FP64 flops.
//  k_main   (HelmholtzDGwithAverJump + HelmholtzIPDGTraceFlux, Sec. 5.1):
//           per element, take u at the Gauss points, its reference gradient
//           (PhysDeriv by collocation), apply kappa G and lambda w|J|, evaluate
//           the SIP flux on its faces from the two sides' traces (Eq. IP: jump,
//           average and penalty), project it back from the shared face rule
//           (TraceIProduct) and extrude it along the normal into the
//           Gauss-point arrays; one transposed gradient + IProduct gives y.
//           Each element writes only its own y: no atomics.
//
// Thread mapping: every stage is a loop over the OUTPUT values of the tile's
// elements (one output per work item), so a stage exposes elements x Q^DIM
// independent items.  The 1D matrices live in shared memory in layouts where
// the lanes of a warp (consecutive outputs) read consecutive addresses.
// Elements are grouped in tiles of equal order (the paper's element groups);
// one CTA per tile and right-hand side; a switch on the order selects the
// compile-time specialisation (Sec. 5.1, "separate kernels for different orders").
#pragma once

#include "common.cuh"

namespace sip {

// contraction style: line per thread (FP32, 3D) or output per thread (otherwise)
template <typename T, int DIM>
__host__ __device__ constexpr bool line_mode() { return DIM == 3 && std::is_same<T, float>::value; }

// ---- per-order compile-time shape
template <int DIM, int N>
struct Shape {
  static constexpr int Q = N + 1;
  static constexpr int NV = cpow(N, DIM);
  static constexpr int QV = cpow(Q, DIM);
  static constexpr int QF1 = cpow(Q, DIM - 1);       // own points on one face
  static constexpr int FMAX = cpow(kQMax, DIM - 1);  // points on one face at the finest rule
  static constexpr int FT = DIM == 3 ? kQMax * Q : 0;
  static constexpr int NFB = faces_per_batch(DIM);
  static constexpr int PER_TRACE = per_elem_trace(DIM, N);
  static constexpr int PER_MAIN = per_elem_main(DIM, N);
};

// Copy this order's 1D tables from __constant__ into the CTA's table block.
template <typename T, int N>
__device__ __forceinline__ void load_tables(T* tb) {
  constexpr int Q = N + 1;
  for (int w = threadIdx.x; w < N * Q; w += blockDim.x) {
    const int q = w / N, i = w - q * N;  // B[q][i]
    const T v = ctab<T>(tab_B(N) + w);
    tb[TabLayout::BT(N) + i * Q + q] = v;
    tb[TabLayout::BB(N) + q * N + i] = v;
  }
  for (int w = threadIdx.x; w < Q * Q; w += blockDim.x) {
    const int q = w / Q, r = w - q * Q;  // D[q][r]
    const T v = ctab<T>(tab_D(Q) + w);
    tb[TabLayout::DT(N) + r * Q + q] = v;
    tb[TabLayout::DD(N) + q * Q + r] = v;
  }
  for (int w = threadIdx.x; w < 4 * Q; w += blockDim.x) tb[TabLayout::LL(N) + w] = ctab<T>(tab_L(Q) + w);
  for (int f = Q + 1; f <= kQMax; ++f) {
    const int io = c_ioff[Q][f];
    for (int w = threadIdx.x; w < f * Q; w += blockDim.x) {
      const int z = w / Q, r = w - z * Q;  // I[z][r]
      const T v = ctab<T>(io + w);
      tb[TabLayout::IT(N, f) + r * f + z] = v;
      tb[TabLayout::II(N, f) + z * Q + r] = v;
    }
  }
  __syncthreads();
}

// out[el][o] (+)= sum_j M[j][k(o)] in[el][line(o) + j SI], one work item per
// output o of every element; in and out are [E2][E1][E0] arrays (E0 fastest)
// whose AX extent is NIN (in) and NOUT (out).  M is a [NIN][NOUT] shared table.
template <typename T, int E0, int E1, int E2, int AX, int NOUT, bool ACC>
__device__ __forceinline__ void cpt(const T* __restrict__ in, T* __restrict__ out, int stride, int ne,
                                    const T* __restrict__ M) {
  constexpr int NIN = AX == 0 ? E0 : (AX == 1 ? E1 : E2);
  constexpr int O0 = AX == 0 ? NOUT : E0;
  constexpr int O1 = AX == 1 ? NOUT : E1;
  constexpr int O2 = AX == 2 ? NOUT : E2;
  constexpr int NO = O0 * O1 * O2;
  constexpr int SI = AX == 0 ? 1 : (AX == 1 ? E0 : E0 * E1);
  for (int w = threadIdx.x; w < ne * NO; w += blockDim.x) {
    const int el = w / NO;
    const int o = w - el * NO;
    const int o0 = o % O0, o1 = (o / O0) % O1, o2 = o / (O0 * O1);
    int k, bi;
    if (AX == 0) { k = o0; bi = o1 * E0 + o2 * E0 * E1; }
    else if (AX == 1) { k = o1; bi = o0 + o2 * E0 * E1; }
    else { k = o2; bi = o0 + o1 * E0; }
    const T* src = in + el * stride + bi;
    T acc = ACC ? out[el * stride + o] : T(0);
#pragma unroll
    for (int j = 0; j < NIN; ++j) acc = fma(M[j * NOUT + k], src[j * SI], acc);
    out[el * stride + o] = acc;
  }
}

// GLL coefficients in bA (N^DIM) -> Gauss values (Q^DIM); bB scratch.  Returns
// the buffer holding the result.
template <typename T, int DIM, int N>
__device__ __forceinline__ T* interp_to_gauss(T* bA, T* bB, int stride, int ne, const T* tb) {
  constexpr int Q = N + 1;
  const T* BT = tb + TabLayout::BT(N);
  if constexpr (DIM == 2) {
    cpt<T, N, N, 1, 0, Q, false>(bA, bB, stride, ne, BT);
    __syncthreads();
    cpt<T, Q, N, 1, 1, Q, false>(bB, bA, stride, ne, BT);
    __syncthreads();
    return bA;
  } else {
    cpt<T, N, N, N, 0, Q, false>(bA, bB, stride, ne, BT);
    __syncthreads();
    cpt<T, Q, N, N, 1, Q, false>(bB, bA, stride, ne, BT);
    __syncthreads();
    cpt<T, Q, Q, N, 2, Q, false>(bA, bB, stride, ne, BT);
    __syncthreads();
    return bB;
  }
}

// tangential axes of the faces normal to axis a (runtime)
template <int DIM>
__device__ __forceinline__ void tang_axes(int a, int& t0, int& t1) {
  if (DIM == 2) { t0 = 1 - a; t1 = -1; }
  else { t0 = a == 0 ? 1 : 0; t1 = a == 2 ? 1 : 2; }
}

// Q^e for e in 0..2
template <int Q>
__device__ __forceinline__ int qpow(int e) { return e == 0 ? 1 : (e == 1 ? Q : Q * Q); }

// ============================================================ trace kernel
// Per-tile copy of the element ids and face slots (kMetaBytes, after the table block).
struct TileMeta {
  int32_t eid[kMaxEpb];
  FaceSlot slot[kMaxEpb * 6];
};

template <int DIM>
__device__ __forceinline__ void load_meta(const int32_t* elist, const FaceSlot* slots, const Tile& t, TileMeta* mt) {
  for (int w = threadIdx.x; w < t.count * 2 * DIM; w += blockDim.x) {
    const int el = w / (2 * DIM), k = w - el * 2 * DIM;
    const int e = elist[t.start + el];
    if (k == 0) mt->eid[el] = e;
    mt->slot[el * 2 * DIM + k] = slots[(int64_t)e * 2 * DIM + k];
  }
}

// Faces K0 .. K0+NFB-1 of every element of the tile, processed together.
template <typename T, int DIM, int N, int K0>
__device__ __forceinline__ void trace_faces(const ApplyArgs<T>& a, const Tile& t, const TileMeta* mt, int rhs,
                                            const T* tb, T* sm, const T* U) {
  using S = Shape<DIM, N>;
  constexpr int Q = S::Q, QF1 = S::QF1, FMAX = S::FMAX, FT = S::FT, NFB = S::NFB, PER = S::PER_TRACE;
  constexpr int FB = 4 * (QF1 + FT + FMAX);  // per face in the batch: Fq [4][QF1], Ft [4][FT], Ff [4][FMAX]
  const int ne = t.count;
  const int qfm = t.flags & kTileQfMask;
  const bool fine = t.flags & kTileFine;
  const bool orth = t.flags & kTileOrth;
  const int npm = DIM == 2 ? qfm : qfm * qfm;
  T* const F0 = sm + 2 * S::QV;
  const T* LL = tb + TabLayout::LL(N);
  const T* DT = tb + TabLayout::DT(N);
  // 1. value and reference normal derivative at the element's own face points
  for (int w = threadIdx.x; w < ne * NFB * QF1; w += blockDim.x) {
    const int el = w / (NFB * QF1);
    const int rem = w - el * NFB * QF1;
    const int fb = rem / QF1, j = rem - fb * QF1;
    const int k = K0 + fb, ax = k >> 1, sd = k & 1;
    int t0, t1;
    tang_axes<DIM>(ax, t0, t1);
    const int j0 = j % Q, j1 = j / Q;
    const int sa = qpow<Q>(ax);
    const T* u = U + el * PER + j0 * qpow<Q>(t0) + (DIM == 3 ? j1 * qpow<Q>(t1) : 0);
    T uf = 0, dn = 0;
#pragma unroll
    for (int r = 0; r < Q; ++r) {
      const T v = u[r * sa];
      uf = fma(LL[sd * Q + r], v, uf);
      dn = fma(LL[(2 + sd) * Q + r], v, dn);
    }
    T* fq = F0 + el * PER + fb * FB;
    fq[j] = uf;
    fq[QF1 + j] = dn;
  }
  __syncthreads();
  // 2. tangential derivatives of the face values (collocation on the Gauss
  //    points); not needed where c has no tangential component
  if (!orth) {
    for (int w = threadIdx.x; w < ne * NFB * (DIM - 1) * QF1; w += blockDim.x) {
      const int el = w / (NFB * (DIM - 1) * QF1);
      const int rem = w - el * NFB * (DIM - 1) * QF1;
      const int fb = rem / ((DIM - 1) * QF1);
      const int r2 = rem - fb * (DIM - 1) * QF1;
      const int m = r2 / QF1, j = r2 - m * QF1;
      const int j0 = j % Q, j1 = j / Q;
      T* fq = F0 + el * PER + fb * FB;
      T d = 0;
      if (m == 0) {
#pragma unroll
        for (int r = 0; r < Q; ++r) d = fma(DT[r * Q + j0], fq[r + Q * j1], d);
      } else {
#pragma unroll
        for (int r = 0; r < Q; ++r) d = fma(DT[r * Q + j1], fq[j0 + Q * r], d);
      }
      fq[(2 + m) * QF1 + j] = d;
    }
    __syncthreads();
  }
  // 3. interpolation to the shared face rule where it is finer (p-non-conforming faces)
  if (fine) {
    const int nfld = orth ? 2 : 4;
    if constexpr (DIM == 2) {
      for (int w = threadIdx.x; w < ne * NFB * nfld * qfm; w += blockDim.x) {
        const int el = w / (NFB * nfld * qfm);
        const int rem = w - el * NFB * nfld * qfm;
        const int fb = rem / (nfld * qfm), r2 = rem - fb * nfld * qfm;
        const int f = r2 / qfm, z = r2 - f * qfm;
        const int qf = mt->slot[el * 2 * DIM + K0 + fb].qf;
        if (qf == Q || z >= qf) continue;
        const T* IT = tb + TabLayout::IT(N, qf);
        T* fq = F0 + el * PER + fb * FB;
        const T* src = fq + f * QF1;
        T s = 0;
#pragma unroll
        for (int r = 0; r < Q; ++r) s = fma(IT[r * qf + z], src[r], s);
        fq[4 * (QF1 + FT) + f * FMAX + z] = s;
      }
      __syncthreads();
    } else {
      for (int w = threadIdx.x; w < ne * NFB * nfld * Q * qfm; w += blockDim.x) {
        const int el = w / (NFB * nfld * Q * qfm);
        const int rem = w - el * NFB * nfld * Q * qfm;
        const int fb = rem / (nfld * Q * qfm), r2 = rem - fb * nfld * Q * qfm;
        const int f = r2 / (Q * qfm), r3 = r2 - f * Q * qfm;
        const int j1 = r3 / qfm, z0 = r3 - j1 * qfm;
        const int qf = mt->slot[el * 2 * DIM + K0 + fb].qf;
        if (qf == Q || z0 >= qf) continue;
        const T* IT = tb + TabLayout::IT(N, qf);
        T* fq = F0 + el * PER + fb * FB;
        const T* src = fq + f * QF1 + j1 * Q;
        T s = 0;
#pragma unroll
        for (int r = 0; r < Q; ++r) s = fma(IT[r * qf + z0], src[r], s);
        fq[4 * QF1 + f * FT + j1 * kQMax + z0] = s;
      }
      __syncthreads();
      for (int w = threadIdx.x; w < ne * NFB * nfld * npm; w += blockDim.x) {
        const int el = w / (NFB * nfld * npm);
        const int rem = w - el * NFB * nfld * npm;
        const int fb = rem / (nfld * npm), r2 = rem - fb * nfld * npm;
        const int f = r2 / npm, zz = r2 - f * npm;
        const int z1 = zz / qfm, z0 = zz - z1 * qfm;
        const int qf = mt->slot[el * 2 * DIM + K0 + fb].qf;
        if (qf == Q || z0 >= qf || z1 >= qf) continue;
        const T* IT = tb + TabLayout::IT(N, qf);
        T* fq = F0 + el * PER + fb * FB;
        const T* src = fq + 4 * QF1 + f * FT + z0;
        T s = 0;
#pragma unroll
        for (int r = 0; r < Q; ++r) s = fma(IT[r * qf + z1], src[r * kQMax], s);
        fq[4 * (QF1 + FT) + f * FMAX + z0 + qf * z1] = s;
      }
      __syncthreads();
    }
  }
  // 4. normal derivative c . grad_ref u, stored in canonical face order
  for (int w = threadIdx.x; w < ne * NFB * npm; w += blockDim.x) {
    const int el = w / (NFB * npm);
    const int rem = w - el * NFB * npm;
    const int fb = rem / npm, zz = rem - fb * npm;
    const int z0 = zz % qfm, z1 = zz / qfm;
    const int k = K0 + fb, ax = k >> 1;
    const FaceSlot sl = mt->slot[el * 2 * DIM + k];
    const int qf = sl.qf;
    if (z0 >= qf || z1 >= qf) continue;
    const int npts = DIM == 2 ? qf : qf * qf;
    const int z = z0 + qf * z1;
    const bool fq_fine = qf != Q;
    const T* fq = F0 + el * PER + fb * FB;
    const T* src = fq_fine ? fq + 4 * (QF1 + FT) : fq;
    const int fs = fq_fine ? FMAX : QF1;
    const int zc = canon(DIM, sl.side, sl.orient, qf, z0, z1);
    const int64_t go = a.f_goff[sl.face];
    const T* c = a.fgeo + go + (int64_t)(1 + sl.side * DIM) * npts + zc;
    T g = c[(int64_t)ax * npts] * src[fs + z];
    if (!orth) {
      int t0, t1;
      tang_axes<DIM>(ax, t0, t1);
      g += c[(int64_t)t0 * npts] * src[2 * fs + z];
      if constexpr (DIM == 3) g += c[(int64_t)t1 * npts] * src[3 * fs + z];
    }
    T* tr = a.trace + rhs * a.trace_stride + 4 * a.f_troff[sl.face] + (int64_t)(2 * sl.side) * npts + zc;
    tr[0] = src[z];
    tr[npts] = g;
  }
  __syncthreads();
}

template <typename T, int DIM, int N>
__device__ void trace_tile(const ApplyArgs<T>& a, const Tile& t, int rhs, T* tb, TileMeta* mt, T* sm) {
  using S = Shape<DIM, N>;
  constexpr int PER = S::PER_TRACE;
  const int ne = t.count;
  load_meta<DIM>(a.elist, a.slots, t, mt);
  load_tables<T, N>(tb);
  for (int w = threadIdx.x; w < ne * S::NV; w += blockDim.x) {
    const int el = w / S::NV, i = w - el * S::NV;
    sm[el * PER + i] = a.x[rhs * a.ndof + a.dof_off[mt->eid[el]] + i];
  }
  __syncthreads();
  // one output per thread (2D, and FP64 in 3D: more parallel work for the narrow
  // FP64 pipe) or one line per thread with the matrices as constant-bank operands
  // (FP32 in 3D: fewer instructions per FMA)
  T* U;
  if constexpr (!line_mode<T, DIM>()) U = interp_to_gauss<T, DIM, N>(sm, sm + S::QV, PER, ne, tb);
  else U = to_gauss<T, DIM, N>(sm, sm + S::QV, PER, ne);
  if (a.ug) {
    for (int w = threadIdx.x; w < ne * S::QV; w += blockDim.x) {
      const int el = w / S::QV, q = w - el * S::QV;
      a.ug[rhs * a.nquad + a.quad_off[mt->eid[el]] + q] = U[el * PER + q];
    }
  }
  if constexpr (DIM == 2) {
    trace_faces<T, DIM, N, 0>(a, t, mt, rhs, tb, sm, U);
  } else {
    trace_faces<T, DIM, N, 0>(a, t, mt, rhs, tb, sm, U);
    trace_faces<T, DIM, N, 1>(a, t, mt, rhs, tb, sm, U);
    trace_faces<T, DIM, N, 2>(a, t, mt, rhs, tb, sm, U);
    trace_faces<T, DIM, N, 3>(a, t, mt, rhs, tb, sm, U);
    trace_faces<T, DIM, N, 4>(a, t, mt, rhs, tb, sm, U);
    trace_faces<T, DIM, N, 5>(a, t, mt, rhs, tb, sm, U);
  }
}

// ============================================================ main kernel
template <typename T, int DIM, int N, int K0>
__device__ __forceinline__ void lift_faces(const ApplyArgs<T>& a, const Tile& t, const TileMeta* mt, int rhs,
                                           const T* tb, T* sm) {
  using S = Shape<DIM, N>;
  constexpr int Q = S::Q, QV = S::QV, QF1 = S::QF1, FMAX = S::FMAX, FT = S::FT, NFB = S::NFB;
  constexpr int PER = S::PER_MAIN, NF = 1 + DIM;  // fields: s, c_0 t, .., c_{d-1} t
  constexpr int FB = NF * (QF1 + FT + FMAX);       // per face: Fq [NF][QF1], Ft [NF][FT], Ff [NF][FMAX]
  const int ne = t.count;
  const int qfm = t.flags & kTileQfMask;
  const bool fine = t.flags & kTileFine;
  const bool orth = t.flags & kTileOrth;  // only s and c_a t are non-zero
  const int npm = DIM == 2 ? qfm : qfm * qfm;
  T* const F0 = sm + (1 + DIM) * QV;
  // a. flux at the shared face points (own point order): s and c_m t
  for (int w = threadIdx.x; w < ne * NFB * npm; w += blockDim.x) {
    const int el = w / (NFB * npm);
    const int rem = w - el * NFB * npm;
    const int fb = rem / npm, zz = rem - fb * npm;
    const int z0 = zz % qfm, z1 = zz / qfm;
    const int k = K0 + fb, ax = k >> 1;
    const FaceSlot sl = mt->slot[el * 2 * DIM + k];
    const int qf = sl.qf;
    if (z0 >= qf || z1 >= qf) continue;
    const int npts = DIM == 2 ? qf : qf * qf;
    const int z = z0 + qf * z1;
    const int zc = canon(DIM, sl.side, sl.orient, qf, z0, z1);
    const T* tr = a.trace + rhs * a.trace_stride + 4 * a.f_troff[sl.face] + zc;
    const int64_t go = a.f_goff[sl.face];
    const T W = a.fgeo[go + zc];
    const T tau = a.f_tau[sl.face];
    const T uo = tr[(int64_t)(2 * sl.side) * npts];
    const T go_ = tr[(int64_t)(2 * sl.side + 1) * npts];
    T s, tt;
    if (sl.flags & kFaceBnd) {
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
    const bool ffine = qf != Q;
    T* fq = F0 + el * PER + fb * FB;
    T* dst = ffine ? fq + NF * (QF1 + FT) : fq;
    const int fs = ffine ? FMAX : QF1;
    dst[z] = s;
    const T* c = a.fgeo + go + (int64_t)(1 + sl.side * DIM) * npts + zc;
#pragma unroll
    for (int m = 0; m < DIM; ++m)
      if (!orth || m == ax) dst[(1 + m) * fs + z] = c[(int64_t)m * npts] * tt;
  }
  __syncthreads();
  // b. projection from the shared rule back to the element's own Gauss points
  if (fine) {
    if constexpr (DIM == 2) {
      for (int w = threadIdx.x; w < ne * NFB * NF * Q; w += blockDim.x) {
        const int el = w / (NFB * NF * Q);
        const int rem = w - el * NFB * NF * Q;
        const int fb = rem / (NF * Q), r2 = rem - fb * NF * Q;
        const int f = r2 / Q, r = r2 - f * Q;
        const int qf = mt->slot[el * 2 * DIM + K0 + fb].qf;
        if (qf == Q || (orth && f != 0 && f != 1 + ((K0 + fb) >> 1))) continue;
        const T* II = tb + TabLayout::II(N, qf);
        T* fq = F0 + el * PER + fb * FB;
        const T* src = fq + NF * (QF1 + FT) + f * FMAX;
        T s = 0;
        for (int z = 0; z < qf; ++z) s = fma(II[z * Q + r], src[z], s);
        fq[f * QF1 + r] = s;
      }
      __syncthreads();
    } else {
      for (int w = threadIdx.x; w < ne * NFB * NF * qfm * Q; w += blockDim.x) {
        const int el = w / (NFB * NF * qfm * Q);
        const int rem = w - el * NFB * NF * qfm * Q;
        const int fb = rem / (NF * qfm * Q), r2 = rem - fb * NF * qfm * Q;
        const int f = r2 / (qfm * Q), r3 = r2 - f * qfm * Q;
        const int z1 = r3 / Q, r0 = r3 - z1 * Q;
        const int qf = mt->slot[el * 2 * DIM + K0 + fb].qf;
        if (qf == Q || z1 >= qf || (orth && f != 0 && f != 1 + ((K0 + fb) >> 1))) continue;
        const T* II = tb + TabLayout::II(N, qf);
        T* fq = F0 + el * PER + fb * FB;
        const T* src = fq + NF * (QF1 + FT) + f * FMAX + qf * z1;
        T s = 0;
        for (int z0 = 0; z0 < qf; ++z0) s = fma(II[z0 * Q + r0], src[z0], s);
        fq[NF * QF1 + f * FT + z1 * Q + r0] = s;
      }
      __syncthreads();
      for (int w = threadIdx.x; w < ne * NFB * NF * QF1; w += blockDim.x) {
        const int el = w / (NFB * NF * QF1);
        const int rem = w - el * NFB * NF * QF1;
        const int fb = rem / (NF * QF1), r2 = rem - fb * NF * QF1;
        const int f = r2 / QF1, r = r2 - f * QF1;
        const int r0 = r % Q, r1 = r / Q;
        const int qf = mt->slot[el * 2 * DIM + K0 + fb].qf;
        if (qf == Q || (orth && f != 0 && f != 1 + ((K0 + fb) >> 1))) continue;
        const T* II = tb + TabLayout::II(N, qf);
        T* fq = F0 + el * PER + fb * FB;
        const T* src = fq + NF * QF1 + f * FT + r0;
        T s = 0;
        for (int z1 = 0; z1 < qf; ++z1) s = fma(II[z1 * Q + r1], src[z1 * Q], s);
        fq[f * QF1 + r] = s;
      }
      __syncthreads();
    }
  }
  // c. extrude along the normal with l_r(+-1) into U (field s) and G_m (fields c_m t)
  const T* LL = tb + TabLayout::LL(N);
  for (int w = threadIdx.x; w < ne * QV; w += blockDim.x) {
    const int el = w / QV, q = w - el * QV;
    T* base = sm + el * PER;
    T acc[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) acc[f] = base[f * QV + q];
#pragma unroll
    for (int fb = 0; fb < NFB; ++fb) {
      const int k = K0 + fb, ax = k >> 1, sd = k & 1;
      int t0, t1;
      tang_axes<DIM>(ax, t0, t1);
      const int qa = (q / qpow<Q>(ax)) % Q;
      const int j = (q / qpow<Q>(t0)) % Q + (DIM == 3 ? Q * ((q / qpow<Q>(t1)) % Q) : 0);
      const T l = LL[sd * Q + qa];
      const T* fq = F0 + el * PER + fb * FB;
      acc[0] = fma(l, fq[j], acc[0]);
#pragma unroll
      for (int m = 0; m < DIM; ++m)
        if (!orth || m == ax) acc[1 + m] = fma(l, fq[(1 + m) * QF1 + j], acc[1 + m]);
    }
#pragma unroll
    for (int f = 0; f < NF; ++f) base[f * QV + q] = acc[f];
  }
  __syncthreads();
}

template <typename T, int DIM, int N>
__device__ void main_tile(const ApplyArgs<T>& a, const Tile& t, int rhs, T* tb, TileMeta* mt, T* sm) {
  using S = Shape<DIM, N>;
  constexpr int Q = S::Q, QV = S::QV, NV = S::NV, PER = S::PER_MAIN;
  const int ne = t.count;
  // per element: U [QV], G_0..G_{DIM-1} [QV each], face buffers
  T* U = sm;
  T* G0 = sm + QV;
  T* G1 = sm + 2 * QV;
  T* G2 = sm + 3 * QV;
  load_meta<DIM>(a.elist, a.slots, t, mt);
  load_tables<T, N>(tb);
  if (a.ug) {
    for (int w = threadIdx.x; w < ne * QV; w += blockDim.x) {
      const int el = w / QV, q = w - el * QV;
      U[el * PER + q] = a.ug[rhs * a.nquad + a.quad_off[mt->eid[el]] + q];
    }
    __syncthreads();
  } else {
    // recompute the Gauss values: 2D G0 -> G1 -> U, 3D G0 -> G1 -> G2 -> U
    for (int w = threadIdx.x; w < ne * NV; w += blockDim.x) {
      const int el = w / NV, i = w - el * NV;
      G0[el * PER + i] = a.x[rhs * a.ndof + a.dof_off[mt->eid[el]] + i];
    }
    __syncthreads();
    const T* BT = tb + TabLayout::BT(N);
    if constexpr (DIM == 2) {
      cpt<T, N, N, 1, 0, Q, false>(G0, G1, PER, ne, BT);
      __syncthreads();
      cpt<T, Q, N, 1, 1, Q, false>(G1, U, PER, ne, BT);
    } else if constexpr (!line_mode<T, DIM>()) {
      cpt<T, N, N, N, 0, Q, false>(G0, G1, PER, ne, BT);
      __syncthreads();
      cpt<T, Q, N, N, 1, Q, false>(G1, G2, PER, ne, BT);
      __syncthreads();
      cpt<T, Q, Q, N, 2, Q, false>(G2, U, PER, ne, BT);
    } else {
      contract<T, N, N, N, 0, Q, tab_B(N), false, false>(G0, G1, PER, ne);
      __syncthreads();
      contract<T, Q, N, N, 1, Q, tab_B(N), false, false>(G1, G2, PER, ne);
      __syncthreads();
      contract<T, Q, Q, N, 2, Q, tab_B(N), false, false>(G2, U, PER, ne);
    }
    __syncthreads();
  }
  // reference gradient by collocation
  {
    const T* DT = tb + TabLayout::DT(N);
    if constexpr (DIM == 2) {
      cpt<T, Q, Q, 1, 0, Q, false>(U, G0, PER, ne, DT);
      cpt<T, Q, Q, 1, 1, Q, false>(U, G1, PER, ne, DT);
    } else if constexpr (!line_mode<T, DIM>()) {
      cpt<T, Q, Q, Q, 0, Q, false>(U, G0, PER, ne, DT);
      cpt<T, Q, Q, Q, 1, Q, false>(U, G1, PER, ne, DT);
      cpt<T, Q, Q, Q, 2, Q, false>(U, G2, PER, ne, DT);
    } else {
      (void)DT;
      contract<T, Q, Q, Q, 0, Q, tab_D(Q), false, false>(U, G0, PER, ne);
      contract<T, Q, Q, Q, 1, Q, tab_D(Q), false, false>(U, G1, PER, ne);
      contract<T, Q, Q, Q, 2, Q, tab_D(Q), false, false>(U, G2, PER, ne);
    }
  }
  __syncthreads();
  // pointwise: q = kappa G grad_ref u, r = lambda w|J| u
  for (int w = threadIdx.x; w < ne * QV; w += blockDim.x) {
    const int el = w / QV, q = w - el * QV;
    const int e = mt->eid[el];
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
  }
  __syncthreads();
  // faces: flux, projection, extrusion into U and G
  if constexpr (DIM == 2) {
    lift_faces<T, DIM, N, 0>(a, t, mt, rhs, tb, sm);
  } else {
    lift_faces<T, DIM, N, 0>(a, t, mt, rhs, tb, sm);
    lift_faces<T, DIM, N, 1>(a, t, mt, rhs, tb, sm);
    lift_faces<T, DIM, N, 2>(a, t, mt, rhs, tb, sm);
    lift_faces<T, DIM, N, 3>(a, t, mt, rhs, tb, sm);
    lift_faces<T, DIM, N, 4>(a, t, mt, rhs, tb, sm);
    lift_faces<T, DIM, N, 5>(a, t, mt, rhs, tb, sm);
  }
  // U += sum_m D_m^T G_m
  if constexpr (line_mode<T, DIM>()) {
    contract<T, Q, Q, Q, 0, Q, tab_D(Q), true, true>(G0, U, PER, ne);
    __syncthreads();
    contract<T, Q, Q, Q, 1, Q, tab_D(Q), true, true>(G1, U, PER, ne);
    __syncthreads();
    contract<T, Q, Q, Q, 2, Q, tab_D(Q), true, true>(G2, U, PER, ne);
    __syncthreads();
  } else {
    // one item per Gauss point reads all DIM fields
    const T* DD = tb + TabLayout::DD(N);
    for (int w = threadIdx.x; w < ne * QV; w += blockDim.x) {
      const int el = w / QV, q = w - el * QV;
      const int q0 = q % Q, q1 = (q / Q) % Q, q2 = q / (Q * Q);
      const T* b = sm + el * PER;
      T acc = b[q];
      const T* g0 = b + QV + q - q0;
#pragma unroll
      for (int r = 0; r < Q; ++r) acc = fma(DD[r * Q + q0], g0[r], acc);
      const T* g1 = b + 2 * QV + q - q1 * Q;
#pragma unroll
      for (int r = 0; r < Q; ++r) acc = fma(DD[r * Q + q1], g1[r * Q], acc);
      if constexpr (DIM == 3) {
        const T* g2 = b + 3 * QV + q - q2 * Q * Q;
#pragma unroll
        for (int r = 0; r < Q; ++r) acc = fma(DD[r * Q + q2], g2[r * Q * Q], acc);
      }
      sm[el * PER + q] = acc;
    }
    __syncthreads();
  }
  // y = (B^T x B^T (x B^T)) U
  const T* BB = tb + TabLayout::BB(N);
  T* res;
  if constexpr (DIM == 2) {
    cpt<T, Q, Q, 1, 0, N, false>(U, G0, PER, ne, BB);
    __syncthreads();
    cpt<T, N, Q, 1, 1, N, false>(G0, G1, PER, ne, BB);
    res = G1;
  } else if constexpr (!line_mode<T, DIM>()) {
    cpt<T, Q, Q, Q, 0, N, false>(U, G0, PER, ne, BB);
    __syncthreads();
    cpt<T, N, Q, Q, 1, N, false>(G0, G1, PER, ne, BB);
    __syncthreads();
    cpt<T, N, N, Q, 2, N, false>(G1, G2, PER, ne, BB);
    res = G2;
  } else {
    (void)BB;
    contract<T, Q, Q, Q, 0, N, tab_B(N), true, false>(U, G0, PER, ne);
    __syncthreads();
    contract<T, N, Q, Q, 1, N, tab_B(N), true, false>(G0, G1, PER, ne);
    __syncthreads();
    contract<T, N, N, Q, 2, N, tab_B(N), true, false>(G1, G2, PER, ne);
    res = G2;
  }
  __syncthreads();
  for (int w = threadIdx.x; w < ne * NV; w += blockDim.x) {
    const int el = w / NV, i = w - el * NV;
    a.y[rhs * a.ndof + a.dof_off[mt->eid[el]] + i] = res[el * PER + i];
  }
}

// Shared memory of a CTA: [table block of its order (table_block_bytes)][TileMeta
// (kMetaBytes)][elements].
#define SIP_ORDER_SWITCH(FN) \
  switch (t.n) {             \
    case 2: FN(2); break;    \
    case 3: FN(3); break;    \
    case 4: FN(4); break;    \
    case 5: FN(5); break;    \
    case 6: FN(6); break;    \
    case 7: FN(7); break;    \
    case 8: FN(8); break;    \
    case 9: FN(9); break;    \
    default: break;          \
  }

template <typename T, int DIM>
__global__ void __launch_bounds__(256) k_trace(ApplyArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Tile t = a.tiles[blockIdx.x];
  const int rhs = blockIdx.y;
  T* tb = reinterpret_cast<T*>(smem_raw);
#define SIP_TRACE_CASE(NN)                                                                              \
  trace_tile<T, DIM, NN>(a, t, rhs, tb, reinterpret_cast<TileMeta*>(smem_raw + table_block_bytes(sizeof(T), NN)), \
                         reinterpret_cast<T*>(smem_raw + table_block_bytes(sizeof(T), NN) + kMetaBytes))
  SIP_ORDER_SWITCH(SIP_TRACE_CASE)
#undef SIP_TRACE_CASE
}

template <typename T, int DIM>
__global__ void __launch_bounds__(256) k_main(ApplyArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Tile t = a.tiles[blockIdx.x];
  const int rhs = blockIdx.y;
  T* tb = reinterpret_cast<T*>(smem_raw);
#define SIP_MAIN_CASE(NN)                                                                              \
  main_tile<T, DIM, NN>(a, t, rhs, tb, reinterpret_cast<TileMeta*>(smem_raw + table_block_bytes(sizeof(T), NN)), \
                        reinterpret_cast<T*>(smem_raw + table_block_bytes(sizeof(T), NN) + kMetaBytes))
  SIP_ORDER_SWITCH(SIP_MAIN_CASE)
#undef SIP_MAIN_CASE
}

}  // namespace sip
