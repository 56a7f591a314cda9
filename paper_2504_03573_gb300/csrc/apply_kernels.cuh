// Matrix-free SIP Helmholtz apply, y = A x, on quad (DIM = 2) and hex
// (DIM = 3) elements with per-element order.  Two phases per apply, run as two
// kernels chained by programmatic dependent launch, or as one cooperative
// kernel (k_apply) with a grid-wide barrier between them (written below for
// Gauss points; the Gauss-Lobatto variant follows further down):
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
// independent items (FP32 in 3D: one line of Q outputs per work item, with the
// matrices as constant-bank operands).  The 1D matrices live in shared memory
// in layouts where the lanes of a warp (consecutive outputs) read consecutive
// addresses.  Elements are grouped in tiles of equal order and point count (the
// paper's element groups); a CTA runs one or more tiles of one (N, Q) per
// right-hand side (grid.y); a switch on (N, Q) selects the compile-time
// specialisation (Sec. 5.1, "separate kernels for different orders").
//
// Point rules: Gauss-Legendre (TracePhysEval / TraceIProduct, Sec. 3.2) or, in
// the translation units built with SIP_TU_RULE = SIP_RULE_GLL, Gauss-Lobatto-
// Legendre points, whose boundary points are the face points: the trace
// kernel then gathers u on the face instead of extrapolating it, and the main
// kernel scatters the flux (s into the mass field, c t into the gradient
// fields) before the one transposed gradient + IProduct (GathrInterp /
// ScatrInterp, Sec. 3.2, Sec. 5.1).  kTileForce sends every face through the
// interpolation path, also where its rule is the element's own (identity
// interpolation): the paper's measure of the cost of non-conforming faces.
//
// Template flag P2P: the point-to-point interpolation variant (Sec. 3.3), where
// each side keeps its own face rule; the shared-rule kernels contain none of
// its code.  Both kernels start with programmatic dependent launch in mind:
// they load their tables, then wait for the previous kernel in the stream
// (griddepcontrol) before reading anything another kernel writes.
#pragma once

#include "common.cuh"

namespace sip {

// contraction style: line per thread (FP32, 3D) or output per thread (otherwise)
template <typename T, int DIM>
__host__ __device__ constexpr bool line_mode() { return DIM == 3 && std::is_same<T, float>::value; }

// face stages of the main kernel over the tile's dense face lists (FP64, where
// every idle lane of an FP64 instruction costs as much as a busy one) or over
// all faces with the others skipped (FP32, where the list's index arithmetic
// costs more than the idle lanes)
template <typename T>
__host__ __device__ constexpr bool dense_faces() { return std::is_same<T, double>::value; }

// ---- per-order compile-time shape
template <int DIM, int N, int Q_>
struct Shape {
  static constexpr int Q = Q_;
  static constexpr int NV = cpow(N, DIM);
  static constexpr int QV = cpow(Q, DIM);
  static constexpr int QF1 = cpow(Q, DIM - 1);       // own points on one face
  static constexpr int FMAX = cpow(kQMax, DIM - 1);  // points on one face at the finest rule
  static constexpr int FT = DIM == 3 ? kQMax * Q : 0;
  static constexpr int NFACE = 2 * DIM;
  static constexpr int PER_TRACE = per_elem_trace(DIM, N, Q_);
  static constexpr int PER_MAIN = per_elem_main(DIM, N, Q_);
};

// Copy this order's 1D tables from __constant__ into the CTA's table block: the
// face-rule interpolations up to the finest rule fmax of the CTA's tiles (from
// the identity F = Q on when interpolation is forced), the weights up to fmax.
// The source is the rule's tables in global memory (gtab: the __constant__
// layout; gw: [kQMax+1][kQMax] weights): consecutive threads read consecutive
// entries, one coalesced round, where the constant bank would serialise the
// warp's 32 different addresses.
template <typename T, int N, int Q>
__device__ __forceinline__ void load_tables(T* tb, int fmax, bool force, const T* __restrict__ gtab,
                                            const T* __restrict__ gw) {
  for (int w = threadIdx.x; w < N * Q; w += blockDim.x) {
    const int q = w / N, i = w - q * N;  // B[q][i]
    const T v = gtab[tab_B(N, Q) + w];
    tb[TabLayout::BT(N, Q) + i * Q + q] = v;
    tb[TabLayout::BB(N, Q) + q * N + i] = v;
  }
  for (int w = threadIdx.x; w < Q * Q; w += blockDim.x) {
    const int q = w / Q, r = w - q * Q;  // D[q][r]
    const T v = gtab[tab_D(Q) + w];
    tb[TabLayout::DT(N, Q) + r * Q + q] = v;
    tb[TabLayout::DD(N, Q) + q * Q + r] = v;
  }
  for (int w = threadIdx.x; w < 4 * Q; w += blockDim.x) tb[TabLayout::LL(N, Q) + w] = gtab[tab_L(Q) + w];
  for (int f = force ? Q : Q + 1; f <= fmax; ++f) {
    const int io = c_ioff[Q][f];  // the same for every thread: a broadcast
    for (int w = threadIdx.x; w < f * Q; w += blockDim.x) {
      const int z = w / Q, r = w - z * Q;  // I[z][r]
      const T v = gtab[io + w];
      tb[TabLayout::IT(N, Q, f) + r * f + z] = v;
      tb[TabLayout::II(N, Q, f) + z * Q + r] = v;
    }
  }
  for (int f = Q; f <= fmax; ++f)
    for (int z = threadIdx.x; z < f; z += blockDim.x) tb[TabLayout::GW(N, Q, f) + z] = gw[f * kQMax + z];
  __syncthreads();
}

// out(el)[o] (+)= sum_j M[j][k(o)] in(el)[line(o) + j SI], one work item per
// output o of every element; in(el) and out(el) give the element's [E2][E1][E0]
// arrays (E0 fastest; shared or global memory) whose AX extent is NIN (in) and
// NOUT (out).  M is a [NIN][NOUT] shared table.
template <typename T, int E0, int E1, int E2, int AX, int NOUT, bool ACC, typename InF, typename OutF>
__device__ __forceinline__ void cpt_io(InF in, OutF out, int ne, const T* __restrict__ M) {
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
    const T* src = in(el) + bi;
    T* dst = out(el);
    T acc = ACC ? dst[o] : T(0);
#pragma unroll
    for (int j = 0; j < NIN; ++j) acc = fma(M[j * NOUT + k], src[j * SI], acc);
    dst[o] = acc;
  }
}

template <typename T, int E0, int E1, int E2, int AX, int NOUT, bool ACC>
__device__ __forceinline__ void cpt(const T* __restrict__ in, T* __restrict__ out, int stride, int ne,
                                    const T* __restrict__ M) {
  cpt_io<T, E0, E1, E2, AX, NOUT, ACC>([&](int el) { return in + el * stride; },
                                       [&](int el) { return out + el * stride; }, ne, M);
}

// GLL coefficients in bA (N^DIM) -> Gauss values (Q^DIM); bB scratch.  Returns
// the buffer holding the result.
template <typename T, int DIM, int N, int Q>
__device__ __forceinline__ T* interp_to_gauss(T* bA, T* bB, int stride, int ne, const T* tb) {
  const T* BT = tb + TabLayout::BT(N, Q);
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

// a face whose rule is the element's own Q-point rule and that skips the
// interpolation path (every face goes through it under kTileForce)
template <int Q>
__device__ __forceinline__ bool own_rule(int qf, bool force) { return qf == Q && !force; }

// ============================================================ trace kernel
// The tile's element and slot descriptors in shared memory (meta_bytes(DIM),
// after the table block): element ids, DOF / geometry / volume-point offsets,
// face slots with their trace and geometry offsets and penalties.
template <int DIM>
struct TileMeta {
  ElemDesc* e_;  // [cmax] in shared memory
  SlotDesc* s_;  // [cmax][2 DIM] in shared memory
  __device__ __forceinline__ const FaceSlot& slot(int i) const { return s_[i].slot; }
  __device__ __forceinline__ int64_t troff(int i) const { return s_[i].troff; }
  __device__ __forceinline__ int64_t goff(int i) const { return s_[i].goff; }
  __device__ __forceinline__ double tau(int i) const { return s_[i].tau; }
  __device__ __forceinline__ int eid(int el) const { return e_[el].eid; }
  __device__ __forceinline__ int aff(int el) const { return e_[el].aff; }
  __device__ __forceinline__ int64_t dof(int el) const { return e_[el].dof_off; }
  __device__ __forceinline__ int64_t vgo(int el) const { return e_[el].vgoff; }
  __device__ __forceinline__ int64_t qoff(int el) const { return e_[el].quad_off; }
};

// Copy the tile's descriptors (two contiguous blocks, 16-byte vector loads) and,
// where the tile has faces on the interpolation path and `list` is given, its
// face list.
template <int DIM>
__device__ __forceinline__ void load_meta(const ElemDesc* desc_e, const SlotDesc* desc_s, const uint16_t* flists,
                                          const Tile& t, TileMeta<DIM>* mt, uint16_t* list) {
  const uint16_t* fl = flists + t.flist;
  const int len = list && (t.flags & kTileFine) ? 3 + 2 * fl[2] + fl[0] + fl[1] : 0;
  constexpr int VE = sizeof(ElemDesc) / 16, VS = sizeof(SlotDesc) / 16;
  const uint4* ge = reinterpret_cast<const uint4*>(desc_e + t.start);
  const uint4* gs = reinterpret_cast<const uint4*>(desc_s + (int64_t)t.start * 2 * DIM);
  uint4* se = reinterpret_cast<uint4*>(mt->e_);
  uint4* ss = reinterpret_cast<uint4*>(mt->s_);
  const int ne = t.count * VE, ns = t.count * 2 * DIM * VS;
  for (int w = threadIdx.x; w < ne + ns; w += blockDim.x) {
    if (w < ne) se[w] = ge[w];
    else ss[w - ne] = gs[w - ne];
  }
  for (int w = threadIdx.x; w < len; w += blockDim.x) list[w] = fl[w];
}

// The tile's faces as dense work lists: the conforming ones, and the ones with
// a finer shared rule grouped by that rule (entries fl_el / fl_k / fl_qf).
struct FaceList {
  const uint16_t* r;
  __device__ __forceinline__ int nconf() const { return r[0]; }
  __device__ __forceinline__ int nfine() const { return r[1]; }
  __device__ __forceinline__ int conf(int i) const { return r[3 + 2 * r[2] + i]; }
  __device__ __forceinline__ int fine(int i) const { return r[3 + 2 * r[2] + r[0] + i]; }
  // work items of all fine faces, items(qf) per face
  template <typename F>
  __device__ __forceinline__ int fine_items(F items) const {
    int n = 0;
    for (int g = 0; g < r[2]; ++g) n += r[4 + 2 * g] * items(r[3 + 2 * g]);
    return n;
  }
  // fine face j and its item u for work item w < fine_items(items)
  template <typename F>
  __device__ __forceinline__ void fine_at(F items, int w, int& j, int& u) const {
    int j0 = 0;
    for (int g = 0; g < r[2]; ++g) {
      const int per = items(r[3 + 2 * g]), cnt = r[4 + 2 * g];
      if (w < cnt * per) {
        const int q = w / per;
        j = j0 + q;
        u = w - q * per;
        return;
      }
      w -= cnt * per;
      j0 += cnt;
    }
    j = 0;
    u = 0;
  }
};

// face geometry at canonical point zc: W, and component m of c on the given side
template <typename T>
struct FaceGeo {
  const T* g;
  int npts, zc, side, dim;
  bool aff;
  T w;  // Gauss weight of the point (affine faces)
  __device__ __forceinline__ T W() const { return aff ? g[0] * w : g[zc]; }
  __device__ __forceinline__ T c(int m) const {
    const int comp = 1 + side * dim + m;
    return aff ? g[comp] : g[(int64_t)comp * npts + zc];
  }
};

// points of one face at a q-point rule per direction
template <int DIM>
__device__ __forceinline__ int face_npts(int q) { return DIM == 2 ? q : q * q; }

// Point-to-point interpolation variant (SIP_FACES_P2P).  Face geometry of an
// interior face: [W-, c-] at the minus side's own points, then [W+, c+] at the
// plus side's (boundary and affine faces as with a shared rule).  Trace slot:
// one block per side, [u, g, u~, g~] at that side's own points, u~ and g~ being
// the other side's values interpolated to them by the other side's trace kernel
// (read from the other side's own block instead where both rules are equal).
template <typename T>
struct FaceGeoP2P {
  const T* g;   // this side's W values (affine: the face's constants)
  const T* gc;  // this side's c values [dim][npts]
  int npts, zc, side, dim;
  bool aff;
  T w;
  __device__ __forceinline__ T W() const { return aff ? g[0] * w : g[zc]; }
  __device__ __forceinline__ T c(int m) const { return aff ? g[1 + side * dim + m] : gc[(int64_t)m * npts + zc]; }
};
// npm: points of the minus side's own rule
template <typename T, int DIM>
__device__ __forceinline__ FaceGeoP2P<T> face_geo_p2p(const ApplyArgs<T>& a, const FaceSlot& sl, int64_t goff, int npts,
                                                      int npm, int zc, T w) {
  const T* g = a.fgeo + goff;
  const bool aff = (sl.flags & kFaceAffine) != 0;
  if (aff) return FaceGeoP2P<T>{g, g, npts, zc, sl.side, DIM, true, w};
  if (sl.flags & kFaceBnd) return FaceGeoP2P<T>{g, g + npts, npts, zc, 0, DIM, false, w};
  const T* gw = g + (int64_t)sl.side * (1 + DIM) * npm;
  return FaceGeoP2P<T>{gw, gw + npts, npts, zc, sl.side, DIM, false, w};
}
// offset of this side's block in the face's trace slot
__device__ __forceinline__ int64_t p2p_own_block(int side, int npm) { return (int64_t)side * 4 * npm; }

// Trace values of all 2 DIM faces of every element of the tile.  Conforming
// faces (shared rule = own Q points) go straight from the per-face buffer to the
// trace; faces with a finer shared rule are interpolated one face at a time in
// the element's scratch.
template <typename T, int DIM, int N, int Q, bool P2P>
__device__ __forceinline__ void trace_all_faces(const ApplyArgs<T>& a, const Tile& t, const TileMeta<DIM>* mt, int rhs,
                                                const T* tb, T* sm, const T* U) {
  using S = Shape<DIM, N, Q>;
  constexpr int QF1 = S::QF1, FMAX = S::FMAX, FT = S::FT, NFACE = S::NFACE, PER = S::PER_TRACE;
  const int ne = t.count;
  const int qfm = t.flags & kTileQfMask;
  const bool fine = t.flags & kTileFine;
  const bool orth = t.flags & kTileOrth;
  const bool force = t.flags & kTileForce;
  const int npm = DIM == 2 ? qfm : qfm * qfm;
  // per element: Fq [NFACE][4][QF1] (u, du/dn_ref, two tangential derivatives), then scratch
  T* const F0 = sm + 2 * S::QV;
  constexpr int SC = NFACE * 4 * QF1;  // scratch offset from F0: Ft [4][FT], Ff [4][FMAX]
  // normal derivative c . grad_ref u from (u, du/dn_ref, tangential derivatives)
  // and store both at canonical point zc
  auto emit_vals = [&](int el, int k, int z0, int z1, T uv, T dn, T d0, T d1) {
    const int si = el * 2 * DIM + k;
    const FaceSlot sl = mt->slot(si);
    const int qf = sl.qf, ax = k >> 1;
    const int npts = DIM == 2 ? qf : qf * qf;
    const int zc = canon(DIM, sl.side, sl.orient, qf, z0, z1);
    if constexpr (P2P) {
      const int npm = face_npts<DIM>(sl.side ? face_oq(sl.flags) : qf);
      const FaceGeoP2P<T> fg = face_geo_p2p<T, DIM>(a, sl, mt->goff(si), npts, npm, zc, T(0));
      T g = fg.c(ax) * dn;
      if (!orth) {
        int t0, t1;
        tang_axes<DIM>(ax, t0, t1);
        g += fg.c(t0) * d0;
        if constexpr (DIM == 3) g += fg.c(t1) * d1;
      }
      T* tr = a.trace + rhs * a.trace_stride + 4 * mt->troff(si) + p2p_own_block(sl.side, npm) + zc;
      tr[0] = uv;
      tr[npts] = g;
    } else {
      FaceGeo<T> fg{a.fgeo + mt->goff(si), npts, zc, sl.side, DIM, (sl.flags & kFaceAffine) != 0, T(0)};
      T g = fg.c(ax) * dn;
      if (!orth) {
        int t0, t1;
        tang_axes<DIM>(ax, t0, t1);
        g += fg.c(t0) * d0;
        if constexpr (DIM == 3) g += fg.c(t1) * d1;
      }
      T* tr = a.trace + rhs * a.trace_stride + 4 * mt->troff(si) + (int64_t)(2 * sl.side) * npts + zc;
      tr[0] = uv;
      tr[npts] = g;
    }
  };
  auto emit = [&](int el, int k, const T* src, int fs, int z0, int z1) {
    const int z = z0 + mt->slot(el * 2 * DIM + k).qf * z1;
    emit_vals(el, k, z0, z1, src[z], src[fs + z], orth ? T(0) : src[2 * fs + z],
              (DIM == 3 && !orth) ? src[3 * fs + z] : T(0));
  };
  const T* LL = tb + TabLayout::LL(N, Q);
  const T* DT = tb + TabLayout::DT(N, Q);
  // 1. value and reference normal derivative at the element's own face points
  //    (orthogonal conforming faces need nothing else and are stored at once)
  for (int w = threadIdx.x; w < ne * NFACE * QF1; w += blockDim.x) {
    const int el = w / (NFACE * QF1);
    const int rem = w - el * NFACE * QF1;
    const int k = rem / QF1, j = rem - k * QF1;
    const int ax = k >> 1, sd = k & 1;
    int t0, t1;
    tang_axes<DIM>(ax, t0, t1);
    const int j0 = j % Q, j1 = j / Q;
    const int sa = qpow<Q>(ax);
    const T* u = U + el * PER + j0 * qpow<Q>(t0) + (DIM == 3 ? j1 * qpow<Q>(t1) : 0);
    T uf = 0, dn = 0;
    if constexpr (kGatherScatter) {
      // the face points are the volume points of this boundary plane: gather
      uf = u[(sd ? Q - 1 : 0) * sa];
#pragma unroll
      for (int r = 0; r < Q; ++r) dn = fma(LL[(2 + sd) * Q + r], u[r * sa], dn);
    } else {
#pragma unroll
      for (int r = 0; r < Q; ++r) {
        const T v = u[r * sa];
        uf = fma(LL[sd * Q + r], v, uf);
        dn = fma(LL[(2 + sd) * Q + r], v, dn);
      }
    }
    if (orth && own_rule<Q>(mt->slot(el * 2 * DIM + k).qf, force)) {
      emit_vals(el, k, j0, j1, uf, dn, T(0), T(0));
      continue;
    }
    T* fq = F0 + el * PER + k * 4 * QF1;
    fq[j] = uf;
    fq[QF1 + j] = dn;
  }
  __syncthreads();
  // 2. tangential derivatives of the face values (collocation on the Gauss points);
  //    not needed where c has no tangential component
  if (!orth) {
    for (int w = threadIdx.x; w < ne * NFACE * (DIM - 1) * QF1; w += blockDim.x) {
      const int el = w / (NFACE * (DIM - 1) * QF1);
      const int rem = w - el * NFACE * (DIM - 1) * QF1;
      const int k = rem / ((DIM - 1) * QF1);
      const int r2 = rem - k * (DIM - 1) * QF1;
      const int m = r2 / QF1, j = r2 - m * QF1;
      const int j0 = j % Q, j1 = j / Q;
      T* fq = F0 + el * PER + k * 4 * QF1;
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
  // 3. conforming faces, all at once (orthogonal ones were stored in step 1)
  for (int w = threadIdx.x; w < (orth ? 0 : ne * NFACE * QF1); w += blockDim.x) {
    const int el = w / (NFACE * QF1);
    const int rem = w - el * NFACE * QF1;
    const int k = rem / QF1, j = rem - k * QF1;
    if (!own_rule<Q>(mt->slot(el * 2 * DIM + k).qf, force)) continue;
    emit(el, k, F0 + el * PER + k * 4 * QF1, QF1, j % Q, j / Q);
  }
  // 4. faces with a finer shared rule (p-non-conforming): NSC faces per round,
  //    each in its own scratch slot
  if (fine) {
    constexpr int NSC = scratch_slots(DIM);
    constexpr int SL = 4 * (FT + FMAX);  // one slot: Ft [4][FT], Ff [4][FMAX]
    // fields to carry to the finer rule: u and du/dn_ref, plus the tangential
    // derivatives (one in 2D, two in 3D) where c has tangential components
    const int nfld = orth ? 2 : 2 + (DIM - 1);
    for (int k0 = 0; k0 < NFACE; k0 += NSC) {
      if constexpr (DIM == 2) {
        for (int w = threadIdx.x; w < ne * NSC * nfld * qfm; w += blockDim.x) {
          const int el = w / (NSC * nfld * qfm);
          const int rem = w - el * NSC * nfld * qfm;
          const int kk = rem / (nfld * qfm), r2 = rem - kk * nfld * qfm;
          const int f = r2 / qfm, z = r2 - f * qfm;
          const int k = k0 + kk;
          const int qf = mt->slot(el * 2 * DIM + k).qf;
          if (own_rule<Q>(qf, force) || z >= qf) continue;
          const T* IT = tb + TabLayout::IT(N, Q, qf);
          const T* src = F0 + el * PER + k * 4 * QF1 + f * QF1;
          T s = 0;
#pragma unroll
          for (int r = 0; r < Q; ++r) s = fma(IT[r * qf + z], src[r], s);
          F0[el * PER + SC + kk * SL + 4 * FT + f * FMAX + z] = s;
        }
        __syncthreads();
      } else {
        for (int w = threadIdx.x; w < ne * NSC * nfld * Q * qfm; w += blockDim.x) {
          const int el = w / (NSC * nfld * Q * qfm);
          const int rem = w - el * NSC * nfld * Q * qfm;
          const int kk = rem / (nfld * Q * qfm), r2 = rem - kk * nfld * Q * qfm;
          const int f = r2 / (Q * qfm), r3 = r2 - f * Q * qfm;
          const int j1 = r3 / qfm, z0 = r3 - j1 * qfm;
          const int k = k0 + kk;
          const int qf = mt->slot(el * 2 * DIM + k).qf;
          if (own_rule<Q>(qf, force) || z0 >= qf) continue;
          const T* IT = tb + TabLayout::IT(N, Q, qf);
          const T* src = F0 + el * PER + k * 4 * QF1 + f * QF1 + j1 * Q;
          T s = 0;
#pragma unroll
          for (int r = 0; r < Q; ++r) s = fma(IT[r * qf + z0], src[r], s);
          F0[el * PER + SC + kk * SL + f * FT + j1 * kQMax + z0] = s;
        }
        __syncthreads();
        for (int w = threadIdx.x; w < ne * NSC * nfld * npm; w += blockDim.x) {
          const int el = w / (NSC * nfld * npm);
          const int rem = w - el * NSC * nfld * npm;
          const int kk = rem / (nfld * npm), r2 = rem - kk * nfld * npm;
          const int f = r2 / npm, zz = r2 - f * npm;
          const int z1 = zz / qfm, z0 = zz - z1 * qfm;
          const int k = k0 + kk;
          const int qf = mt->slot(el * 2 * DIM + k).qf;
          if (own_rule<Q>(qf, force) || z0 >= qf || z1 >= qf) continue;
          const T* IT = tb + TabLayout::IT(N, Q, qf);
          const T* src = F0 + el * PER + SC + kk * SL + f * FT + z0;
          T s = 0;
#pragma unroll
          for (int r = 0; r < Q; ++r) s = fma(IT[r * qf + z1], src[r * kQMax], s);
          F0[el * PER + SC + kk * SL + 4 * FT + f * FMAX + z0 + qf * z1] = s;
        }
        __syncthreads();
      }
      for (int w = threadIdx.x; w < ne * NSC * npm; w += blockDim.x) {
        const int el = w / (NSC * npm), r2 = w - el * NSC * npm;
        const int kk = r2 / npm, zz = r2 - kk * npm;
        const int z0 = zz % qfm, z1 = zz / qfm;
        const int k = k0 + kk;
        const int qf = mt->slot(el * 2 * DIM + k).qf;
        if (own_rule<Q>(qf, force) || z0 >= qf || z1 >= qf) continue;
        emit(el, k, F0 + el * PER + SC + kk * SL + 4 * FT, FMAX, z0, z1);
      }
      __syncthreads();
    }
  }
  __syncthreads();
}

// Point-to-point interpolation (Sec. 3.3): on every interior face whose other
// side has another rule, this side's u and g, stored just before at its own Q
// points (canonical order), are interpolated to the other side's own oq-point
// rule and written into the other side's block, where its main kernel reads
// them as the neighbour's trace.  The stored values are read back from global
// memory, visible to the whole CTA after the barrier that ends the face stages.
template <typename T, int DIM, int N, int Q>
__device__ __forceinline__ void p2p_send(const ApplyArgs<T>& a, const Tile& t, const TileMeta<DIM>* mt, int rhs) {
  constexpr int NFACE = 2 * DIM, FMAX = cpow(kQMax, DIM - 1), NP = cpow(Q, DIM - 1);
  const int ne = t.count;
  for (int w = threadIdx.x; w < ne * NFACE * FMAX; w += blockDim.x) {
    const int el = w / (NFACE * FMAX), rem = w - el * NFACE * FMAX;
    const int k = rem / FMAX, z = rem - k * FMAX;
    const FaceSlot sl = mt->slot(el * 2 * DIM + k);
    const int oq = face_oq(sl.flags);
    const int npo = face_npts<DIM>(oq);
    if ((sl.flags & kFaceBnd) || oq == Q || z >= npo) continue;
    const int npm = sl.side ? npo : NP;
    T* base = a.trace + rhs * a.trace_stride + 4 * mt->troff(el * 2 * DIM + k);
    const T* src = base + (int64_t)sl.side * 4 * npm;                // own [u][g], Q points
    T* dst = base + (sl.side ? 0 : (int64_t)4 * npm) + 2 * npo;      // the other side's [u~][g~]
    const T* I = a.p2p_I + (Q * (kQMax + 1) + oq) * (kQMax * kQMax);  // Q-point rule -> oq-point rule
    T u = 0, g = 0;
    if constexpr (DIM == 2) {
#pragma unroll 1
      for (int r = 0; r < Q; ++r) {
        const T wv = I[z * kQMax + r];
        u = fma(wv, src[r], u);
        g = fma(wv, src[NP + r], g);
      }
    } else {
      const int z0 = z % oq, z1 = z / oq;
#pragma unroll 1
      for (int r1 = 0; r1 < Q; ++r1) {
        T su = 0, sg = 0;
#pragma unroll 1
        for (int r0 = 0; r0 < Q; ++r0) {
          const T wv = I[z0 * kQMax + r0];
          su = fma(wv, src[r0 + Q * r1], su);
          sg = fma(wv, src[NP + r0 + Q * r1], sg);
        }
        const T w1 = I[z1 * kQMax + r1];
        u = fma(w1, su, u);
        g = fma(w1, sg, g);
      }
    }
    dst[z] = u;
    dst[npo + z] = g;
  }
}

template <typename T, int DIM, int N, int Q, bool P2P>
__device__ void trace_tile(const ApplyArgs<T>& a, const Tile& t, int rhs, T* tb, TileMeta<DIM>* mt, T* sm,
                           bool meta_loaded) {
  using S = Shape<DIM, N, Q>;
  constexpr int PER = S::PER_TRACE;
  const int ne = t.count;
  if (!meta_loaded) {
    load_meta<DIM>(a.desc_e, a.desc_s, a.flists, t, mt, nullptr);
    __syncthreads();
  }
  // one output per thread (2D, and FP64 in 3D: more parallel work for the narrow
  // FP64 pipe) or one line per thread with the matrices as constant-bank operands
  // (FP32 in 3D: fewer instructions per FMA)
  T* U;
  if constexpr (!line_mode<T, DIM>()) {
    // first contraction reads the coefficients straight from global memory
    constexpr int Q = S::Q;
    const T* BT = tb + TabLayout::BT(N, Q);
    T* bA = sm;
    T* bB = sm + S::QV;
    auto gx = [&](int el) { return a.x + rhs * a.ndof + mt->dof(el); };
    if constexpr (DIM == 2) {
      cpt_io<T, N, N, 1, 0, Q, false>(gx, [&](int el) { return bB + el * PER; }, ne, BT);
      __syncthreads();
      cpt<T, Q, N, 1, 1, Q, false>(bB, bA, PER, ne, BT);
      __syncthreads();
      U = bA;
    } else {
      cpt_io<T, N, N, N, 0, Q, false>(gx, [&](int el) { return bB + el * PER; }, ne, BT);
      __syncthreads();
      cpt<T, Q, N, N, 1, Q, false>(bB, bA, PER, ne, BT);
      __syncthreads();
      cpt<T, Q, Q, N, 2, Q, false>(bA, bB, PER, ne, BT);
      __syncthreads();
      U = bB;
    }
  } else {
    for (int w = threadIdx.x; w < ne * S::NV; w += blockDim.x) {
      const int el = w / S::NV, i = w - el * S::NV;
      sm[el * PER + i] = a.x[rhs * a.ndof + mt->dof(el) + i];
    }
    __syncthreads();
    U = to_gauss<T, DIM, N, Q>(sm, sm + S::QV, PER, ne);
  }
  if (a.ug) {
    for (int w = threadIdx.x; w < ne * S::QV; w += blockDim.x) {
      const int el = w / S::QV, q = w - el * S::QV;
      a.ug[rhs * a.nquad + t.qbase + (int64_t)el * S::QV + q] = U[el * PER + q];
    }
  }
  trace_all_faces<T, DIM, N, Q, P2P>(a, t, mt, rhs, tb, sm, U);
  if constexpr (P2P) p2p_send<T, DIM, N, Q>(a, t, mt, rhs);
}

// ============================================================ main kernel
// SIP flux of face k of element el at its shared point (z0, z1) (own order):
// writes s and c_m t (m = 0..DIM-1; only c_a t where the tile is orthogonal) to
// dst[f * fs + z0 + qf z1].
template <typename T, int DIM, int N, int Q>
__device__ __forceinline__ void face_flux_p2p(const ApplyArgs<T>& a, const TileMeta<DIM>* mt, int rhs, const T* tb,
                                              bool orth, int el, int k, int z0, int z1, T* dst, int fs);

template <typename T, int DIM, int N, int Q, bool P2P>
__device__ __forceinline__ void face_flux(const ApplyArgs<T>& a, const TileMeta<DIM>* mt, int rhs, const T* tb,
                                          bool orth, int el, int k, int z0, int z1, T* dst, int fs) {
  if constexpr (P2P) {
    face_flux_p2p<T, DIM, N, Q>(a, mt, rhs, tb, orth, el, k, z0, z1, dst, fs);
    return;
  }
  const int si = el * 2 * DIM + k;
  const FaceSlot sl = mt->slot(si);
  const int qf = sl.qf, ax = k >> 1;
  const int npts = DIM == 2 ? qf : qf * qf;
  const int z = z0 + qf * z1;
  const int zc = canon(DIM, sl.side, sl.orient, qf, z0, z1);
  const T* tr = a.trace + rhs * a.trace_stride + 4 * mt->troff(si) + zc;
  const bool faff = (sl.flags & kFaceAffine) != 0;
  const T* GWf = tb + TabLayout::GW(N, Q, qf);
  const T wz = faff ? (DIM == 2 ? GWf[zc] : GWf[zc % qf] * GWf[zc / qf]) : T(0);
  FaceGeo<T> fg{a.fgeo + mt->goff(si), npts, zc, sl.side, DIM, faff, wz};
  const T W = fg.W();
  const T tau = (T)mt->tau(si);
  // traces come from other CTAs (in the single-launch apply, of the same
  // kernel): read them at L2
  const T uo = __ldcg(tr + (int64_t)(2 * sl.side) * npts);
  const T go_ = __ldcg(tr + (int64_t)(2 * sl.side + 1) * npts);
  T s, tt;
  if (sl.flags & kFaceBnd) {
    // Nitsche: -(grad v.n, u) - (v, grad u.n) + tau (v, u)
    if (!a.transpose) { s = W * (tau * uo - go_); tt = -W * uo; }
    else { s = W * tau * uo - W * go_; tt = -(W * uo); }
  } else {
    const int oth = 1 - sl.side;
    const T un = __ldcg(tr + (int64_t)(2 * oth) * npts);
    const T gn = __ldcg(tr + (int64_t)(2 * oth + 1) * npts);
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
  dst[z] = s;
#pragma unroll
  for (int m = 0; m < DIM; ++m)
    if (!orth || m == ax) dst[(1 + m) * fs + z] = fg.c(m) * tt;
}

// The same flux with point-to-point interpolation: this side's own rule, the
// other side's values already interpolated to its points by the other side's
// trace kernel (rows only; the transpose apply is not defined for this variant).
template <typename T, int DIM, int N, int Q>
__device__ __forceinline__ void face_flux_p2p(const ApplyArgs<T>& a, const TileMeta<DIM>* mt, int rhs, const T* tb,
                                              bool orth, int el, int k, int z0, int z1, T* dst, int fs) {
  const int si = el * 2 * DIM + k;
  const FaceSlot sl = mt->slot(si);
  const int qf = sl.qf, ax = k >> 1;
  const int npts = DIM == 2 ? qf : qf * qf;
  const int z = z0 + qf * z1;
  const int zc = canon(DIM, sl.side, sl.orient, qf, z0, z1);
  const int oq = face_oq(sl.flags);
  const int npm = face_npts<DIM>(sl.side ? oq : qf);
  const bool faff = (sl.flags & kFaceAffine) != 0;
  const T* GWf = tb + TabLayout::GW(N, Q, qf);
  const T wz = faff ? (DIM == 2 ? GWf[zc] : GWf[zc % qf] * GWf[zc / qf]) : T(0);
  const FaceGeoP2P<T> fg = face_geo_p2p<T, DIM>(a, sl, mt->goff(si), npts, npm, zc, wz);
  const T* trf = a.trace + rhs * a.trace_stride + 4 * mt->troff(si);
  const T* tr = trf + p2p_own_block(sl.side, npm) + zc;
  const T W = fg.W();
  const T tau = (T)mt->tau(si);
  const T uo = __ldcg(tr);
  const T go_ = __ldcg(tr + npts);
  T s, tt;
  if (sl.flags & kFaceBnd) {
    s = W * (tau * uo - go_);
    tt = -W * uo;
  } else {
    const T* trn = oq == qf ? trf + p2p_own_block(1 - sl.side, npm) + zc : tr + 2 * npts;
    const T un = __ldcg(trn);
    const T gn = __ldcg(trn + npts);
    const T jmp = uo - un;
    const T avg = T(0.5) * (go_ - gn);
    s = W * (tau * jmp - avg);
    tt = T(-0.5) * W * jmp;
  }
  dst[z] = s;
#pragma unroll
  for (int m = 0; m < DIM; ++m)
    if (!orth || m == ax) dst[(1 + m) * fs + z] = fg.c(m) * tt;
}

// Flux of faces with a finer shared rule (p-non-conforming), SC slots per
// round: flux at the shared points, then projection back to the element's own
// face points (TraceIProduct) into the per-face buffers.
template <typename T, int DIM, int N, int Q, bool P2P>
__device__ __forceinline__ void lift_fine_faces(const ApplyArgs<T>& a, const Tile& t, const TileMeta<DIM>* mt,
                                                const uint16_t* flist, int rhs,
                                                const T* tb, T* F0, int per, bool orth) {
  using S = Shape<DIM, N, Q>;
  constexpr int QF1 = S::QF1, FMAX = S::FMAX, FT = S::FT, NFACE = S::NFACE, NF = 1 + DIM;
  constexpr int SC = NFACE * NF * QF1;
  constexpr int NSC = scratch_slots(DIM);
  constexpr int SL = NF * (FT + FMAX);  // one slot: Ft [NF][FT], Ff [NF][FMAX]
  const int ne = t.count;
  const int qfm = t.flags & kTileQfMask;
  const bool force = t.flags & kTileForce;
  const int npm = DIM == 2 ? qfm : qfm * qfm;
  if constexpr (DIM == 2 && dense_faces<T>()) {
    // one scratch slot per face (slot k): all fine faces at once, as dense work
    // lists grouped by the shared rule
    static_assert(DIM != 2 || NSC == NFACE, "2D keeps one scratch slot per face");
    const FaceList fl{flist};
    auto per_f = [&](int qf) { return qf; };
    for (int w = threadIdx.x; w < fl.fine_items(per_f); w += blockDim.x) {
      int j, z;
      fl.fine_at(per_f, w, j, z);
      const int e = fl.fine(j), el = fl_el(e), k = fl_k(e);
      face_flux<T, DIM, N, Q, P2P>(a, mt, rhs, tb, orth, el, k, z, 0, F0 + el * per + SC + k * SL + NF * FT, FMAX);
    }
    __syncthreads();
    // projection of the fields in use (s and c_a t where the tile is orthogonal)
    const int nfu = orth ? 2 : NF;
    for (int w = threadIdx.x; w < fl.nfine() * nfu * Q; w += blockDim.x) {
      const int j = w / (nfu * Q), r2 = w - j * nfu * Q;
      const int fi = r2 / Q, r = r2 - fi * Q;
      const int e = fl.fine(j), el = fl_el(e), k = fl_k(e), qf = fl_qf(e);
      const int f = orth && fi == 1 ? 1 + (k >> 1) : fi;
      const T* II = tb + TabLayout::II(N, Q, qf);
      const T* src = F0 + el * per + SC + k * SL + NF * FT + f * FMAX;
      T s = 0;
      for (int z = 0; z < qf; ++z) s = fma(II[z * Q + r], src[z], s);
      F0[el * per + k * NF * QF1 + f * QF1 + r] = s;
    }
    __syncthreads();
  } else {
    for (int k0 = 0; k0 < NFACE; k0 += NSC) {
      for (int w = threadIdx.x; w < ne * NSC * npm; w += blockDim.x) {
        const int el = w / (NSC * npm), r2 = w - el * NSC * npm;
        const int kk = r2 / npm, zz = r2 - kk * npm;
        const int z0 = zz % qfm, z1 = zz / qfm;
        const int k = k0 + kk;
        const int qf = mt->slot(el * 2 * DIM + k).qf;
        if (own_rule<Q>(qf, force) || z0 >= qf || z1 >= qf) continue;
        face_flux<T, DIM, N, Q, P2P>(a, mt, rhs, tb, orth, el, k, z0, z1, F0 + el * per + SC + kk * SL + NF * FT, FMAX);
      }
      __syncthreads();
      if constexpr (DIM == 2) {
        for (int w = threadIdx.x; w < ne * NSC * NF * Q; w += blockDim.x) {
          const int el = w / (NSC * NF * Q);
          const int rem = w - el * NSC * NF * Q;
          const int kk = rem / (NF * Q), r2 = rem - kk * NF * Q;
          const int f = r2 / Q, r = r2 - f * Q;
          const int k = k0 + kk;
          const int qf = mt->slot(el * 2 * DIM + k).qf;
          if (own_rule<Q>(qf, force) || (orth && f != 0 && f != 1 + (k >> 1))) continue;
          const T* II = tb + TabLayout::II(N, Q, qf);
          const T* src = F0 + el * per + SC + kk * SL + NF * FT + f * FMAX;
          T s = 0;
          for (int z = 0; z < qf; ++z) s = fma(II[z * Q + r], src[z], s);
          F0[el * per + k * NF * QF1 + f * QF1 + r] = s;
        }
        __syncthreads();
      } else {
        for (int w = threadIdx.x; w < ne * NSC * NF * qfm * Q; w += blockDim.x) {
          const int el = w / (NSC * NF * qfm * Q);
          const int rem = w - el * NSC * NF * qfm * Q;
          const int kk = rem / (NF * qfm * Q), r2 = rem - kk * NF * qfm * Q;
          const int f = r2 / (qfm * Q), r3 = r2 - f * qfm * Q;
          const int z1 = r3 / Q, r0 = r3 - z1 * Q;
          const int k = k0 + kk;
          const int qf = mt->slot(el * 2 * DIM + k).qf;
          if (own_rule<Q>(qf, force) || z1 >= qf || (orth && f != 0 && f != 1 + (k >> 1))) continue;
          const T* II = tb + TabLayout::II(N, Q, qf);
          const T* src = F0 + el * per + SC + kk * SL + NF * FT + f * FMAX + qf * z1;
          T s = 0;
          for (int z0 = 0; z0 < qf; ++z0) s = fma(II[z0 * Q + r0], src[z0], s);
          F0[el * per + SC + kk * SL + f * FT + z1 * Q + r0] = s;
        }
        __syncthreads();
        for (int w = threadIdx.x; w < ne * NSC * NF * QF1; w += blockDim.x) {
          const int el = w / (NSC * NF * QF1);
          const int rem = w - el * NSC * NF * QF1;
          const int kk = rem / (NF * QF1), r2 = rem - kk * NF * QF1;
          const int f = r2 / QF1, r = r2 - f * QF1;
          const int r0 = r % Q, r1 = r / Q;
          const int k = k0 + kk;
          const int qf = mt->slot(el * 2 * DIM + k).qf;
          if (own_rule<Q>(qf, force) || (orth && f != 0 && f != 1 + (k >> 1))) continue;
          const T* II = tb + TabLayout::II(N, Q, qf);
          const T* src = F0 + el * per + SC + kk * SL + f * FT + r0;
          T s = 0;
          for (int z1 = 0; z1 < qf; ++z1) s = fma(II[z1 * Q + r1], src[z1 * Q], s);
          F0[el * per + k * NF * QF1 + f * QF1 + r] = s;
        }
        __syncthreads();
      }
    }
  }
}

template <typename T, int DIM, int N, int Q, bool P2P>
__device__ void main_tile(const ApplyArgs<T>& a, const Tile& t, int rhs, T* tb, TileMeta<DIM>* mt, T* sm,
                          bool meta_loaded) {
  using S = Shape<DIM, N, Q>;
  constexpr int QV = S::QV, NV = S::NV, QF1 = S::QF1, NFACE = S::NFACE, PER = S::PER_MAIN;
  constexpr int NF = 1 + DIM;
  const int ne = t.count;
  const bool fine = t.flags & kTileFine;
  const bool orth = t.flags & kTileOrth;
  const bool force = t.flags & kTileForce;
  // per element: U [QV], G_0..G_{DIM-1} [QV each], R [QV], face buffers Fq
  // [NFACE][NF][QF1] (fields s, c_0 t, .., c_{d-1} t) and scratch
  T* U = sm;
  T* G0 = sm + QV;
  T* G1 = sm + 2 * QV;
  T* G2 = sm + 3 * QV;
  T* R = sm + (1 + DIM) * QV;
  T* const F0 = sm + (2 + DIM) * QV;
  // the face list follows the element buffers (kFaceListBytes, FP64 only)
  uint16_t* flist = dense_faces<T>() ? reinterpret_cast<uint16_t*>(sm + ne * PER) : nullptr;
  if (!meta_loaded) load_meta<DIM>(a.desc_e, a.desc_s, a.flists, t, mt, flist);
  if (a.ug) {
    // the trace phase stored the tile's volume-point values contiguously (the
    // tile's own range of the hand-off buffer), so they load in the same stage as
    // the descriptors, with no lookup
    const T* ug = a.ug + rhs * a.nquad + t.qbase;
    for (int w = threadIdx.x; w < ne * QV; w += blockDim.x) U[(w / QV) * PER + w % QV] = __ldcg(ug + w);
    __syncthreads();
  } else {
    __syncthreads();
    // recompute the Gauss values: 2D G0 -> G1 -> U, 3D G0 -> G1 -> G2 -> U
    for (int w = threadIdx.x; w < ne * NV; w += blockDim.x) {
      const int el = w / NV, i = w - el * NV;
      G0[el * PER + i] = a.x[rhs * a.ndof + mt->dof(el) + i];
    }
    __syncthreads();
    const T* BT = tb + TabLayout::BT(N, Q);
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
      contract<T, N, N, N, 0, Q, tab_B(N, Q), false, false>(G0, G1, PER, ne);
      __syncthreads();
      contract<T, Q, N, N, 1, Q, tab_B(N, Q), false, false>(G1, G2, PER, ne);
      __syncthreads();
      contract<T, Q, Q, N, 2, Q, tab_B(N, Q), false, false>(G2, U, PER, ne);
    }
    __syncthreads();
  }
  if constexpr (line_mode<T, DIM>()) {
    // reference gradient, one line per thread
    contract<T, Q, Q, Q, 0, Q, tab_D(Q), false, false>(U, G0, PER, ne);
    contract<T, Q, Q, Q, 1, Q, tab_D(Q), false, false>(U, G1, PER, ne);
    contract<T, Q, Q, Q, 2, Q, tab_D(Q), false, false>(U, G2, PER, ne);
    __syncthreads();
  }
  // volume pointwise terms (with the collocation gradient computed in place in
  // output-per-thread mode) and the flux of the conforming faces, in one pass:
  //   G_m = kappa (G grad_ref u)_m,  R = lambda w|J| u,  Fq[k] = (s, c_m t)
  {
    const T* DT = tb + TabLayout::DT(N, Q);
    const int nvol = ne * QV;
    // two copies of the pass: the FP32 one over all faces with the others skipped
    // (the shape its compiled code is fastest in), the FP64 one over the tile's
    // list of conforming faces where the tile has finer rules
    if constexpr (!dense_faces<T>()) {
      for (int w = threadIdx.x; w < nvol + ne * NFACE * QF1; w += blockDim.x) {
        if (w >= nvol) {
          const int v = w - nvol;
          const int el = v / (NFACE * QF1);
          const int rem = v - el * NFACE * QF1;
          const int k = rem / QF1, j = rem - k * QF1;
          if (!own_rule<Q>(mt->slot(el * 2 * DIM + k).qf, force)) continue;
          face_flux<T, DIM, N, Q, P2P>(a, mt, rhs, tb, orth, el, k, j % Q, j / Q, F0 + el * PER + k * NF * QF1, QF1);
          continue;
        }
        const int el = w / QV, q = w - el * QV;
        T* b = sm + el * PER;
        T g[DIM];
        if constexpr (line_mode<T, DIM>()) {
  #pragma unroll
          for (int m = 0; m < DIM; ++m) g[m] = b[(1 + m) * QV + q];
        } else {
          const int qc[3] = {q % Q, (q / Q) % Q, DIM == 3 ? q / (Q * Q) : 0};
  #pragma unroll
          for (int m = 0; m < DIM; ++m) {
            const int sm_ = m == 0 ? 1 : (m == 1 ? Q : Q * Q);
            const T* u = b + q - qc[m] * sm_;
            T acc = 0;
  #pragma unroll
            for (int r = 0; r < Q; ++r) acc = fma(DT[r * Q + qc[m]], u[r * sm_], acc);
            g[m] = acc;
          }
        }
        // deformed element: factors per point; affine element: constants times the
        // Gauss weight.  The gradient is scaled first (kappa, weight), so that each
        // multiply that is 1 is skipped.
        const bool eaf = mt->aff(el) != 0;
        const T* geo = a.vgeo + mt->vgo(el) + (eaf ? 0 : q);
        const int gs = eaf ? 1 : QV;
        T lwj = a.lambda * geo[DIM == 2 ? 3 * gs : 6 * gs];
        if (eaf || a.kappa) {
          T wk = T(1);
          if (eaf) {
            const T* gw = tb + TabLayout::GW(N, Q, Q);
            T wq = gw[q % Q] * gw[(q / Q) % Q];
            if constexpr (DIM == 3) wq *= gw[q / (Q * Q)];
            lwj *= wq;
            wk = wq;
          }
          if (a.kappa) wk = eaf ? wk * a.kappa[mt->qoff(el) + q] : a.kappa[mt->qoff(el) + q];
  #pragma unroll
          for (int m = 0; m < DIM; ++m) g[m] *= wk;
        }
        if constexpr (DIM == 2) {
          b[QV + q] = geo[0] * g[0] + geo[gs] * g[1];
          b[2 * QV + q] = geo[gs] * g[0] + geo[2 * gs] * g[1];
        } else {
          const T a00 = geo[0], a01 = geo[gs], a02 = geo[2 * gs], a11 = geo[3 * gs], a12 = geo[4 * gs],
                  a22 = geo[5 * gs];
          b[QV + q] = a00 * g[0] + a01 * g[1] + a02 * g[2];
          b[2 * QV + q] = a01 * g[0] + a11 * g[1] + a12 * g[2];
          b[3 * QV + q] = a02 * g[0] + a12 * g[1] + a22 * g[2];
        }
        b[(1 + DIM) * QV + q] = lwj * b[q];
      }
    } else {
      const FaceList fl{flist};
      // conforming faces: every face of a tile without finer rules; otherwise the
      // tile's list of them
      const bool dense = fine;
      const int nfi = dense ? fl.nconf() * QF1 : ne * NFACE * QF1;
      for (int w = threadIdx.x; w < nvol + nfi; w += blockDim.x) {
        if (w >= nvol) {
          const int v = w - nvol;
          int el, k, j;
          if (dense) {
            const int i = v / QF1, e = fl.conf(i);
            j = v - i * QF1;
            el = fl_el(e);
            k = fl_k(e);
          } else {
            el = v / (NFACE * QF1);
            const int rem = v - el * NFACE * QF1;
            k = rem / QF1;
            j = rem - k * QF1;
            if (fine && !own_rule<Q>(mt->slot(el * 2 * DIM + k).qf, force)) continue;
          }
          face_flux<T, DIM, N, Q, P2P>(a, mt, rhs, tb, orth, el, k, j % Q, j / Q, F0 + el * PER + k * NF * QF1, QF1);
          continue;
        }
        const int el = w / QV, q = w - el * QV;
        T* b = sm + el * PER;
        T g[DIM];
        if constexpr (line_mode<T, DIM>()) {
  #pragma unroll
          for (int m = 0; m < DIM; ++m) g[m] = b[(1 + m) * QV + q];
        } else {
          const int qc[3] = {q % Q, (q / Q) % Q, DIM == 3 ? q / (Q * Q) : 0};
  #pragma unroll
          for (int m = 0; m < DIM; ++m) {
            const int sm_ = m == 0 ? 1 : (m == 1 ? Q : Q * Q);
            const T* u = b + q - qc[m] * sm_;
            T acc = 0;
  #pragma unroll
            for (int r = 0; r < Q; ++r) acc = fma(DT[r * Q + qc[m]], u[r * sm_], acc);
            g[m] = acc;
          }
        }
        // deformed element: factors per point; affine element: constants times the
        // Gauss weight.  The gradient is scaled first (kappa, weight), so that each
        // multiply that is 1 is skipped.
        const bool eaf = mt->aff(el) != 0;
        const T* geo = a.vgeo + mt->vgo(el) + (eaf ? 0 : q);
        const int gs = eaf ? 1 : QV;
        T lwj = a.lambda * geo[DIM == 2 ? 3 * gs : 6 * gs];
        if (eaf || a.kappa) {
          T wk = T(1);
          if (eaf) {
            const T* gw = tb + TabLayout::GW(N, Q, Q);
            T wq = gw[q % Q] * gw[(q / Q) % Q];
            if constexpr (DIM == 3) wq *= gw[q / (Q * Q)];
            lwj *= wq;
            wk = wq;
          }
          if (a.kappa) wk = eaf ? wk * a.kappa[mt->qoff(el) + q] : a.kappa[mt->qoff(el) + q];
  #pragma unroll
          for (int m = 0; m < DIM; ++m) g[m] *= wk;
        }
        if constexpr (DIM == 2) {
          b[QV + q] = geo[0] * g[0] + geo[gs] * g[1];
          b[2 * QV + q] = geo[gs] * g[0] + geo[2 * gs] * g[1];
        } else {
          const T a00 = geo[0], a01 = geo[gs], a02 = geo[2 * gs], a11 = geo[3 * gs], a12 = geo[4 * gs],
                  a22 = geo[5 * gs];
          b[QV + q] = a00 * g[0] + a01 * g[1] + a02 * g[2];
          b[2 * QV + q] = a01 * g[0] + a11 * g[1] + a12 * g[2];
          b[3 * QV + q] = a02 * g[0] + a12 * g[1] + a22 * g[2];
        }
        b[(1 + DIM) * QV + q] = lwj * b[q];
      }
    }
  }
  __syncthreads();
  if (fine) lift_fine_faces<T, DIM, N, Q, P2P>(a, t, mt, flist, rhs, tb, F0, PER, orth);
  const T* DD = tb + TabLayout::DD(N, Q);
  if constexpr (kGatherScatter) {
    // ScatrInterp: the face points are volume points of the element's boundary
    // planes, so each face adds s to R and c_m t to G_m there; the one
    // transposed gradient + IProduct below then lifts both.  One work item per
    // volume point, summing the faces through it (no two items write the same
    // point).
    for (int w = threadIdx.x; w < ne * QV; w += blockDim.x) {
      const int el = w / QV, q = w - el * QV;
      const int qc[3] = {q % Q, (q / Q) % Q, DIM == 3 ? q / (Q * Q) : 0};
      bool edge = false;
#pragma unroll
      for (int ax = 0; ax < DIM; ++ax) edge = edge || qc[ax] == 0 || qc[ax] == Q - 1;
      if (!edge) continue;
      T* b = sm + el * PER;
      const T* fel = F0 + el * PER;
      T r = b[(1 + DIM) * QV + q];
      T g[DIM];
#pragma unroll
      for (int m = 0; m < DIM; ++m) g[m] = b[(1 + m) * QV + q];
#pragma unroll
      for (int ax = 0; ax < DIM; ++ax) {
        const int j = DIM == 2 ? qc[1 - ax] : (ax == 0 ? qc[1] + Q * qc[2] : (ax == 1 ? qc[0] + Q * qc[2] : qc[0] + Q * qc[1]));
#pragma unroll
        for (int sd = 0; sd < 2; ++sd) {
          if (qc[ax] != (sd ? Q - 1 : 0)) continue;
          const T* fq = fel + (2 * ax + sd) * NF * QF1 + j;
          r += fq[0];
#pragma unroll
          for (int m = 0; m < DIM; ++m)
            if (!orth || m == ax) g[m] += fq[(1 + m) * QF1];
        }
      }
      b[(1 + DIM) * QV + q] = r;
#pragma unroll
      for (int m = 0; m < DIM; ++m) b[(1 + m) * QV + q] = g[m];
    }
    __syncthreads();
  } else if (!orth) {
    // face field P = s + sum_{tangential m} D_m^T (c_m t) on the face (the
    // tangential part of the lift after the transposed gradient); c_a t stays
    // as is and is lifted with l'(+-1)
    for (int w = threadIdx.x; w < ne * NFACE * QF1; w += blockDim.x) {
      const int el = w / (NFACE * QF1);
      const int rem = w - el * NFACE * QF1;
      const int k = rem / QF1, j = rem - k * QF1;
      const int ax = k >> 1;
      int t0, t1;
      tang_axes<DIM>(ax, t0, t1);
      const int j0 = j % Q, j1 = j / Q;
      T* fq = F0 + el * PER + k * NF * QF1;
      T p = fq[j];
      const T* f0 = fq + (1 + t0) * QF1 + Q * j1;
#pragma unroll
      for (int r = 0; r < Q; ++r) p = fma(DD[r * Q + j0], f0[r], p);
      if constexpr (DIM == 3) {
        const T* f1 = fq + (1 + t1) * QF1 + j0;
#pragma unroll
        for (int r = 0; r < Q; ++r) p = fma(DD[r * Q + j1], f1[r * Q], p);
      }
      fq[j] = p;
    }
    __syncthreads();
  }
  // H = R + sum_m D_m^T G_m + sum_faces [ l(+-1) P + l'(+-1) c_a t ] (into U);
  // with gathered / scattered traces the faces are already in R and G
  {
    const T* LL = tb + TabLayout::LL(N, Q);
    for (int w = threadIdx.x; w < ne * QV; w += blockDim.x) {
      const int el = w / QV, q = w - el * QV;
      const int qc[3] = {q % Q, (q / Q) % Q, DIM == 3 ? q / (Q * Q) : 0};
      const T* b = sm + el * PER;
      const T* fel = F0 + el * PER;
      T acc = b[(1 + DIM) * QV + q];
      if constexpr (!line_mode<T, DIM>()) {
#pragma unroll
        for (int m = 0; m < DIM; ++m) {
          const int sm_ = m == 0 ? 1 : (m == 1 ? Q : Q * Q);
          const T* g = b + (1 + m) * QV + q - qc[m] * sm_;
#pragma unroll
          for (int r = 0; r < Q; ++r) acc = fma(DD[r * Q + qc[m]], g[r * sm_], acc);
        }
      }
#pragma unroll
      for (int ax = 0; ax < (kGatherScatter ? 0 : DIM); ++ax) {
        const int j = DIM == 2 ? qc[1 - ax] : (ax == 0 ? qc[1] + Q * qc[2] : (ax == 1 ? qc[0] + Q * qc[2] : qc[0] + Q * qc[1]));
#pragma unroll
        for (int sd = 0; sd < 2; ++sd) {
          const T* fq = fel + (2 * ax + sd) * NF * QF1 + j;
          acc = fma(LL[sd * Q + qc[ax]], fq[0], acc);
          acc = fma(LL[(2 + sd) * Q + qc[ax]], fq[(1 + ax) * QF1], acc);
        }
      }
      sm[el * PER + q] = acc;
    }
  }
  __syncthreads();
  if constexpr (line_mode<T, DIM>()) {
    contract<T, Q, Q, Q, 0, Q, tab_D(Q), true, true>(G0, U, PER, ne);
    __syncthreads();
    contract<T, Q, Q, Q, 1, Q, tab_D(Q), true, true>(G1, U, PER, ne);
    __syncthreads();
    contract<T, Q, Q, Q, 2, Q, tab_D(Q), true, true>(G2, U, PER, ne);
    __syncthreads();
  }
  // y = (B^T x B^T (x B^T)) H; the last contraction writes y in global memory
  const T* BB = tb + TabLayout::BB(N, Q);
  auto gy = [&](int el) { return a.y + rhs * a.ndof + mt->dof(el); };
  T* res = nullptr;
  if constexpr (DIM == 2) {
    cpt<T, Q, Q, 1, 0, N, false>(U, G0, PER, ne, BB);
    __syncthreads();
    cpt_io<T, N, Q, 1, 1, N, false>([&](int el) { return G0 + el * PER; }, gy, ne, BB);
  } else if constexpr (!line_mode<T, DIM>()) {
    cpt<T, Q, Q, Q, 0, N, false>(U, G0, PER, ne, BB);
    __syncthreads();
    cpt<T, N, Q, Q, 1, N, false>(G0, G1, PER, ne, BB);
    __syncthreads();
    cpt_io<T, N, N, Q, 2, N, false>([&](int el) { return G1 + el * PER; }, gy, ne, BB);
  } else {
    (void)BB;
    contract<T, Q, Q, Q, 0, N, tab_B(N, Q), true, false>(U, G0, PER, ne);
    __syncthreads();
    contract<T, N, Q, Q, 1, N, tab_B(N, Q), true, false>(G0, G1, PER, ne);
    __syncthreads();
    contract<T, N, N, Q, 2, N, tab_B(N, Q), true, false>(G1, G2, PER, ne);
    res = G2;
  }
  if constexpr (line_mode<T, DIM>()) {
    __syncthreads();
    for (int w = threadIdx.x; w < ne * NV; w += blockDim.x) {
      const int el = w / NV, i = w - el * NV;
      a.y[rhs * a.ndof + mt->dof(el) + i] = res[el * PER + i];
    }
  } else {
    (void)res;
    (void)NV;
  }
}

// Shared memory of a CTA: [table block of its order up to the finest face rule
// of its tiles (table_block_bytes)][descriptors of its largest tile (meta_bytes)][elements].  A CTA runs a list of tiles of one order (its share
// of the launch, tiles cta_off[b] .. cta_off[b+1]-1) one after the other, with the
// order's tables loaded once.
// The (N, Q) of the CTA's tiles selects the compile-time specialisation: the
// standard pairs Q = N + 1, and in the Gauss-Lobatto units the extra pairs
// of kExtraPairs (elements whose points do not follow their order).
#define SIP_PAIR_KEY(n, q) ((n) * 16 + (q))
#define SIP_EXTRA_CASES(FN)                                        \
  case SIP_PAIR_KEY(2, 4): if constexpr (kGatherScatter) FN(2, 4); break; \
  case SIP_PAIR_KEY(2, 5): if constexpr (kGatherScatter) FN(2, 5); break; \
  case SIP_PAIR_KEY(3, 5): if constexpr (kGatherScatter) FN(3, 5); break;
#define SIP_ORDER_SWITCH(FN)                        \
  switch (SIP_PAIR_KEY(t.n, t.q)) {                 \
    case SIP_PAIR_KEY(2, 3): FN(2, 3); break;       \
    case SIP_PAIR_KEY(3, 4): FN(3, 4); break;       \
    case SIP_PAIR_KEY(4, 5): FN(4, 5); break;       \
    case SIP_PAIR_KEY(5, 6): FN(5, 6); break;       \
    case SIP_PAIR_KEY(6, 7): FN(6, 7); break;       \
    case SIP_PAIR_KEY(7, 8): FN(7, 8); break;       \
    case SIP_PAIR_KEY(8, 9): FN(8, 9); break;       \
    case SIP_PAIR_KEY(9, 10): FN(9, 10); break;     \
    case SIP_PAIR_KEY(10, 11): FN(10, 11); break;   \
    case SIP_PAIR_KEY(11, 12): FN(11, 12); break;   \
    SIP_EXTRA_CASES(FN)                             \
    default: break;                                 \
  }
static_assert(kNumExtra == 3 && extra_pair(2, 4) == 0 && extra_pair(2, 5) == 1 && extra_pair(3, 5) == 2,
              "the extra cases of SIP_ORDER_SWITCH list kExtraPairs");

// Grid-wide barrier of the single-launch apply: every CTA of the cooperative
// launch (all resident at once) arrives once; the last one to arrive opens the
// next generation.  A wait gives up after a bounded number of polls (about a
// second), sets the status word and lets the CTA go on, so the kernel always
// ends; the solver reports a set status as an error.
__device__ __forceinline__ void grid_barrier(unsigned int* gbar) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int* vgen = gbar + 1;
    const unsigned int gen = *vgen;
    __threadfence();
    const unsigned int total = gridDim.x * gridDim.y;
    if (atomicAdd(gbar, 1u) + 1u == total) {
      gbar[0] = 0u;
      __threadfence();
      atomicAdd(gbar + 1, 1u);
    } else {
      unsigned int polls = 0;
      while (*vgen == gen) {
        if (++polls > (1u << 24)) {
          atomicExch(gbar + 2, 1u);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
}

// MODE: 0 the trace phase, 1 the main phase, 2 both in one launch with a grid
// barrier between them (the tables are loaded once)
template <typename T, int DIM, int N, int Q, int MODE, bool P2P>
__device__ __forceinline__ void run_tiles(const ApplyArgs<T>& a, int ti0, int ti1, int rhs, unsigned char* smem_raw) {
  // finest face rule and largest tile of the CTA's tiles: the extents of its
  // table block and descriptor block
  int fmax = Q, cmax = 1;
  bool force = false;
  for (int ti = ti0; ti < ti1; ++ti) {
    const Tile t = a.tiles[ti];
    fmax = max(fmax, t.flags & kTileQfMask);
    cmax = max(cmax, t.count);
    force = force || (t.flags & kTileForce);
  }
  const int tbytes = table_block_bytes(sizeof(T), N, Q, fmax);
  T* tb = reinterpret_cast<T*>(smem_raw);
  TileMeta<DIM> meta;
  meta.e_ = reinterpret_cast<ElemDesc*>(smem_raw + tbytes);
  meta.s_ = reinterpret_cast<SlotDesc*>(meta.e_ + cmax);
  TileMeta<DIM>* mt = &meta;
  T* sm = reinterpret_cast<T*>(smem_raw + tbytes + meta_bytes(DIM, cmax));
  // the first tile's descriptors (and, for the main phase, its face list) are
  // static data: copy them before the wait too, so that their latency overlaps
  // the previous kernel's tail (load_tables ends with the barrier that makes them
  // visible)
  {
    const Tile t0 = a.tiles[ti0];
    uint16_t* fl0 = MODE == 1 && dense_faces<T>()
                        ? reinterpret_cast<uint16_t*>(sm + t0.count * Shape<DIM, N, Q>::PER_MAIN)
                        : nullptr;
    load_meta<DIM>(a.desc_e, a.desc_s, a.flists, t0, mt, fl0);
  }
  load_tables<T, N, Q>(tb, fmax, force, a.gtab, a.ggw);
  grid_dep_wait();  // before anything that another kernel writes
  if constexpr (MODE != 1) {
    for (int ti = ti0; ti < ti1; ++ti) {
      if (ti > ti0) __syncthreads();  // the previous tile's last stage still reads shared memory
      trace_tile<T, DIM, N, Q, P2P>(a, a.tiles[ti], rhs, tb, mt, sm, ti == ti0);
    }
  }
  if constexpr (MODE == 2) grid_barrier(a.gbar);  // every trace is written (and visible)
  if constexpr (MODE != 0) {
    for (int ti = ti0; ti < ti1; ++ti) {
      if (ti > ti0 || MODE == 2) __syncthreads();
      main_tile<T, DIM, N, Q, P2P>(a, a.tiles[ti], rhs, tb, mt, sm, MODE == 1 && ti == ti0);
    }
  }
}

// P2P: the point-to-point interpolation variant (SIP_FACES_P2P); the shared-rule
// kernels are compiled without any of its code.
// RULE: the translation unit's point rule (kTuRule), part of the kernel's name
// so that the Gauss and the Gauss-Lobatto instantiations stay distinct.
template <typename T, int DIM, bool P2P, int RULE>
__global__ void __launch_bounds__(256) k_trace(ApplyArgs<T> a) {
  static_assert(RULE == kTuRule, "kernel instantiated in a unit of another rule");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  grid_dep_launch_next();  // k_main may load its tables meanwhile
  const int ti0 = a.cta_off[blockIdx.x], ti1 = a.cta_off[blockIdx.x + 1];
  if (ti0 >= ti1) return;
  const Tile t = a.tiles[ti0];  // every tile of the CTA has this (N, Q)
#define SIP_TRACE_CASE(NN, QQ) run_tiles<T, DIM, NN, QQ, 0, P2P>(a, ti0, ti1, blockIdx.y, smem_raw)
  SIP_ORDER_SWITCH(SIP_TRACE_CASE)
#undef SIP_TRACE_CASE
}

// Launch bounds of the main kernel, set by the translation unit that
// instantiates it: FP64 asks for registers for 4 resident CTAs per SM (room for
// the wider values without spilling), FP32 gives no hint, which keeps its
// register count and so its occupancy highest.
#ifndef SIP_MAIN_LAUNCH_BOUNDS
#define SIP_MAIN_LAUNCH_BOUNDS 256
#endif

template <typename T, int DIM, bool P2P, int RULE>
__global__ void __launch_bounds__(SIP_MAIN_LAUNCH_BOUNDS) k_main(ApplyArgs<T> a) {
  static_assert(RULE == kTuRule, "kernel instantiated in a unit of another rule");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int ti0 = a.cta_off[blockIdx.x], ti1 = a.cta_off[blockIdx.x + 1];
  if (ti0 >= ti1) return;
  const Tile t = a.tiles[ti0];
#define SIP_MAIN_CASE(NN, QQ) run_tiles<T, DIM, NN, QQ, 1, P2P>(a, ti0, ti1, blockIdx.y, smem_raw)
  SIP_ORDER_SWITCH(SIP_MAIN_CASE)
#undef SIP_MAIN_CASE
}

// The whole apply in one cooperative launch of persistent CTAs: trace phase,
// grid barrier, main phase.  Every CTA of a persistent schedule has tiles; one
// without would still take part in the barrier.
template <typename T, int DIM, bool P2P, int RULE>
__global__ void __launch_bounds__(SIP_MAIN_LAUNCH_BOUNDS) k_apply(ApplyArgs<T> a) {
  static_assert(RULE == kTuRule, "kernel instantiated in a unit of another rule");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int ti0 = a.cta_off[blockIdx.x], ti1 = a.cta_off[blockIdx.x + 1];
  if (ti0 >= ti1) {
    grid_barrier(a.gbar);
    return;
  }
  const Tile t = a.tiles[ti0];
  bool ran = false;
#define SIP_APPLY_CASE(NN, QQ) (run_tiles<T, DIM, NN, QQ, 2, P2P>(a, ti0, ti1, blockIdx.y, smem_raw), ran = true)
  SIP_ORDER_SWITCH(SIP_APPLY_CASE)
#undef SIP_APPLY_CASE
  if (!ran) grid_barrier(a.gbar);  // (no such tile is built) keep the barrier whole
}

}  // namespace sip
