// Internal definitions shared by the host plan builder, the C-ABI layer and
// the CUDA kernels.  Not part of the public ABI.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/sip.h"

namespace sip {

constexpr int kMaxOrder = SIP_MAX_ORDER;  // P in 1..10
constexpr int kNMin = 2;                  // N = P + 1
constexpr int kNMax = kMaxOrder + 1;      // 11
constexpr int kQMin = kNMin + 1;          // Q = P + 2 (qvol_extra = 2)
constexpr int kQMax = kNMax + 1;          // 12; also the largest face rule

// ---------------------------------------------------------------------------
// 1D table layout, identical on host (filling) and device (__constant__ reads).
// One set per point rule R (Gauss-Legendre or Gauss-Lobatto-Legendre, chosen per
// handle; each kernel translation unit holds the set of its rule):
//   B_N   [Q][N]  B[q][i]  = l^GLL_N,i (xi^R_Q,q)       (interpolation nodes -> rule points)
//   D_Q   [Q][Q]  D[q][r]  = l^R_Q,r ' (xi^R_Q,q)        (collocation derivative)
//   L_Q   [4][Q]  rows l_r(-1), l_r(+1), l_r'(-1), l_r'(+1) of the rule's Lagrange basis
//   I_Q,F [F][Q]  I[z][r]  = l^R_Q,r (xi^R_F,z), F in Q..kQMax (face rule interpolation;
//                 F = Q is the identity, used when interpolation is forced on every face)
// B for Q = N + 1 (the standard (P+2)-point rules) and for the extra (N, Q) pairs
// below; D, L and I for every Q.
// ---------------------------------------------------------------------------

// Elements whose points do not follow their order (Q != N + 1): the pairs the
// Gauss-Lobatto kernels are also built for.  They carry the transition layer of
// Sec. 3.3 (the coefficients of one order, the points of a higher one, e.g.
// P2Q5 between P4Q5 and P2Q3 in the paper's counts) and Table 2's P3Q5.
struct NQ { int n, q; };
constexpr NQ kExtraPairs[] = {{2, 4}, {2, 5}, {3, 5}};
constexpr int kNumExtra = (int)(sizeof(kExtraPairs) / sizeof(kExtraPairs[0]));
constexpr int extra_pair(int n, int q) {
  for (int i = 0; i < kNumExtra; ++i)
    if (kExtraPairs[i].n == n && kExtraPairs[i].q == q) return i;
  return -1;
}
// an (N, Q) pair the kernels of a rule are built for
constexpr bool pair_supported(int rule, int n, int q) {
  return (q == n + 1 && n >= kNMin && n <= kNMax) || (rule == SIP_RULE_GLL && extra_pair(n, q) >= 0);
}

constexpr int tab_B(int N, int Q) {
  int off = 0;
  if (Q == N + 1) {
    for (int n = kNMin; n < N; ++n) off += (n + 1) * n;
    return off;
  }
  for (int n = kNMin; n <= kNMax; ++n) off += (n + 1) * n;
  for (int i = 0; i < kNumExtra && !(kExtraPairs[i].n == N && kExtraPairs[i].q == Q); ++i)
    off += kExtraPairs[i].n * kExtraPairs[i].q;
  return off;
}
constexpr int tab_B(int N) { return tab_B(N, N + 1); }
constexpr int kTabBEnd = tab_B(0, 0);   // past the last extra pair
constexpr int tab_D(int Q) {
  int off = kTabBEnd;
  for (int q = kQMin; q < Q; ++q) off += q * q;
  return off;
}
constexpr int kTabDEnd = tab_D(kQMax + 1);
constexpr int tab_L(int Q) {
  int off = kTabDEnd;
  for (int q = kQMin; q < Q; ++q) off += 4 * q;
  return off;
}
constexpr int kTabLEnd = tab_L(kQMax + 1);
constexpr int tab_I(int Q, int F) {
  int off = kTabLEnd;
  for (int q = kQMin; q <= kQMax; ++q)
    for (int f = q; f <= kQMax; ++f) {
      if (q == Q && f == F) return off;
      off += f * q;
    }
  return off;
}
constexpr int kTabSize = tab_I(kQMax + 1, kQMax + 2);

// ---------------------------------------------------------------------------
// Shared-memory layout of the apply kernels (host computes launch sizes, device
// indexes with the same constexpr functions).
//
// Per-CTA table block for one (N, Q), laid out so that a warp whose lanes compute
// consecutive outputs reads consecutive addresses:
//   BT [N][Q]  B[q][i] at i*Q + q      forward interpolation nodes -> rule points
//   BB [Q][N]  B[q][i] at q*N + i      transposed interpolation
//   DT [Q][Q]  D[q][r] at r*Q + q      collocation derivative
//   DD [Q][Q]  D[q][r] at q*Q + r      transposed derivative
//   LL [4][Q]  l(-1), l(+1), l'(-1), l'(+1)
//   for F = Q .. kQMax:    GW_F [F] weights of the F-point rule
//   for F = Q .. kQMax:    IT_F [Q][F] (I[z][r] at r*F + z), II_F [F][Q] (I[z][r] at z*Q + r)
// A CTA holds (and loads) the block only up to the finest face rule fmax of its
// tiles: the element buffers follow at table_block_bytes(bytes, n, fmax).
// ---------------------------------------------------------------------------
struct TabLayout {
  static constexpr int BT(int, int) { return 0; }
  static constexpr int BB(int n, int q) { return n * q; }
  static constexpr int DT(int n, int q) { return 2 * n * q; }
  static constexpr int DD(int n, int q) { return DT(n, q) + q * q; }
  static constexpr int LL(int n, int q) { return DD(n, q) + q * q; }
  // weights of the F-point rules, F = Q .. kQMax (affine geometry)
  static constexpr int GW(int n, int q, int f) {
    int o = LL(n, q) + 4 * q;
    for (int g = q; g < f; ++g) o += g;
    return o;
  }
  static constexpr int IT(int n, int q, int f) {
    int o = GW(n, q, kQMax + 1);
    for (int g = q; g < f; ++g) o += 2 * g * q;
    return o;
  }
  static constexpr int II(int n, int q, int f) { return IT(n, q, f) + f * q; }
  // entries up to and including the interpolation to the fmax-point rule
  static constexpr int size(int n, int q, int fmax) { return IT(n, q, fmax + 1); }
};

constexpr int cpow(int b, int e) { return e == 0 ? 1 : b * cpow(b, e - 1); }

// per-element shared memory (in elements of T) of the trace and main kernels:
// face values of all 2*dim faces at the element's own face points
// [2 dim][fields][Q^(dim-1)], plus scratch for faces with a finer shared rule,
// [slots][fields][FT + kQMax^(dim-1)] (FT = kQMax Q in 3D, 0 in 2D): one slot per
// face in 2D (all processed together), one slot in 3D (one face at a time)
constexpr int scratch_slots(int dim) { return dim == 2 ? 4 : 1; }
constexpr int face_buf(int dim, int q, int fields) {
  return 2 * dim * fields * cpow(q, dim - 1) +
         scratch_slots(dim) * fields * ((dim == 3 ? kQMax * q : 0) + cpow(kQMax, dim - 1));
}
// (the volume buffers hold Q^dim values; N <= Q, so the N^dim coefficients fit)
constexpr int per_elem_trace(int dim, int n, int q) { return (void)n, 2 * cpow(q, dim) + face_buf(dim, q, 4); }
constexpr int per_elem_main(int dim, int n, int q) { return (void)n, (2 + dim) * cpow(q, dim) + face_buf(dim, q, 1 + dim); }
// bytes of the CTA's table block (padded to 16) that precedes the element buffers,
// for tiles whose finest face rule is fmax (at most kQMax)
constexpr int table_block_bytes(int bytes_per, int n, int q, int fmax = kQMax) {
  return ((TabLayout::size(n, q, fmax) * bytes_per + 15) / 16) * 16;
}

// ---------------------------------------------------------------------------
// Per element local face slot (2*dim per element; local face k = 2*axis + side).
// ---------------------------------------------------------------------------
constexpr int kFaceBnd = 1;     // boundary face
constexpr int kFaceOrth = 2;    // c = J^-1 n has no tangential component on either side
constexpr int kFaceAffine = 4;  // both sides affine: geometry stored as constants (W without the weight)

// bits 3-6 of the slot flags: points per direction of the OTHER side's rule
// (equal to qf with a shared rule; the neighbour's own rule with point-to-point
// interpolation, SIP_FACES_P2P)
constexpr int kFaceOqShift = 3;
constexpr int8_t face_oq_bits(int q) { return (int8_t)(q << kFaceOqShift); }
constexpr int face_oq(int flags) { return (flags >> kFaceOqShift) & 15; }

struct FaceSlot {  // 8 bytes
  int32_t face;    // face id
  int8_t side;     // 0: minus side (or boundary), 1: plus side
  int8_t orient;   // plus side: bit0 flip t0, bit1 flip t1, bit2 transpose; else 0
  int8_t qf;       // points per direction of this side's face rule (the shared rule,
                   // or with SIP_FACES_P2P this element's own Q)
  int8_t flags;    // kFaceBnd | kFaceOrth | kFaceAffine | face_oq_bits(other side's rule)
};

constexpr int kTileQfMask = 0xff;  // bits 0-7: largest face rule of the tile
constexpr int kTileFine = 1 << 8;  // some face of the tile goes through the interpolation path
                                   // (a finer shared rule than Q, or kTileForce)
constexpr int kTileOrth = 1 << 9;  // every face of the tile is orthogonal (kFaceOrth)
constexpr int kTileForce = 1 << 10;  // every face goes through the shared-rule interpolation
                                     // path, also where its rule is the element's own
constexpr int kMaxEpb = 32;        // elements per tile, at most

struct Tile {
  int32_t n;       // nodes per direction (P + 1) of every element of the tile
  int32_t q;       // volume points per direction of every element of the tile
  int32_t start;   // first index into the order-sorted element list
  int32_t count;   // elements in the tile
  int32_t flags;   // kTileQfMask | kTileFine | kTileOrth | kTileForce
  int32_t flist;   // offset of the tile's face list (16-bit words)
  int64_t qbase;   // first volume point of the tile in the element-list order of the
                   // volume-point hand-off buffer (ug): the tile's points are contiguous there
};
static_assert(sizeof(Tile) == 32, "tile layout");

// Face list of a tile, so that face stages run over dense work items:
// [nconf, nfine, ngroups, (qf, count) x ngroups, nconf conforming entries
// (shared rule = own Q points), nfine entries with a finer shared rule in
// ascending qf (the groups)]; entry = el | k << 5 | qf << 8.
constexpr int kFaceListMax = 3 + 2 * 16 + kMaxEpb * 6;  // at most 16 groups (qf <= 16)
constexpr int fl_el(int e) { return e & 31; }
constexpr int fl_k(int e) { return (e >> 5) & 7; }
constexpr int fl_qf(int e) { return e >> 8; }

// What the kernels look up per element and per face slot, packed in the order of
// the order-sorted element list (elist), so that a tile's descriptors are two
// contiguous blocks read with one round of coalesced loads instead of chains of
// dependent lookups (element id -> offsets, face id -> offsets and penalty).
struct ElemDesc {     // 32 bytes
  int64_t dof_off;    // first DOF of the element
  int64_t vgoff;      // volume geometry offset
  int64_t quad_off;   // first volume point (kappa, Gauss-point values)
  int32_t eid;        // element id
  int32_t aff;        // 1: volume geometry stored as constants
};
struct SlotDesc {     // 32 bytes
  FaceSlot slot;      // the element's local face slot
  int64_t troff;      // trace offset of the face (points)
  int64_t goff;       // face geometry offset
  double tau;         // penalty of the face
};
static_assert(sizeof(ElemDesc) == 32 && sizeof(SlotDesc) == 32, "descriptor layout");

// per-tile copy of the element and slot descriptors in shared memory, after the
// table block, sized for the largest tile (cmax elements) of the CTA; the face
// list, where used, follows the element buffers
constexpr int meta_bytes(int dim, int cmax = kMaxEpb) {
  return cmax * ((int)sizeof(ElemDesc) + 2 * dim * (int)sizeof(SlotDesc));
}
constexpr int kMetaBytes = meta_bytes(3);
constexpr int kFaceListBytes = ((2 * kFaceListMax + 15) / 16) * 16;

// Host plan: everything the device needs, in FP64.
struct Plan {
  int dim = 0;
  int64_t E = 0, ndof = 0, nquad = 0;
  sip_options opt{};
  std::vector<int32_t> P;
  std::vector<int32_t> Q;       // volume points per direction of each element
  std::vector<int64_t> dof_off, quad_off;
  std::vector<int8_t> affine;
  // volume geometry: per element nG comps x Q^dim points, comp-major:
  // 2D: G00 G01 G11 wJ, 3D: G00 G01 G02 G11 G12 G22 wJ with G = w|J| J^-1 J^-T;
  // affine elements store the nG constants without the weight w (|J| J^-1 J^-T, |J|)
  std::vector<int64_t> vgoff;
  std::vector<double> vgeo;
  std::vector<double> xq;       // physical Gauss points [nquad][dim]
  std::vector<double> vol;      // |K|
  // faces
  int64_t n_int = 0, n_bnd = 0, n_nonconf = 0;
  std::vector<int32_t> f_em, f_km, f_ep, f_kp, f_orient, f_qf;  // ep = -1 on the boundary
  std::vector<int64_t> f_troff;  // trace offset (in points; 4 values per point slot group)
  std::vector<int64_t> f_goff;   // face geometry offset
  std::vector<double> f_tau;
  // face geometry, canonical point order (minus side's parametrisation):
  // interior: W, c-_0..c-_{d-1}, c+_0..c+_{d-1}; boundary: W, c_0..c_{d-1};
  // SIP_FACES_P2P interior faces: W-, c- at the minus side's own Q- points, then
  // W+, c+ at the plus side's own Q+ points
  // each comp holds npts = qf^(dim-1) values; c = J^-1 n of that side;
  // affine faces (kFaceAffine) store one value per comp, W without the weight w_z
  std::vector<double> fgeo;
  int64_t trace_points = 0;
  std::vector<FaceSlot> slots;   // [E][2 dim]
  // elements sorted by order (stable); tiles are cut from this list per precision
  std::vector<int32_t> elist;
  // descriptors in elist order: [E] and [E][2 dim]
  std::vector<ElemDesc> desc_e;
  std::vector<SlotDesc> desc_s;
  // volume points before each position of the element list ([E+1], prefix sums of Q^dim)
  std::vector<int64_t> qpos;
  int64_t orient_hist[8] = {0};
};

int build_plan(const sip_mesh* mesh, const int32_t* orders, const sip_options* opt, Plan& plan,
               std::string& err);

// host 1D rules (own implementation, FP64)
void gauss_legendre(int q, std::vector<double>& x, std::vector<double>& w);
void gauss_lobatto(int n, std::vector<double>& x, std::vector<double>& w);
// the q-point rule of the volume and face points: SIP_RULE_GAUSS or SIP_RULE_GLL
void point_rule(int rule, int q, std::vector<double>& x, std::vector<double>& w);
double lagrange(const std::vector<double>& nodes, int j, double x);
double lagrange_deriv(const std::vector<double>& nodes, int j, double x);
void fill_tables(int rule, std::vector<double>& tab);

// elements per tile for the apply kernels (host choice), per-element flops, and
// the tiles with the CTA that runs each (tiles cta_off[b] .. cta_off[b+1]-1, one
// order per CTA)
int apply_epb(int dim, int n, int q, int precision, int threads);
void element_flops(const Plan& p, int64_t e, double& ft, double& fm);
void build_tiles(const Plan& p, int precision, const int* epb_override, int threads, int nctas, bool persistent,
                 std::vector<Tile>& tiles, std::vector<int32_t>& cta_off, std::vector<uint16_t>& flists);

}  // namespace sip
