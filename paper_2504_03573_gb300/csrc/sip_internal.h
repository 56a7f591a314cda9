// Internal definitions shared by the host plan builder, the C-ABI layer and
// the CUDA kernels.  Not part of the public ABI.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/sip.h"

namespace sip {

constexpr int kMaxOrder = SIP_MAX_ORDER;  // P in 1..8
constexpr int kNMin = 2;                  // N = P + 1
constexpr int kNMax = kMaxOrder + 1;      // 9
constexpr int kQMin = kNMin + 1;          // Q = P + 2 (qvol_extra = 2)
constexpr int kQMax = kNMax + 1;          // 10; also the largest face rule

// ---------------------------------------------------------------------------
// 1D table layout, identical on host (filling) and device (__constant__ reads).
//   B_N   [Q][N]  B[q][i]  = l^GLL_N,i (xi^G_Q,q)       (interpolation GLL -> Gauss)
//   D_Q   [Q][Q]  D[q][r]  = l^G_Q,r ' (xi^G_Q,q)        (Gauss collocation derivative)
//   L_Q   [4][Q]  rows l_r(-1), l_r(+1), l_r'(-1), l_r'(+1) of the Gauss-Q Lagrange basis
//   I_Q,F [F][Q]  I[z][r]  = l^G_Q,r (xi^G_F,z), F in Q+1..kQMax (face rule interpolation)
// with Q = N + 1.
// ---------------------------------------------------------------------------
constexpr int tab_B(int N) {
  int off = 0;
  for (int n = kNMin; n < N; ++n) off += (n + 1) * n;
  return off;
}
constexpr int kTabBEnd = tab_B(kNMax + 1);
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
    for (int f = q + 1; f <= kQMax; ++f) {
      if (q == Q && f == F) return off;
      off += f * q;
    }
  return off;
}
constexpr int kTabSize = tab_I(kQMax + 1, kQMax + 2);

// ---------------------------------------------------------------------------
// Per element local face slot (2*dim per element; local face k = 2*axis + side).
// ---------------------------------------------------------------------------
struct FaceSlot {
  int32_t face;    // face id
  int8_t side;     // 0: minus side (or boundary), 1: plus side
  int8_t orient;   // plus side: bit0 flip t0, bit1 flip t1, bit2 transpose; else 0
  int8_t qf;       // points per direction of the shared face rule
  int8_t bnd;      // 1: boundary face
};

struct Tile {
  int32_t n;       // nodes per direction (P + 1) of every element of the tile
  int32_t start;   // first index into the order-sorted element list
  int32_t count;   // elements in the tile
  int32_t pad;
};

// Host plan: everything the device needs, in FP64.
struct Plan {
  int dim = 0;
  int64_t E = 0, ndof = 0, nquad = 0;
  sip_options opt{};
  std::vector<int32_t> P;
  std::vector<int64_t> dof_off, quad_off;
  std::vector<int8_t> affine;
  // volume geometry: per element nG comps x Q^dim points, comp-major:
  // 2D: G00 G01 G11 wJ, 3D: G00 G01 G02 G11 G12 G22 wJ with G = w|J| J^-1 J^-T
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
  // interior: W, c-_0..c-_{d-1}, c+_0..c+_{d-1}; boundary: W, c_0..c_{d-1}
  // each comp holds npts = qf^(dim-1) values; c = J^-1 n of that side
  std::vector<double> fgeo;
  int64_t trace_points = 0;
  std::vector<FaceSlot> slots;   // [E][2 dim]
  // order buckets
  std::vector<int32_t> elist;
  std::vector<Tile> tiles;
  int64_t orient_hist[8] = {0};
};

int build_plan(const sip_mesh* mesh, const int32_t* orders, const sip_options* opt, Plan& plan,
               std::string& err);

// host 1D rules (own implementation, FP64)
void gauss_legendre(int q, std::vector<double>& x, std::vector<double>& w);
void gauss_lobatto(int n, std::vector<double>& x, std::vector<double>& w);
double lagrange(const std::vector<double>& nodes, int j, double x);
double lagrange_deriv(const std::vector<double>& nodes, int j, double x);
void fill_tables(std::vector<double>& tab);

// elements per tile for the apply kernels (host choice, also used by launchers)
int apply_epb(int dim, int n, int precision);

}  // namespace sip
