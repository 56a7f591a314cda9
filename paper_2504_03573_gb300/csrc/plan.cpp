// Host mesh analysis for the SIP apply: face pairing, plus-side orientation,
// geometric factors at volume and face quadrature points, penalties, order
// buckets.  Runs once per mesh (the paper's preprocessing: traces and
// trace-conforming elements of Sec. 3.3, orientations of Sec. 5.1, element
// groups of equal order of Sec. 5.1).
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <numeric>
#include <string>
#include <thread>
#include <utility>
#include <vector>

#include "sip_internal.h"

namespace sip {

namespace {

// point rules (Gauss-Legendre or Gauss-Lobatto-Legendre) of every size the plan
// uses, computed once
struct PointRules {
  std::vector<double> x[kQMax + 1], w[kQMax + 1];
  explicit PointRules(int rule) {
    for (int q = 2; q <= kQMax; ++q) point_rule(rule, q, x[q], w[q]);
  }
};

// body(i0, i1) over [0, n) split into contiguous chunks on the host's cores;
// the first failure (nonzero return) of any chunk is returned with its message
template <typename F>
int parallel_chunks(int64_t n, F body, std::string& err) {
  const int64_t min_chunk = 256;
  int nt = (int)std::min<int64_t>(std::max(1u, std::thread::hardware_concurrency()), 64);
  nt = (int)std::max<int64_t>(1, std::min<int64_t>(nt, (n + min_chunk - 1) / min_chunk));
  if (nt == 1) return body(0, n, err);
  std::vector<std::thread> th;
  std::vector<std::string> errs(nt);
  std::vector<int> rcs(nt, 0);
  for (int t = 0; t < nt; ++t)
    th.emplace_back([&, t]() { rcs[t] = body(n * t / nt, n * (t + 1) / nt, errs[t]); });
  for (auto& x : th) x.join();
  for (int t = 0; t < nt; ++t)
    if (rcs[t]) {
      err = errs[t];
      return rcs[t];
    }
  return 0;
}

struct Geo {
  double x[3];
  double J[3][3];   // J[i][m] = d x_i / d xi_m
  double Ji[3][3];  // inverse: Ji[m][i] = d xi_m / d x_i
  double det;
};

// multilinear map of one element at reference point xi
void eval_map(int dim, const double* v /* [2^dim][dim] */, const double* xi, Geo& g) {
  for (int i = 0; i < 3; ++i) {
    g.x[i] = 0.0;
    for (int m = 0; m < 3; ++m) g.J[i][m] = 0.0;
  }
  const int nc = 1 << dim;
  for (int c = 0; c < nc; ++c) {
    double n[3], dn[3];
    for (int k = 0; k < dim; ++k) {
      const int b = (c >> k) & 1;
      n[k] = b ? 0.5 * (1.0 + xi[k]) : 0.5 * (1.0 - xi[k]);
      dn[k] = b ? 0.5 : -0.5;
    }
    double shape = 1.0;
    for (int k = 0; k < dim; ++k) shape *= n[k];
    for (int i = 0; i < dim; ++i) g.x[i] += shape * v[c * dim + i];
    for (int m = 0; m < dim; ++m) {
      double ds = dn[m];
      for (int k = 0; k < dim; ++k)
        if (k != m) ds *= n[k];
      for (int i = 0; i < dim; ++i) g.J[i][m] += ds * v[c * dim + i];
    }
  }
  if (dim == 2) {
    g.det = g.J[0][0] * g.J[1][1] - g.J[0][1] * g.J[1][0];
    const double id = 1.0 / g.det;
    g.Ji[0][0] = g.J[1][1] * id;
    g.Ji[0][1] = -g.J[0][1] * id;
    g.Ji[1][0] = -g.J[1][0] * id;
    g.Ji[1][1] = g.J[0][0] * id;
  } else {
    const auto& a = g.J;
    const double c00 = a[1][1] * a[2][2] - a[1][2] * a[2][1];
    const double c01 = a[1][2] * a[2][0] - a[1][0] * a[2][2];
    const double c02 = a[1][0] * a[2][1] - a[1][1] * a[2][0];
    g.det = a[0][0] * c00 + a[0][1] * c01 + a[0][2] * c02;
    const double id = 1.0 / g.det;
    g.Ji[0][0] = c00 * id;
    g.Ji[1][0] = c01 * id;
    g.Ji[2][0] = c02 * id;
    g.Ji[0][1] = (a[0][2] * a[2][1] - a[0][1] * a[2][2]) * id;
    g.Ji[1][1] = (a[0][0] * a[2][2] - a[0][2] * a[2][0]) * id;
    g.Ji[2][1] = (a[0][1] * a[2][0] - a[0][0] * a[2][1]) * id;
    g.Ji[0][2] = (a[0][1] * a[1][2] - a[0][2] * a[1][1]) * id;
    g.Ji[1][2] = (a[0][2] * a[1][0] - a[0][0] * a[1][2]) * id;
    g.Ji[2][2] = (a[0][0] * a[1][1] - a[0][1] * a[1][0]) * id;
  }
}

// local corner of face (axis a, side s) with tangential bits b0 (+ b1)
int face_corner(int dim, int a, int s, int b0, int b1) {
  int t[2], nt = 0;
  for (int k = 0; k < dim; ++k)
    if (k != a) t[nt++] = k;
  int c = s << a;
  c |= b0 << t[0];
  if (dim == 3) c |= b1 << t[1];
  return c;
}

struct FaceKey {
  std::array<int64_t, 4> v;
  int32_t e, k;
  bool operator<(const FaceKey& o) const {
    if (v != o.v) return v < o.v;
    if (e != o.e) return e < o.e;
    return k < o.k;
  }
};

// plus-side own tangential index j -> canonical (minus) index z, per orientation
inline void orient_map(int dim, int code, int qf, const int j[2], int z[2]) {
  if (dim == 2) {
    z[0] = (code & 1) ? qf - 1 - j[0] : j[0];
    z[1] = 0;
    return;
  }
  const int perm0 = (code & 4) ? 1 : 0, perm1 = (code & 4) ? 0 : 1;
  z[perm0] = (code & 1) ? qf - 1 - j[0] : j[0];
  z[perm1] = (code & 2) ? qf - 1 - j[1] : j[1];
}

}  // namespace

int build_plan(const sip_mesh* mesh, const int32_t* orders, const sip_options* opt_in, Plan& p,
               std::string& err) {
  if (!mesh || !orders) { err = "null mesh or orders"; return SIP_ERR_ARG; }
  const int dim = mesh->dim;
  if (dim != 2 && dim != 3) { err = "dim must be 2 or 3"; return SIP_ERR_ARG; }
  if (mesh->n_elem < 1 || mesh->n_vert < 1 || !mesh->vert || !mesh->elem_vert) {
    err = "empty mesh or null arrays"; return SIP_ERR_ARG;
  }
  sip_options opt;
  if (opt_in) opt = *opt_in; else sip_options_default(&opt);
  if (opt.qvol_extra != 2) { err = "only qvol_extra = 2 (Q = P + 2) is supported"; return SIP_ERR_ARG; }
  if (!(opt.tau_scale > 0.0)) { err = "tau_scale must be > 0"; return SIP_ERR_ARG; }
  if (opt.quad_rule != SIP_RULE_GAUSS && opt.quad_rule != SIP_RULE_GLL) {
    err = "quad_rule must be SIP_RULE_GAUSS or SIP_RULE_GLL";
    return SIP_ERR_ARG;
  }
  if (opt.force_interp != 0 && opt.force_interp != 1) { err = "force_interp must be 0 or 1"; return SIP_ERR_ARG; }
  if (opt.force_interp && opt.face_scheme != SIP_FACES_SHARED) {
    err = "force_interp applies to the shared-rule face scheme only";
    return SIP_ERR_ARG;
  }
  if (opt.face_scheme != SIP_FACES_SHARED && opt.face_scheme != SIP_FACES_P2P) {
    err = "face_scheme must be SIP_FACES_SHARED or SIP_FACES_P2P";
    return SIP_ERR_ARG;
  }
  const bool p2p = opt.face_scheme == SIP_FACES_P2P;
  p.opt = opt;
  p.dim = dim;
  const int64_t E = mesh->n_elem;
  p.E = E;
  const int nc = 1 << dim, nf = 2 * dim;
  for (int64_t e = 0; e < E; ++e) {
    if (orders[e] < 1 || orders[e] > kMaxOrder) {
      err = "element " + std::to_string(e) + ": order outside 1.." + std::to_string(kMaxOrder);
      return SIP_ERR_ARG;
    }
    for (int c = 0; c < nc; ++c) {
      int64_t v = mesh->elem_vert[e * nc + c];
      if (v < 0 || v >= mesh->n_vert) {
        err = "element " + std::to_string(e) + ": vertex id out of range"; return SIP_ERR_ARG;
      }
    }
  }
  p.P.assign(orders, orders + E);
  // volume points per direction: P + 2, or the caller's per-element counts
  p.Q.resize(E);
  for (int64_t e = 0; e < E; ++e) {
    const int q = opt.qorders ? opt.qorders[e] : p.P[e] + 2;
    if (!pair_supported(opt.quad_rule, p.P[e] + 1, q)) {
      err = "element " + std::to_string(e) + ": " + std::to_string(q) + " points per direction for order " +
            std::to_string(p.P[e]) + " is not supported with this rule (P + 2 always; with Gauss-Lobatto points "
            "also (P, Q) = (1, 4), (1, 5), (2, 5))";
      return SIP_ERR_ARG;
    }
    p.Q[e] = q;
  }
  p.dof_off.assign(E + 1, 0);
  p.quad_off.assign(E + 1, 0);
  for (int64_t e = 0; e < E; ++e) {
    int64_t n = p.P[e] + 1, q = p.Q[e];
    p.dof_off[e + 1] = p.dof_off[e] + (dim == 2 ? n * n : n * n * n);
    p.quad_off[e + 1] = p.quad_off[e] + (dim == 2 ? q * q : q * q * q);
  }
  p.ndof = p.dof_off[E];
  p.nquad = p.quad_off[E];

  // element corner coordinates
  std::vector<double> ev((size_t)E * nc * dim);
  for (int64_t e = 0; e < E; ++e)
    for (int c = 0; c < nc; ++c)
      for (int i = 0; i < dim; ++i)
        ev[(e * nc + c) * dim + i] = mesh->vert[mesh->elem_vert[e * nc + c] * dim + i];

  // ---- volume geometry (elements in parallel)
  const PointRules rules(opt.quad_rule);
  const int nG = dim == 2 ? 4 : 7;
  p.vgoff.assign(E + 1, 0);
  for (int64_t e = 0; e < E; ++e) p.vgoff[e + 1] = p.vgoff[e] + (int64_t)nG * (p.quad_off[e + 1] - p.quad_off[e]);
  p.vgeo.assign(p.vgoff[E], 0.0);
  p.xq.assign((size_t)p.nquad * dim, 0.0);
  p.vol.assign(E, 0.0);
  p.affine.assign(E, 0);
  int vrc = parallel_chunks(E, [&](int64_t e0, int64_t e1, std::string& verr) -> int {
  for (int64_t e = e0; e < e1; ++e) {
    const int Q = p.Q[e];
    const std::vector<double>& xg = rules.x[Q];
    const std::vector<double>& wg = rules.w[Q];
    const double* v = &ev[(size_t)e * nc * dim];
    const int nq = dim == 2 ? Q * Q : Q * Q * Q;
    double* G = &p.vgeo[p.vgoff[e]];
    double vol = 0.0;
    for (int q = 0; q < nq; ++q) {
      int qi[3] = {q % Q, (q / Q) % Q, q / (Q * Q)};
      double xi[3], w = 1.0;
      for (int k = 0; k < dim; ++k) { xi[k] = xg[qi[k]]; w *= wg[qi[k]]; }
      Geo g;
      eval_map(dim, v, xi, g);
      if (!(g.det > 0.0)) {
        verr = "element " + std::to_string(e) + ": non-positive Jacobian at a volume Gauss point";
        return SIP_ERR_MESH;
      }
      const double wj = w * g.det;
      vol += wj;
      // G = w|J| Ji Ji^T  (Ji[m][i] = d xi_m / d x_i)
      double Gm[3][3];
      for (int a = 0; a < dim; ++a)
        for (int b = 0; b < dim; ++b) {
          double s = 0.0;
          for (int i = 0; i < dim; ++i) s += g.Ji[a][i] * g.Ji[b][i];
          Gm[a][b] = wj * s;
        }
      if (dim == 2) {
        G[0 * nq + q] = Gm[0][0]; G[1 * nq + q] = Gm[0][1]; G[2 * nq + q] = Gm[1][1];
        G[3 * nq + q] = wj;
      } else {
        G[0 * nq + q] = Gm[0][0]; G[1 * nq + q] = Gm[0][1]; G[2 * nq + q] = Gm[0][2];
        G[3 * nq + q] = Gm[1][1]; G[4 * nq + q] = Gm[1][2]; G[5 * nq + q] = Gm[2][2];
        G[6 * nq + q] = wj;
      }
      for (int i = 0; i < dim; ++i) p.xq[(size_t)(p.quad_off[e] + q) * dim + i] = g.x[i];
    }
    p.vol[e] = vol;
    // affine iff every mixed (bi/tri-linear) coefficient of the map vanishes
    double hmax = 0.0, mixed = 0.0;
    for (int c = 1; c < nc; ++c)
      for (int i = 0; i < dim; ++i) hmax = std::max(hmax, std::fabs(v[c * dim + i] - v[i]));
    for (int m = 3; m < nc; ++m) {
      if ((m & (m - 1)) == 0) continue;  // single-axis terms are the linear part
      for (int i = 0; i < dim; ++i) {
        double s = 0.0;
        for (int c = 0; c < nc; ++c) {
          if ((c & ~m) != 0) continue;   // corners inside the sub-cube spanned by m
          const int par = __builtin_popcount((unsigned)(m & ~c)) & 1;
          s += par ? -v[c * dim + i] : v[c * dim + i];
        }
        mixed = std::max(mixed, std::fabs(s));
      }
    }
    p.affine[e] = mixed <= 1e-13 * hmax ? 1 : 0;
  }
  return 0;
  }, err);
  if (vrc) return vrc;

  // ---- face pairing by vertex sets
  const int nfc = 1 << (dim - 1);
  std::vector<FaceKey> keys;
  keys.reserve((size_t)E * nf);
  for (int64_t e = 0; e < E; ++e)
    for (int k = 0; k < nf; ++k) {
      const int a = k / 2, s = k % 2;
      FaceKey fk;
      fk.v = {-1, -1, -1, -1};
      for (int c = 0; c < nfc; ++c) {
        const int lc = face_corner(dim, a, s, c & 1, (c >> 1) & 1);
        fk.v[c] = mesh->elem_vert[e * nc + lc];
      }
      std::sort(fk.v.begin(), fk.v.begin() + nfc);
      for (int c = 1; c < nfc; ++c)
        if (fk.v[c] == fk.v[c - 1]) {
          err = "element " + std::to_string(e) + ": degenerate face (repeated vertex)";
          return SIP_ERR_MESH;
        }
      fk.e = (int32_t)e;
      fk.k = k;
      keys.push_back(fk);
    }
  std::sort(keys.begin(), keys.end());
  struct Pair { int32_t em, km, ep, kp; };
  std::vector<Pair> inter, bnd;
  for (size_t i = 0; i < keys.size();) {
    size_t j = i + 1;
    while (j < keys.size() && keys[j].v == keys[i].v) ++j;
    if (j - i == 1) bnd.push_back({keys[i].e, keys[i].k, -1, -1});
    else if (j - i == 2) {
      if (keys[i].e == keys[i + 1].e) { err = "element glued to itself"; return SIP_ERR_MESH; }
      inter.push_back({keys[i].e, keys[i].k, keys[i + 1].e, keys[i + 1].k});
    } else {
      err = "non-manifold face shared by more than two elements"; return SIP_ERR_MESH;
    }
    i = j;
  }
  auto cmp = [](const Pair& a, const Pair& b) { return a.em != b.em ? a.em < b.em : a.km < b.km; };
  std::sort(inter.begin(), inter.end(), cmp);
  std::sort(bnd.begin(), bnd.end(), cmp);
  p.n_int = (int64_t)inter.size();
  p.n_bnd = (int64_t)bnd.size();
  const int64_t F = p.n_int + p.n_bnd;
  p.f_em.resize(F); p.f_km.resize(F); p.f_ep.resize(F); p.f_kp.resize(F);
  p.f_orient.assign(F, 0); p.f_qf.resize(F);
  p.f_troff.assign(F + 1, 0); p.f_goff.assign(F + 1, 0); p.f_tau.assign(F, 0.0);
  p.slots.assign((size_t)E * nf, FaceSlot{-1, 0, 0, 0, 0});
  for (int64_t f = 0; f < F; ++f) {
    const Pair& pr = f < p.n_int ? inter[f] : bnd[f - p.n_int];
    p.f_em[f] = pr.em; p.f_km[f] = pr.km; p.f_ep[f] = pr.ep; p.f_kp[f] = pr.kp;
    const int qm = p.Q[pr.em];
    const int qp = pr.ep >= 0 ? p.Q[pr.ep] : qm;
    const int qf = std::max(qm, qp);
    p.f_qf[f] = qf;
    if (pr.ep >= 0 && p.P[pr.ep] != p.P[pr.em]) ++p.n_nonconf;
    const int64_t npts = dim == 2 ? qf : (int64_t)qf * qf;
    if (p2p && pr.ep >= 0) {
      // each side's own rule: trace [u-, g-, u+~, g+~] at qm points then
      // [u+, g+, u-~, g-~] at qp points (~: the other side's values interpolated
      // to these points); geometry [W-, c-] then [W+, c+]
      const int64_t npm = dim == 2 ? qm : (int64_t)qm * qm, npp = dim == 2 ? qp : (int64_t)qp * qp;
      p.f_troff[f + 1] = p.f_troff[f] + npm + npp;
      p.f_goff[f + 1] = p.f_goff[f] + (npm + npp) * (1 + dim);
    } else {
      p.f_troff[f + 1] = p.f_troff[f] + npts;
      p.f_goff[f + 1] = p.f_goff[f] + npts * (pr.ep >= 0 ? 1 + 2 * dim : 1 + dim);
    }
    // rule of each side's own points (qf: the shared rule), and the other side's
    // rule in the slot flags
    const int q_own_m = p2p ? qm : qf, q_own_p = p2p ? qp : qf;
    if (pr.ep >= 0) {
      // orientation: plus corner (beta0, beta1) must carry the same vertex as minus
      // corner b with b_perm[m] = beta_m xor flip_m
      const int am = pr.km / 2, sm = pr.km % 2, ap = pr.kp / 2, sp = pr.kp % 2;
      int64_t gm[4], gp[4];
      for (int c = 0; c < nfc; ++c) {
        gm[c] = mesh->elem_vert[(int64_t)pr.em * nc + face_corner(dim, am, sm, c & 1, (c >> 1) & 1)];
        gp[c] = mesh->elem_vert[(int64_t)pr.ep * nc + face_corner(dim, ap, sp, c & 1, (c >> 1) & 1)];
      }
      int found = -1;
      const int ncode = dim == 2 ? 2 : 8;
      for (int code = 0; code < ncode && found < 0; ++code) {
        bool ok = true;
        for (int c = 0; c < nfc && ok; ++c) {
          int beta[2] = {c & 1, (c >> 1) & 1}, b[2] = {0, 0};
          if (dim == 2) b[0] = beta[0] ^ (code & 1);
          else {
            const int p0 = (code & 4) ? 1 : 0, p1 = (code & 4) ? 0 : 1;
            b[p0] = beta[0] ^ (code & 1);
            b[p1] = beta[1] ^ ((code >> 1) & 1);
          }
          ok = gm[b[0] + 2 * b[1]] == gp[c];
        }
        if (ok) found = code;
      }
      if (found < 0) { err = "face " + std::to_string(f) + ": no orientation matches"; return SIP_ERR_MESH; }
      p.f_orient[f] = found;
      p.orient_hist[found] += 1;
      p.slots[(size_t)pr.em * nf + pr.km] = FaceSlot{(int32_t)f, 0, 0, (int8_t)q_own_m, face_oq_bits(q_own_p)};
      p.slots[(size_t)pr.ep * nf + pr.kp] = FaceSlot{(int32_t)f, 1, (int8_t)found, (int8_t)q_own_p, face_oq_bits(q_own_m)};
    } else {
      p.slots[(size_t)pr.em * nf + pr.km] = FaceSlot{(int32_t)f, 0, 0, (int8_t)qf, (int8_t)(kFaceBnd | face_oq_bits(qf))};
    }
  }
  p.trace_points = p.f_troff[F];

  // ---- face geometry in canonical (minus side) point order
  // W = w |J| |J^-T e_a| and c = J^-1 n of the minus side (cm) and of the plus
  // side (cp, c+ = J+^-1 (-n)) at the canonical points of the q-point Gauss rule
  // of face f; W [npts], cm and cp [dim][npts], nullptr where not wanted.
  // Returns the face area by that rule, or -1 if the two sides do not coincide.
  auto eval_face = [&](int64_t f, int qf, double* Wo, double* cmo, double* cpo) -> double {
    const std::vector<double>& xgq = rules.x[qf];
    const std::vector<double>& wgq = rules.w[qf];
    const int npts = dim == 2 ? qf : qf * qf;
    const int em = p.f_em[f], km = p.f_km[f], ep = p.f_ep[f], kp = p.f_kp[f];
    const int am = km / 2, sm = km % 2;
    int tm[2], ntm = 0;
    for (int k = 0; k < dim; ++k) if (k != am) tm[ntm++] = k;
    double area = 0.0;
    for (int z = 0; z < npts; ++z) {
      const int zi[2] = {z % qf, z / qf};
      double xi[3];
      xi[am] = sm ? 1.0 : -1.0;
      double w = 1.0;
      for (int m = 0; m < dim - 1; ++m) { xi[tm[m]] = xgq[zi[m]]; w *= wgq[zi[m]]; }
      Geo g;
      eval_map(dim, &ev[(size_t)em * nc * dim], xi, g);
      double nraw[3], nn = 0.0;
      for (int i = 0; i < dim; ++i) { nraw[i] = (sm ? 1.0 : -1.0) * g.Ji[am][i]; nn += nraw[i] * nraw[i]; }
      nn = std::sqrt(nn);
      double n[3];
      for (int i = 0; i < dim; ++i) n[i] = nraw[i] / nn;
      const double W = w * std::fabs(g.det) * nn;
      area += W;
      if (Wo) Wo[z] = W;
      if (cmo)
        for (int m = 0; m < dim; ++m) {
          double c = 0.0;
          for (int i = 0; i < dim; ++i) c += g.Ji[m][i] * n[i];
          cmo[m * npts + z] = c;
        }
      if (ep >= 0) {
        // plus-side reference point of the same physical point: invert orient_map
        const int ap = kp / 2, sp = kp % 2;
        int tp[2], ntp = 0;
        for (int k = 0; k < dim; ++k) if (k != ap) tp[ntp++] = k;
        const int code = p.f_orient[f];
        int jj[2] = {0, 0};
        // find plus index j with orient_map(j) == zi (qf^(dim-1) candidates at most 100)
        bool hit = false;
        for (int j1 = 0; j1 < (dim == 3 ? qf : 1) && !hit; ++j1)
          for (int j0 = 0; j0 < qf && !hit; ++j0) {
            int jt[2] = {j0, j1}, zz[2];
            orient_map(dim, code, qf, jt, zz);
            if (zz[0] == zi[0] && (dim == 2 || zz[1] == zi[1])) { jj[0] = j0; jj[1] = j1; hit = true; }
          }
        double xip[3];
        xip[ap] = sp ? 1.0 : -1.0;
        for (int m = 0; m < dim - 1; ++m) xip[tp[m]] = xgq[jj[m]];
        Geo gp;
        eval_map(dim, &ev[(size_t)ep * nc * dim], xip, gp);
        double dx = 0.0, h = 0.0;
        for (int i = 0; i < dim; ++i) {
          dx = std::max(dx, std::fabs(gp.x[i] - g.x[i]));
          h = std::max(h, std::fabs(g.J[i][0]) + std::fabs(g.J[i][1]) + (dim == 3 ? std::fabs(g.J[i][2]) : 0.0));
        }
        if (dx > 1e-11 * h) return -1.0;
        if (cpo)
          for (int m = 0; m < dim; ++m) {
            double c = 0.0;
            for (int i = 0; i < dim; ++i) c -= gp.Ji[m][i] * n[i];   // c+ = J+^-1 (-n)
            cpo[m * npts + z] = c;
          }
      }
    }
    return area;
  };
  p.fgeo.assign(p.f_goff[F], 0.0);
  // faces in parallel: each writes only its own geometry, penalty and the flags
  // of its own two slots
  int frc = parallel_chunks(F, [&](int64_t f0, int64_t f1, std::string& ferr) -> int {
  std::vector<double> shared_tmp;
  for (int64_t f = f0; f < f1; ++f) {
    const int qf = p.f_qf[f];
    const int npts = dim == 2 ? qf : qf * qf;
    const int em = p.f_em[f], km = p.f_km[f], ep = p.f_ep[f], kp = p.f_kp[f];
    const int am = km / 2;
    double* fg = &p.fgeo[p.f_goff[f]];
    // the shared rule's [W, c-, c+] (for the area, hence tau, and the orthogonality
    // test): stored as is, or (point-to-point) a temporary beside each side's own
    // rule [W-, c-] at Q- points then [W+, c+] at Q+ points
    const bool own = p2p && ep >= 0;
    if (own) shared_tmp.assign((size_t)(1 + 2 * dim) * npts, 0.0);
    double* sg = own ? shared_tmp.data() : fg;
    const double area = eval_face(f, qf, sg, sg + npts, ep >= 0 ? sg + (1 + dim) * npts : nullptr);
    bool ok = area > 0.0;
    if (own && ok) {
      const int qm = p.Q[em], qp = p.Q[ep];
      const int npm = dim == 2 ? qm : qm * qm, npp = dim == 2 ? qp : qp * qp;
      ok = eval_face(f, qm, fg, fg + npm, nullptr) > 0.0;
      double* fp = fg + (1 + dim) * npm;
      ok = ok && eval_face(f, qp, fp, nullptr, fp + npp) > 0.0;
    }
    if (!ok) {
      ferr = "face " + std::to_string(f) + ": sides do not coincide (mesh not conforming)";
      return SIP_ERR_MESH;
    }
    // orthogonal face: c has no tangential component on either side
    {
      bool orth = true;
      for (int z = 0; z < npts && orth; ++z) {
        const double cn = std::fabs(sg[(1 + am) * npts + z]);
        for (int m = 0; m < dim; ++m)
          if (m != am && std::fabs(sg[(1 + m) * npts + z]) > 1e-13 * cn) orth = false;
        if (ep >= 0) {
          const int ap = kp / 2;
          const double cp = std::fabs(sg[(1 + dim + ap) * npts + z]);
          for (int m = 0; m < dim; ++m)
            if (m != ap && std::fabs(sg[(1 + dim + m) * npts + z]) > 1e-13 * cp) orth = false;
        }
      }
      if (orth) {
        p.slots[(size_t)em * 2 * dim + km].flags |= kFaceOrth;
        if (ep >= 0) p.slots[(size_t)ep * 2 * dim + kp].flags |= kFaceOrth;
      }
    }
    const double vmin = ep >= 0 ? std::min(p.vol[em], p.vol[ep]) : p.vol[em];
    const double hf = vmin / area;
    const int pmax = ep >= 0 ? std::max(p.P[em], p.P[ep]) : p.P[em];
    p.f_tau[f] = opt.tau_scale * (pmax + 1.0) * (pmax + 1.0) / hf;
    if (ep < 0 && !opt.boundary)  // pure-Neumann variant: boundary faces contribute nothing
      for (int z = 0; z < npts; ++z) fg[z] = 0.0;
  }
  return 0;
  }, err);
  if (frc) return frc;

  // ---- regular (affine) elements and faces keep constants only (Sec. 5.1: regular
  // vs deformed elements): the kernels multiply by the Gauss weights themselves
  {
    std::vector<double> wv, wq;
    std::vector<int64_t> vnew(E + 1, 0);
    for (int64_t e = 0; e < E; ++e)
      vnew[e + 1] = vnew[e] + (p.affine[e] ? nG : p.vgoff[e + 1] - p.vgoff[e]);
    std::vector<double> vg(vnew[E]);
    for (int64_t e = 0; e < E; ++e) {
      const int64_t nq = p.quad_off[e + 1] - p.quad_off[e];
      const double* src = &p.vgeo[p.vgoff[e]];
      if (p.affine[e]) {
        const std::vector<double>& wq = rules.w[p.Q[e]];
        double w0 = 1.0;
        for (int k = 0; k < dim; ++k) w0 *= wq[0];
        for (int c = 0; c < nG; ++c) vg[vnew[e] + c] = src[c * nq] / w0;
      } else {
        std::copy(src, src + nG * nq, vg.begin() + vnew[e]);
      }
    }
    p.vgeo.swap(vg);
    p.vgoff.swap(vnew);
    std::vector<int64_t> fnew(F + 1, 0);
    std::vector<char> faff(F, 0);
    for (int64_t f = 0; f < F; ++f) {
      const bool aff = p.affine[p.f_em[f]] && (p.f_ep[f] < 0 || p.affine[p.f_ep[f]]);
      faff[f] = aff;
      const int ncomp = p.f_ep[f] >= 0 ? 1 + 2 * dim : 1 + dim;
      fnew[f + 1] = fnew[f] + (aff ? ncomp : p.f_goff[f + 1] - p.f_goff[f]);
    }
    std::vector<double> fgn(fnew[F]);
    for (int64_t f = 0; f < F; ++f) {
      const double* src = &p.fgeo[p.f_goff[f]];
      const int qf = p.f_qf[f];
      const int npts = dim == 2 ? qf : qf * qf;
      const int ncomp = p.f_ep[f] >= 0 ? 1 + 2 * dim : 1 + dim;
      if (faff[f] && p2p && p.f_ep[f] >= 0) {
        // own rules: [W-, c-] at Q- points, [W+, c+] at Q+ points -> the same
        // constants as a shared face (W without the weight, c-, c+)
        const int qm = p.Q[p.f_em[f]], qp = p.Q[p.f_ep[f]];
        const int npm = dim == 2 ? qm : qm * qm, npp = dim == 2 ? qp : qp * qp;
        const std::vector<double>& wq = rules.w[qm];
        const double wz = dim == 2 ? wq[0] : wq[0] * wq[0];
        fgn[fnew[f]] = src[0] / wz;
        for (int m = 0; m < dim; ++m) {
          fgn[fnew[f] + 1 + m] = src[(1 + m) * npm];
          fgn[fnew[f] + 1 + dim + m] = src[(1 + dim) * npm + (1 + m) * npp];
        }
        p.slots[(size_t)p.f_em[f] * 2 * dim + p.f_km[f]].flags |= kFaceAffine;
        p.slots[(size_t)p.f_ep[f] * 2 * dim + p.f_kp[f]].flags |= kFaceAffine;
      } else if (faff[f]) {
        const std::vector<double>& wq = rules.w[qf];
        const double wz = dim == 2 ? wq[0] : wq[0] * wq[0];
        fgn[fnew[f]] = src[0] / wz;
        for (int c = 1; c < ncomp; ++c) fgn[fnew[f] + c] = src[c * npts];
        p.slots[(size_t)p.f_em[f] * 2 * dim + p.f_km[f]].flags |= kFaceAffine;
        if (p.f_ep[f] >= 0) p.slots[(size_t)p.f_ep[f] * 2 * dim + p.f_kp[f]].flags |= kFaceAffine;
      } else {
        std::copy(src, src + (p.f_goff[f + 1] - p.f_goff[f]), fgn.begin() + fnew[f]);
      }
    }
    p.fgeo.swap(fgn);
    p.f_goff.swap(fnew);
  }

  // ---- elements sorted by order (the paper's element groups)
  p.elist.resize(E);
  std::iota(p.elist.begin(), p.elist.end(), 0);
  std::stable_sort(p.elist.begin(), p.elist.end(), [&](int32_t a, int32_t b) {
    return p.P[a] != p.P[b] ? p.P[a] < p.P[b] : p.Q[a] < p.Q[b];
  });
  p.desc_e.resize(E);
  p.desc_s.resize((size_t)E * nf);
  p.qpos.assign(E + 1, 0);
  for (int64_t i = 0; i < E; ++i) p.qpos[i + 1] = p.qpos[i] + (p.quad_off[p.elist[i] + 1] - p.quad_off[p.elist[i]]);
  for (int64_t i = 0; i < E; ++i) {
    const int32_t e = p.elist[i];
    p.desc_e[i] = ElemDesc{p.dof_off[e], p.vgoff[e], p.quad_off[e], e, (int32_t)p.affine[e]};
    for (int k = 0; k < nf; ++k) {
      const FaceSlot& sl = p.slots[(size_t)e * nf + k];
      p.desc_s[(size_t)i * nf + k] = SlotDesc{sl, p.f_troff[sl.face], p.f_goff[sl.face], p.f_tau[sl.face]};
    }
  }
  return SIP_OK;
}

// Flops (FMA = 2) of one element in the trace and main kernels: the work model
// of the apply and the cost that the CTA schedule balances.
void element_flops(const Plan& p, int64_t e, double& ft, double& fm) {
  const int d = p.dim;
  const double N = p.P[e] + 1, Q = p.Q[e];
  const double QV = d == 2 ? Q * Q : Q * Q * Q;
  const double QF1 = d == 2 ? Q : Q * Q;
  // one sum-factorised interpolation GLL -> Gauss
  const double interp = 2.0 * (d == 2 ? (N * N * Q + N * Q * Q) : (N * N * N * Q + N * N * Q * Q + N * Q * Q * Q));
  const double grad = 2.0 * d * QV * Q;
  const bool gll = p.opt.quad_rule == SIP_RULE_GLL;  // traces gathered, fluxes scattered
  const bool force = p.opt.force_interp != 0;
  ft = interp;
  fm = grad + (2.0 * d * d + d + 2.0) * QV + grad + interp;  // gradient, pointwise, D^T, B^T
  for (int k = 0; k < 2 * d; ++k) {
    const FaceSlot& sl = p.slots[(size_t)e * 2 * d + k];
    const bool orth = sl.flags & kFaceOrth;  // tangential terms vanish identically
    const double qf = sl.qf;
    const double np = d == 2 ? qf : qf * qf;
    const double nfl_t = orth ? 2.0 : 1.0 + d, nfl_m = orth ? 2.0 : 1.0 + d;
    double interp_t = 0.0, interp_m = 0.0;
    if (sl.qf != (int)Q || force) {
      const double per_field = 2.0 * (d == 2 ? qf * Q : (Q * qf * Q + qf * qf * Q));
      interp_t = nfl_t * per_field;
      interp_m = nfl_m * per_field;
    }
    // value (extrapolated, or gathered from the boundary plane) and normal
    // derivative at the element's own face points, tangential derivatives,
    // interpolation to the shared rule, c . grad
    ft += (gll ? 2.0 : 4.0) * QF1 * Q + (orth ? 0.0 : 2.0 * (d - 1) * QF1 * Q) + interp_t + 2.0 * (orth ? 1.0 : d) * np;
    // flux and projection; then either the scatter into the boundary plane
    // (1 + (1 or d) adds per point) or the tangential transposed derivative on the
    // face (P) and the lift l(+-1) P + l'(+-1) c_a t at every volume point
    fm += 12.0 * np + (orth ? 1.0 : d) * np + interp_m +
          (gll ? (1.0 + (orth ? 1.0 : d)) * QF1 : (orth ? 0.0 : 2.0 * (d - 1) * Q * QF1) + 2.0 * 2.0 * QV);
    // point-to-point interpolation of this side's two trace scalars from its own
    // rule to the other side's oq-point rule
    const int oq = face_oq(sl.flags);
    if (!(sl.flags & kFaceBnd) && oq != sl.qf)
      ft += (d == 2 ? oq : oq * oq) * 2.0 * 2.0 * (d == 2 ? qf : qf * (qf + 1.0));
  }
}

namespace {

// tile of elist[s0, s1) (n nodes and q points per direction) with its face list
// appended to fl
Tile make_tile(const Plan& p, int n, int q, int64_t s0, int64_t s1, std::vector<uint16_t>& fl) {
  int qfm = q;
  bool orth = true;
  const bool force = p.opt.force_interp != 0;
  std::vector<uint16_t> conf, fine;
  for (int64_t s = s0; s < s1; ++s)
    for (int f = 0; f < 2 * p.dim; ++f) {
      const FaceSlot& sl = p.slots[(size_t)p.elist[s] * 2 * p.dim + f];
      qfm = std::max(qfm, (int)sl.qf);
      orth = orth && (sl.flags & kFaceOrth);
      const uint16_t e = (uint16_t)((s - s0) | (f << 5) | (sl.qf << 8));
      (sl.qf == q && !force ? conf : fine).push_back(e);
    }
  std::stable_sort(fine.begin(), fine.end(), [](uint16_t a, uint16_t b) { return fl_qf(a) < fl_qf(b); });
  std::vector<std::pair<int, int>> groups;  // (qf, count)
  for (uint16_t e : fine) {
    if (groups.empty() || groups.back().first != fl_qf(e)) groups.emplace_back(fl_qf(e), 0);
    ++groups.back().second;
  }
  const int32_t off = (int32_t)fl.size();
  fl.push_back((uint16_t)conf.size());
  fl.push_back((uint16_t)fine.size());
  fl.push_back((uint16_t)groups.size());
  for (auto& g : groups) {
    fl.push_back((uint16_t)g.first);
    fl.push_back((uint16_t)g.second);
  }
  fl.insert(fl.end(), conf.begin(), conf.end());
  fl.insert(fl.end(), fine.begin(), fine.end());
  const int flags = qfm | (qfm > q || force ? kTileFine : 0) | (orth ? kTileOrth : 0) | (force ? kTileForce : 0);
  return Tile{n, q, (int32_t)s0, (int32_t)(s1 - s0), flags, off, p.qpos[s0]};
}

}  // namespace

// Tiles cut from the order-sorted element list, and the CTA that runs each.  A
// run of cnt elements of one order, whose flops are C_n of the apply's C:
//  * nctas <= 0: ceil(cnt / epb) tiles of equal size, one CTA each;
//  * persistent = false: max(ceil(cnt / epb), round(nctas C_n / C)) tiles, one CTA
//    each: with nctas = the CTAs resident at once, every tile not capped by epb
//    carries the same flops, so one wave of CTAs keeps every SM busy to the end
//    (larger meshes get more tiles than that and the hardware balances the waves);
//  * persistent = true: k_n = round(nctas C_n / C) CTAs (1 .. cnt), each an equal
//    share of the run cut into tiles of at most epb elements and run one after
//    the other.
void build_tiles(const Plan& p, int precision, const int* epb_override, int threads, int nctas, bool persistent,
                 std::vector<Tile>& tiles, std::vector<int32_t>& cta_off, std::vector<uint16_t>& flists) {
  tiles.clear();
  flists.clear();
  cta_off.assign(1, 0);
  const int64_t E = p.E;
  double C = 0.0;
  std::vector<double> ce(E);
  for (int64_t i = 0; i < E; ++i) {
    double ft = 0.0, fm = 0.0;
    element_flops(p, p.elist[i], ft, fm);
    ce[i] = ft + fm;
    C += ce[i];
  }
  for (int64_t i = 0; i < E;) {
    // a run of elements with the same (N, Q)
    const int n = p.P[p.elist[i]] + 1, q = p.Q[p.elist[i]];
    int64_t j = i;
    double Cn = 0.0;
    while (j < E && p.P[p.elist[j]] + 1 == n && p.Q[p.elist[j]] == q) Cn += ce[j++];
    int epb = epb_override && epb_override[n] > 0 ? epb_override[n] : apply_epb(p.dim, n, q, precision, threads);
    epb = std::max(1, std::min(epb, kMaxEpb));
    const int64_t cnt = j - i;
    const int64_t share = nctas > 0 ? std::max<int64_t>(1, std::llround(nctas * Cn / C)) : 0;
    // CTAs of this run and tiles per CTA
    int64_t kc = (cnt + epb - 1) / epb;
    if (nctas > 0) kc = persistent ? share : std::max(kc, share);
    kc = std::min(kc, cnt);
    for (int64_t c = 0; c < kc; ++c) {
      const int64_t r0 = i + (cnt * c) / kc, r1 = i + (cnt * (c + 1)) / kc;
      const int64_t m = r1 - r0, nt = (m + epb - 1) / epb;
      for (int64_t k = 0; k < nt; ++k)
        tiles.push_back(make_tile(p, n, q, r0 + (m * k) / nt, r0 + (m * (k + 1)) / nt, flists));
      cta_off.push_back((int32_t)tiles.size());
    }
    i = j;
  }
}

}  // namespace sip
