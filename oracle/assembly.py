"""Element-by-element, face-by-face assembly of the SIP Helmholtz matrix.

Follows the primal bilinear form of Sec. 2.2 (Eq. primal), read from the
element view of Eq. IP and the block layout of Appendix A:

    a(v, u) = sum_K [ (kappa grad v, grad u)_K + lambda (v, u)_K ]
            - ({grad v}, [[u]])_Gamma - ([[v]], {grad u})_Gamma
            + tau_F ([[u]], [[v]])_Gamma

with {w} = (w- + w+)/2 and [[u]] = u- n- + u+ n+ (Sec. 2.2, average and jump).

* Basis: tensor-product Lagrange polynomials on N = P+1 Gauss-Lobatto-Legendre
  nodes per direction (Table 1, Lagrange-GLL; Eq. expansion), DOFs element
  major, node index i0 + N i1 (+ N^2 i2).
* Volume quadrature: Q = P + qvol_extra Gauss-Legendre points per direction
  (Eq. iproduct).
* Interior faces: ONE shared Gauss rule with Q_F = max(Q-, Q+) points per
  face direction, placed in the face parametrisation of the minus side (the
  lower element id) and located in the plus element by Newton inversion of its
  geometric map (the shared trace space of Sec. 3.3; evaluating each side's
  own polynomial at the shared points is the mortar-equivalent of Sec. 3.3,
  Eq. after "mortar project").
* Point-to-point variant (``face_scheme="p2p"``, the comparison method of
  Sec. 3.3, "Point-to-point interpolation", and Table 2): each side of an
  interior face integrates on its OWN face rule (Q of that element), with the
  other side's trace values Lagrange-interpolated from the other side's own
  face points to its points; the rows of each element are then tested and
  lifted on its own rule.  The transferred quantities are the two scalars of
  the trace exchange (u and grad u . n, n the minus side's unit normal at the
  source point; Sec. 5.1 exchanges two scalars per trace point), which equals
  the paper's interpolated gradient wherever n is constant over the face.
* ``rule="gll"`` swaps every Gauss rule (volume and face) for the
  Gauss-Lobatto-Legendre rule with the same number of points (the set-up of
  Table 2), and ``qorders`` sets Q per element.
* Boundary faces: Nitsche weak Dirichlet with g = 0, i.e. [[u]] = u n and
  {grad u} = grad u on the boundary (reading of "u+ from boundary
  conditions", Sec. 2.2).
* Penalty tau_F = tau_scale (max(P-, P+) + 1)^2 / h_F with
  h_F = min(|K-|, |K+|) / |F| (|K+| omitted on the boundary); the paper leaves
  tau and h_F undefined, this is the reading used throughout.
* Optional diffusivity kappa per volume quadrature point multiplies the
  volume diffusion term only.

Everything is dense linear algebra on small per-element / per-face matrices;
no sum factorisation.  FP64.
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp

from .quadrature import gauss_legendre, gauss_lobatto, lagrange_matrix, lagrange_deriv_matrix


# ---------------------------------------------------------------- reference data

def _tensor_points(x1d, w1d, dim):
    """Tensor rule, lexicographic with coordinate 0 fastest: pts [P, dim], w [P]."""
    grids = list(itertools.product(range(len(x1d)), repeat=dim))
    pts = np.array([[x1d[g[dim - 1 - k]] for k in range(dim)] for g in grids])
    w = np.array([np.prod([w1d[gi] for gi in g]) for g in grids])
    return pts, w


_GLL = {}


def _gll_nodes(n):
    if n not in _GLL:
        _GLL[n] = gauss_lobatto(n)[0]
    return _GLL[n]


def basis_at(n_nodes: int, xi: np.ndarray):
    """phi[p, i] and reference gradient dphi[p, k, i] of the tensor Lagrange-GLL
    basis with n_nodes per direction at reference points xi [P, dim]."""
    dim = xi.shape[1]
    nodes = _gll_nodes(n_nodes)
    L = [lagrange_matrix(nodes, xi[:, k]) for k in range(dim)]
    dL = [lagrange_deriv_matrix(nodes, xi[:, k]) for k in range(dim)]
    nb = n_nodes ** dim
    phi = np.ones((xi.shape[0], nb))
    dphi = np.ones((xi.shape[0], dim, nb))
    for i in range(nb):
        ik = [(i // n_nodes ** k) % n_nodes for k in range(dim)]
        for k in range(dim):
            phi[:, i] *= L[k][:, ik[k]]
            for m in range(dim):
                dphi[:, m, i] *= (dL if m == k else L)[k][:, ik[k]]
    return phi, dphi


# ---------------------------------------------------------------- geometry

def _map(vert_e: np.ndarray, xi: np.ndarray):
    """Multilinear map of one element: x [P, dim] and J [P, dim(x), dim(xi)]."""
    dim = xi.shape[1]
    P = xi.shape[0]
    x = np.zeros((P, dim))
    J = np.zeros((P, dim, dim))
    for c in range(2 ** dim):
        bits = [(c >> k) & 1 for k in range(dim)]
        n = [(1.0 + xi[:, k]) / 2 if bits[k] else (1.0 - xi[:, k]) / 2 for k in range(dim)]
        dn = [0.5 if bits[k] else -0.5 for k in range(dim)]
        shape = np.prod(n, axis=0)
        x += shape[:, None] * vert_e[c][None, :]
        for m in range(dim):
            dshape = dn[m] * np.prod([n[k] for k in range(dim) if k != m], axis=0) if dim > 1 else np.full(P, dn[m])
            J[:, :, m] += dshape[:, None] * vert_e[c][None, :]
    return x, J


def _locate(vert_e: np.ndarray, x_target: np.ndarray, axis: int, side: int):
    """Reference coordinates in one element of physical points lying on its face
    (axis, side), by Newton's method on the multilinear map."""
    dim = x_target.shape[1]
    xi = np.zeros_like(x_target)
    xi[:, axis] = 1.0 if side else -1.0
    for _ in range(40):
        x, J = _map(vert_e, xi)
        r = x - x_target
        d = np.linalg.solve(J, -r[:, :, None])[:, :, 0]
        xi = xi + d
        if np.max(np.abs(d)) < 1e-14:
            break
    x, _ = _map(vert_e, xi)
    scale = np.max(np.abs(vert_e.max(0) - vert_e.min(0)))
    if np.max(np.abs(x - x_target)) > 1e-12 * scale or np.max(np.abs(np.abs(xi[:, axis]) - 1.0)) > 1e-10:
        raise RuntimeError("face point not found on the neighbour face")
    xi[:, axis] = 1.0 if side else -1.0
    return xi


# ---------------------------------------------------------------- oracle

class SipOracle:
    """FP64 assembly of the SIP Helmholtz matrix for one mesh.

    mesh: object with dim, vert [nv, dim], elem_vert [E, 2^dim], orders [E].
    kappa: None (= 1) or a sequence of per-element arrays of Q_e^dim values.
    boundary: False drops boundary faces (pure-Neumann variant, for tests).
    face_scheme: "shared" (one shared rule per face, Sec. 3.3) or "p2p"
        (point-to-point interpolation between the two sides' own rules).
    rule: "gauss" or "gll" quadrature points (volume and faces).
    qorders: quadrature points per direction of each element (default P + qvol_extra).
    """

    def __init__(self, mesh, lam: float = 1.0, tau_scale: float = 2.0, qvol_extra: int = 2,
                 kappa=None, boundary: bool = True, face_scheme: str = "shared", rule: str = "gauss",
                 qorders=None):
        if face_scheme not in ("shared", "p2p"):
            raise ValueError("face_scheme must be 'shared' or 'p2p'")
        if rule not in ("gauss", "gll"):
            raise ValueError("rule must be 'gauss' or 'gll'")
        self.face_scheme = face_scheme
        self.rule = rule
        self.dim = int(mesh.dim)
        self.vert = np.asarray(mesh.vert, dtype=np.float64)
        self.elem_vert = np.asarray(mesh.elem_vert, dtype=np.int64)
        self.P = np.asarray(mesh.orders, dtype=np.int64)
        self.E = self.elem_vert.shape[0]
        self.N = self.P + 1
        self.Q = self.P + qvol_extra if qorders is None else np.asarray(qorders, dtype=np.int64)
        self.lam = float(lam)
        self.tau_scale = float(tau_scale)
        self.boundary = boundary
        nb = self.N ** self.dim
        self.off = np.concatenate([[0], np.cumsum(nb)]).astype(np.int64)
        self.ndof = int(self.off[-1])
        self.kappa = kappa
        self._ref = {}
        self._vol_cache = {}
        self._build_faces()

    def volume(self, e):
        """|K| by the element's own Gauss rule."""
        if e not in self._vol_cache:
            self._vol_cache[e] = self._element_geometry(e)[4].sum()
        return self._vol_cache[e]

    # ---- reference data per (N, Q)
    def _rule_1d(self, q, rule=None):
        return (gauss_lobatto if (rule or self.rule) == "gll" else gauss_legendre)(q)

    def _ref_volume(self, n, q, rule=None):
        key = ("vol", n, q, rule or self.rule)
        if key not in self._ref:
            x1, w1 = self._rule_1d(q, rule)
            pts, w = _tensor_points(x1, w1, self.dim)
            phi, dphi = basis_at(n, pts)
            self._ref[key] = (pts, w, phi, dphi)
        return self._ref[key]

    def _element_geometry(self, e, q=None, rule=None):
        n = int(self.N[e])
        q = int(self.Q[e]) if q is None else q
        pts, w, phi, dphi = self._ref_volume(n, q, rule)
        x, J = _map(self.vert[self.elem_vert[e]], pts)
        det = np.linalg.det(J)
        if np.any(det <= 0):
            raise ValueError(f"element {e}: non-positive Jacobian")
        Jinv = np.linalg.inv(J)
        # physical gradient: grad phi = J^{-T} grad_ref phi
        gphys = np.einsum("pki,pkb->pib", Jinv, dphi)
        return x, phi, gphys, det, w * det

    # ---- faces
    def _face_corners(self, e, k):
        a, side = divmod(k, 2)
        loc = [c for c in range(2 ** self.dim) if ((c >> a) & 1) == side]
        return [int(self.elem_vert[e, c]) for c in loc]

    def _build_faces(self):
        table = {}
        for e in range(self.E):
            for k in range(2 * self.dim):
                key = tuple(sorted(self._face_corners(e, k)))
                table.setdefault(key, []).append((e, k))
        self.interior = []
        self.bfaces = []
        for key, lst in table.items():
            if len(lst) == 2:
                (e0, k0), (e1, k1) = sorted(lst)
                if e0 == e1:
                    raise ValueError("element glued to itself")
                self.interior.append(((e0, k0), (e1, k1)))
            elif len(lst) == 1:
                self.bfaces.append(lst[0])
            else:
                raise ValueError("non-manifold face (more than two elements)")
        self.interior.sort()
        self.bfaces.sort()

    def _face_rule(self, q):
        key = ("face", q, self.rule)
        if key not in self._ref:
            x1, w1 = self._rule_1d(q)
            if self.dim == 2:
                self._ref[key] = (x1[:, None], w1)
            else:
                self._ref[key] = _tensor_points(x1, w1, 2)
        return self._ref[key]

    def _side_values(self, e, k, xi):
        """phi, physical gradient at xi of element e."""
        n = int(self.N[e])
        phi, dphi = basis_at(n, xi)
        _, J = _map(self.vert[self.elem_vert[e]], xi)
        Jinv = np.linalg.inv(J)
        gphys = np.einsum("pki,pkb->pib", Jinv, dphi)
        return phi, gphys, J, Jinv

    def face_data(self, pair, qf=None):
        """Quadrature data of one interior face: W [Z], n [Z, d], tau, and for each
        side (phi, gphys·n) at the points of the qf-point face rule (default: the
        shared rule, qf = max(Q-, Q+)), placed in the minus side's face
        parametrisation.  tau always comes from the shared rule's area."""
        (em, km), (ep, kp) = pair
        qshared = int(max(self.Q[em], self.Q[ep]))
        if qf is None:
            qf = qshared
        zs, wz = self._face_rule(qf)
        am, sm = divmod(km, 2)
        xi_m = np.zeros((zs.shape[0], self.dim))
        tang = [b for b in range(self.dim) if b != am]
        xi_m[:, am] = 1.0 if sm else -1.0
        for j, b in enumerate(tang):
            xi_m[:, b] = zs[:, j]
        phim, gm, Jm, Jinvm = self._side_values(em, km, xi_m)
        xphys, _ = _map(self.vert[self.elem_vert[em]], xi_m)
        ap, sp_ = divmod(kp, 2)
        xi_p = _locate(self.vert[self.elem_vert[ep]], xphys, ap, sp_)
        phip, gp, _, _ = self._side_values(ep, kp, xi_p)
        nraw = (1.0 if sm else -1.0) * Jinvm[:, am, :]
        nrm = np.linalg.norm(nraw, axis=1)
        nvec = nraw / nrm[:, None]
        W = wz * np.abs(np.linalg.det(Jm)) * nrm
        area = W.sum() if qf == qshared else self.face_data(pair)[0].sum()
        h = min(self.volume(em), self.volume(ep)) / area
        tau = self.tau_scale * (max(self.P[em], self.P[ep]) + 1) ** 2 / h
        dnm = np.einsum("pib,pi->pb", gm, nvec)
        dnp = np.einsum("pib,pi->pb", gp, nvec)
        return W, nvec, tau, (phim, dnm), (phip, dnp)

    def boundary_face_data(self, e, k):
        a, s = divmod(k, 2)
        qf = int(self.Q[e])
        zs, wz = self._face_rule(qf)
        xi = np.zeros((zs.shape[0], self.dim))
        tang = [b for b in range(self.dim) if b != a]
        xi[:, a] = 1.0 if s else -1.0
        for j, b in enumerate(tang):
            xi[:, b] = zs[:, j]
        phi, g, J, Jinv = self._side_values(e, k, xi)
        nraw = (1.0 if s else -1.0) * Jinv[:, a, :]
        nrm = np.linalg.norm(nraw, axis=1)
        nvec = nraw / nrm[:, None]
        W = wz * np.abs(np.linalg.det(J)) * nrm
        h = self.volume(e) / W.sum()
        tau = self.tau_scale * (self.P[e] + 1) ** 2 / h
        dn = np.einsum("pib,pi->pb", g, nvec)
        return W, nvec, tau, phi, dn

    # ---- local blocks
    def element_block(self, e):
        """Volume block: sum_q w|J| [kappa grad phi_i . grad phi_j + lambda phi_i phi_j]."""
        _, phi, g, _, wdet = self._element_geometry(e)
        kap = np.ones_like(wdet) if self.kappa is None else np.asarray(self.kappa[e], dtype=np.float64)
        K = np.einsum("p,pib,pic->bc", wdet * kap, g, g)
        M = np.einsum("p,pb,pc->bc", wdet, phi, phi)
        return K + self.lam * M

    def _face_interp(self, q_from, q_to):
        """Lagrange interpolation on the face from the q_from-point rule to the
        q_to-point rule: [q_to^(d-1), q_from^(d-1)], face points z0 + q z1."""
        x_from, _ = self._rule_1d(q_from)
        x_to, _ = self._rule_1d(q_to)
        L = lagrange_matrix(x_from, x_to)
        return L if self.dim == 2 else np.kron(L, L)

    @staticmethod
    def _sip_face_block(W, tau, pv, dv, sv, pw, dw, sw):
        """sum_z W [ -1/2 s_w (dn_v)_i phi_w_j - 1/2 s_v phi_v_i (dn_w)_j + tau s_v s_w phi_v_i phi_w_j ]."""
        return (-0.5 * sw * np.einsum("z,zi,zj->ij", W, dv, pw)
                - 0.5 * sv * np.einsum("z,zi,zj->ij", W, pv, dw)
                + tau * sv * sw * np.einsum("z,zi,zj->ij", W, pv, pw))

    def interior_face_blocks(self, pair):
        """Blocks {(v, w): A_vw} of one interior face, v, w in {0 (minus), 1 (plus)}:
        sum_z W [ -1/2 s_w (dn_v)_i phi_w_j - 1/2 s_v phi_v_i (dn_w)_j + tau s_v s_w phi_v_i phi_w_j ],
        s_minus = +1, s_plus = -1, normal derivatives along the minus side's normal.

        Shared scheme: one rule for all four blocks.  Point-to-point scheme: the
        rows of side v use side v's own rule, with side w's values (phi_w,
        dn_w) taken at side w's own points and interpolated to side v's."""
        if self.face_scheme == "shared":
            W, _, tau, (phim, dnm), (phip, dnp) = self.face_data(pair)
            sides = [(phim, dnm, 1.0), (phip, dnp, -1.0)]
            out = {}
            for v in range(2):
                for w in range(2):
                    pv, dv, sv = sides[v]
                    pw, dw, sw = sides[w]
                    out[(v, w)] = self._sip_face_block(W, tau, pv, dv, sv, pw, dw, sw)
            return out
        (em, _), (ep, _) = pair
        q = (int(self.Q[em]), int(self.Q[ep]))
        # each side's data at its own rule: W, and (phi, dn) of that side
        own = []
        for v in range(2):
            W, _, tau, side_m, side_p = self.face_data(pair, qf=q[v])
            own.append((W, side_m if v == 0 else side_p))
        sgn = (1.0, -1.0)
        out = {}
        for v in range(2):
            Wv, (pv, dv) = own[v]
            for w in range(2):
                if w == v:
                    pw, dw = pv, dv
                else:
                    L = self._face_interp(q[w], q[v])
                    pw, dw = L @ own[w][1][0], L @ own[w][1][1]
                out[(v, w)] = self._sip_face_block(Wv, tau, pv, dv, sgn[v], pw, dw, sgn[w])
        return out

    def boundary_face_block(self, e, k):
        """Nitsche block: sum_z W [ -(dn)_i phi_j - phi_i (dn)_j + tau phi_i phi_j ]."""
        W, _, tau, phi, dn = self.boundary_face_data(e, k)
        return (-np.einsum("z,zi,zj->ij", W, dn, phi) - np.einsum("z,zi,zj->ij", W, phi, dn)
                + tau * np.einsum("z,zi,zj->ij", W, phi, phi))

    # ---- global objects
    def _emit(self, rows, cols, vals, e_r, e_c, blk, row_map=None):
        r0, c0 = self.off[e_r], self.off[e_c]
        nr, nc = blk.shape
        rr = np.repeat(np.arange(nr), nc)
        cc = np.tile(np.arange(nc), nr)
        if row_map is None:
            rows.append(r0 + rr)
        else:
            rows.append(row_map[e_r] + rr)
        cols.append(c0 + cc)
        vals.append(blk.ravel())

    def assemble(self):
        """Global sparse matrix A (CSR, ndof x ndof)."""
        rows, cols, vals = [], [], []
        for e in range(self.E):
            self._emit(rows, cols, vals, e, e, self.element_block(e))
        for pair in self.interior:
            blks = self.interior_face_blocks(pair)
            es = (pair[0][0], pair[1][0])
            for (v, w), blk in blks.items():
                self._emit(rows, cols, vals, es[v], es[w], blk)
        if self.boundary:
            for (e, k) in self.bfaces:
                self._emit(rows, cols, vals, e, e, self.boundary_face_block(e, k))
        A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(self.ndof, self.ndof))
        return A.tocsr()

    def rows_for_elements(self, elems):
        """Rows of A belonging to the DOFs of ``elems`` (in that order): CSR
        [sum_e N_e^d, ndof].  Only the blocks those rows need are built."""
        elems = [int(e) for e in elems]
        row_map = {}
        acc = 0
        for e in elems:
            row_map[e] = acc
            acc += int(self.off[e + 1] - self.off[e])
        rows, cols, vals = [], [], []
        wanted = set(elems)
        for e in elems:
            self._emit(rows, cols, vals, e, e, self.element_block(e), row_map)
        for pair in self.interior:
            es = (pair[0][0], pair[1][0])
            if es[0] not in wanted and es[1] not in wanted:
                continue
            blks = self.interior_face_blocks(pair)
            for (v, w), blk in blks.items():
                if es[v] in wanted:
                    self._emit(rows, cols, vals, es[v], es[w], blk, row_map)
        if self.boundary:
            for (e, k) in self.bfaces:
                if e in wanted:
                    self._emit(rows, cols, vals, e, e, self.boundary_face_block(e, k), row_map)
        return sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                             shape=(acc, self.ndof)).tocsr()

    def dofs_of(self, elems):
        return np.concatenate([np.arange(self.off[e], self.off[e + 1]) for e in elems])

    def mass_matrix(self):
        rows, cols, vals = [], [], []
        for e in range(self.E):
            _, phi, _, _, wdet = self._element_geometry(e)
            self._emit(rows, cols, vals, e, e, np.einsum("p,pb,pc->bc", wdet, phi, phi))
        return sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                             shape=(self.ndof, self.ndof)).tocsr()

    def quad_points(self, e):
        """Physical coordinates of element e's volume Gauss points [Q^d, d]."""
        return self._element_geometry(e)[0]

    def rhs(self, f):
        """b_i = sum_q w_q |J_q| phi_i(x_q) f(x_q) (Eq. iproduct)."""
        b = np.zeros(self.ndof)
        for e in range(self.E):
            x, phi, _, _, wdet = self._element_geometry(e)
            b[self.off[e]:self.off[e + 1]] = phi.T @ (wdet * f(x))
        return b

    def l2_error(self, uh, u_exact, extra=4):
        """sqrt( sum_K int_K (u_h - u)^2 ) with a (P + extra)-point Gauss rule."""
        err = 0.0
        for e in range(self.E):
            x, phi, _, _, wdet = self._element_geometry(e, q=int(self.P[e]) + extra, rule="gauss")
            diff = phi @ uh[self.off[e]:self.off[e + 1]] - u_exact(x)
            err += np.sum(wdet * diff * diff)
        return np.sqrt(err)

    def interpolate(self, u):
        """Nodal values of a function at every element's GLL nodes (the DOFs)."""
        out = np.zeros(self.ndof)
        for e in range(self.E):
            n = int(self.N[e])
            nodes, _ = gauss_lobatto(n)
            pts, _ = _tensor_points(nodes, np.ones(n), self.dim)
            x, _ = _map(self.vert[self.elem_vert[e]], pts)
            out[self.off[e]:self.off[e + 1]] = u(x)
        return out

    def kappa_gradient(self, ybar, x, elements=None):
        """d(ybar^T A(kappa) x)/d kappa_q = w_q |J_q| grad ybar_h(x_q) . grad x_h(x_q),
        one array of Q_e^d values per element (of ``elements``, default all)."""
        out = []
        for e in (range(self.E) if elements is None else elements):
            _, _, g, _, wdet = self._element_geometry(e)
            s = slice(self.off[e], self.off[e + 1])
            gy = np.einsum("pib,b->pi", g, ybar[s])
            gx = np.einsum("pib,b->pi", g, x[s])
            out.append(wdet * np.sum(gy * gx, axis=1))
        return out

    def n_quad(self):
        return int(np.sum(self.Q ** self.dim))
