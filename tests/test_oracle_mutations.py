"""Planted mistakes: each plausible error in the face terms of the oracle must
break at least one of the invariants that pin it (symmetry, Galerkin
consistency, penalty closed form).  Mistakes are planted in a subclass of the
oracle, on the CPU only."""
import numpy as np
import pytest

import sip_inputs as si
from oracle import SipOracle
from test_oracle_operator import _bubble, _rel_asym


class Mutant(SipOracle):
    def __init__(self, mesh, mutation, **kw):
        self.mutation = mutation
        super().__init__(mesh, **kw)

    def interior_face_blocks(self, pair):
        W, _, tau, (phim, dnm), (phip, dnp) = self.face_data(pair)
        mu = self.mutation
        if mu == "plus_normal_flipped":
            dnp = -dnp
        sides = [(phim, dnm, 1.0), (phip, dnp, -1.0)]
        half_sym = 1.0 if mu == "no_half_in_symmetry_term" else 0.5
        cons_sign = 1.0 if mu == "consistency_sign" else -1.0
        tau_f = 2.0 * tau if mu == "double_tau" else tau
        out = {}
        for v in range(2):
            for w in range(2):
                pv, dv, sv = sides[v]
                pw, dw, sw = sides[w]
                out[(v, w)] = (-half_sym * sw * np.einsum("z,zi,zj->ij", W, dv, pw)
                               + cons_sign * 0.5 * sv * np.einsum("z,zi,zj->ij", W, pv, dw)
                               + tau_f * sv * sw * np.einsum("z,zi,zj->ij", W, pv, pw))
        return out


def _checks(orc, m, amat, bvec, lam):
    A = orc.assemble()
    u, neg_lap = _bubble(amat, bvec, m.dim)
    lhs = A @ orc.interpolate(u)
    rhs = orc.rhs(lambda x: neg_lap(x) + lam * u(x))
    consistent = np.max(np.abs(lhs - rhs)) <= 1e-12 * np.max(np.abs(rhs))
    symmetric = _rel_asym(A) <= 1e-13
    # penalty closed form on a uniform grid (amat = identity here)
    n = int(round(np.sqrt(m.n_elem)))
    h = 1.0 / n
    pen_ok = True
    for e in range(m.n_elem):
        ex, ey = e % n, e // n
        expect = lam * h * h
        for ax, idx in enumerate((ex, ey)):
            for d in (-1, 1):
                j = idx + d
                nb = e + d * n ** ax
                pmax = max(m.orders[e], m.orders[nb]) if 0 <= j < n else m.orders[e]
                expect += 2.0 * (pmax + 1) ** 2
        ind = np.zeros(orc.ndof)
        ind[orc.off[e]:orc.off[e + 1]] = 1.0
        pen_ok &= abs(ind @ (A @ ind) - expect) <= 1e-12 * expect
    return consistent, symmetric, pen_ok


MESH = dict(dim=2, n=3, seed=8, order_range=(2, 4))


def test_unmutated_passes_all():
    m = si.rotate_elements(si.structured_mesh(**MESH), 2)
    lam = 1.1
    assert all(_checks(Mutant(m, "none", lam=lam), m, np.eye(2), np.zeros(2), lam))


@pytest.mark.parametrize("mutation", ["plus_normal_flipped", "no_half_in_symmetry_term",
                                      "consistency_sign", "double_tau"])
def test_planted_mistake_is_caught(mutation):
    m = si.rotate_elements(si.structured_mesh(**MESH), 2)
    lam = 1.1
    res = _checks(Mutant(m, mutation, lam=lam), m, np.eye(2), np.zeros(2), lam)
    assert not all(res), (mutation, res)


class P2PMutant(SipOracle):
    """The point-to-point variant with one planted mistake (a copy of the
    variant's block formula with the mistake switched in)."""

    def __init__(self, mesh, mutation, **kw):
        self.mutation = mutation
        super().__init__(mesh, face_scheme="p2p", **kw)

    def interior_face_blocks(self, pair):
        (em, _), (ep, _) = pair
        q = (int(self.Q[em]), int(self.Q[ep]))
        own = []
        for v in range(2):
            W, _, tau, side_m, side_p = self.face_data(pair, qf=q[v])
            phi, dn = side_m if v == 0 else side_p
            if v == 1 and self.mutation == "plus_normal_flipped":
                dn = -dn
            own.append((W, (phi, dn)))
        sgn = (1.0, -1.0)
        half = 1.0 if self.mutation == "no_half_in_consistency" else 0.5
        out = {}
        for v in range(2):
            Wv, (pv, dv) = own[v]
            for w in range(2):
                if w == v:
                    pw, dw = pv, dv
                else:
                    L = self._face_interp(q[w], q[v])
                    pw, dw = L @ own[w][1][0], L @ own[w][1][1]
                out[(v, w)] = (-0.5 * sgn[w] * np.einsum("z,zi,zj->ij", Wv, dv, pw)
                               - half * sgn[v] * np.einsum("z,zi,zj->ij", Wv, pv, dw)
                               + tau * sgn[v] * sgn[w] * np.einsum("z,zi,zj->ij", Wv, pv, pw))
        return out


@pytest.mark.parametrize("mutation", ["plus_normal_flipped", "no_half_in_consistency"])
def test_planted_p2p_mistake_is_caught(mutation):
    """The variant's pins: it equals the shared-rule operator wherever the lower
    order's rule is exact (here orders 2 and 4 with Gauss rules, Q = P + 2)."""
    m = si.structured_mesh(2, 4, jitter=0.0, seed=3, order_range=(2, 4))
    S = SipOracle(m).assemble().toarray()
    good = P2PMutant(m, "none").assemble().toarray()
    assert np.abs(good - S).max() <= 1e-13 * np.abs(S).max()
    bad = P2PMutant(m, mutation).assemble().toarray()
    assert np.abs(bad - S).max() > 1e-6 * np.abs(S).max()


# ---------------------------------------------------------------- non-affine face geometry
# Mistakes that leave every affine pin intact (there the Jacobian is one constant
# per element), caught by the jittered pins of test_oracle_nonaffine.py.

class FaceGradMutant(SipOracle):
    """Face gradients with the inverse Jacobian of the element centre instead
    of the one at each face point."""

    def _side_values(self, e, k, xi):
        from oracle.assembly import basis_at, _map
        phi, dphi = basis_at(int(self.N[e]), xi)
        _, J = _map(self.vert[self.elem_vert[e]], xi)
        _, Jc = _map(self.vert[self.elem_vert[e]], np.zeros((1, self.dim)))
        Jinv_c = np.repeat(np.linalg.inv(Jc), xi.shape[0], axis=0)
        gphys = np.einsum("pki,pkb->pib", Jinv_c, dphi)
        return phi, gphys, J, np.linalg.inv(J)


class PlusAreaMutant(SipOracle):
    """Face area element W built from the plus side's |det J| (at the located
    points) instead of the minus side's."""

    def face_data(self, pair, qf=None):
        from oracle.assembly import _locate, _map
        (em, km), (ep, kp) = pair
        qf = int(max(self.Q[em], self.Q[ep])) if qf is None else qf
        zs, wz = self._face_rule(qf)
        am, sm = divmod(km, 2)
        xi_m = np.zeros((zs.shape[0], self.dim))
        xi_m[:, am] = 1.0 if sm else -1.0
        for j, b in enumerate([b for b in range(self.dim) if b != am]):
            xi_m[:, b] = zs[:, j]
        phim, gm, Jm, Jinvm = self._side_values(em, km, xi_m)
        xphys, _ = _map(self.vert[self.elem_vert[em]], xi_m)
        ap, sp_ = divmod(kp, 2)
        xi_p = _locate(self.vert[self.elem_vert[ep]], xphys, ap, sp_)
        phip, gp, Jp, _ = self._side_values(ep, kp, xi_p)
        nraw = (1.0 if sm else -1.0) * Jinvm[:, am, :]
        nrm = np.linalg.norm(nraw, axis=1)
        nvec = nraw / nrm[:, None]
        W = wz * np.abs(np.linalg.det(Jp)) * nrm
        h = min(self.volume(em), self.volume(ep)) / W.sum()
        tau = self.tau_scale * (max(self.P[em], self.P[ep]) + 1) ** 2 / h
        return (W, nvec, tau, (phim, np.einsum("pib,pi->pb", gm, nvec)),
                (phip, np.einsum("pib,pi->pb", gp, nvec)))


def test_face_gradient_mistake_caught_only_on_jittered_meshes():
    from test_oracle_nonaffine import _consistency_residual, _dirichlet_case
    # invisible to the affine pins: symmetry, affine consistency, uniform penalty
    m = si.rotate_elements(si.structured_mesh(**MESH), 2)
    assert all(_checks(FaceGradMutant(m, lam=1.1), m, np.eye(2), np.zeros(2), 1.1))
    # caught by consistency on a jittered mesh
    mj, _, u, f = _dirichlet_case(2, 3, (4, 6), 0.2, 21)
    assert _rel_asym(FaceGradMutant(mj, lam=1.3).assemble()) <= 1e-13
    assert _consistency_residual(FaceGradMutant(mj, lam=1.3), u, f) > 1e-6


def test_plus_side_area_mistake_caught_by_3d_jittered_penalty():
    from test_oracle_nonaffine import _indicator_energies, _penalty_expectations_3d
    # uniform hexahedra: both sides have the same Jacobian, nothing changes
    mu = si.rotate_elements(si.structured_mesh(3, 2, seed=2, order_range=(1, 2)), 5)
    good = _indicator_energies(SipOracle(mu, lam=0.7))
    assert np.allclose(_indicator_energies(PlusAreaMutant(mu, lam=0.7)), good, rtol=1e-12, atol=0)
    # jittered hexahedra: the closed form with independent areas and volumes fails
    mj = si.rotate_elements(si.structured_mesh(3, 2, jitter=0.25, seed=41, order_range=(1, 2)), 42)
    expect, _, _ = _penalty_expectations_3d(mj, 0.7)
    assert np.max(np.abs(_indicator_energies(SipOracle(mj, lam=0.7)) - expect) / expect) <= 1e-12
    got = _indicator_energies(PlusAreaMutant(mj, lam=0.7))
    assert np.max(np.abs(got - expect) / expect) > 1e-6
