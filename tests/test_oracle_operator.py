"""Pins of the oracle's SIP matrix against what the paper and the mathematics fix.

* symmetry of A, also across p-non-conforming faces and arbitrary relative
  element orientations (Sec. 2.2 / Appendix A: symmetric iff both sides use
  the same face quadrature);
* the penalty closed form 1_K^T A 1_K = lambda |K| + sum_F tau_F |F|, with
  |K| and |F| from elementary geometry (a constant has no gradient, so only
  the mass and the tau([[u]],[[v]]) term of Eq. primal survive);
* Galerkin consistency: for a global polynomial u of degree <= min P that
  vanishes on the boundary, A I(u) equals the load vector of
  f = -lap u + lambda u (integration by parts of Eq. primal; every face term
  must cancel exactly for this to hold);
* the constant mode spans the kernel of the pure-Neumann stiffness;
* positive definiteness; sum of the mass matrix = |Omega|;
* the P+2 Gauss rule is exact on affine meshes (over-integration changes
  nothing);
* invariance under relabelling the local vertices of every element;
* manufactured-solution convergence at order P+1 in L2 (Sec. 4.2).
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import sip_inputs as si
from oracle import SipOracle
from oracle.quadrature import gauss_legendre


def _rel_asym(A):
    D = A - A.T
    return abs(D).max() / abs(A).max()


def test_symmetry_c1():
    A = SipOracle(si.workload("c1_2d_4x4_p3")).assemble()
    assert _rel_asym(A) <= 1e-13


@pytest.mark.parametrize("dim,n,orders,jit,seed", [
    (2, 6, (1, 5), 0.2, 11),
    (2, 5, (2, 6), 0.15, 12),
    (3, 3, (1, 3), 0.15, 13),
])
def test_symmetry_nonconforming_rotated(dim, n, orders, jit, seed):
    m = si.structured_mesh(dim, n, jitter=jit, seed=seed, order_range=orders)
    m = si.rotate_elements(m, seed + 100)
    assert len(set(m.orders.tolist())) > 1
    A = SipOracle(m).assemble()
    assert _rel_asym(A) <= 1e-13


def _shoelace(pts):
    x, y = pts[:, 0], pts[:, 1]
    return 0.5 * abs(np.dot(x, np.roll(y, -1)) - np.dot(y, np.roll(x, -1)))


def test_penalty_closed_form_2d_jittered():
    m = si.structured_mesh(2, 5, jitter=0.2, seed=3, order_range=(1, 5))
    m = si.rotate_elements(m, 4)
    lam = 0.7
    orc = SipOracle(m, lam=lam)
    A = orc.assemble()
    # elementary geometry, independent of the oracle
    area = []
    for e in range(m.n_elem):
        c = m.vert[m.elem_vert[e]]
        area.append(_shoelace(c[[0, 1, 3, 2]]))
    edges = {}
    for e in range(m.n_elem):
        ev = m.elem_vert[e]
        for a, b in ((0, 1), (2, 3), (0, 2), (1, 3)):
            key = tuple(sorted((int(ev[a]), int(ev[b]))))
            edges.setdefault(key, []).append(e)
    for e in range(m.n_elem):
        expect = lam * area[e]
        for key, els in edges.items():
            if e not in els:
                continue
            length = np.linalg.norm(m.vert[key[0]] - m.vert[key[1]])
            if len(els) == 2:
                pmax = max(m.orders[els[0]], m.orders[els[1]])
                h = min(area[els[0]], area[els[1]]) / length
            else:
                pmax = m.orders[e]
                h = area[e] / length
            expect += 2.0 * (pmax + 1) ** 2 / h * length
        ind = np.zeros(orc.ndof)
        ind[orc.off[e]:orc.off[e + 1]] = 1.0
        got = ind @ (A @ ind)
        assert abs(got - expect) <= 1e-12 * expect


def test_penalty_closed_form_3d_uniform():
    n = 3
    m = si.structured_mesh(3, n, seed=2, order_range=(1, 3))
    m = si.rotate_elements(m, 5)
    orc = SipOracle(m, lam=1.0)
    A = orc.assemble()
    h = 1.0 / n
    for e in range(m.n_elem):
        ex, ey, ez = e % n, (e // n) % n, e // (n * n)
        expect = h ** 3
        for ax, idx in enumerate((ex, ey, ez)):
            for d in (-1, 1):
                j = idx + d
                if 0 <= j < n:
                    nb = e + d * n ** ax
                    pmax = max(m.orders[e], m.orders[nb])
                else:
                    pmax = m.orders[e]
                expect += 2.0 * (pmax + 1) ** 2 / h * h * h
        ind = np.zeros(orc.ndof)
        ind[orc.off[e]:orc.off[e + 1]] = 1.0
        assert abs(ind @ (A @ ind) - expect) <= 1e-12 * expect


def _bubble(amat, bvec, dim):
    """u = prod_k s_k (1 - s_k), s = amat^{-1}(x - b): a degree-2 polynomial in x
    vanishing on the mapped unit square/cube; returns u and -lap u."""
    C = np.linalg.inv(amat)
    CC = C @ C.T

    def s_of(x):
        return (x - bvec) @ C.T

    def u(x):
        s = s_of(x)
        return np.prod(s * (1 - s), axis=1)

    def neg_lap(x):
        s = s_of(x)
        g = s * (1 - s)
        g1 = 1 - 2 * s
        out = np.zeros(x.shape[0])
        for k in range(dim):
            for l in range(dim):
                if k == l:
                    term = -2.0 * np.prod(np.delete(g, k, axis=1), axis=1)
                else:
                    term = g1[:, k] * g1[:, l] * np.prod(np.delete(g, [k, l], axis=1), axis=1)
                out += CC[k, l] * term
        return -out

    return u, neg_lap


@pytest.mark.parametrize("dim,n,orders,seed", [(2, 4, (2, 5), 1), (2, 3, (2, 2), 2), (3, 2, (2, 3), 3)])
def test_galerkin_consistency_affine(dim, n, orders, seed):
    amat = np.array([[1.2, 0.3], [-0.2, 0.9]]) if dim == 2 else np.array([[1.1, 0.2, -0.1], [0.1, 0.9, 0.2], [-0.15, 0.05, 1.3]])
    bvec = np.full(dim, 0.25)
    m = si.structured_mesh(dim, n, seed=seed, order_range=orders)
    m = si.affine_map_vertices(si.rotate_elements(m, seed + 7), amat, bvec)
    lam = 1.3
    orc = SipOracle(m, lam=lam)
    A = orc.assemble()
    u, neg_lap = _bubble(amat, bvec, dim)
    lhs = A @ orc.interpolate(u)
    rhs = orc.rhs(lambda x: neg_lap(x) + lam * u(x))
    assert np.max(np.abs(lhs - rhs)) <= 1e-12 * np.max(np.abs(rhs))
    # the identity is sensitive: a wrong face term breaks it
    orc_bad = SipOracle(m, lam=lam, tau_scale=2.0)
    orc_bad.boundary = False
    lhs_bad = orc_bad.assemble() @ orc.interpolate(u)
    assert np.max(np.abs(lhs_bad - rhs)) > 1e-6 * np.max(np.abs(rhs))


@pytest.mark.parametrize("dim,n,orders,jit", [(2, 5, (1, 6), 0.2), (3, 2, (1, 3), 0.1)])
def test_constant_in_neumann_kernel(dim, n, orders, jit):
    m = si.rotate_elements(si.structured_mesh(dim, n, jitter=jit, seed=9, order_range=orders), 10)
    A = SipOracle(m, lam=0.0, boundary=False).assemble()
    one = np.ones(A.shape[0])
    assert np.max(np.abs(A @ one)) <= 1e-12 * abs(A).max()


def test_spd_c1():
    A = SipOracle(si.workload("c1_2d_4x4_p3")).assemble().toarray()
    ev = np.linalg.eigvalsh(0.5 * (A + A.T))
    assert ev.min() > 0


def test_mass_sums_to_area():
    m = si.structured_mesh(2, 6, jitter=0.2, seed=1, order_range=(2, 6))
    M = SipOracle(m).mass_matrix()
    assert abs(M.sum() - 1.0) < 1e-13
    m3 = si.structured_mesh(3, 2, jitter=0.1, seed=1, order_range=(1, 3))
    M3 = SipOracle(m3).mass_matrix()
    assert abs(M3.sum() - 1.0) < 1e-13


@pytest.mark.parametrize("dim,n,orders", [(2, 4, (3, 3)), (2, 4, (1, 6)), (3, 2, (1, 3))])
def test_gauss_rule_exact_on_affine(dim, n, orders):
    m = si.rotate_elements(si.structured_mesh(dim, n, seed=4, order_range=orders), 3)
    amat = np.eye(dim) + 0.2 * np.tri(dim, dim, -1)
    m = si.affine_map_vertices(m, amat)
    A = SipOracle(m).assemble()
    A8 = SipOracle(m, qvol_extra=8).assemble()
    assert abs(A - A8).max() <= 1e-12 * abs(A).max()


def test_orientation_invariance():
    base = si.structured_mesh(2, 4, jitter=0.2, seed=5, order_range=(2, 4))
    rot = si.rotate_elements(base, 6)
    g = lambda x: np.exp(x[:, 0]) * np.cos(2 * x[:, 1])
    res = []
    for m in (base, rot):
        orc = SipOracle(m)
        r = orc.assemble() @ orc.interpolate(g)
        # physical position of every DOF
        pos = []
        from oracle.assembly import _map, _tensor_points, _gll_nodes
        for e in range(m.n_elem):
            nodes = _gll_nodes(int(orc.N[e]))
            pts, _ = _tensor_points(nodes, np.ones(nodes.size), 2)
            x, _ = _map(m.vert[m.elem_vert[e]], pts)
            pos.append(x)
        res.append((r, pos, orc.off))
    (r0, p0, o0), (r1, p1, o1) = res
    for e in range(base.n_elem):
        a = np.lexsort(np.round(p0[e], 12).T[::-1])
        b = np.lexsort(np.round(p1[e], 12).T[::-1])
        assert np.allclose(p0[e][a], p1[e][b], atol=1e-13)
        assert np.allclose(r0[o0[e]:o0[e + 1]][a], r1[o1[e]:o1[e + 1]][b], rtol=0, atol=1e-11)


def _sine_error(dim, n, P, rotate=False, lam=1.0):
    m = si.structured_mesh(dim, n, order=P)
    if rotate:
        m = si.rotate_elements(m, 1)
    orc = SipOracle(m, lam=lam)
    A = orc.assemble()
    ue = lambda x: np.prod(np.sin(np.pi * x), axis=1)
    b = orc.rhs(lambda x: (lam + dim * np.pi ** 2) * ue(x))
    uh = spla.spsolve(A.tocsc(), b)
    return orc.l2_error(uh, ue)


@pytest.mark.parametrize("P", [2, 3])
def test_convergence_order_2d(P):
    errs = [_sine_error(2, n, P, rotate=(P == 3)) for n in (4, 8, 16)]
    rates = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert rates[-1] >= P + 1 - 0.2, (errs, rates)


def test_convergence_order_3d():
    errs = [_sine_error(3, n, 2) for n in (2, 4, 6)]
    rate = np.log(errs[1] / errs[2]) / np.log(6 / 4)
    assert rate >= 3 - 0.2, (errs, rate)


@pytest.mark.parametrize("P", [2, 3])
def test_half_domain_p_refinement(P):
    """Sec. 4.2: with half of the domain one order higher (sin(2 pi x) sin(2 pi y),
    k = 2 pi), the L2 error converges at the rate of the lower order, P + 1,
    like the unrefined mesh, and is only somewhat lower than its error (the
    lower-order half dominates)."""
    k = 2 * np.pi

    def err(n, p_left, p_right):
        m = si.structured_mesh(2, n, order=1)
        left = m.vert[m.elem_vert].mean(axis=1)[:, 0] < 0.5
        m.orders = np.where(left, p_left, p_right).astype(np.int32)
        orc = SipOracle(m)
        ue = lambda x: np.prod(np.sin(k * x), axis=1)
        uh = spla.spsolve(orc.assemble().tocsc(), orc.rhs(lambda x: (1 + 2 * k * k) * ue(x)))
        return orc.l2_error(uh, ue)

    uni = [err(n, P, P) for n in (4, 8, 16)]
    half = [err(n, P, P + 1) for n in (4, 8, 16)]
    rate = np.log2(half[1] / half[2])
    assert abs(rate - np.log2(uni[1] / uni[2])) <= 0.2 and rate >= P + 1 - 0.2, (half, uni)
    for h, u in zip(half, uni):
        assert 0.4 * u <= h < u
