"""Pins of the oracle's face geometry on non-affine (bilinear / trilinear)
elements: jittered meshes, where the Jacobian varies from point to point.

Galerkin consistency holds EXACTLY (to rounding) on such meshes, not only up
to a quadrature error.  Let u be a polynomial in the physical coordinates and
F the multilinear map of an element.  Every coordinate of F has degree <= 1
in each reference variable, so u o F lies in Q_P as soon as P >= deg u, and the
nodal interpolant reproduces u.  The integrands of a(v, u) and of the load
(v, f) (Sec. 2.2, Eq. primal) are then polynomials in the reference
coordinates:

* volume:  w |J| J^-1 J^-T grad_ref(u o F) = w adj(J) grad_x u, with
  adj(J) = |J| J^-1 a polynomial for a multilinear map;
* faces:   W grad u . n = w |J| |J^-T e_a| (J^-T e_a / |J^-T e_a|) . grad_x u
           = w (adj(J)^T e_a) . grad_x u;
* load:    v f |J| with f polynomial.

Their degrees stay within what the (P+2)-point Gauss rules integrate exactly,
so A I(u) = b(-lap u + lambda u) to rounding.  A mistake in the pointwise face
Jacobian, normal, area element, the inverse Jacobian of the face gradients or
the location of the shared points in the neighbour breaks the identity; the
affine pins of test_oracle_operator.py cannot see any of these, because there
the Jacobian is one constant per element.

The penalty closed form 1_K^T A 1_K = lambda |K| + sum_F tau_F |F| is checked
on jittered hexahedra as well, with |K| from the test's own integration of
det J and |F| from the test's own cross product of the face parametrisation,
which pins h_F = min(|K-|, |K+|) / |F| on warped faces (the reading of the
undefined penalty length, with |F| by the face's shared Gauss rule).
"""
import itertools

import numpy as np
import pytest
from numpy.polynomial.legendre import leggauss

import sip_inputs as si
from oracle import SipOracle
from test_oracle_operator import _bubble


def _consistency_residual(orc, u, f):
    lhs = orc.assemble() @ orc.interpolate(u)
    rhs = orc.rhs(f)
    return np.max(np.abs(lhs - rhs)) / np.max(np.abs(rhs))


def _dirichlet_case(dim, n, orders, jitter, seed, lam=1.3, **kw):
    m = si.rotate_elements(si.structured_mesh(dim, n, jitter=jitter, seed=seed, order_range=orders), seed + 1)
    u, neg_lap = _bubble(np.eye(dim), np.zeros(dim), dim)
    orc = SipOracle(m, lam=lam, **kw)
    return m, orc, u, (lambda x: neg_lap(x) + lam * u(x))


def _neumann_poly(dim):
    """u = sum_k g(x_k), g(s) = s^2 (3 - 2 s): degree 3, grad u . n = 0 on the
    faces of the unit square / cube (g'(0) = g'(1) = 0); -lap u = -sum_k (6 - 12 x_k)."""
    def u(x):
        return np.sum(x * x * (3.0 - 2.0 * x), axis=1)

    def neg_lap(x):
        return -np.sum(6.0 - 12.0 * x, axis=1)
    return u, neg_lap


@pytest.mark.parametrize("n,orders,jitter,seed", [(3, (4, 6), 0.2, 21), (4, (4, 5), 0.25, 23)])
def test_consistency_jittered_2d(n, orders, jitter, seed):
    m, orc, u, f = _dirichlet_case(2, n, orders, jitter, seed)
    assert len(set(m.orders.tolist())) > 1
    assert _consistency_residual(orc, u, f) <= 1e-12


def test_consistency_jittered_3d_dirichlet():
    """Trilinear hexahedra with Nitsche boundary faces: the bubble has degree 2
    in each coordinate, so P = 6."""
    m, orc, u, f = _dirichlet_case(3, 2, (6, 6), 0.2, 31)
    assert _consistency_residual(orc, u, f) <= 1e-12


def test_consistency_jittered_3d_neumann_nonconforming():
    """Trilinear hexahedra with p-non-conforming faces (orders 3 and 4) on the
    pure-Neumann operator, where a degree-3 polynomial with zero normal
    derivative on the boundary makes the identity exact."""
    m = si.rotate_elements(si.structured_mesh(3, 3, jitter=0.2, seed=33, order_range=(3, 4)), 34)
    assert len(set(m.orders.tolist())) > 1
    lam = 0.8
    u, neg_lap = _neumann_poly(3)
    orc = SipOracle(m, lam=lam, boundary=False)
    assert _consistency_residual(orc, u, lambda x: neg_lap(x) + lam * u(x)) <= 1e-12


def test_consistency_jittered_2d_neumann_nonconforming():
    m = si.rotate_elements(si.structured_mesh(2, 5, jitter=0.25, seed=35, order_range=(3, 6)), 36)
    lam = 0.8
    u, neg_lap = _neumann_poly(2)
    orc = SipOracle(m, lam=lam, boundary=False)
    assert _consistency_residual(orc, u, lambda x: neg_lap(x) + lam * u(x)) <= 1e-12


def test_consistency_is_exact_not_converging():
    """Over-integration (Q = P + 6) leaves the residual at rounding level: the
    identity above is exact with the standard rules, so a residual that only
    shrank with more points would point at a wrong integrand."""
    m, orc, u, f = _dirichlet_case(2, 3, (4, 5), 0.2, 25)
    r2 = _consistency_residual(orc, u, f)
    r6 = _consistency_residual(SipOracle(m, lam=1.3, qvol_extra=6), u, f)
    assert r2 <= 1e-12 and r6 <= 1e-12


# ---------------------------------------------------------------- 3D penalty closed form

def _trilinear_jacobian(c, xi):
    """d x / d xi of the trilinear map through corners c [8, 3] (corner bit k
    = side along reference axis k) at reference points xi [P, 3]."""
    J = np.zeros((xi.shape[0], 3, 3))
    for k in range(8):
        b = [(k >> a) & 1 for a in range(3)]
        lin = [(1.0 + xi[:, a]) / 2 if b[a] else (1.0 - xi[:, a]) / 2 for a in range(3)]
        for m in range(3):
            d = (0.5 if b[m] else -0.5) * np.prod([lin[a] for a in range(3) if a != m], axis=0)
            J[:, :, m] += d[:, None] * c[k][None, :]
    return J


def _hex_volume(c):
    """|K| = int det J over the reference cube; det J of a trilinear map has
    degree <= 2 in each variable, so 3 Gauss points per direction are exact."""
    x, w = leggauss(3)
    pts = np.array(list(itertools.product(x, x, x)))
    wts = np.array([a * b * d for a, b, d in itertools.product(w, w, w)])
    return float(np.sum(wts * np.linalg.det(_trilinear_jacobian(c, pts))))


def _face_area(c4, q):
    """Area of the bilinear face through corners c4 [4, 3] (bit 0: first
    tangential side, bit 1: second) by the q-point Gauss rule per direction,
    area element |x_s x x_t|."""
    x, w = leggauss(q)
    area = 0.0
    for (s, ws), (t, wt) in itertools.product(zip(x, w), zip(x, w)):
        ls = [(1 - s) / 2, (1 + s) / 2]
        lt = [(1 - t) / 2, (1 + t) / 2]
        xs = sum((-0.5 if (k & 1) == 0 else 0.5) * lt[k >> 1] * c4[k] for k in range(4))
        xt = sum((-0.5 if (k >> 1) == 0 else 0.5) * ls[k & 1] * c4[k] for k in range(4))
        area += ws * wt * np.linalg.norm(np.cross(xs, xt))
    return area


def _face_corners(m, e, a, s):
    tang = [b for b in range(3) if b != a]
    out = []
    for k in range(4):
        c = (s << a) | ((k & 1) << tang[0]) | (((k >> 1) & 1) << tang[1])
        out.append(int(m.elem_vert[e, c]))
    return out


def _penalty_expectations_3d(m, lam, qvol_extra=2):
    vol = [_hex_volume(m.vert[m.elem_vert[e]]) for e in range(m.n_elem)]
    faces = {}
    for e in range(m.n_elem):
        for a in range(3):
            for s in range(2):
                cs = _face_corners(m, e, a, s)
                faces.setdefault(tuple(sorted(cs)), []).append((e, cs))
    expect = [lam * v for v in vol]
    for lst in faces.values():
        els = [e for e, _ in lst]
        pmax = max(int(m.orders[e]) for e in els)
        qf = max(int(m.orders[e]) + qvol_extra for e in els)   # the shared face rule
        area = _face_area(m.vert[lst[0][1]], qf)
        h = min(vol[e] for e in els) / area
        for e in els:
            expect[e] += 2.0 * (pmax + 1) ** 2 / h * area
    return np.array(expect), vol, faces


def _indicator_energies(orc):
    A = orc.assemble()
    out = []
    for e in range(orc.E):
        ind = np.zeros(orc.ndof)
        ind[orc.off[e]:orc.off[e + 1]] = 1.0
        out.append(ind @ (A @ ind))
    return np.array(out)


def test_penalty_closed_form_3d_jittered():
    m = si.rotate_elements(si.structured_mesh(3, 3, jitter=0.25, seed=41, order_range=(1, 3)), 42)
    lam = 0.7
    expect, vol, faces = _penalty_expectations_3d(m, lam)
    # the mesh really has warped faces: the rule's area differs from the exact one
    warped = [abs(_face_area(m.vert[lst[0][1]], 2) - _face_area(m.vert[lst[0][1]], 30)) for lst in faces.values()]
    assert max(warped) > 1e-8
    got = _indicator_energies(SipOracle(m, lam=lam))
    assert np.max(np.abs(got - expect) / expect) <= 1e-12
