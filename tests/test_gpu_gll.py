"""Gauss-Lobatto-Legendre point sets on the GPU (sip_options.quad_rule =
SIP_RULE_GLL; Sec. 3.2 "Gather & interpolate trace data", Sec. 5.1): the P+2
volume points per direction include the endpoints, so the trace kernel gathers
u on a face and the main kernel scatters the flux back before the one
IProduct.  Parity with the oracle's rule="gll" assembly at 1e-12 (FP64) and
1e-5 (FP32); forced interpolation on every face gives the same operator; the
point-to-point variant with these rules reproduces Table 2's classification on
the GPU; and the largest orders (9, 10) of the default rule are checked
against the oracle's rows.
"""
import numpy as np
import pytest

import sip_inputs as si
from oracle import SipOracle
from test_gpu_apply import TOL32, TOL64, gpu_apply, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    from conftest import build_library
    return build_library()


MESHES = {
    "2d_rot_jitter_p1to8": si.rotate_elements(si.structured_mesh(2, 7, jitter=0.2, seed=71, order_range=(1, 8)), 72),
    "2d_conforming_p4": si.structured_mesh(2, 4, jitter=0.15, seed=73, order=4),
    "3d_rot_jitter_p1to5": si.rotate_elements(si.structured_mesh(3, 3, jitter=0.15, seed=74, order_range=(1, 5)), 75),
    "3d_affine_p3": si.structured_mesh(3, 3, order=3),
}


def _gll_op(pkg, m, **kw):
    return pkg.SipOperator.from_mesh(m, opts=pkg.options(quad_rule=pkg.SIP_RULE_GLL, **kw))


@pytest.mark.parametrize("name", list(MESHES))
def test_gll_apply_parity(pkg, name):
    m = MESHES[name]
    A = SipOracle(m, lam=m.lam, rule="gll").assemble()
    op = _gll_op(pkg, m)
    x = si.random_vector(A.shape[0], 0)
    yr = A @ x
    y = gpu_apply(op, x)
    assert rel(y, yr) <= TOL64, rel(y, yr)
    scale = np.abs(A) @ np.abs(x)
    assert np.max(np.abs(y - yr) / scale) <= 1e-13
    assert rel(gpu_apply(op, x, transpose=True), A.T @ x) <= TOL64
    assert rel(gpu_apply(op, x, "f32"), yr) <= TOL32
    # on deformed elements the Gauss-Legendre operator is another discretisation
    # (the integrands are rational); on affine ones both (P+2)-point rules are
    # exact and the operators coincide
    yg = gpu_apply(pkg.SipOperator.from_mesh(m), x)
    if "affine" in name:
        assert rel(yg, yr) <= TOL64
    else:
        assert rel(yg, yr) > 1e-8


@pytest.mark.parametrize("rule", ["gauss", "gll"])
@pytest.mark.parametrize("name", ["2d_rot_jitter_p1to8", "3d_rot_jitter_p1to5"])
def test_forced_interpolation_same_operator(pkg, name, rule):
    """Interpolation to the shared rule on every face (identity where the rules
    match) changes the work, not the operator."""
    m = MESHES[name]
    r = pkg.SIP_RULE_GLL if rule == "gll" else pkg.SIP_RULE_GAUSS
    x = si.random_vector(si.ndof(m.orders, m.dim), 1)
    y0 = gpu_apply(pkg.SipOperator.from_mesh(m, opts=pkg.options(quad_rule=r)), x)
    opf = pkg.SipOperator.from_mesh(m, opts=pkg.options(quad_rule=r, force_interp=1))
    y1 = gpu_apply(opf, x)
    assert rel(y1, y0) <= 1e-13
    assert rel(gpu_apply(opf, x, transpose=True), y0) <= 1e-12
    assert rel(gpu_apply(opf, x, "f32"), y0) <= TOL32
    w0 = pkg.SipOperator.from_mesh(m, opts=pkg.options(quad_rule=r)).work_model()
    assert opf.work_model()["flops_trace"] > w0["flops_trace"]


def test_gll_symmetry_and_cg(pkg):
    import torch
    m = MESHES["2d_rot_jitter_p1to8"]
    orc = SipOracle(m, rule="gll")
    A = orc.assemble()
    op = _gll_op(pkg, m)
    x1, x2 = si.random_vector(orc.ndof, 2), si.random_vector(orc.ndof, 3)
    y1, y2 = gpu_apply(op, x1), gpu_apply(op, x2)
    assert abs(x2 @ y1 - x1 @ y2) <= 1e-13 * np.linalg.norm(x1) * np.linalg.norm(y2)
    b = orc.rhs(lambda p: (1 + 2 * np.pi ** 2) * np.prod(np.sin(np.pi * p), axis=1))
    for mode in (pkg.SIP_CG_FP64, pkg.SIP_CG_FP32_REFINED):
        u, st = op.cg_solve(torch.tensor(b, device="cuda"), mode=mode, rtol=1e-10)
        u = u.cpu().numpy()
        assert np.linalg.norm(b - A @ u) <= 1e-10 * np.linalg.norm(b)


def test_gll_quadrature_points_and_iproduct(pkg):
    """The auxiliary kernels use the same rule: sip_quad_points returns the GLL
    points of each element, sip_iproduct the oracle's load vector."""
    import torch
    m = MESHES["3d_rot_jitter_p1to5"]
    orc = SipOracle(m, rule="gll")
    op = _gll_op(pkg, m)
    xq = op.quad_points().cpu().numpy()
    ref = np.concatenate([orc.quad_points(e) for e in range(m.n_elem)])
    assert np.max(np.abs(xq - ref)) <= 1e-14
    f = lambda p: np.cos(p[:, 0]) + p[:, 1] * p[:, 2]
    b = op.iproduct(torch.tensor(f(xq), device="cuda")).cpu().numpy()
    assert rel(b, orc.rhs(f)) <= 1e-13


def _half_mesh(dim, n, p_low, p_high, jitter=0.0, seed=1):
    mm = si.structured_mesh(dim, n, jitter=jitter, seed=seed, order=1)
    left = mm.vert[mm.elem_vert].mean(axis=1)[:, 0] < 0.5
    mm.orders = np.where(left, p_low, p_high).astype(np.int32)
    return mm


def _asym(op, ndof, pkg):
    """max over a few vector pairs of |x1^T A x2 - x2^T A x1| / (|x1| |A x2|),
    measured through the GPU apply."""
    worst = 0.0
    for s in range(3):
        x1, x2 = si.random_vector(ndof, 10 + s), si.random_vector(ndof, 20 + s)
        y1, y2 = gpu_apply(op, x1), gpu_apply(op, x2)
        worst = max(worst, abs(x2 @ y1 - x1 @ y2) / (np.linalg.norm(x1) * np.linalg.norm(y2)))
    return worst


@pytest.mark.parametrize("deg_low,deg_high,jitter,symmetric", [
    (2, 4, 0.0, False),    # P3Q4-P5Q6 (coefficient counts): the low side's 4 GLL points are not exact
    (3, 4, 0.0, True),     # P4Q5-P5Q6 on affine geometry: exact, symmetric
    (3, 4, 0.2, False),    # P4Q5-P5Q6 on trilinear geometry (p_geom = 1): not exact
])
def test_table2_point_to_point_on_gpu(pkg, deg_low, deg_high, jitter, symmetric):
    """Table 2 (Sec. 4.1) with the paper's rules, GLL with Q = P + 2 points
    (counts P+1 coefficients, P+2 points), on 2^3 hexahedra: the GPU's
    point-to-point operator equals the oracle's, is symmetric exactly where the
    lower side's rule integrates the face term exactly, and the shared-rule
    operator (the method) is symmetric in every case."""
    m = _half_mesh(3, 2, deg_low, deg_high, jitter=jitter, seed=1)
    orc = SipOracle(m, rule="gll", face_scheme="p2p")
    A = orc.assemble()
    op = pkg.SipOperator.from_mesh(m, opts=pkg.options(quad_rule=pkg.SIP_RULE_GLL, face_scheme=pkg.SIP_FACES_P2P))
    x = si.random_vector(orc.ndof, 5)
    assert rel(gpu_apply(op, x), A @ x) <= TOL64
    a = _asym(op, orc.ndof, pkg)
    if symmetric:
        assert a <= 1e-13, a
    else:
        assert a >= 5e-5, a
    assert _asym(_gll_op(pkg, m), orc.ndof, pkg) <= 1e-13


def test_orders_9_and_10_against_oracle_rows(pkg):
    """The largest orders: one element of order 10 and one of order 9 among
    order-3 neighbours (p-non-conforming faces with 12-point shared rules), 3D
    jittered, and a 2D mesh with every order 1..10; rows of the oracle."""
    m3 = si.structured_mesh(3, 2, jitter=0.1, seed=77, order=3)
    m3.orders[0], m3.orders[7] = 10, 9
    orc = SipOracle(m3)
    op = pkg.SipOperator.from_mesh(m3)
    x = si.random_vector(orc.ndof, 6)
    y = gpu_apply(op, x)
    for e in (0, 7):
        R = orc.rows_for_elements([e])
        assert rel(y[orc.off[e]:orc.off[e + 1]], R @ x) <= TOL64
    y32 = gpu_apply(op, x, "f32")
    assert rel(y32, y) <= TOL32
    m2 = si.rotate_elements(si.structured_mesh(2, 6, jitter=0.15, seed=78, order_range=(1, 10)), 79)
    assert {9, 10} <= set(m2.orders.tolist())
    A2 = SipOracle(m2).assemble()
    x2 = si.random_vector(A2.shape[0], 7)
    op2 = pkg.SipOperator.from_mesh(m2)
    assert rel(gpu_apply(op2, x2), A2 @ x2) <= TOL64
    assert rel(gpu_apply(op2, x2, transpose=True), A2.T @ x2) <= TOL64
    assert rel(gpu_apply(op2, x2, "f32"), A2 @ x2) <= TOL32


def _column_mesh(n, spec):
    """n x n quads of the unit square; column c (along x) gets (degree, points)
    spec[c] (the paper's counts are coefficients: degree = count - 1)."""
    mm = si.structured_mesh(2, n, order=1)
    col = (mm.vert[mm.elem_vert].mean(axis=1)[:, 0] * n).astype(int)
    mm.orders = np.array([spec[c][0] for c in col], dtype=np.int32)
    return mm, np.array([spec[c][1] for c in col], dtype=np.int32)


def test_transition_layer_on_gpu(pkg):
    """Sec. 3.3's transition layer with the point-to-point variant: a P4Q5
    element (4 coefficients, 5 GLL points) next to P2Q3 ones is not
    symmetric; a layer of P2Q5 elements (the lower order's coefficients, the
    higher order's points) between them makes both interfaces exact and the
    operator symmetric.  GPU against the oracle's assembly with the same
    per-element point counts, and the symmetry measured through the GPU apply."""
    high, trans, low = (3, 5), (1, 5), (1, 3)
    res = {}
    for name, n, spec in (("direct", 2, [high, low]), ("layered", 3, [high, trans, low])):
        m, q = _column_mesh(n, spec)
        orc = SipOracle(m, face_scheme="p2p", rule="gll", qorders=q)
        A = orc.assemble()
        op = pkg.SipOperator.from_mesh(m, opts=pkg.options(quad_rule=pkg.SIP_RULE_GLL, face_scheme=pkg.SIP_FACES_P2P,
                                                           qorders=q))
        x = si.random_vector(orc.ndof, 8)
        assert rel(gpu_apply(op, x), A @ x) <= TOL64
        assert rel(gpu_apply(op, x, "f32"), A @ x) <= TOL32
        res[name] = _asym(op, orc.ndof, pkg)
        # the shared-rule operator with the same point counts
        S = SipOracle(m, rule="gll", qorders=q).assemble()
        ops = pkg.SipOperator.from_mesh(m, opts=pkg.options(quad_rule=pkg.SIP_RULE_GLL, qorders=q))
        assert rel(gpu_apply(ops, x), S @ x) <= TOL64
        assert rel(gpu_apply(ops, x, transpose=True), S.T @ x) <= TOL64
    assert res["direct"] >= 1e-4, res
    assert res["layered"] <= 1e-13, res


def test_table2_p3q5_on_gpu(pkg):
    """Table 2's P3Q5-P5Q6 (degree 2 on 5 GLL points, degree 4 on 6): the
    lower side's own rule is exact, so the point-to-point operator is
    symmetric; GPU against the oracle."""
    m = _half_mesh(3, 2, 2, 4)
    left = m.vert[m.elem_vert].mean(axis=1)[:, 0] < 0.5
    q = np.where(left, 5, 6).astype(np.int32)
    orc = SipOracle(m, rule="gll", face_scheme="p2p", qorders=q)
    A = orc.assemble()
    op = pkg.SipOperator.from_mesh(m, opts=pkg.options(quad_rule=pkg.SIP_RULE_GLL, face_scheme=pkg.SIP_FACES_P2P,
                                                       qorders=q))
    x = si.random_vector(orc.ndof, 9)
    assert rel(gpu_apply(op, x), A @ x) <= TOL64
    assert _asym(op, orc.ndof, pkg) <= 1e-13

