"""Parity of the CUDA point-to-point interpolation variant (SIP_FACES_P2P;
Sec. 3.3 "Point-to-point interpolation", Table 2) with the oracle's variant,
and the paper's finding on the GPU: the variant loses symmetry where the
lower-order side's own rule is not exact for the face integrand, while the
shared-rule operator stays symmetric.  Tolerances as for the shared-rule
apply: 1e-12 relative in FP64, 1e-5 in FP32."""
import numpy as np
import pytest

import sip_inputs as si
from oracle import SipOracle

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 1e-5


@pytest.fixture(scope="module")
def pkg():
    from conftest import build_library
    return build_library()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _half(dim, n, p_low, p_high, jitter=0.0, seed=1):
    m = si.structured_mesh(dim, n, jitter=jitter, seed=seed, order=1)
    left = m.vert[m.elem_vert].mean(axis=1)[:, 0] < 0.5
    m.orders = np.where(left, p_low, p_high).astype(np.int32)
    return m


MESHES = {
    "2d_rot_jitter_p1to8": si.rotate_elements(si.structured_mesh(2, 9, jitter=0.2, seed=21, order_range=(1, 8)), 22),
    "2d_half_p2_p6": _half(2, 4, 2, 6),
    "3d_rot_jitter_p1to5": si.rotate_elements(si.structured_mesh(3, 3, jitter=0.15, seed=23, order_range=(1, 5)), 24),
    "3d_rot_p2to8": si.rotate_elements(si.structured_mesh(3, 2, jitter=0.1, seed=25, order_range=(2, 8)), 26),
    "3d_half_p2_p7_affine": _half(3, 2, 2, 7),
    "2d_affine_skew": si.affine_map_vertices(si.rotate_elements(si.structured_mesh(2, 5, seed=27, order_range=(2, 7)), 28),
                                             np.array([[1.1, 0.4], [-0.3, 0.8]])),
}


def _op(pkg, m, scheme):
    return pkg.SipOperator.from_mesh(m, opts=pkg.options(face_scheme=scheme))


def _apply(op, x, dtype):
    import torch
    y = op.apply(torch.tensor(x, device="cuda", dtype=dtype))
    torch.cuda.synchronize()
    return y.double().cpu().numpy()


@pytest.mark.parametrize("name", list(MESHES))
def test_p2p_apply_parity(pkg, name):
    import torch
    m = MESHES[name]
    A = SipOracle(m, lam=m.lam, face_scheme="p2p").assemble()
    op = _op(pkg, m, pkg.SIP_FACES_P2P)
    x = si.random_vector(A.shape[0], 0)
    yr = A @ x
    y = _apply(op, x, torch.float64)
    assert rel(y, yr) <= TOL64, rel(y, yr)
    scale = np.abs(A) @ np.abs(x)
    assert np.max(np.abs(y - yr) / scale) <= 1e-13
    y32 = _apply(op, x, torch.float32)
    assert rel(y32, yr) <= TOL32, rel(y32, yr)
    # multi-RHS launch: every column as its own apply
    X = si.random_rhs_batch(3, A.shape[0], 5)
    Y = op.apply(torch.tensor(X, device="cuda")).cpu().numpy()
    for r in range(3):
        assert rel(Y[r], A @ X[r]) <= TOL64


def test_p2p_equals_shared_on_conforming_mesh(pkg):
    import torch
    m = si.rotate_elements(si.structured_mesh(3, 3, jitter=0.15, seed=31, order=4), 32)
    x = si.random_vector(si.ndof(m.orders, 3), 0)
    a = _apply(_op(pkg, m, pkg.SIP_FACES_P2P), x, torch.float64)
    b = _apply(_op(pkg, m, pkg.SIP_FACES_SHARED), x, torch.float64)
    assert rel(a, b) <= 1e-15


def test_symmetry_lost_only_by_p2p_c2(pkg):
    """64x64 jittered quads, orders 2..6: faces between orders 2 and 6 need a
    rule exact to degree 8 on the order-2 side, whose own 4-point Gauss rule is
    exact to 7, so the point-to-point operator is not symmetric; the shared-rule
    operator is, to rounding (Sec. 3.3, Sec. 4.1)."""
    import torch
    m = si.workload("c2_2d_64x64_jitter_p2to6")
    asym = {}
    for scheme in (pkg.SIP_FACES_SHARED, pkg.SIP_FACES_P2P):
        op = _op(pkg, m, scheme)
        n = op.ndof
        x1 = torch.tensor(si.random_vector(n, 0), device="cuda")
        x2 = torch.tensor(si.random_vector(n, 1), device="cuda")
        a = float(x1 @ op.apply(x2))
        b = float(x2 @ op.apply(x1))
        asym[scheme] = abs(a - b) / float(torch.linalg.norm(x1) * torch.linalg.norm(op.apply(x2)))
    assert asym[pkg.SIP_FACES_SHARED] <= 1e-13
    assert asym[pkg.SIP_FACES_P2P] >= 1e-8


def test_p2p_rejects_transpose_and_solves(pkg):
    import torch
    m = MESHES["2d_half_p2_p6"]
    op = _op(pkg, m, pkg.SIP_FACES_P2P)
    x = torch.tensor(si.random_vector(op.ndof, 0), device="cuda")
    with pytest.raises(pkg.SipError) as e:
        op.apply_transpose(x)
    assert e.value.code == pkg._lib.SIP_ERR_ARG
    with pytest.raises(pkg.SipError):
        op.cg_solve(x)
