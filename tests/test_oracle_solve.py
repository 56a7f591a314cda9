"""Oracle CG and adjoint gradients, pinned by a direct sparse solve and by
central finite differences of the oracle's own assembly (a different code
path from the adjoint formulas)."""
import numpy as np
import scipy.sparse.linalg as spla

import sip_inputs as si
from oracle import SipOracle
from oracle.solve import cg, apply_gradients, solve_gradients


def test_cg_matches_direct_solve():
    orc = SipOracle(si.workload("c1_2d_4x4_p3"))
    A = orc.assemble()
    ue = lambda x: np.prod(np.sin(np.pi * x), axis=1)
    b = orc.rhs(lambda x: (1 + 2 * np.pi ** 2) * ue(x))
    x, it, res = cg(A, b, rtol=1e-10)
    assert res <= 1e-10 and it > 0
    xd = spla.spsolve(A.tocsc(), b)
    assert np.linalg.norm(x - xd) <= 1e-8 * np.linalg.norm(xd)


def _kappa_mesh():
    m = si.structured_mesh(2, 3, jitter=0.15, seed=2, order_range=(2, 3))
    rng = np.random.default_rng(3)
    kap = [np.exp(0.3 * rng.standard_normal((int(p) + 2) ** 2)) for p in m.orders]
    return m, kap


def test_apply_gradients_vs_central_fd():
    m, kap = _kappa_mesh()
    lam = 0.8
    orc = SipOracle(m, lam=lam, kappa=kap)
    A, M = orc.assemble(), orc.mass_matrix()
    rng = np.random.default_rng(0)
    x = rng.standard_normal(orc.ndof)
    ybar = rng.standard_normal(orc.ndof)
    xbar, lbar, kbar = apply_gradients(orc, A, M, x, ybar)
    L = lambda A_: ybar @ (A_ @ x)
    # A is affine in lambda and kappa, so a central difference is exact up to
    # rounding for any step; a large step keeps rounding small
    eps = 1e-2
    # lambda
    fd = (L(SipOracle(m, lam=lam + eps, kappa=kap).assemble()) - L(SipOracle(m, lam=lam - eps, kappa=kap).assemble())) / (2 * eps)
    assert abs(fd - lbar) <= 1e-6 * abs(lbar)
    # kappa direction
    dk = [rng.standard_normal(k.size) for k in kap]
    kp = [k + eps * d for k, d in zip(kap, dk)]
    km = [k - eps * d for k, d in zip(kap, dk)]
    fd = (L(SipOracle(m, lam=lam, kappa=kp).assemble()) - L(SipOracle(m, lam=lam, kappa=km).assemble())) / (2 * eps)
    an = sum(float(g @ d) for g, d in zip(kbar, dk))
    assert abs(fd - an) <= 1e-6 * abs(an)
    # x
    dx = rng.standard_normal(orc.ndof)
    assert abs(ybar @ (A @ dx) - xbar @ dx) <= 1e-12 * abs(xbar @ dx)


def test_solve_gradients_vs_central_fd():
    m, kap = _kappa_mesh()
    lam = 1.0
    orc = SipOracle(m, lam=lam, kappa=kap)
    A, M = orc.assemble(), orc.mass_matrix()
    rng = np.random.default_rng(1)
    b = rng.standard_normal(orc.ndof)
    ut = rng.standard_normal(orc.ndof) * 0.1

    def loss(lam_, kap_, b_):
        A_ = SipOracle(m, lam=lam_, kappa=kap_).assemble()
        u_ = spla.spsolve(A_.tocsc(), b_)
        return np.sum((u_ - ut) ** 2)

    u = spla.spsolve(A.tocsc(), b)
    bbar, lbar, kbar = solve_gradients(orc, A, M, u, 2 * (u - ut))
    eps = 1e-6
    fd = (loss(lam + eps, kap, b) - loss(lam - eps, kap, b)) / (2 * eps)
    assert abs(fd - lbar) <= 1e-5 * abs(lbar)
    dk = [rng.standard_normal(k.size) for k in kap]
    fd = (loss(lam, [k + eps * d for k, d in zip(kap, dk)], b) - loss(lam, [k - eps * d for k, d in zip(kap, dk)], b)) / (2 * eps)
    an = sum(float(g @ d) for g, d in zip(kbar, dk))
    assert abs(fd - an) <= 1e-5 * abs(an)
    db = rng.standard_normal(orc.ndof)
    fd = (loss(lam, kap, b + eps * db) - loss(lam, kap, b - eps * db)) / (2 * eps)
    assert abs(fd - bbar @ db) <= 1e-5 * abs(bbar @ db)
