"""Diffusivity, IProduct, mass products and adjoint gradients on the GPU.

Against the oracle (kappa in the volume term, kappa gradient, mass matrix,
load vector, quadrature points) and against central finite differences of
GPU solves for the gradients through the CG solve (the 16^3 hexes with P = 5
and a smoothed log-normal kappa, where the kappa gradient is also compared
with the oracle's formula on sampled elements, and a small analogue that the
oracle solves directly)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import sip_inputs as si
from oracle import SipOracle
from oracle.solve import apply_gradients, solve_gradients

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    from conftest import build_library
    return build_library()


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


MESHES = {
    "2d": si.rotate_elements(si.structured_mesh(2, 5, jitter=0.15, seed=41, order_range=(1, 6)), 42),
    "3d": si.rotate_elements(si.structured_mesh(3, 2, jitter=0.1, seed=43, order_range=(2, 5)), 44),
}


def kappa_for(m, seed):
    rng = np.random.default_rng(seed)
    return [np.exp(0.3 * rng.standard_normal((int(p) + 2) ** m.dim)) for p in m.orders]


@pytest.mark.parametrize("name", list(MESHES))
def test_kappa_apply_grad_mass_iproduct(pkg, name):
    import torch
    m = MESHES[name]
    kap = kappa_for(m, 1)
    orc = SipOracle(m, kappa=kap)
    A = orc.assemble()
    M = orc.mass_matrix()
    op = pkg.SipOperator.from_mesh(m)
    kt = torch.tensor(np.concatenate(kap), device="cuda")
    op.set_kappa(kt)
    x = si.random_vector(orc.ndof, 0)
    ybar = si.random_vector(orc.ndof, 1)
    xt = torch.tensor(x, device="cuda")
    yt = torch.tensor(ybar, device="cuda")
    assert rel(op.apply(xt).cpu().numpy(), A @ x) <= 1e-12
    assert rel(op.apply(xt.float()).double().cpu().numpy(), A @ x) <= 1e-5
    # kappa gradient
    kg = op.grad_kappa(yt, xt).cpu().numpy()
    assert rel(kg, np.concatenate(orc.kappa_gradient(ybar, x))) <= 1e-12
    kg2 = op.grad_kappa(yt, xt, out=torch.tensor(kg, device="cuda"), accumulate=True).cpu().numpy()
    assert rel(kg2, 2 * kg) <= 1e-15
    # mass inner product
    assert abs(float(op.mass_dot(yt, xt)) - ybar @ (M @ x)) <= 1e-12 * abs(ybar @ (M @ x))
    # quadrature points and IProduct
    xq = op.quad_points().cpu().numpy()
    assert np.allclose(xq, np.concatenate([orc.quad_points(e) for e in range(m.n_elem)]), atol=1e-15)
    f = np.cos(3 * xq[:, 0]) * np.exp(xq[:, 1])
    fn = lambda p: np.cos(3 * p[:, 0]) * np.exp(p[:, 1])
    assert rel(op.iproduct(torch.tensor(f, device="cuda")).cpu().numpy(), orc.rhs(fn)) <= 1e-13
    # reset to kappa = 1
    op.set_kappa(None)
    A1 = SipOracle(m).assemble()
    assert rel(op.apply(xt).cpu().numpy(), A1 @ x) <= 1e-12


def test_apply_autograd_vs_oracle(pkg):
    import torch
    m = MESHES["3d"]
    kap = kappa_for(m, 2)
    lam = 0.7
    orc = SipOracle(m, lam=lam, kappa=kap)
    A, M = orc.assemble(), orc.mass_matrix()
    op = pkg.SipOperator.from_mesh(m)
    x = si.random_vector(orc.ndof, 3)
    t = si.random_vector(orc.ndof, 4)
    xt = torch.tensor(x, device="cuda", requires_grad=True)
    lt = torch.tensor(lam, dtype=torch.float64, device="cuda", requires_grad=True)
    kt = torch.tensor(np.concatenate(kap), device="cuda", requires_grad=True)
    y = pkg.SipApplyFn.apply(op, xt, lt, kt)
    loss = torch.sum((y - torch.tensor(t, device="cuda")) ** 2)
    loss.backward()
    ybar = 2 * (A @ x - t)
    xbar, lbar, kbar = apply_gradients(orc, A, M, x, ybar)
    assert rel(xt.grad.cpu().numpy(), xbar) <= 1e-12
    assert abs(float(lt.grad) - lbar) <= 1e-11 * abs(lbar)
    assert rel(kt.grad.cpu().numpy(), np.concatenate(kbar)) <= 1e-11


def test_solve_autograd_small_vs_oracle_and_fd(pkg):
    """Small 4^3 analogue of the differentiation workload (P = 5 is replaced
    by P = 3 so the oracle can solve directly)."""
    import torch
    m = si.structured_mesh(3, 3, order=3)
    q = 5
    kap_all = si.kappa_lattice_field(3, q, seed=5)
    kap = [kap_all[e] for e in range(m.n_elem)]
    orc = SipOracle(m, kappa=kap)
    A, M = orc.assemble(), orc.mass_matrix()
    b = orc.rhs(lambda p: (1 + 3 * np.pi ** 2) * np.prod(np.sin(np.pi * p), axis=1))
    ut = spla.spsolve(SipOracle(m).assemble().tocsc(), b)   # target: the solve at kappa = 1
    op = pkg.SipOperator.from_mesh(m)
    bt = torch.tensor(b, device="cuda", requires_grad=True)
    lt = torch.tensor(1.0, dtype=torch.float64, device="cuda", requires_grad=True)
    kt = torch.tensor(np.concatenate(kap), device="cuda", requires_grad=True)
    u = pkg.SipSolveFn.apply(op, bt, lt, kt, 0, 1e-13)
    loss = torch.sum((u - torch.tensor(ut, device="cuda")) ** 2)
    loss.backward()
    u_np = spla.spsolve(A.tocsc(), b)
    bbar, lbar, kbar = solve_gradients(orc, A, M, u_np, 2 * (u_np - ut))
    assert rel(bt.grad.cpu().numpy(), bbar) <= 1e-8
    assert abs(float(lt.grad) - lbar) <= 1e-8 * abs(lbar)
    assert rel(kt.grad.cpu().numpy(), np.concatenate(kbar)) <= 1e-8


def _loss_at(op, b, ut, lam, kap):
    import torch
    op.set_lambda(lam)
    op.set_kappa(kap)
    # FP64 CG to a 1e-12 residual (near the rounding floor of the FP64 residual
    # b - A x at this conditioning, where FP32-apply refinement gains nothing)
    u, st = op.cg_solve(b, mode=0, rtol=1e-12)
    return float(torch.sum((u - ut) ** 2))


def test_solve_gradients_fd_full_c5(pkg):
    """16^3 hexes, P = 5, kappa = exp(0.5 g): gradients of L = ||u - u_target||^2
    w.r.t. kappa, lambda and the right-hand side by the adjoint solve, with the
    forward CG checkpointed every 16 iterations, against central differences
    (step 1e-6) on random directions."""
    import torch
    m = si.workload("c5_3d_16cube_p5")
    opts = pkg.options(checkpoint_every=16, max_iter=50000)
    op = pkg.SipOperator(m.dim, m.vert, m.elem_vert, m.orders, 1.0, opts)
    kap = torch.tensor(si.kappa_lattice_field(16, 7, seed=5).ravel(), device="cuda")
    xq = op.quad_points()
    f = (1.0 + 3 * np.pi ** 2) * torch.prod(torch.sin(np.pi * xq), dim=1)
    b = op.iproduct(f.contiguous())
    ut, _ = op.cg_solve(b, mode=0, rtol=1e-12)     # target: kappa = 1
    bt = b.clone().requires_grad_(True)
    lt = torch.tensor(1.0, dtype=torch.float64, device="cuda", requires_grad=True)
    kt = kap.clone().requires_grad_(True)
    u = pkg.SipSolveFn.apply(op, bt, lt, kt, 0, 1e-12)
    loss = torch.sum((u - ut) ** 2)
    loss.backward()
    assert op.checkpoint_count() > 0
    gk, gl, gb = kt.grad.clone(), float(lt.grad), bt.grad.clone()
    # the oracle's kappa gradient -w|J| grad psi . grad u on sampled elements, with
    # the GPU's u and adjoint psi (= dL/db, exactly the psi the backward used)
    orc = SipOracle(m)
    psi, u_np = gb.cpu().numpy(), u.detach().cpu().numpy()
    qoff = np.concatenate([[0], np.cumsum((m.orders + 2) ** 3)])
    sample = sorted(set(np.random.default_rng(21).choice(m.n_elem, 24, replace=False).tolist()) | {0, m.n_elem - 1})
    ref = orc.kappa_gradient(psi, u_np, elements=sample)
    gk_np = gk.cpu().numpy()
    for e, r in zip(sample, ref):
        assert rel(gk_np[qoff[e]:qoff[e + 1]], -r) <= 1e-10, e
    eps = 1e-6
    rng = np.random.default_rng(20)
    ndir = 20
    errs = []
    for i in range(ndir):
        kind = i % 3
        if kind == 0:
            d = torch.tensor(rng.standard_normal(op.nquad), device="cuda") * kap
            fp = _loss_at(op, b, ut, 1.0, (kap + eps * d).contiguous())
            fm = _loss_at(op, b, ut, 1.0, (kap - eps * d).contiguous())
            an = float(gk @ d)
        elif kind == 1:
            fp = _loss_at(op, b, ut, 1.0 + eps, kap)
            fm = _loss_at(op, b, ut, 1.0 - eps, kap)
            an = gl
        else:
            d = torch.tensor(rng.standard_normal(op.ndof), device="cuda") * b.abs().max()
            fp = _loss_at(op, (b + eps * d).contiguous(), ut, 1.0, kap)
            fm = _loss_at(op, (b - eps * d).contiguous(), ut, 1.0, kap)
            an = float(gb @ d)
        fd = (fp - fm) / (2 * eps)
        errs.append(abs(fd - an) / abs(an))
    assert max(errs) <= 1e-5, errs
