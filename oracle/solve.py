"""Plain conjugate gradients and adjoint gradients on the oracle's matrix.

CG (Sec. 2.2: the symmetric SIP system is solved by conjugate gradients):
x0 = 0, no preconditioner, stopping on the TRUE relative residual
||b - A x|| / ||b|| <= rtol (checked whenever the recursive residual passes).

Adjoint gradients of a loss through the apply y = A x and through the solve
u = A^{-1} b (the paper has no gradients; these are the standard adjoint
identities):

* apply: xbar = A^T ybar, lambdabar = ybar^T M x,
  kappabar_q = w_q |J_q| grad ybar_h(x_q) . grad x_h(x_q);
* solve: psi = A^{-T} ubar, bbar = psi, lambdabar = -psi^T M u,
  kappabar_q = -w_q |J_q| grad psi_h(x_q) . grad u_h(x_q).
"""
from __future__ import annotations

import numpy as np


def cg(A, b, rtol=1e-10, max_iter=100000, x0=None):
    """Returns (x, iterations, true relative residual)."""
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    bn = np.linalg.norm(b)
    if bn == 0.0:
        return np.zeros_like(b), 0, 0.0
    r = b - A @ x
    p = r.copy()
    rr = r @ r
    it = 0
    while it < max_iter:
        if np.sqrt(rr) <= rtol * bn:
            true = np.linalg.norm(b - A @ x) / bn
            if true <= rtol:
                return x, it, true
            r = b - A @ x
            p = r.copy()
            rr = r @ r
        Ap = A @ p
        pAp = p @ Ap
        if pAp <= 0.0:
            raise FloatingPointError("CG breakdown: p^T A p <= 0")
        alpha = rr / pAp
        x += alpha * p
        r -= alpha * Ap
        rr_new = r @ r
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
    return x, it, np.linalg.norm(b - A @ x) / bn


def apply_gradients(orc, A, M, x, ybar):
    """Gradients of L(y), y = A x, given ybar = dL/dy."""
    xbar = A.T @ ybar
    lbar = float(ybar @ (M @ x))
    kbar = orc.kappa_gradient(ybar, x)
    return xbar, lbar, kbar


def solve_gradients(orc, A, M, u, ubar, solver=None):
    """Gradients of L(u), u = A^{-1} b, given ubar = dL/du."""
    if solver is None:
        import scipy.sparse.linalg as spla
        psi = spla.spsolve(A.T.tocsc(), ubar)
    else:
        psi = solver(A.T, ubar)
    bbar = psi
    lbar = -float(psi @ (M @ u))
    kbar = [-k for k in orc.kappa_gradient(psi, u)]
    return bbar, lbar, kbar
