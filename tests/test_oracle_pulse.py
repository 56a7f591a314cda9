"""Local p-refinement on the Gaussian-pulse problem (Sec. 4.2, with the
exponent's sign read as exp(-r^2/a^2)): the cube [-1,1]^d, a = 0.2, the
elements inside [-0.5,0.5]^d at the higher order.  The paper's finding: with
the refinement where the solution lives, the error is close to that of the
uniformly high-order mesh at a fraction of its degrees of freedom.  Checked
here on the oracle with a direct sparse solve (2D, 8x8 quads, orders 2 | 5)."""
import numpy as np
import scipy.sparse.linalg as spla

import sip_inputs as si
from oracle import SipOracle

A_PULSE = 0.2


def u_pulse(x):
    return np.exp(-np.sum(x * x, axis=1) / A_PULSE ** 2)


def f_pulse(x, dim, lam=1.0):
    """-Laplace u + lam u for the pulse: (2d/a^2 - 4 r^2/a^4 + lam) u."""
    r2 = np.sum(x * x, axis=1)
    return (2 * dim / A_PULSE ** 2 - 4 * r2 / A_PULSE ** 4 + lam) * u_pulse(x)


def _solve(m):
    o = SipOracle(m)
    A = o.assemble()
    b = o.rhs(lambda x: f_pulse(x, m.dim))
    u = spla.spsolve(A.tocsc(), b)
    return o.ndof, o.l2_error(u, u_pulse)


def test_local_refinement_matches_uniform_high_order():
    n_low, e_low = _solve(si.pulse_refined_mesh(2, 8, 2, 2))
    n_loc, e_loc = _solve(si.pulse_refined_mesh(2, 8, 2, 5))
    n_high, e_high = _solve(si.pulse_refined_mesh(2, 8, 5, 5))
    assert n_loc < 0.5 * n_high
    assert e_loc < 3.0 * e_high
    assert e_loc < e_low / 50
