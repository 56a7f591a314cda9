"""Pin of the oracle's diffusivity term: kappa multiplies the volume diffusion
integrand at every volume Gauss point, so that the assembled operator is the
SIP discretisation of -div(kappa grad u) + lambda u.

The paper has no kappa; what it fixes is the volume term of the Helmholtz
operator (Sec. 2.2, Eq. IP).  With kappa - 1 vanishing on every element face,
the face terms see kappa = 1 whichever way a face treatment of kappa would be
read, and Galerkin consistency is exact:

    A(kappa) I(u) = b(-div(kappa grad u) + lambda u)

for the pure-Neumann operator and a polynomial u with zero normal derivative
on the boundary, because every integrand is a polynomial that the (P+2)-point
Gauss rules integrate exactly (uniform grid: kappa - 1 = c prod_k x_k (x_k -
1/2) (1 - x_k) on the 2^d grid has degree 3 per variable).  A kappa applied at
the wrong point, squared, left out of one gradient component or applied to the
mass term breaks the identity.
"""
import numpy as np
import pytest

import sip_inputs as si
from oracle import SipOracle

# kappa - 1 reaches about 0.05 (2D) and 0.2 (3D) of kappa = 1
C_K = {2: 20.0, 3: 2000.0}


def _kappa(x):
    return 1.0 + C_K[x.shape[1]] * np.prod(x * (x - 0.5) * (1.0 - x), axis=1)


def _grad_kappa(x):
    f = x * (x - 0.5) * (1.0 - x)
    df = -3.0 * x * x + 3.0 * x - 0.5          # d/ds of s (s - 1/2) (1 - s)
    out = np.zeros_like(x)
    for k in range(x.shape[1]):
        out[:, k] = C_K[x.shape[1]] * df[:, k] * np.prod(np.delete(f, k, axis=1), axis=1)
    return out


def _u(x):
    return np.sum(x * x * (3.0 - 2.0 * x), axis=1)       # grad u . n = 0 on the boundary


def _grad_u(x):
    return 6.0 * x * (1.0 - x)


def _lap_u(x):
    return np.sum(6.0 - 12.0 * x, axis=1)


@pytest.mark.parametrize("dim,orders", [(2, (3, 5)), (3, (3, 4))])
def test_kappa_volume_term_consistency(dim, orders):
    lam = 0.6
    m = si.rotate_elements(si.structured_mesh(dim, 2, seed=61, order_range=orders), 62)
    probe = SipOracle(m, lam=lam, boundary=False)
    kappa = [_kappa(probe.quad_points(e)) for e in range(m.n_elem)]
    assert max(np.max(np.abs(k - 1.0)) for k in kappa) > 1e-2     # kappa really varies
    orc = SipOracle(m, lam=lam, boundary=False, kappa=kappa)

    def f(x):
        return -(np.sum(_grad_kappa(x) * _grad_u(x), axis=1) + _kappa(x) * _lap_u(x)) + lam * _u(x)

    lhs = orc.assemble() @ orc.interpolate(_u)
    rhs = orc.rhs(f)
    assert np.max(np.abs(lhs - rhs)) <= 1e-12 * np.max(np.abs(rhs))
    # the identity distinguishes kappa from 1: without kappa it fails
    lhs1 = SipOracle(m, lam=lam, boundary=False).assemble() @ orc.interpolate(_u)
    assert np.max(np.abs(lhs1 - rhs)) > 1e-4 * np.max(np.abs(rhs))
