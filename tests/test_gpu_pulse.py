"""Local p-refinement on the Gaussian-pulse problem (Sec. 4.2) solved on the
GPU: the CG solution of the refined mesh agrees with the oracle's direct solve
(2D), and in 3D (8^3 hexahedra of [-1,1]^3, orders 2 | 5 inside [-0.5,0.5]^3)
the refined mesh reaches close to the uniform order-5 error with far fewer
degrees of freedom, in FP64 CG and in FP32-refined CG.  Errors are measured by
the oracle's L2 norm on the downloaded solution."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import sip_inputs as si
from oracle import SipOracle
from test_oracle_pulse import f_pulse, u_pulse

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    from conftest import build_library
    return build_library()


def _gpu_solve(pkg, m, mode):
    import torch
    op = pkg.SipOperator.from_mesh(m)
    xq = op.quad_points().cpu().numpy()
    f = torch.tensor(f_pulse(xq, m.dim), device="cuda")
    b = op.iproduct(f)
    u, st = op.cg_solve(b, mode=mode, rtol=1e-10)
    assert st["converged"] == 1 and st["rel_residual"] <= 1e-10
    return op.ndof, u.cpu().numpy()


def test_pulse_2d_gpu_solution_matches_oracle(pkg):
    m = si.pulse_refined_mesh(2, 8, 2, 5)
    o = SipOracle(m)
    ud = spla.spsolve(o.assemble().tocsc(), o.rhs(lambda x: f_pulse(x, 2)))
    for mode in (pkg.SIP_CG_FP64, pkg.SIP_CG_FP32_REFINED):
        _, u = _gpu_solve(pkg, m, mode)
        assert np.linalg.norm(u - ud) <= 1e-7 * np.linalg.norm(ud)


def test_pulse_3d_local_refinement(pkg):
    res = {}
    for key, (pl, ph) in {"low": (2, 2), "local": (2, 5), "high": (5, 5)}.items():
        m = si.pulse_refined_mesh(3, 8, pl, ph)
        n, u = _gpu_solve(pkg, m, pkg.SIP_CG_FP64)
        res[key] = (n, SipOracle(m).l2_error(u, u_pulse))
        if key == "local":
            _, u32 = _gpu_solve(pkg, m, pkg.SIP_CG_FP32_REFINED)
            assert abs(SipOracle(m).l2_error(u32, u_pulse) - res[key][1]) <= 1e-3 * res[key][1]
    assert res["local"][0] < 0.5 * res["high"][0]
    assert res["local"][1] < 3.0 * res["high"][1]
    assert res["local"][1] < res["low"][1] / 20
