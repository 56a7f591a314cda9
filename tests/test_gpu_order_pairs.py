"""Every pair of neighbouring orders against the oracle: two elements that share
one face, orders (P-, P+) for all P in 1..8 in 2D and for P <= 6 (plus the
highest pairs) in 3D, moved interior vertex (non-affine elements) and random
rotations of each element's reference frame (every face orientation).  The
apply, the transpose apply and the FP32 apply each match the oracle's
assembled matrix: 1e-12 relative (FP64), 1e-5 (FP32)."""
import dataclasses

import numpy as np
import pytest

import sip_inputs as si
from oracle import SipOracle

pytestmark = pytest.mark.gpu

PAIRS_2D = [(p, q) for p in range(1, 9) for q in range(1, 9)]
PAIRS_3D = [(p, q) for p in range(1, 7) for q in range(1, 7)] + [(1, 8), (8, 3), (7, 8)]


@pytest.fixture(scope="module")
def pkg():
    from conftest import build_library
    return build_library()


def pair_mesh(dim, p1, p2, seed):
    """Elements 0 and 1 of the 2^dim grid of [0,1]^dim (neighbours along x),
    the grid's interior vertex moved, then each element relabelled by a random
    rotation."""
    m = si.structured_mesh(dim, 2, jitter=0.2, seed=seed, order=1)
    m = dataclasses.replace(m, elem_vert=m.elem_vert[[0, 1]], orders=np.array([p1, p2], dtype=np.int32))
    return si.rotate_elements(m, seed + 1)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("dim,pairs", [(2, PAIRS_2D), (3, PAIRS_3D)])
def test_order_pairs(pkg, dim, pairs):
    import torch
    worst = {}
    for p1, p2 in pairs:
        m = pair_mesh(dim, p1, p2, 10 * p1 + p2)
        A = SipOracle(m).assemble()
        op = pkg.SipOperator.from_mesh(m)
        x = si.random_vector(A.shape[0], p1 * 9 + p2)
        xt = torch.tensor(x, device="cuda")
        yr = A @ x
        e64 = rel(op.apply(xt).cpu().numpy(), yr)
        et = rel(op.apply_transpose(xt).cpu().numpy(), A.T @ x)
        e32 = rel(op.apply(xt.float()).double().cpu().numpy(), yr)
        worst[(p1, p2)] = (e64, et, e32)
    bad = {k: v for k, v in worst.items() if v[0] > 1e-12 or v[1] > 1e-12 or v[2] > 1e-5}
    assert not bad, bad
