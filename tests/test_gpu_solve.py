"""CG on the GPU (FP64, and FP32 apply inside FP64 refinement) against the
oracle: true residual of the FP64 oracle matrix <= 1e-10, agreement with a
direct sparse solve, multi-RHS, determinism, checkpoint replay, the transpose
solve, and the error paths (not converged, non-finite input, breakdown)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import sip_inputs as si
from oracle import SipOracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    from conftest import build_library
    return build_library()


def sine_rhs(orc, dim, lam=1.0):
    return orc.rhs(lambda p: (lam + dim * np.pi ** 2) * np.prod(np.sin(np.pi * p), axis=1))


def true_res(A, b, x):
    return float(np.linalg.norm(b - A @ x) / np.linalg.norm(b))


MESH_2D = si.rotate_elements(si.structured_mesh(2, 8, jitter=0.15, seed=31, order_range=(2, 6)), 32)
MESH_3D = si.rotate_elements(si.structured_mesh(3, 3, jitter=0.1, seed=33, order_range=(1, 4)), 34)


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("which", ["c1", "2d", "3d"])
def test_cg_modes_reach_1e10(pkg, mode, which):
    import torch
    m = {"c1": si.workload("c1_2d_4x4_p3"), "2d": MESH_2D, "3d": MESH_3D}[which]
    orc = SipOracle(m)
    A = orc.assemble()
    b = sine_rhs(orc, m.dim)
    op = pkg.SipOperator.from_mesh(m)
    x, st = op.cg_solve(torch.tensor(b, device="cuda"), mode=mode, rtol=1e-10)
    x = x.cpu().numpy()
    assert true_res(A, b, x) <= 1e-10, (true_res(A, b, x), st)
    assert st["converged"] == 1 and st["rel_residual"] <= 1e-10
    xd = spla.spsolve(A.tocsc(), b)
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) <= 1e-6
    if mode == 1:
        assert st["refinements"] >= 1 and st["applies_fp32"] > 0


def test_cg_multi_rhs_and_determinism(pkg):
    import torch
    m = MESH_3D
    orc = SipOracle(m)
    A = orc.assemble()
    B = si.random_rhs_batch(4, orc.ndof, 7)
    B[2] *= 1e3
    op = pkg.SipOperator.from_mesh(m)
    Bt = torch.tensor(B, device="cuda")
    for mode in (0, 1):
        X, st = op.cg_solve(Bt, mode=mode, rtol=1e-10)
        X2, _ = op.cg_solve(Bt, mode=mode, rtol=1e-10)
        assert torch.equal(X, X2), "solves are not bit-reproducible"
        Xn = X.cpu().numpy()
        for r in range(4):
            assert true_res(A, B[r], Xn[r]) <= 1e-10


def test_transpose_solve(pkg):
    import torch
    m = MESH_2D
    orc = SipOracle(m)
    A = orc.assemble()
    b = si.random_vector(orc.ndof, 2)
    op = pkg.SipOperator.from_mesh(m)
    bt = torch.tensor(b, device="cuda")
    x, _ = op.cg_solve(bt, rtol=1e-11)
    xt, _ = op.cg_solve(bt, rtol=1e-11, transpose=True)
    assert true_res(A.T, b, xt.cpu().numpy()) <= 1e-11
    assert float(torch.linalg.norm(x - xt) / torch.linalg.norm(x)) <= 1e-8


def test_checkpoint_replay_bit_exact(pkg):
    import torch
    m = MESH_2D
    orc = SipOracle(m)
    b = sine_rhs(orc, 2)
    opts = pkg.options(checkpoint_every=16, checkpoint_slots=64)
    op = pkg.SipOperator(m.dim, m.vert, m.elem_vert, m.orders, 1.0, opts)
    bt = torch.tensor(b, device="cuda")
    x, st = op.cg_solve(bt, rtol=1e-10)
    n = op.checkpoint_count()
    assert n >= 3 and st["checkpoints"] == n
    x0, r0, p0, rr0, k0 = op.checkpoint(0)
    x1, r1, p1, rr1, k1 = op.checkpoint(1)
    assert k1 - k0 == 16
    rr = op.replay(x0, r0, p0, rr0, 16)
    torch.cuda.synchronize()
    assert torch.equal(x0, x1) and torch.equal(r0, r1) and torch.equal(p0, p1)
    assert rr == rr1
    # checkpointing does not change the result
    op2 = pkg.SipOperator.from_mesh(m)
    x2, _ = op2.cg_solve(bt, rtol=1e-10)
    assert torch.equal(x, x2)


@pytest.mark.parametrize("mode,nrhs", [(1, 1), (0, 4), (1, 4)])
def test_checkpoint_replay_refined_and_batched(pkg, mode, nrhs):
    """Checkpoints of the FP32 recurrence of the refined solve and of batched
    solves: continuing a checkpoint's recurrence to the next checkpoint (no
    refinement or residual replacement in between) reproduces that
    checkpoint's FP64 iterate bit for bit, and checkpointing leaves the
    solution unchanged."""
    import torch
    m = MESH_2D
    orc = SipOracle(m)
    b = sine_rhs(orc, 2)
    B = torch.tensor(b if nrhs == 1 else si.random_rhs_batch(nrhs, orc.ndof, 7), device="cuda")
    op = pkg.SipOperator(m.dim, m.vert, m.elem_vert, m.orders, 1.0,
                         pkg.options(checkpoint_every=16, checkpoint_slots=256))
    x, st = op.cg_solve(B, mode=mode, rtol=1e-10)
    n = op.checkpoint_count()
    assert n >= 3 and st["checkpoints"] == n
    info = [op.checkpoint_info(i) for i in range(n)]
    assert all(c["nrhs"] == nrhs for c in info)
    keys = ("mode", "refinements", "restarts")
    pairs = [(i, i + 1) for i in range(n - 1)
             if all(info[i][k] == info[i + 1][k] for k in keys) and info[i]["mode"] == mode]
    assert len(pairs) >= 2
    for i, j in pairs[:4]:
        xr = op.checkpoint_replay(i, info[j]["iteration"] - info[i]["iteration"])
        assert torch.equal(xr, op.checkpoint_iterate(j)), (i, j, info[i], info[j])
    x2, _ = pkg.SipOperator.from_mesh(m).cg_solve(B, mode=mode, rtol=1e-10)
    assert torch.equal(x, x2)


def test_error_paths(pkg):
    import torch
    m = si.workload("c1_2d_4x4_p3")
    orc = SipOracle(m)
    b = torch.tensor(sine_rhs(orc, 2), device="cuda")
    op = pkg.SipOperator(m.dim, m.vert, m.elem_vert, m.orders, 1.0, pkg.options(max_iter=5))
    with pytest.raises(pkg.SipError) as e:
        op.cg_solve(b)
    assert e.value.code == 6
    _, st = op.cg_solve(b, raise_on_fail=False)
    assert st["converged"] == 0 and st["iterations"] <= 5 + 16
    bad = b.clone()
    bad[3] = float("nan")
    op2 = pkg.SipOperator.from_mesh(m)
    with pytest.raises(pkg.SipError) as e:
        op2.cg_solve(bad)
    assert e.value.code == 5
    # a penalty far too small makes the SIP matrix indefinite: CG must stop with an error
    opts = pkg.options(tau_scale=1e-3)
    A_bad = SipOracle(m, tau_scale=1e-3).assemble().toarray()
    assert np.linalg.eigvalsh(0.5 * (A_bad + A_bad.T)).min() < 0
    op3 = pkg.SipOperator(m.dim, m.vert, m.elem_vert, m.orders, 1.0, opts)
    with pytest.raises(pkg.SipError) as e:
        op3.cg_solve(torch.tensor(si.random_vector(op3.ndof, 1), device="cuda"))
    assert e.value.code in (6, 7)


def test_precision_config_c3(pkg):
    """32^3 hexes, P = 4: FP64 CG and FP32-refined CG both reach 1e-10 and agree."""
    import torch
    m = si.workload("c3_3d_32cube_p4")
    op = pkg.SipOperator.from_mesh(m)
    xq = op.quad_points()
    f = (1.0 + 3 * np.pi ** 2) * torch.prod(torch.sin(np.pi * xq), dim=1)
    b = op.iproduct(f.contiguous())
    x64, s64 = op.cg_solve(b, mode=0, rtol=1e-10)
    x32, s32 = op.cg_solve(b, mode=1, rtol=1e-10)
    for x in (x64, x32):
        r = b - op.apply(x)
        assert float(torch.linalg.norm(r) / torch.linalg.norm(b)) <= 1e-10
    assert float(torch.linalg.norm(x64 - x32) / torch.linalg.norm(x64)) <= 1e-7
    assert s32["refinements"] >= 2


def test_batched_rhs_c4_full_mesh(pkg):
    """24^3 jittered hexes, orders 2..7, a batch of right-hand sides from the
    seed-4 N(0,1) batch: FP64 CG and FP32-refined CG, all columns to 1e-10,
    each column's residual checked with a separate FP64 apply."""
    import torch
    m = si.workload("c4_3d_24cube_jitter_p2to7")
    op = pkg.SipOperator.from_mesh(m)
    B = torch.tensor(si.random_rhs_batch(32, op.ndof, 4)[:4], device="cuda")
    X32, s32 = op.cg_solve(B, mode=1, rtol=1e-10)
    X64, s64 = op.cg_solve(B, mode=0, rtol=1e-10)
    for X in (X32, X64):
        R = B - op.apply(X)
        rel = torch.linalg.norm(R, dim=1) / torch.linalg.norm(B, dim=1)
        assert float(rel.max()) <= 1e-10
    assert s32["converged"] == 1 and s64["converged"] == 1
