"""Parity of the CUDA apply (y = A x, and A^T x) with the FP64 oracle.

Small meshes are compared element by element on every output; the full-size
workloads (the 64x64 jittered p-non-conforming quads, the 32^3, 24^3 and
16^3 hexes) on the rows of a sample of elements, which the oracle computes
one block row at a time.  Tolerances: 1e-12 relative (2-norm) in FP64,
1e-5 relative in FP32.
"""
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


def gpu_apply(op, x, precision="f64", transpose=False):
    import torch
    dt = torch.float64 if precision == "f64" else torch.float32
    xt = torch.tensor(x, dtype=dt, device="cuda")
    y = op.apply(xt, transpose=transpose)
    torch.cuda.synchronize()
    return y.double().cpu().numpy()


def small_meshes():
    out = {
        "c1": si.workload("c1_2d_4x4_p3"),
        "2d_rot_jitter_p1to8": si.rotate_elements(si.structured_mesh(2, 9, jitter=0.2, seed=21, order_range=(1, 8)), 22),
        "2d_single_p5": si.structured_mesh(2, 1, order=5),
        "3d_rot_jitter_p1to5": si.rotate_elements(si.structured_mesh(3, 3, jitter=0.15, seed=23, order_range=(1, 5)), 24),
        "3d_rot_p6to8": si.rotate_elements(si.structured_mesh(3, 2, jitter=0.1, seed=25, order_range=(6, 8)), 26),
        "3d_single_p3": si.structured_mesh(3, 1, order=3),
        "2d_affine_skew": si.affine_map_vertices(si.rotate_elements(si.structured_mesh(2, 5, seed=27, order_range=(2, 5)), 28),
                                                 np.array([[1.1, 0.4], [-0.3, 0.8]])),
        "3d_affine_skew": si.affine_map_vertices(si.structured_mesh(3, 3, seed=29, order_range=(2, 4)),
                                                 np.array([[1.0, 0.3, 0.1], [0.0, 0.9, -0.2], [0.2, 0.0, 1.2]])),
    }
    return out


MESHES = small_meshes()


@pytest.mark.parametrize("name", list(MESHES))
def test_apply_fp64_full_parity(pkg, name):
    m = MESHES[name]
    orc = SipOracle(m, lam=m.lam)
    A = orc.assemble()
    op = pkg.SipOperator.from_mesh(m)
    x = si.random_vector(orc.ndof, 0)
    y = gpu_apply(op, x)
    yr = A @ x
    assert rel(y, yr) <= TOL64, rel(y, yr)
    # element-wise, scaled by the row magnitude
    scale = np.abs(A) @ np.abs(x)
    assert np.max(np.abs(y - yr) / scale) <= 1e-13
    yt = gpu_apply(op, x, transpose=True)
    assert rel(yt, A.T @ x) <= TOL64
    y32 = gpu_apply(op, x, "f32")
    assert rel(y32, yr) <= TOL32, rel(y32, yr)


@pytest.mark.parametrize("name", ["2d_rot_jitter_p1to8", "3d_rot_jitter_p1to5"])
def test_neumann_variant_and_lambda_zero(pkg, name):
    m = MESHES[name]
    opts = pkg.options(boundary=0)
    op = pkg.SipOperator(m.dim, m.vert, m.elem_vert, m.orders, 0.0, opts)
    orc = SipOracle(m, lam=0.0, boundary=False)
    A = orc.assemble()
    x = si.random_vector(orc.ndof, 3)
    assert rel(gpu_apply(op, x), A @ x) <= TOL64
    # the constant is in the kernel of the pure-Neumann stiffness
    one = np.ones(orc.ndof)
    y1 = gpu_apply(op, one)
    assert np.max(np.abs(y1)) <= 1e-11 * np.max(np.abs(A).sum(axis=1))


def test_multi_rhs(pkg):
    import torch
    m = MESHES["3d_rot_jitter_p1to5"]
    orc = SipOracle(m)
    A = orc.assemble()
    op = pkg.SipOperator.from_mesh(m)
    X = si.random_rhs_batch(5, orc.ndof, 9)
    Y = op.apply(torch.tensor(X, device="cuda")).cpu().numpy()
    for r in range(5):
        assert rel(Y[r], A @ X[r]) <= TOL64
    Y32 = op.apply(torch.tensor(X, device="cuda", dtype=torch.float32)).double().cpu().numpy()
    for r in range(5):
        assert rel(Y32[r], A @ X[r]) <= TOL32


def _sample_elements(m, k, seed):
    rng = np.random.default_rng(seed)
    E = m.n_elem
    s = set(rng.choice(E, size=min(k, E), replace=False).tolist())
    s.update({0, E - 1})
    # one element of every order present
    for p in np.unique(m.orders):
        s.add(int(np.flatnonzero(m.orders == p)[0]))
    return sorted(s)


@pytest.mark.parametrize("name,k", [("c2_2d_64x64_jitter_p2to6", 48), ("c3_3d_32cube_p4", 12),
                                    ("c4_3d_24cube_jitter_p2to7", 12), ("c5_3d_16cube_p5", 12)])
def test_full_size_sampled_rows(pkg, name, k):
    import torch
    m = si.workload(name)
    op = pkg.SipOperator.from_mesh(m)
    orc = SipOracle(m)
    sample = _sample_elements(m, k, 5)
    R = orc.rows_for_elements(sample)
    dofs = orc.dofs_of(sample)
    nrhs = 32 if name.startswith("c4") else 1
    X = si.random_rhs_batch(nrhs, orc.ndof, 4) if nrhs > 1 else si.random_vector(orc.ndof, 0)[None]
    Xt = torch.tensor(X, device="cuda")
    Y = op.apply(Xt if nrhs > 1 else Xt[0]).reshape(nrhs, -1).cpu().numpy()
    X32 = Xt.float()
    Y32 = op.apply(X32 if nrhs > 1 else X32[0]).reshape(nrhs, -1).double().cpu().numpy()
    for r in ([0, nrhs // 2, nrhs - 1] if nrhs > 1 else [0]):
        yr = R @ X[r]
        assert rel(Y[r][dofs], yr) <= TOL64, (r, rel(Y[r][dofs], yr))
        assert rel(Y32[r][dofs], yr) <= TOL32, (r, rel(Y32[r][dofs], yr))


def test_symmetry_c2_via_gpu(pkg):
    import torch
    m = si.workload("c2_2d_64x64_jitter_p2to6")
    op = pkg.SipOperator.from_mesh(m)
    n = op.ndof
    x1 = torch.tensor(si.random_vector(n, 0), device="cuda")
    x2 = torch.tensor(si.random_vector(n, 1), device="cuda")
    a = float(x1 @ op.apply(x2))
    b = float(x2 @ op.apply(x1))
    den = float(torch.linalg.norm(x1) * torch.linalg.norm(op.apply(x2)))
    assert abs(a - b) / den <= 1e-13
    # A^T x via the transpose apply equals A x to rounding
    y = op.apply(x1)
    yt = op.apply_transpose(x1)
    assert float(torch.linalg.norm(y - yt) / torch.linalg.norm(y)) <= 1e-13


def test_apply_host_matches_device(pkg):
    """sip_apply_host (host vectors in and out) gives the same bits as sip_apply
    on device copies, FP64 and FP32, one and several right-hand sides, with x and
    y each pinned (read / written in place by the kernels) or pageable (staged
    through device buffers), on hexes and on quads."""
    import torch
    for name in ("3d_rot_jitter_p1to5", "2d_rot_jitter_p1to8"):
        op = pkg.SipOperator.from_mesh(MESHES[name])
        X = torch.tensor(si.random_rhs_batch(3, op.ndof, 11))
        Yd = op.apply(X.cuda()).cpu()
        for x_pin in (False, True):
            for y_pin in (False, True):
                xh = X.pin_memory() if x_pin else X.clone()
                yh = torch.empty_like(X).pin_memory() if y_pin else torch.empty_like(X)
                yh.fill_(float("nan"))
                assert torch.equal(op.apply_host(xh, out=yh), Yd), (name, x_pin, y_pin)
                # twice in a row into the same buffers
                assert torch.equal(op.apply_host(xh, out=yh), Yd), (name, x_pin, y_pin)
        assert torch.equal(op.apply_host(X[0].clone()), Yd[0])
        assert torch.equal(op.apply_host(X[1].clone().pin_memory()), Yd[1])
        X32 = X.float()
        Y32 = op.apply(X32.cuda()).cpu()
        assert torch.equal(op.apply_host(X32), Y32)
        assert torch.equal(op.apply_host(X32.pin_memory(), out=torch.empty_like(X32).pin_memory()), Y32)
    with pytest.raises(pkg.SipError):
        op.apply_host(X.cuda())


def test_bad_inputs_raise(pkg):
    import torch
    m = MESHES["c1"]
    op = pkg.SipOperator.from_mesh(m)
    with pytest.raises(pkg.SipError):
        op.apply(torch.zeros(op.ndof + 1, dtype=torch.float64, device="cuda"))
    with pytest.raises(pkg.SipError):
        op.apply(torch.zeros(op.ndof, dtype=torch.float64))


@pytest.mark.parametrize("name", ["2d_rot_jitter_p1to8", "3d_rot_jitter_p1to5"])
def test_autotuned_tiles_keep_parity(pkg, name):
    import torch
    m = MESHES[name]
    orc = SipOracle(m)
    A = orc.assemble()
    op = pkg.SipOperator.from_mesh(m)
    x = si.random_vector(orc.ndof, 0)
    for prec, dt, tol in ((pkg.SIP_FP64, torch.float64, TOL64), (pkg.SIP_FP32, torch.float32, TOL32)):
        before = op.tiling(prec)
        after = op.autotune(prec, reps=2)
        assert after["ntiles"] > 0
        assert [b > 0 for b in before["epb_by_order"]] == [a > 0 for a in after["epb_by_order"]]
        y = op.apply(torch.tensor(x, device="cuda", dtype=dt)).double().cpu().numpy()
        assert rel(y, A @ x) <= tol


@pytest.mark.parametrize("name", ["2d_rot_jitter_p1to8", "3d_rot_jitter_p1to5", "c2_2d_64x64_jitter_p2to6"])
def test_tilings_give_identical_results(pkg, name):
    """Each element's arithmetic does not depend on how elements are grouped in
    tiles: every tiling gives the same bits (and, on the small meshes, parity)."""
    import torch
    small = name in MESHES
    m = MESHES[name] if small else si.workload(name)
    A = SipOracle(m).assemble() if small else None
    op = pkg.SipOperator.from_mesh(m)
    x = si.random_vector(op.ndof, 0)
    P1 = pkg._lib.SIP_MAX_ORDER + 1
    for prec, dt, tol in ((pkg.SIP_FP64, torch.float64, TOL64), (pkg.SIP_FP32, torch.float32, TOL32)):
        xt = torch.tensor(x, device="cuda", dtype=dt)
        ref = op.apply(xt)
        if small:
            assert rel(ref.double().cpu().numpy(), A @ x) <= tol
        ntiles = set()
        big = 32 if m.dim == 2 else 4
        smm = pkg.SIP_CTAS_SM_MAJOR   # the non-default block order
        for epb, per_sm, pers, thr, lay in (([1] * P1, 0, False, 256, 0), ([1] * P1, 0, False, 256, smm),
                                            ([big] * P1, 0, False, 256, 0), ([big] * P1, 1, True, 256, smm),
                                            (None, 1, False, 128, 0), (None, 3, True, 64, 0),
                                            ([2] * P1, 8, True, 128, smm), ([2] * P1, 8, False, 64, 0),
                                            (None, 0, 2, 256, 0), (None, 0, 2, 256, smm), ([2] * P1, 2, 2, 128, 0),
                                            (None, 1, 2, 32, 0)):
            info = op.set_tiling(prec, epb, per_sm, pers, thr, lay)
            assert info["persistent"] == pers and info["threads"] == thr
            assert info["cta_layout"] == (lay or pkg.SIP_CTAS_SEQUENTIAL)
            assert 1 <= info["nctas"] <= len(m.orders) and info["ctas_per_sm"] >= 1
            if epb is not None and epb[0] == 1:
                assert info["ntiles"] == len(m.orders)
            if not pers:
                assert info["nctas"] == info["ntiles"]
            if pers == 2:   # one cooperative launch per apply: trace phase, grid barrier, main phase
                op.set_timing(True)
                assert torch.equal(op.apply(xt), ref)
                tr_ms, main_ms = op.last_kernel_ms()
                assert tr_ms < 0.02 and main_ms > 0.0   # no separate trace kernel
                op.set_timing(False)
            ntiles.add(info["ntiles"])
            assert torch.equal(op.apply(xt), ref), (epb, per_sm, pers, thr, lay, info)
        if not small:
            assert len(ntiles) >= 3
        op.set_tiling(prec)  # back to the defaults
        assert torch.equal(op.apply(xt), ref)


def test_single_launch_apply(pkg):
    """The whole apply as one cooperative launch (schedule mode 2): the same
    bits as the two-kernel apply for several right-hand sides, the transpose,
    the point-to-point variant and Gauss-Lobatto points, the CG solve on top of
    it, and the two-kernel fallback when the CTAs of all right-hand sides do not
    fit on the device at once."""
    import torch
    P1 = pkg._lib.SIP_MAX_ORDER + 1
    m = MESHES["3d_rot_jitter_p1to5"]
    for kw in ({}, {"face_scheme": pkg.SIP_FACES_P2P}, {"quad_rule": pkg.SIP_RULE_GLL}):
        op = pkg.SipOperator.from_mesh(m, opts=pkg.options(**kw) if kw else None)
        X = torch.tensor(si.random_rhs_batch(3, op.ndof, 11), device="cuda")
        for prec, dt in ((pkg.SIP_FP64, torch.float64), (pkg.SIP_FP32, torch.float32)):
            Xp = X.to(dt)
            ref = op.apply(Xp)
            reft = None if kw.get("face_scheme") else op.apply(Xp, transpose=True)
            info = op.set_tiling(prec, None, 0, 2, 256)
            assert info["persistent"] == 2
            assert torch.equal(op.apply(Xp), ref)
            if reft is not None:
                assert torch.equal(op.apply(Xp, transpose=True), reft)
            op.set_tiling(prec)
    # CG on the single-launch apply gives the default solve's bits
    op = pkg.SipOperator.from_mesh(m)
    b = torch.tensor(si.random_vector(op.ndof, 12), device="cuda")
    x0, _ = op.cg_solve(b, mode=0, rtol=1e-10)
    x1r, _ = op.cg_solve(b, mode=1, rtol=1e-10)
    op.set_tiling(pkg.SIP_FP64, [1] * P1, 0, 2, 256)
    op.set_tiling(pkg.SIP_FP32, [1] * P1, 0, 2, 256)
    x1, st = op.cg_solve(b, mode=0, rtol=1e-10)
    assert torch.equal(x0, x1) and st["converged"] == 1
    x2r, _ = op.cg_solve(b, mode=1, rtol=1e-10)
    assert torch.equal(x1r, x2r)
    # more right-hand sides than fit at once: the two kernels run instead
    nctas = op.tiling(pkg.SIP_FP64)["nctas"]
    nr = 152 * 64 // nctas + 2
    Xb = torch.tensor(si.random_rhs_batch(nr, op.ndof, 13), device="cuda")
    Yb = op.apply(Xb)
    op.set_tiling(pkg.SIP_FP64)
    assert torch.equal(op.apply(Xb), Yb)


def test_set_tiling_rejects_bad_values(pkg):
    m = MESHES["2d_rot_jitter_p1to8"]
    op = pkg.SipOperator.from_mesh(m)
    before = op.tiling(pkg.SIP_FP64)
    P1 = pkg._lib.SIP_MAX_ORDER + 1
    with pytest.raises(pkg.SipError):
        op.set_tiling(pkg.SIP_FP64, [33] * P1, 0)
    with pytest.raises(pkg.SipError):
        op.set_tiling(pkg.SIP_FP64, None, -1)
    with pytest.raises(pkg.SipError):
        op.set_tiling(pkg.SIP_FP64, None, 0, False, 96)
    with pytest.raises(pkg.SipError):
        op.set_tiling(pkg.SIP_FP64, None, 0, False, 256, 3)
    with pytest.raises(ValueError):
        op.set_tiling(pkg.SIP_FP64, [1, 2], 0)
    assert op.tiling(pkg.SIP_FP64) == before
