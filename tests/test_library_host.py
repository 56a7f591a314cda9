"""CPU-side checks of the C ABI library: it loads, exports every function that
include/sip.h declares, and its host-side mesh analysis (face pairing,
orientation, geometry, penalties, argument and mesh errors) is right.  No GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import sip_inputs as si

HERE = os.path.dirname(os.path.abspath(__file__))
HEADER = os.path.join(HERE, "..", "include", "sip.h")


@pytest.fixture(scope="module")
def pkg():
    from conftest import build_library
    return build_library()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s+\**(sip_[a-z0-9_]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(pkg):
    names = declared_functions()
    assert len(names) >= 25, names
    so = C.CDLL(pkg._lib.LIB_PATH)
    for n in names:
        assert hasattr(so, n), n
    # and the binding wraps exactly the declared set
    assert set(names) == set(pkg._lib.SIGNATURES), set(names) ^ set(pkg._lib.SIGNATURES)


def test_defaults(pkg):
    o = pkg.options()
    assert o.tau_scale == 2.0 and o.qvol_extra == 2 and o.boundary == 1
    assert o.inner_rtol == 1e-5 and o.check_every == 16


def _info(pkg, m, **kw):
    return pkg.plan_info(m.dim, m.vert, m.elem_vert, m.orders, pkg.options(**kw) if kw else None)


def test_plan_counts_c1(pkg):
    m = si.workload("c1_2d_4x4_p3")
    i = _info(pkg, m)
    assert i["ndof"] == 256 and i["nquad"] == 16 * 25
    assert i["n_faces_interior"] == 24 and i["n_faces_boundary"] == 16
    assert i["n_elem_affine"] == 16 and i["n_faces_nonconforming"] == 0
    assert abs(i["min_h_face"] - 0.25) < 1e-14
    assert abs(i["max_tau"] - 2 * 16 / 0.25) < 1e-10


def test_plan_counts_c2(pkg):
    m = si.workload("c2_2d_64x64_jitter_p2to6")
    i = _info(pkg, m)
    assert i["n_faces_interior"] == 8064 and i["n_faces_boundary"] == 256
    assert i["ndof"] == si.ndof(m.orders, 2)
    # non-conforming faces counted independently
    n = 64
    o = m.orders.reshape(n, n)
    nc = int(np.sum(o[:, 1:] != o[:, :-1]) + np.sum(o[1:, :] != o[:-1, :]))
    assert i["n_faces_nonconforming"] == nc
    assert i["n_elem_affine"] == 0
    # trace points: sum over faces of (max(P-,P+)+2)
    q = o + 2
    tp = int(np.sum(np.maximum(q[:, 1:], q[:, :-1])) + np.sum(np.maximum(q[1:, :], q[:-1, :])))
    tp += int(np.sum(q[:, 0]) + np.sum(q[:, -1]) + np.sum(q[0, :]) + np.sum(q[-1, :]))
    assert i["trace_points"] == tp


@pytest.mark.parametrize("dim,n", [(2, 5), (3, 3)])
def test_orientations_cover_rotations(pkg, dim, n):
    m = si.rotate_elements(si.structured_mesh(dim, n, jitter=0.1, seed=2, order_range=(1, 4)), 7)
    i = _info(pkg, m)
    hist = i["orient_hist"]
    assert sum(hist) == i["n_faces_interior"]
    used = sum(1 for h in hist if h > 0)
    assert used == (2 if dim == 2 else 8)
    plain = _info(pkg, si.structured_mesh(dim, n, jitter=0.1, seed=2, order_range=(1, 4)))
    assert plain["orient_hist"][0] == plain["n_faces_interior"]


def test_face_counts_match_oracle(pkg):
    from oracle import SipOracle
    m = si.rotate_elements(si.structured_mesh(3, 3, jitter=0.1, seed=4, order_range=(1, 3)), 1)
    orc = SipOracle(m)
    i = _info(pkg, m)
    assert i["n_faces_interior"] == len(orc.interior)
    assert i["n_faces_boundary"] == len(orc.bfaces)


def test_errors(pkg):
    m = si.workload("c1_2d_4x4_p3")
    bad = m.orders.copy()
    bad[3] = 0
    with pytest.raises(pkg.SipError) as e:
        pkg.plan_info(2, m.vert, m.elem_vert, bad)
    assert e.value.code == 1
    bad[3] = pkg._lib.SIP_MAX_ORDER + 1
    with pytest.raises(pkg.SipError) as e:
        pkg.plan_info(2, m.vert, m.elem_vert, bad)
    assert e.value.code == 1
    with pytest.raises(pkg.SipError) as e:
        pkg.plan_info(2, m.vert, m.elem_vert, m.orders, pkg.options(qvol_extra=3))
    assert e.value.code == 1
    for bad_opt in (dict(quad_rule=2), dict(force_interp=2), dict(force_interp=1, face_scheme=pkg.SIP_FACES_P2P)):
        with pytest.raises(pkg.SipError) as e:
            pkg.plan_info(2, m.vert, m.elem_vert, m.orders, pkg.options(**bad_opt))
        assert e.value.code == 1
    # inverted element: swap two corners -> non-positive Jacobian
    ev = m.elem_vert.copy()
    ev[5, [0, 1]] = ev[5, [1, 0]]
    with pytest.raises(pkg.SipError) as e:
        pkg.plan_info(2, m.vert, ev, m.orders)
    assert e.value.code == 2
    # three elements on one face: duplicate an element
    ev = np.vstack([m.elem_vert, m.elem_vert[6:7]])
    with pytest.raises(pkg.SipError) as e:
        pkg.plan_info(2, m.vert, ev, np.append(m.orders, 3))
    assert e.value.code == 2
    # vertex id out of range
    ev = m.elem_vert.copy()
    ev[0, 0] = 10 ** 6
    with pytest.raises(pkg.SipError) as e:
        pkg.plan_info(2, m.vert, ev, m.orders)
    assert e.value.code == 1


def test_create_without_gpu_fails_loudly(pkg):
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    m = si.workload("c1_2d_4x4_p3")
    with pytest.raises(pkg.SipError):
        pkg.SipOperator.from_mesh(m)


def test_p2p_plan(pkg):
    """Point-to-point variant: each interior face holds one trace block per side
    at that side's own (P+2)-point rule, [u, g, u~, g~] (4 values per point);
    boundary faces as with the shared rule.  Penalties do not change."""
    m = si.rotate_elements(si.structured_mesh(3, 3, jitter=0.1, seed=3, order_range=(1, 6)), 4)
    a = _info(pkg, m)
    b = _info(pkg, m, face_scheme=pkg.SIP_FACES_P2P)
    orc_faces = __import__("oracle").SipOracle(m)
    q = m.orders + 2
    shared = sum(max(q[em], q[ep]) ** 2 for (em, _), (ep, _) in orc_faces.interior) + sum(q[e] ** 2 for e, _ in orc_faces.bfaces)
    own = sum(q[em] ** 2 + q[ep] ** 2 for (em, _), (ep, _) in orc_faces.interior) + sum(q[e] ** 2 for e, _ in orc_faces.bfaces)
    assert a["trace_points"] == shared
    assert b["trace_points"] == own
    for k in ("max_tau", "min_h_face", "n_faces_interior", "n_faces_nonconforming", "ndof", "nquad"):
        assert a[k] == b[k], k
    with pytest.raises(pkg.SipError):
        _info(pkg, m, face_scheme=2)


def test_header_is_plain_c_and_links(pkg, tmp_path):
    """include/sip.h compiles as C99 and a C program linked against libsip.so
    runs the host-only plan analysis through the ABI."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "abi.c"
    src.write_text(r'''
#include <stdio.h>
#include "sip.h"
int main(void) {
    /* 2 x 1 quads of [0,2] x [0,1], orders 2 and 3 */
    const double vert[] = {0,0, 1,0, 2,0, 0,1, 1,1, 2,1};
    const int64_t ev[] = {0,1,3,4, 1,2,4,5};
    const int32_t orders[] = {2, 3};
    sip_mesh m = {2, 6, vert, 2, ev};
    sip_options o;
    sip_options_default(&o);
    sip_plan* p = NULL;
    if (sip_plan_create(&m, orders, &o, &p) != SIP_OK) { printf("error %s\n", sip_last_error()); return 1; }
    sip_plan_info info;
    sip_plan_info_get(p, &info);
    printf("%lld %lld %lld %lld\n", (long long)info.ndof, (long long)info.n_faces_interior,
           (long long)info.n_faces_boundary, (long long)info.n_faces_nonconforming);
    sip_plan_destroy(p);
    return 0;
}
''')
    lib = pkg._lib.LIB_PATH
    exe = tmp_path / "abi"
    inc = os.path.join(HERE, "..", "include")
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", inc, str(src), lib, "-o", str(exe),
                        "-Wl,-rpath," + os.path.dirname(lib)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.split() == ["25", "1", "6", "1"]


def test_binding_structs_match_the_header(pkg, tmp_path):
    """Every ctypes structure of the binding has the size and field offsets of
    its C declaration in include/sip.h (compiled and printed by gcc)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = [getattr(pkg._lib, n) for n in ("sip_mesh", "sip_options", "sip_stats", "sip_plan_info",
                                               "sip_tiling", "sip_checkpoint_info", "sip_work")]
    lines = []
    for st in structs:
        lines.append('printf("%s size %%zu\\n", sizeof(%s));' % (st.__name__, st.__name__))
        for f in st._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (st.__name__, f[0], st.__name__, f[0]))
    src = tmp_path / "layout.c"
    src.write_text("#include <stddef.h>\n#include <stdio.h>\n#include \"sip.h\"\nint main(void) {\n"
                   + "\n".join(lines) + "\nreturn 0;\n}\n")
    exe = tmp_path / "layout"
    inc = os.path.join(HERE, "..", "include")
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", inc, str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, check=True)
    got = {tuple(line.split()[:2]): int(line.split()[2]) for line in r.stdout.splitlines()}
    for st in structs:
        assert got[(st.__name__, "size")] == C.sizeof(st), st.__name__
        for f in st._fields_:
            assert got[(st.__name__, f[0])] == getattr(st, f[0]).offset, (st.__name__, f[0])


def test_qorders_option(pkg):
    """Per-element point counts (sip_options.qorders): the plan takes the
    supported (P, Q) pairs, sizes the volume-point arrays by them and rejects
    the others (the extra pairs only with Gauss-Lobatto points)."""
    m = si.structured_mesh(2, 3, order=1)
    col = (m.vert[m.elem_vert].mean(axis=1)[:, 0] * 3).astype(int)
    m.orders = np.array([(3, 1, 1)[c] for c in col], dtype=np.int32)
    q = np.array([(5, 5, 3)[c] for c in col], dtype=np.int32)
    info = pkg.plan_info(2, m.vert, m.elem_vert, m.orders, pkg.options(quad_rule=pkg.SIP_RULE_GLL, qorders=q))
    assert info["nquad"] == int(np.sum(q.astype(np.int64) ** 2))
    bad = q.copy()
    bad[0] = 7
    for opts in (pkg.options(quad_rule=pkg.SIP_RULE_GLL, qorders=bad), pkg.options(qorders=q)):
        with pytest.raises(pkg.SipError) as e:
            pkg.plan_info(2, m.vert, m.elem_vert, m.orders, opts)
        assert e.value.code == 1
