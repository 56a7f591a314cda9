"""The seeded synthetic workloads: sizes, draw order and value ranges of the
five benchmark meshes and of the helpers (the input recipe of the workloads;
no SIP arithmetic is involved)."""
import numpy as np
import pytest

import sip_inputs as si


@pytest.mark.parametrize("name,dim,n_elem,ndof,orders", [
    ("c1_2d_4x4_p3", 2, 16, 256, {3}),
    ("c2_2d_64x64_jitter_p2to6", 2, 4096, None, {2, 3, 4, 5, 6}),
    ("c3_3d_32cube_p4", 3, 32768, 4_096_000, {4}),
    ("c4_3d_24cube_jitter_p2to7", 3, 13824, None, {2, 3, 4, 5, 6, 7}),
    ("c5_3d_16cube_p5", 3, 4096, 884_736, {5}),
])
def test_workload_sizes(name, dim, n_elem, ndof, orders):
    m = si.workload(name)
    assert m.dim == dim and m.n_elem == n_elem and m.lam == 1.0
    assert set(np.unique(m.orders).tolist()) == orders
    if ndof is not None:
        assert si.ndof(m.orders, dim) == ndof
    lo, hi = m.vert.min(axis=0), m.vert.max(axis=0)
    assert np.allclose(lo, 0.0) and np.allclose(hi, 1.0)


@pytest.mark.parametrize("dim,n,c,seed,rng_orders", [(2, 64, 0.15, 1, (2, 6)), (3, 24, 0.1, 3, (2, 7))])
def test_jitter_then_orders_draw_order(dim, n, c, seed, rng_orders):
    """Jitter uniform(-c h, c h) per interior vertex and coordinate in
    lexicographic vertex order, then the orders, from one default_rng(seed)."""
    m = si.structured_mesh(dim, n, jitter=c, seed=seed, order_range=rng_orders)
    h = 1.0 / n
    idx = np.rint(m.vert / h)
    interior = np.all((idx > 0) & (idx < n), axis=1)
    # the grid is recovered by rounding only because the jitter stays below h/2
    d = m.vert - idx * h
    assert np.all(np.abs(d[~interior]) == 0.0)
    assert np.all(np.abs(d[interior]) <= c * h)
    rng = np.random.default_rng(seed)
    jit = rng.uniform(-c * h, c * h, (int(interior.sum()), dim))
    assert np.allclose(d[interior], jit, rtol=0, atol=1e-15)
    assert np.array_equal(m.orders, rng.integers(rng_orders[0], rng_orders[1] + 1, m.n_elem).astype(np.int32))


def test_vectors_and_batches():
    assert np.array_equal(si.random_vector(10, 0), np.random.default_rng(0).standard_normal(10))
    b = si.random_rhs_batch(32, 7, 4)
    assert b.shape == (32, 7) and np.array_equal(b, np.random.default_rng(4).standard_normal((32, 7)))
    off = si.dof_offsets(np.array([1, 2, 3]), 2)
    assert off.tolist() == [0, 4, 13, 29] and si.ndof(np.array([1, 2, 3]), 2) == 29


def test_kappa_field_layout_and_smoothing():
    n, q = 3, 2
    k = si.kappa_lattice_field(n, q, seed=5, dim=3)
    assert k.shape == (n ** 3, q ** 3) and np.all(k > 0)
    # rebuild the smoothed lattice directly and read element (ex, ey, ez) = (1, 0, 2)
    m = n * q
    g = np.random.default_rng(5).standard_normal((m, m, m))
    for ax in range(3):
        gp = np.pad(g, [(1, 1) if a == ax else (0, 0) for a in range(3)], mode="edge")
        g = sum(np.take(gp, np.arange(s, s + m), axis=ax) for s in range(3)) / 3.0
    ex, ey, ez = 1, 0, 2
    e = ex + n * ey + n * n * ez
    blk = np.exp(0.5 * g[ez * q:(ez + 1) * q, ey * q:(ey + 1) * q, ex * q:(ex + 1) * q])
    assert np.allclose(k[e], blk.reshape(-1))


@pytest.mark.parametrize("dim", [2, 3])
def test_rotations_keep_elements(dim):
    m = si.structured_mesh(dim, 3, jitter=0.1, seed=2, order=2)
    r = si.rotate_elements(m, 7)
    for e in range(m.n_elem):
        assert set(m.elem_vert[e]) == set(r.elem_vert[e])
    assert np.any(r.elem_vert != m.elem_vert)


def test_pulse_mesh():
    m = si.pulse_refined_mesh(3, 8, 2, 5)
    assert np.allclose(m.vert.min(axis=0), -1.0) and np.allclose(m.vert.max(axis=0), 1.0)
    cent = m.vert[m.elem_vert].mean(axis=1)
    inside = np.all(np.abs(cent) < 0.5, axis=1)
    assert inside.sum() == 4 ** 3
    assert np.all(m.orders[inside] == 5) and np.all(m.orders[~inside] == 2)
