"""Seeded synthetic workloads for the SIP Helmholtz apply.

This module holds no SIP arithmetic.  It only produces the *inputs* that the
oracle and the CUDA library both consume:

* structured quad/hex meshes of [0,1]^d: vertex coordinates (optionally
  jittered) and element-to-vertex connectivity (2^d vertices per element,
  lexicographic local order, x fastest);
* per-element polynomial orders (constant or i.i.d. uniform);
* random DOF vectors and right-hand-side batches;
* a smoothed log-normal diffusivity field on the volume-quadrature lattice.

Draw order (one ``numpy.random.default_rng(seed)`` stream per mesh): first the
interior-vertex jitter ``uniform(-c h, c h, (n_interior, d))`` in lexicographic
vertex order, then the orders ``integers(Pmin, Pmax + 1, E)``.

The five named workloads follow the configurations the method is measured on
(Sec. 4 uses structured meshes treated as unstructured; the meshes here are
structured grids passed to the library as plain unstructured connectivity).
"""
from __future__ import annotations

import dataclasses
import itertools

import numpy as np

__all__ = [
    "Mesh", "structured_mesh", "workload", "WORKLOADS", "ndof", "dof_offsets",
    "random_vector", "random_rhs_batch", "kappa_lattice_field", "rotate_elements",
    "affine_map_vertices", "pulse_refined_mesh",
]


@dataclasses.dataclass
class Mesh:
    """An unstructured-style quad/hex mesh plus per-element orders.

    vert:      float64 [n_vert, dim]
    elem_vert: int64   [n_elem, 2**dim]  local vertex c has bit k = corner side along axis k
    orders:    int32   [n_elem]          polynomial degree P_e of each element
    """
    dim: int
    vert: np.ndarray
    elem_vert: np.ndarray
    orders: np.ndarray
    lam: float = 1.0
    name: str = ""

    @property
    def n_elem(self) -> int:
        return int(self.elem_vert.shape[0])

    @property
    def n_vert(self) -> int:
        return int(self.vert.shape[0])


def structured_mesh(dim: int, n: int, *, jitter: float = 0.0, seed: int | None = None,
                    order: int | None = None, order_range: tuple[int, int] | None = None,
                    lam: float = 1.0, name: str = "") -> Mesh:
    """n^dim grid of [0,1]^dim.

    jitter = c moves every interior vertex by uniform(-c h, c h) per coordinate,
    h = 1/n.  Orders: ``order`` for all elements, or i.i.d. uniform integers in
    ``order_range`` (inclusive) drawn from the same generator after the jitter.
    """
    if dim not in (2, 3):
        raise ValueError("dim must be 2 or 3")
    rng = np.random.default_rng(seed)
    h = 1.0 / n
    nv = (n + 1) ** dim
    v = np.arange(nv, dtype=np.int64)
    # lexicographic vertex order, x fastest: v = ix + (n+1) iy + (n+1)^2 iz
    idx = np.stack([(v // (n + 1) ** k) % (n + 1) for k in range(dim)], axis=1)
    vert = idx.astype(np.float64) * h
    if jitter > 0.0:
        interior = np.all((idx > 0) & (idx < n), axis=1)
        n_int = int(interior.sum())
        d = rng.uniform(-jitter * h, jitter * h, (n_int, dim))
        vert[interior] += d
    # elements, lexicographic, x fastest: e = ex + n ey + n^2 ez
    ne = n ** dim
    e = np.arange(ne, dtype=np.int64)
    eidx = np.stack([(e // n ** k) % n for k in range(dim)], axis=1)
    base = sum(eidx[:, k] * (n + 1) ** k for k in range(dim))
    elems = np.empty((ne, 2 ** dim), dtype=np.int64)
    for c in range(2 ** dim):
        off = sum(((c >> k) & 1) * (n + 1) ** k for k in range(dim))
        elems[:, c] = base + off
    elem_vert = np.asarray(elems, dtype=np.int64)
    E = elem_vert.shape[0]
    if order_range is not None:
        lo, hi = order_range
        orders = rng.integers(lo, hi + 1, E).astype(np.int32)
    else:
        orders = np.full(E, 3 if order is None else order, dtype=np.int32)
    return Mesh(dim=dim, vert=vert, elem_vert=elem_vert, orders=orders, lam=lam, name=name)


def ndof(orders: np.ndarray, dim: int) -> int:
    return int(np.sum((np.asarray(orders, dtype=np.int64) + 1) ** dim))


def dof_offsets(orders: np.ndarray, dim: int) -> np.ndarray:
    n = (np.asarray(orders, dtype=np.int64) + 1) ** dim
    return np.concatenate([[0], np.cumsum(n)]).astype(np.int64)


def random_vector(n: int, seed: int = 0) -> np.ndarray:
    """One N(0,1) float64 value per DOF."""
    return np.random.default_rng(seed).standard_normal(n)


def random_rhs_batch(nrhs: int, n: int, seed: int = 4) -> np.ndarray:
    """[nrhs, n] N(0,1) float64 batch."""
    return np.random.default_rng(seed).standard_normal((nrhs, n))


def kappa_lattice_field(n: int, q: int, seed: int = 5, dim: int = 3) -> np.ndarray:
    """Diffusivity kappa = exp(0.5 g) per volume-quadrature point.

    g is i.i.d. N(0,1) on the global (n q)^dim lattice (x fastest), smoothed by
    one [1,1,1]/3 box filter along each axis with edge-replicate boundaries.
    Element (ex, ey, ez) (x fastest, as in ``structured_mesh``) owns the lattice
    block [ex q:(ex+1) q] x ...; its q^dim values are returned in lexicographic
    local order (x fastest).  Result: float64 [n^dim, q^dim].
    """
    m = n * q
    g = np.random.default_rng(seed).standard_normal((m,) * dim)  # axis order (z, y, x): x fastest in memory
    for ax in range(dim):
        pad = [(0, 0)] * dim
        pad[ax] = (1, 1)
        gp = np.pad(g, pad, mode="edge")
        sl = lambda a, b: tuple(slice(a, b) if k == ax else slice(None) for k in range(dim))
        g = (gp[sl(0, m)] + gp[sl(1, m + 1)] + gp[sl(2, m + 2)]) / 3.0
    kap = np.exp(0.5 * g)
    if dim == 3:
        k = kap.reshape(n, q, n, q, n, q)          # (ez, qz, ey, qy, ex, qx)
        k = k.transpose(0, 2, 4, 1, 3, 5)           # (ez, ey, ex, qz, qy, qx)
        return np.ascontiguousarray(k.reshape(n ** 3, q ** 3))
    k = kap.reshape(n, q, n, q).transpose(0, 2, 1, 3)
    return np.ascontiguousarray(k.reshape(n ** 2, q ** 2))


def _proper_rotations(dim: int):
    """Signed axis permutations with determinant +1 (4 in 2D, 24 in 3D)."""
    out = []
    for perm in itertools.permutations(range(dim)):
        for flips in itertools.product((0, 1), repeat=dim):
            m = np.zeros((dim, dim))
            for k in range(dim):
                m[k, perm[k]] = -1.0 if flips[k] else 1.0
            if np.linalg.det(m) > 0:
                out.append((perm, flips))
    return out


def rotate_elements(mesh: Mesh, seed: int) -> Mesh:
    """Relabel each element's local vertices by a random proper rotation of the
    reference square/cube, so that neighbouring elements meet in arbitrary
    relative orientations (an unstructured mesh in all but name).  New local
    corner c' takes the old corner c with c_{perm[k]} = c'_k xor flip_k.
    """
    rng = np.random.default_rng(seed)
    rots = _proper_rotations(mesh.dim)
    choice = rng.integers(0, len(rots), mesh.n_elem)
    ev = np.empty_like(mesh.elem_vert)
    d = mesh.dim
    for e in range(mesh.n_elem):
        perm, flips = rots[choice[e]]
        for cn in range(2 ** d):
            c = 0
            for k in range(d):
                bit = ((cn >> k) & 1) ^ flips[k]
                c |= bit << perm[k]
            ev[e, cn] = mesh.elem_vert[e, c]
    return dataclasses.replace(mesh, elem_vert=ev)


def affine_map_vertices(mesh: Mesh, a: np.ndarray, b: np.ndarray | None = None) -> Mesh:
    """Apply x -> a x + b to every vertex (keeps elements affine)."""
    v = mesh.vert @ np.asarray(a, dtype=np.float64).T
    if b is not None:
        v = v + np.asarray(b, dtype=np.float64)
    return dataclasses.replace(mesh, vert=v)


def pulse_refined_mesh(dim: int, n: int, p_low: int, p_high: int, box: float = 0.5) -> Mesh:
    """Local p-refinement set-up of the Gaussian-pulse study: the cube [-1,1]^dim
    as an n^dim grid, elements whose centre lies in [-box, box]^dim at order
    p_high, the others at p_low."""
    m = structured_mesh(dim, n, order=p_low)
    m = affine_map_vertices(m, 2.0 * np.eye(dim), -np.ones(dim))
    cent = m.vert[m.elem_vert].mean(axis=1)
    inside = np.all(np.abs(cent) < box, axis=1)
    orders = np.where(inside, p_high, p_low).astype(np.int32)
    return dataclasses.replace(m, orders=orders, name=f"pulse_{dim}d_{n}_p{p_low}_{p_high}")


WORKLOADS = {
    # 2D 4x4 uniform quads, P=3, lambda=1
    "c1_2d_4x4_p3": dict(dim=2, n=4, order=3),
    # 2D 64x64 quads, interior jitter +-0.15h (seed 1), orders U{2..6}
    "c2_2d_64x64_jitter_p2to6": dict(dim=2, n=64, jitter=0.15, seed=1, order_range=(2, 6)),
    # 3D 32^3 uniform hexes, P=4
    "c3_3d_32cube_p4": dict(dim=3, n=32, order=4),
    # 3D 24^3 hexes, jitter +-0.1h (seed 3), orders U{2..7}; 32 right-hand sides (seed 4)
    "c4_3d_24cube_jitter_p2to7": dict(dim=3, n=24, jitter=0.1, seed=3, order_range=(2, 7)),
    # 3D 16^3 uniform hexes, P=5, kappa field (seed 5)
    "c5_3d_16cube_p5": dict(dim=3, n=16, order=5),
}


def workload(name: str) -> Mesh:
    kw = dict(WORKLOADS[name])
    return structured_mesh(lam=1.0, name=name, **kw)
