"""Seeded synthetic meshes and upstream gradients.

This module only *generates inputs*: structured simplex meshes, vertex jitter,
sliver elements, per-element coefficients and upstream gradients.  It holds
none of the integration arithmetic, and both the CUDA path and the FP64
oracle consume its arrays, so it is the one piece of code the two share.

Workload shapes follow the paper's test problems (Sec. 5: the 2D and 3D P1
Laplacian and P1 elasticity) at the sizes of the benchmark configurations:

* ``square_tri_mesh``  unit square, n x n cells, each split along its
  (0,0)-(1,1) diagonal into two counter-clockwise triangles; vertex id
  ``j*(n+1)+i`` at ``(i h, j h)``; interior vertices jittered U(-j h, j h).
* ``cube_tet_mesh``    unit cube, n^3 cells, each split into the 6 Kuhn
  (Freudenthal) tetrahedra ``v000 -> +e_p1 -> +e_p2 -> +e_p3`` for the six
  axis permutations p (odd permutations get their last two vertices swapped so
  every element is positively oriented); vertex id ``(k(n+1)+j)(n+1)+i``;
  elements in cell-major lexicographic order; interior vertices jittered.
  Optionally a fraction of elements becomes slivers: for each chosen element
  one local vertex gets a private copy moved along the normal of its opposite
  face until its height is r times the original, r = 10^-U(2,4); the copy is
  appended to the vertex array and the element is rewired to it.
* ``mixed_batch``      96 meshes of log-uniform size in [1e3, 2e6] elements,
  six (shape, form) kinds, 16 of each in a seeded order.

Seeds: ``numpy.random.Generator(PCG64(11030066 + k))`` for workload k.
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 11030066

# form ids, identical to the C ABI's enum
LAPLACE_P1, LAPLACE_P2, ELASTIC_P1 = 0, 1, 2


def rng_for(k: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED_BASE + k))


@dataclass
class Mesh:
    dim: int
    coords: np.ndarray            # [V][dim] float32 or float64
    conn: np.ndarray              # [E][dim+1] int32
    sliver: np.ndarray = field(default=None)  # [E] bool, True for sliver elements

    @property
    def n_elem(self) -> int:
        return int(self.conn.shape[0])

    @property
    def n_vert(self) -> int:
        return int(self.coords.shape[0])


def _boundary_mask(idx: np.ndarray, n: int) -> np.ndarray:
    return (idx == 0) | (idx == n)


def square_tri_mesh(n: int, jitter: float = 0.2, rng: np.random.Generator | None = None,
                    dtype=np.float64) -> Mesh:
    """n x n cells of the unit square, 2 triangles per cell."""
    h = 1.0 / n
    j, i = np.meshgrid(np.arange(n + 1), np.arange(n + 1), indexing="ij")
    xy = np.stack([i.ravel() * h, j.ravel() * h], axis=1)
    if jitter and rng is not None:
        interior = ~(_boundary_mask(i.ravel(), n) | _boundary_mask(j.ravel(), n))
        d = rng.uniform(-jitter * h, jitter * h, size=(int(interior.sum()), 2))
        xy[interior] += d
    cj, ci = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    v00 = (cj * (n + 1) + ci).ravel()
    v10, v01 = v00 + 1, v00 + (n + 1)
    v11 = v01 + 1
    t0 = np.stack([v00, v10, v11], axis=1)
    t1 = np.stack([v00, v11, v01], axis=1)
    conn = np.stack([t0, t1], axis=1).reshape(-1, 3).astype(np.int32)
    return Mesh(2, xy.astype(dtype), conn, np.zeros(conn.shape[0], bool))


_PERMS = list(itertools.permutations(range(3)))  # lexicographic


def _perm_parity(p) -> int:
    inv = sum(1 for a in range(3) for b in range(a + 1, 3) if p[a] > p[b])
    return inv % 2


def cube_tet_mesh(n: int, jitter: float = 0.15, rng: np.random.Generator | None = None,
                  sliver_frac: float = 0.0, dtype=np.float32) -> Mesh:
    """n^3 cells of the unit cube, 6 Kuhn tetrahedra per cell, optional slivers."""
    h = 1.0 / n
    m = n + 1
    k, j, i = np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij")
    xyz = np.stack([i.ravel() * h, j.ravel() * h, k.ravel() * h], axis=1)
    if jitter and rng is not None:
        interior = ~(_boundary_mask(i.ravel(), n) | _boundary_mask(j.ravel(), n)
                     | _boundary_mask(k.ravel(), n))
        d = rng.uniform(-jitter * h, jitter * h, size=(int(interior.sum()), 3))
        xyz[interior] += d
    ck, cj, ci = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    base = ((ck * m + cj) * m + ci).ravel().astype(np.int64)
    step = np.array([1, m, m * m], dtype=np.int64)
    tets = []
    for p in _PERMS:
        v0 = base
        v1 = v0 + step[p[0]]
        v2 = v1 + step[p[1]]
        v3 = v2 + step[p[2]]
        if _perm_parity(p):
            v2, v3 = v3, v2
        tets.append(np.stack([v0, v1, v2, v3], axis=1))
    conn = np.stack(tets, axis=1).reshape(-1, 4).astype(np.int32)
    coords = xyz.astype(dtype)
    sliver = np.zeros(conn.shape[0], bool)
    if sliver_frac > 0.0:
        assert rng is not None
        coords, conn, sliver = _add_slivers(coords, conn, sliver_frac, rng)
    return Mesh(3, coords, conn, sliver)


def _heights(P: np.ndarray, k: np.ndarray):
    """Height of local vertex k above the plane of the opposite face, the face's
    unit normal (pointing to the vertex side) and a point of the face (FP64)."""
    E = P.shape[0]
    others = np.array([[1, 2, 3], [0, 2, 3], [0, 1, 3], [0, 1, 2]])[k]
    a = P[np.arange(E), others[:, 0]]
    b = P[np.arange(E), others[:, 1]]
    c = P[np.arange(E), others[:, 2]]
    nrm = np.cross(b - a, c - a)
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    x = P[np.arange(E), k]
    H = np.einsum("ij,ij->i", x - a, nrm)
    flip = H < 0
    nrm[flip] *= -1.0
    H = np.abs(H)
    return H, nrm, a


def _add_slivers(coords, conn, frac, rng, r_lo=5e-5, r_hi=2e-2):
    E = conn.shape[0]
    ns = int(round(frac * E))
    chosen = np.sort(rng.choice(E, size=ns, replace=False))
    kloc = rng.integers(0, 4, size=ns)
    P = coords[conn[chosen]].astype(np.float64)          # [ns][4][3]
    H, nrm, a = _heights(P, kloc)
    x = P[np.arange(ns), kloc]
    newx = np.empty((ns, 3), dtype=coords.dtype)
    todo = np.arange(ns)
    for _ in range(100):
        r = 10.0 ** (-rng.uniform(2.0, 4.0, size=todo.size))
        cand = (x[todo] - ((1.0 - r) * H[todo])[:, None] * nrm[todo]).astype(coords.dtype)
        # re-measure after rounding to the storage type
        Pc = P[todo].copy()
        Pc[np.arange(todo.size), kloc[todo]] = cand.astype(np.float64)
        Hc = np.einsum("ij,ij->i", cand.astype(np.float64) - a[todo], nrm[todo])
        rr = Hc / H[todo]
        ok = (rr >= r_lo) & (rr <= r_hi) & (np.linalg.det(Pc[:, 1:] - Pc[:, :1]) > 0)
        newx[todo[ok]] = cand[ok]
        todo = todo[~ok]
        if todo.size == 0:
            break
    assert todo.size == 0, "sliver resampling did not converge"
    V0 = coords.shape[0]
    coords = np.concatenate([coords, newx], axis=0)
    conn = conn.copy()
    conn[chosen, kloc] = (V0 + np.arange(ns)).astype(np.int32)
    sliver = np.zeros(E, bool)
    sliver[chosen] = True
    return coords, conn, sliver


def check_orientation(mesh: Mesh) -> None:
    """Assert every element is positively oriented (input validity check)."""
    P = mesh.coords[mesh.conn].astype(np.float64)
    det = np.linalg.det(P[:, 1:] - P[:, :1])
    assert np.all(det > 0), f"{int((det <= 0).sum())} inverted or flat elements"


def shuffled(mesh: Mesh, rng: np.random.Generator, elements: bool = True,
             vertices: bool = True) -> tuple[Mesh, np.ndarray]:
    """The same mesh with its elements in a seeded random order and its
    vertices renumbered at random.  Each element keeps its local vertex order,
    so orientation and every element matrix are unchanged; only the order in
    which elements come and the numbers of their vertices differ.  This is how
    a mesh from an unstructured mesh generator looks to the kernels:
    consecutive elements share few vertices, so a 32-element tile touches up
    to 4 x 32 distinct vertices and the coordinate gather loses its locality.

    Returns (mesh, order): new element k is old element order[k] (apply it to
    any per-element array, e.g. coef[order])."""
    E, V = mesh.n_elem, mesh.n_vert
    order = rng.permutation(E) if elements else np.arange(E)
    new_id = rng.permutation(V) if vertices else np.arange(V)   # old vertex v -> new_id[v]
    coords = np.empty_like(mesh.coords)
    coords[new_id] = mesh.coords
    conn = new_id[mesh.conn[order]].astype(np.int32)
    sliver = None if mesh.sliver is None else mesh.sliver[order]
    return Mesh(mesh.dim, coords, np.ascontiguousarray(conn), sliver), order


def lognormal_coef(rng: np.random.Generator, E: int) -> np.ndarray:
    return np.exp(rng.standard_normal(E)).astype(np.float32)


def upstream(rng: np.random.Generator, E: int, n: int) -> np.ndarray:
    return rng.standard_normal((E, n, n), dtype=np.float32)


def form_n(form: int, dim: int) -> int:
    nb = dim + 1 if form != LAPLACE_P2 else (dim + 1) * (dim + 2) // 2
    return nb * (dim if form == ELASTIC_P1 else 1)


# ---------------------------------------------------------------- workloads

def workload_tri_p1_fp64() -> Mesh:
    """P1 Laplacian on triangles: 64x64 square, 8,192 elements, FP64 coordinates."""
    return square_tri_mesh(64, 0.2, rng_for(1), np.float64)


def workload_tet_slivers(n: int = 128, k: int = 2) -> Mesh:
    """128^3 Kuhn cube (12,582,912 tets), jitter 0.15h, 5% slivers, FP32 coordinates."""
    return cube_tet_mesh(n, 0.15, rng_for(k), 0.05, np.float32)


def _warp(x: np.ndarray, eps: float) -> np.ndarray:
    """A smooth map of the unit square / cube onto itself plus a bulge:
    x + eps * (product of sines of the other coordinates), per component."""
    x = np.asarray(x, dtype=np.float64)
    s = np.sin(np.pi * x)
    out = x.copy()
    if x.shape[-1] == 2:
        out[..., 0] += eps * s[..., 1]
        out[..., 1] += eps * s[..., 0]
    else:
        out[..., 0] += eps * s[..., 1] * s[..., 2]
        out[..., 1] += eps * s[..., 2] * s[..., 0]
        out[..., 2] += eps * s[..., 0] * s[..., 1]
    return out


def edge_pairs(dim: int):
    """Local vertex pairs of the element's edges, in the P2 (lexicographic) order."""
    return [(a, b) for a in range(dim + 1) for b in range(a + 1, dim + 1)]


def curved_mesh(mesh: Mesh, eps: float = 0.05, dtype=np.float32) -> tuple[Mesh, np.ndarray]:
    """Quadratic (non-affine) elements from a straight-sided mesh: the vertices
    and the midpoints of every element's straight edges are mapped by a smooth
    warp, so each element's edges become curves through the warped midpoints.
    Returns the mesh with warped vertices and mid [E][n_edges][dim] (the
    edge-midpoint nodes, element by element; shared edges get equal nodes)."""
    X = np.asarray(mesh.coords, dtype=np.float64)
    P = X[mesh.conn]                                            # [E][dim+1][dim]
    pairs = edge_pairs(mesh.dim)
    M = np.stack([0.5 * (P[:, a] + P[:, b]) for a, b in pairs], axis=1)
    curved = Mesh(mesh.dim, _warp(X, eps).astype(dtype), mesh.conn, mesh.sliver)
    return curved, _warp(M, eps).astype(dtype)


def workload_tet_shuffled(n: int = 128, k: int = 2, ks: int = 12) -> Mesh:
    """The 128^3 sliver cube of workload_tet_slivers with its elements in a
    random order and its vertices renumbered at random (seed 11030066 + ks)."""
    return shuffled(workload_tet_slivers(n, k), rng_for(ks))[0]


def workload_curved_tets(n: int = 64, k: int = 6, eps: float = 0.05):
    """n^3 Kuhn cube, jitter 0.15 h, no slivers, warped into quadratic elements."""
    base = cube_tet_mesh(n, 0.15, rng_for(k), 0.0, np.float32)
    return curved_mesh(base, eps)


@dataclass
class BatchItem:
    form: int
    mesh: Mesh
    coef: np.ndarray
    dA: np.ndarray


BATCH_KINDS = [(2, LAPLACE_P1), (2, LAPLACE_P2), (2, ELASTIC_P1),
               (3, LAPLACE_P1), (3, LAPLACE_P2), (3, ELASTIC_P1)]


def _first_elements(mesh: Mesh, E: int) -> Mesh:
    conn = mesh.conn[:E]
    used, inv = np.unique(conn.ravel(), return_inverse=True)
    return Mesh(mesh.dim, np.ascontiguousarray(mesh.coords[used]),
                inv.reshape(conn.shape).astype(np.int32), np.zeros(E, bool))


def mixed_batch(n_meshes: int = 96, e_lo: float = 1e3, e_hi: float = 2e6, k: int = 5,
                scale: float = 1.0, shuffle: bool = False) -> list[BatchItem]:
    """96 meshes, E_m = round(exp(U(ln e_lo, ln e_hi))) (times ``scale`` for
    shrunken test batches), kinds cycling over a seeded shuffle of BATCH_KINDS.
    shuffle=True puts each mesh's elements in a random order and renumbers its
    vertices (``shuffled``)."""
    rng = rng_for(k)
    sizes = np.round(np.exp(rng.uniform(math.log(e_lo), math.log(e_hi), size=n_meshes)))
    sizes = np.maximum(1, np.round(sizes * scale)).astype(np.int64)
    order = rng.permutation(len(BATCH_KINDS))
    items = []
    for m in range(n_meshes):
        dim, form = BATCH_KINDS[order[m % len(BATCH_KINDS)]]
        E = int(sizes[m])
        if dim == 2:
            nc = max(1, math.ceil(math.sqrt(E / 2.0)))
            full = square_tri_mesh(nc, 0.2, rng, np.float32)
        else:
            nc = max(1, math.ceil((E / 6.0) ** (1.0 / 3.0)))
            full = cube_tet_mesh(nc, 0.15, rng, 0.0, np.float32)
        mesh = _first_elements(full, E)
        if shuffle:
            mesh = shuffled(mesh, rng)[0]
        n = form_n(form, dim)
        items.append(BatchItem(form, mesh, lognormal_coef(rng, E), upstream(rng, E, n)))
    return items
