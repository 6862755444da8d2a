"""Pins for the oracle's global assembly A = sum_e P_e^T A_e P_e (no GPU).

Checks that do not trust the oracle: brute-force dense assembly, the
Laplacian's symmetry, zero row sums and exactness on linear fields (interior
rows of A u vanish, u^T A u is the exact Dirichlet energy), and for P1
elasticity the rigid modes in the null space of the assembled matrix and the
exact energy of a linear displacement."""
import numpy as np
import pytest

from paper_1103_0066_gb300 import meshgen as mg

LP1, EP1 = 0, 2


def _mesh(dim):
    if dim == 2:
        return mg.square_tri_mesh(3, 0.2, mg.rng_for(61), np.float64)
    return mg.cube_tet_mesh(2, 0.15, mg.rng_for(62), 0.0, np.float64)


def _volume(mesh):
    P = mesh.coords[mesh.conn]
    d = mesh.dim
    return np.abs(np.linalg.det(P[:, 1:] - P[:, :1])).sum() / (2 if d == 2 else 6)


def _interior(mesh):
    x = mesh.coords
    return np.all((x > 1e-12) & (x < 1 - 1e-12), axis=1)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("form", [LP1, EP1])
def test_assembly_equals_brute_force(orc, dim, form):
    mesh = _mesh(dim)
    A, _ = orc.integrate(dim, form, mesh.conn, mesh.coords)
    M = orc.assemble(dim, form, mesh.conn, mesh.n_vert, A).toarray()
    b = dim if form == EP1 else 1
    D = np.zeros_like(M)
    nv = dim + 1
    for e in range(mesh.n_elem):
        for I in range(nv * b):
            c, i = divmod(I, nv)
            for J in range(nv * b):
                c2, j = divmod(J, nv)
                D[mesh.conn[e, i] * b + c, mesh.conn[e, j] * b + c2] += A[e, I, J]
    assert np.array_equal(M, D) or np.abs(M - D).max() <= 1e-15 * np.abs(D).max()


@pytest.mark.parametrize("dim", [2, 3])
def test_assembled_laplacian_identities(orc, dim):
    mesh = _mesh(dim)
    A, _ = orc.integrate(dim, LP1, mesh.conn, mesh.coords)
    M = orc.assemble(dim, LP1, mesh.conn, mesh.n_vert, A)
    Md = M.toarray()
    assert np.abs(Md - Md.T).max() <= 1e-14 * np.abs(Md).max()
    assert np.abs(Md.sum(1)).max() <= 1e-13 * np.abs(Md).max()
    b = np.array([0.7, -1.3, 0.4][:dim])
    u = mesh.coords @ b + 0.25
    r = M @ u
    assert np.abs(r[_interior(mesh)]).max() <= 1e-12          # linear fields are exact
    assert abs(u @ r - b @ b * _volume(mesh)) <= 1e-12 * b @ b  # exact Dirichlet energy


@pytest.mark.parametrize("dim", [2, 3])
def test_assembled_elasticity_rigid_modes_and_energy(orc, dim):
    mesh = _mesh(dim)
    A, _ = orc.integrate(dim, EP1, mesh.conn, mesh.coords)
    M = orc.assemble(dim, EP1, mesh.conn, mesh.n_vert, A)
    x = mesh.coords
    modes = [np.tile(np.eye(dim)[c], mesh.n_vert) for c in range(dim)]  # translations, node-major
    pairs = [(0, 1)] if dim == 2 else [(0, 1), (0, 2), (1, 2)]
    for a, b in pairs:  # infinitesimal rotations in the (a, b) plane
        r = np.zeros((mesh.n_vert, dim))
        r[:, a], r[:, b] = -x[:, b], x[:, a]
        modes.append(r.ravel())
    scale = np.abs(M).max()
    for m in modes:
        assert np.abs(M @ m).max() <= 1e-12 * scale * np.abs(m).max()
    B = np.random.default_rng(63).standard_normal((dim, dim))
    u = (x @ B.T).ravel()
    S = 0.5 * (B + B.T)
    assert abs(u @ (M @ u) - _volume(mesh) * np.sum(S * S)) <= 1e-11 * np.sum(S * S)


LP2 = 1


@pytest.mark.parametrize("dim", [2, 3])
def test_p2_assembly_equals_brute_force(orc, dim):
    """The P2 unknowns numbered by explicit loops (vertices, then the edges in
    increasing (lower, higher) vertex order) and a dense sum of the element
    matrices give the oracle's matrix."""
    mesh = _mesh(dim)
    A, _ = orc.integrate(dim, LP2, mesh.conn, mesh.coords)
    M = orc.assemble(dim, LP2, mesh.conn, mesh.n_vert, A).toarray()
    pairs = mg.edge_pairs(dim)
    edges = sorted({(min(c[a], c[b]), max(c[a], c[b])) for c in mesh.conn.tolist() for a, b in pairs})
    number = {ed: mesh.n_vert + k for k, ed in enumerate(edges)}
    N = mesh.n_vert + len(edges)
    D = np.zeros((N, N))
    for e, c in enumerate(mesh.conn.tolist()):
        g = c + [number[(min(c[a], c[b]), max(c[a], c[b]))] for a, b in pairs]
        for i, gi in enumerate(g):
            for j, gj in enumerate(g):
                D[gi, gj] += A[e, i, j]
    assert M.shape == (N, N)
    assert np.abs(M - D).max() <= 1e-15 * np.abs(D).max()


@pytest.mark.parametrize("dim", [2, 3])
def test_assembled_p2_laplacian_identities(orc, dim):
    """Symmetric, zero row sums, and the exact Dirichlet energy of a quadratic
    field interpolated at the vertices and the edge midpoints."""
    mesh = _mesh(dim)
    A, _ = orc.integrate(dim, LP2, mesh.conn, mesh.coords)
    M = orc.assemble(dim, LP2, mesh.conn, mesh.n_vert, A)
    Md = M.toarray()
    assert np.abs(Md - Md.T).max() <= 1e-14 * np.abs(Md).max()
    assert np.abs(Md.sum(1)).max() <= 1e-13 * np.abs(Md).max()
    dofs, N = orc.p2_dofs(dim, mesh.conn, mesh.n_vert)
    pts = np.zeros((N, dim))
    pts[:mesh.n_vert] = mesh.coords
    for q, (a, b) in enumerate(mg.edge_pairs(dim)):
        pts[dofs[:, dim + 1 + q]] = 0.5 * (mesh.coords[mesh.conn[:, a]] + mesh.coords[mesh.conn[:, b]])
    # u = x_0^2 (in P2 on affine elements): int |grad u|^2 = int 4 x_0^2 over the mesh
    u = pts[:, 0] ** 2
    P = mesh.coords[mesh.conn]
    vol = np.abs(np.linalg.det(P[:, 1:] - P[:, :1])) / (2 if dim == 2 else 6)
    # exact int x^2 over a simplex: vol/((d+1)(d+2)) (sum x_i^2 + (sum x_i)^2) for vertex coordinates x_i
    x0 = P[:, :, 0]
    ex = (vol / ((dim + 1) * (dim + 2)) * ((x0 ** 2).sum(1) + x0.sum(1) ** 2)).sum()
    assert abs(u @ (M @ u) - 4 * ex) <= 1e-12 * 4 * ex
