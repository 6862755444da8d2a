"""GPU parity of the global assembly (-m gpu).

* The pattern (row_ptr, col_idx) equals the oracle's CSR structure exactly;
  for the P2 forms so do the unknowns (vertices, then edges in increasing
  (lower, higher) vertex order) of every element.
* The values equal, bit for bit, float32 sums of the same GPU element matrices
  in the order the library defines (numpy's unbuffered np.add.at): for the
  scalar P1 forms, per 32-element tile the contributions in element order,
  then those tile sums in tile order; for P1 elasticity's blocks and the P2
  forms, all contributions in element order.
* Against the FP64 oracle (oracle element matrices, assembled by the oracle):
  per row v, max |a_gpu - a_ref| <= 1e-5 * sum over the elements e at v of
  max |A_e| -- the element tolerance carried through the sum (a row of a
  sliver's neighbour holds entries far below that sliver's largest ones)."""
import numpy as np
import pytest
import torch

from paper_1103_0066_gb300 import meshgen as mg

pytestmark = pytest.mark.gpu
LP1, LP2, EP1, LP1W = 0, 1, 2, 3
DEV = "cuda:0"
TOL = 1e-5


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _mesh(dim, extra_vertices=0):
    if dim == 2:
        m = mg.square_tri_mesh(13, 0.2, mg.rng_for(71), np.float32)
    else:
        m = mg.cube_tet_mesh(7, 0.15, mg.rng_for(72), 0.05, np.float32)
    if extra_vertices:  # unused vertices: empty rows
        m.coords = np.vstack([m.coords, np.full((extra_vertices, dim), 0.5, np.float32)])
    return m


def _global_index(conn, dim, form):
    if form == EP1:
        return (conn[:, None, :].astype(np.int64) * dim + np.arange(dim)[None, :, None]).reshape(conn.shape[0], -1)
    return conn.astype(np.int64)


def _expand(row_ptr, col_idx, vals, b, n_vert):
    """BSR (b x b blocks) or CSR values -> dense [V*b][V*b] float64."""
    D = np.zeros((n_vert * b, n_vert * b))
    vals = vals.reshape(-1, b, b)
    for v in range(n_vert):
        for k in range(row_ptr[v], row_ptr[v + 1]):
            w = col_idx[k]
            D[v * b:(v + 1) * b, w * b:(w + 1) * b] = vals[k]
    return D


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("form", [LP1, EP1, LP1W])
def test_assembly_bitwise_and_oracle(gfem, orc, dim, form):
    mesh = _mesh(dim, extra_vertices=3)
    coords, conn = _t(mesh.coords), _t(mesh.conn)
    coef = (mg.lognormal_coef(mg.rng_for(73), mesh.n_vert) if form == LP1W
            else mg.lognormal_coef(mg.rng_for(74), mesh.n_elem))
    A = gfem.integrate_fwd(coords, conn, form, _t(coef))
    asm = gfem.Assembly(coords, conn, form)
    vals = asm.assemble(A)
    torch.cuda.synchronize()
    b = dim if form == EP1 else 1
    row_ptr = asm.row_ptr.cpu().numpy()
    col_idx = asm.col_idx.cpu().numpy()
    # pattern: the oracle's vertex graph
    P = orc.assemble(dim, LP1, mesh.conn, mesh.n_vert, np.ones((mesh.n_elem, dim + 1, dim + 1)))
    assert np.array_equal(row_ptr, P.indptr) and np.array_equal(col_idx, P.indices)
    assert asm.nnz == P.nnz and np.all(np.diff(row_ptr)[-3:] == 0)
    # bitwise: float32 sums in increasing element order at the same positions
    Ah = A.cpu().numpy()
    g = _global_index(mesh.conn, dim, form)
    n = g.shape[1]
    pos = {}
    for v in range(mesh.n_vert):
        for k in range(row_ptr[v], row_ptr[v + 1]):
            pos[(v, col_idx[k])] = k
    slot = np.empty((mesh.n_elem, n, n), np.int64)
    for e in range(mesh.n_elem):
        for I in range(n):
            for J in range(n):
                vi, vj = g[e, I] // b, g[e, J] // b
                slot[e, I, J] = pos[(vi, vj)] * b * b + (g[e, I] % b) * b + g[e, J] % b
    ref32 = np.zeros(asm.nnz * b * b, np.float32)
    if b == 1:
        ent = slot.reshape(-1)
        tile = np.repeat(np.arange(mesh.n_elem) // 32, n * n)
        keys, inv = np.unique(tile * ref32.size + ent, return_inverse=True)
        part = np.zeros(keys.size, np.float32)
        np.add.at(part, inv, Ah.reshape(-1))              # per (tile, entry), element order
        np.add.at(ref32, keys % ref32.size, part)          # keys ascend: tile order per entry
        assert asm.n_records == keys.size                  # one record per distinct (tile, entry)
    else:
        assert asm.n_records == 0
        np.add.at(ref32, slot.ravel(), Ah.reshape(-1))
    got = vals.cpu().numpy().reshape(-1)
    assert np.array_equal(got, ref32)
    # FP64 oracle, per row
    if form == LP1W:
        Ar, _ = orc.integrate_w1(dim, LP1, mesh.conn, mesh.coords, coef)
        Mr = orc.assemble(dim, LP1, mesh.conn, mesh.n_vert, Ar).toarray()
    else:
        Ar, _ = orc.integrate(dim, form, mesh.conn, mesh.coords, coef)
        Mr = orc.assemble(dim, form, mesh.conn, mesh.n_vert, Ar).toarray()
    D = _expand(row_ptr, col_idx, got.astype(np.float64), b, mesh.n_vert)
    elmax = np.abs(Ar).reshape(mesh.n_elem, -1).max(1)
    bound = np.zeros(mesh.n_vert)
    for i in range(dim + 1):
        np.add.at(bound, mesh.conn[:, i], elmax)
    bound = np.repeat(bound, b)
    live = bound > 0
    err = np.abs(D - Mr).max(1)
    assert np.all(err[live] <= TOL * bound[live]), float((err[live] / bound[live]).max())
    assert np.all(D[~live] == 0)


def test_assembly_deterministic_and_repeatable(gfem):
    mesh = _mesh(3)
    coords, conn = _t(mesh.coords), _t(mesh.conn)
    A = gfem.integrate_fwd(coords, conn, LP1)
    a1 = gfem.Assembly(coords, conn, LP1)
    v1 = a1.assemble(A).clone()
    a2 = gfem.Assembly(coords, conn, LP1)  # rebuilt maps: same pattern, same bits
    v2 = a2.assemble(A)
    torch.cuda.synchronize()
    assert torch.equal(a1.row_ptr, a2.row_ptr) and torch.equal(a1.col_idx, a2.col_idx) and torch.equal(v1, v2)


def test_assembly_errors_and_empty(gfem):
    mesh = _mesh(2)
    coords, conn = _t(mesh.coords), _t(mesh.conn)
    with pytest.raises(gfem.FemError):
        gfem.Assembly(coords, conn, 7)  # a coupling block is rectangular: not assembled
    rep = mesh.conn.copy()
    rep[4, 1] = rep[4, 0]
    with pytest.raises(gfem.FemError):
        gfem.Assembly(coords, _t(rep), LP2)  # an element repeating a vertex has no edge there
    bad = mesh.conn.copy()
    bad[4, 1] = mesh.n_vert + 2
    with pytest.raises(gfem.FemError):
        gfem.Assembly(coords, _t(bad), LP1)
    empty = gfem.Assembly(coords, conn[:0], LP1)
    assert empty.nnz == 0 and torch.all(empty.row_ptr == 0)
    vals = empty.assemble(torch.empty((0, 3, 3), device=DEV))
    assert vals.numel() == 0


def _p2_expected(dofs, A, n_rows):
    """float32 sums of the element entries in element order (np.add.at is unbuffered, in index order)."""
    E, n = dofs.shape
    rows = np.repeat(dofs, n, axis=1).ravel()
    cols = np.tile(dofs, (1, n)).ravel()
    key = rows.astype(np.int64) * n_rows + cols
    uk, inv = np.unique(key, return_inverse=True)
    vals = np.zeros(len(uk), np.float32)
    np.add.at(vals, inv, A.reshape(-1).astype(np.float32))
    return uk // n_rows, uk % n_rows, vals


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("form", [LP2, 4, 6])
@pytest.mark.parametrize("shuffle", [False, True])
def test_p2_assembly_bitwise_and_oracle(gfem, orc, dim, form, shuffle):
    """P2 Laplacian (per-element, P1-coefficient and curved): unknowns, pattern
    and values against the oracle's P2 numbering and assembly."""
    mesh = _mesh(dim, extra_vertices=2)
    if shuffle:
        mesh, _ = mg.shuffled(mesh, mg.rng_for(74))
    coords, conn = _t(mesh.coords), _t(mesh.conn)
    V = mesh.n_vert
    if form == LP2:
        coef = mg.lognormal_coef(mg.rng_for(75), mesh.n_elem)
        A = gfem.integrate_fwd(coords, conn, form, _t(coef))
    elif form == 4:
        A = gfem.integrate_fwd(coords, conn, form, _t(mg.lognormal_coef(mg.rng_for(76), V)))
    else:
        cm, mid = mg.curved_mesh(mesh, 0.03)
        A = gfem.integrate_fwd_iso(_t(cm.coords), conn, _t(mid), form)
    asm = gfem.Assembly(coords, conn, form)
    vals = asm.assemble(A)
    torch.cuda.synchronize()
    dofs_ref, N = orc.p2_dofs(dim, mesh.conn, V)
    assert asm.n_rows == N
    assert np.array_equal(asm.dofs.cpu().numpy(), dofs_ref)
    An = A.cpu().numpy()
    M = orc.assemble(dim, LP2, mesh.conn, V, An.astype(np.float64))
    rp, ci = asm.row_ptr.cpu().numpy(), asm.col_idx.cpu().numpy()
    assert np.array_equal(rp, M.indptr) and np.array_equal(ci, M.indices)
    r, c, v = _p2_expected(dofs_ref, An, N)
    assert np.array_equal(ci, c) and np.array_equal(vals.cpu().numpy(), v)   # element order, float32: same bits
    assert asm.nnz == len(v)
    v2 = asm.assemble(A)
    assert torch.equal(vals, v2)


def test_p2_assembly_energy_of_a_quadratic(gfem):
    """The assembled P2 Laplacian of the GPU element matrices gives the exact
    Dirichlet energy of x_0^2 (interpolated at vertices and edge midpoints) to
    FP32 accuracy."""
    mesh = mg.cube_tet_mesh(6, 0.15, mg.rng_for(77), 0.0, np.float32)
    coords, conn = _t(mesh.coords), _t(mesh.conn)
    A = gfem.integrate_fwd(coords, conn, LP2)
    asm = gfem.Assembly(coords, conn, LP2)
    vals = asm.assemble(A).double().cpu().numpy()
    dofs = asm.dofs.cpu().numpy()
    pts = np.zeros((asm.n_rows, 3))
    X = mesh.coords.astype(np.float64)
    pts[:mesh.n_vert] = X
    for q, (a, b) in enumerate(mg.edge_pairs(3)):
        pts[dofs[:, 4 + q]] = 0.5 * (X[mesh.conn[:, a]] + X[mesh.conn[:, b]])
    u = pts[:, 0] ** 2
    rp, ci = asm.row_ptr.cpu().numpy(), asm.col_idx.cpu().numpy()
    Ku = np.zeros_like(u)
    for i in range(asm.n_rows):
        Ku[i] = vals[rp[i]:rp[i + 1]] @ u[ci[rp[i]:rp[i + 1]]]
    P = X[mesh.conn]
    vol = np.abs(np.linalg.det(P[:, 1:] - P[:, :1])) / 6
    x0 = P[:, :, 0]
    exact = 4 * (vol / 20 * ((x0 ** 2).sum(1) + x0.sum(1) ** 2)).sum()
    assert abs(u @ Ku - exact) <= 1e-5 * exact
