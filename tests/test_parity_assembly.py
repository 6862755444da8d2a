"""GPU parity of the global assembly (-m gpu).

* The pattern (row_ptr, col_idx) equals the oracle's CSR structure exactly.
* The values equal, bit for bit, float32 sums of the same GPU element matrices
  in the order the library defines (numpy's unbuffered np.add.at): for the
  scalar forms, per 32-element tile the contributions in element order, then
  those tile sums in tile order; for P1 elasticity's blocks, all contributions
  in element order.
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
        gfem.Assembly(coords, conn, LP2)  # P2 unknowns include edges: unsupported
    bad = mesh.conn.copy()
    bad[4, 1] = mesh.n_vert + 2
    with pytest.raises(gfem.FemError):
        gfem.Assembly(coords, _t(bad), LP1)
    empty = gfem.Assembly(coords, conn[:0], LP1)
    assert empty.nnz == 0 and torch.all(empty.row_ptr == 0)
    vals = empty.assemble(torch.empty((0, 3, 3), device=DEV))
    assert vals.numel() == 0
