"""fem_mesh_order / fem_mesh_renumber (-m gpu): a locality numbering for
unstructured meshes.  The orders are integer work, so they are compared
exactly with a NumPy restatement of their definition (Z-order codes of
positions and centroids on a grid over the bounding box, ties by old number,
FP32 arithmetic in the same order).  The renumbered mesh gives the same
element matrices bit for bit, the same coefficient gradients bit for bit, and
the same vertex gradients up to the reduction's summation order; it has far
fewer adjoint records than the shuffled mesh it came from."""
import numpy as np
import pytest
import torch

from paper_1103_0066_gb300 import meshgen as mg

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _spread(x, bits, d):
    r = np.zeros_like(x, dtype=np.int64)
    for i in range(bits):
        r |= ((x >> i) & 1) << (d * i)
    return r


def _codes(p, lo, hi, bits):
    """Z-order code of points p [n][d] (FP32) on 2^bits cells per axis."""
    d = p.shape[1]
    cells = np.float32(1 << bits)
    key = np.zeros(p.shape[0], np.int64)
    for a in range(d):
        s = cells / (hi[a] - lo[a]) if hi[a] > lo[a] else np.float32(0)
        q = np.floor((p[:, a] - lo[a]) * np.float32(s)).astype(np.float32)
        q = np.minimum(np.maximum(q, np.float32(0)), cells - np.float32(1)).astype(np.int64)
        key |= _spread(q, bits, d) << a
    return key


def _expected(mesh):
    d = mesh.dim
    bits = 7 if d == 3 else 10
    x = mesh.coords.astype(np.float32)
    lo, hi = x.min(0), x.max(0)
    vk = _codes(x, lo, hi, bits)
    c = np.zeros((mesh.n_elem, d), np.float32)
    for k in range(d + 1):
        c = (c + x[mesh.conn[:, k]]).astype(np.float32)
    c = (c * (np.float32(1) / np.float32(d + 1))).astype(np.float32)
    ek = _codes(c, lo, hi, bits)
    return (np.lexsort((np.arange(mesh.n_elem), ek)).astype(np.int32),
            np.lexsort((np.arange(mesh.n_vert), vk)).astype(np.int32))


def _meshes():
    tet = mg.shuffled(mg.cube_tet_mesh(12, 0.15, mg.rng_for(101), 0.05, np.float32), mg.rng_for(102))[0]
    tri = mg.shuffled(mg.square_tri_mesh(40, 0.2, mg.rng_for(103), np.float32), mg.rng_for(104))[0]
    return {"tet": tet, "tri": tri}


@pytest.mark.parametrize("which", ["tet", "tri"])
def test_order_equals_its_definition(gfem, which):
    mesh = _meshes()[which]
    ep, vp = gfem.mesh_order(_t(mesh.coords), _t(mesh.conn))
    ep_ref, vp_ref = _expected(mesh)
    assert np.array_equal(ep.cpu().numpy(), ep_ref)
    assert np.array_equal(vp.cpu().numpy(), vp_ref)


@pytest.mark.parametrize("which", ["tet", "tri"])
def test_renumbered_mesh_same_matrices_and_gradients(gfem, which):
    mesh = _meshes()[which]
    d = mesh.dim
    n = d + 1
    coords, conn = _t(mesh.coords), _t(mesh.conn)
    coef = _t(mg.lognormal_coef(mg.rng_for(105), mesh.n_elem))
    dA = _t(mg.upstream(mg.rng_for(106), mesh.n_elem, n))
    ep, vp = gfem.mesh_order(coords, conn)
    c2, k2 = gfem.renumber(coords, conn, ep, vp)
    epl, vpl = ep.long(), vp.long()
    assert torch.equal(c2, coords[vpl])
    inv = torch.empty_like(vpl)
    inv[vpl] = torch.arange(mesh.n_vert, device=DEV)
    assert torch.equal(k2.long(), inv[conn[epl].long()])
    A = gfem.integrate_fwd(coords, conn, 0, coef)
    A2 = gfem.integrate_fwd(c2, k2, 0, coef[epl].contiguous())
    assert torch.equal(A2, A[epl])
    dx, dw = gfem.integrate_bwd(coords, conn, 0, dA, coef)
    dx2, dw2 = gfem.integrate_bwd(c2, k2, 0, dA[epl].contiguous(), coef[epl].contiguous())
    assert torch.equal(dw2, dw[epl])
    assert float((dx2 - dx[vpl]).abs().max()) <= 1e-5 * float(dx.abs().max())


def test_renumbering_restores_record_sharing(gfem):
    """On the shuffled cube a 32-element tile shares few vertices; in the new
    order it shares most of them again."""
    mesh = _meshes()["tet"]
    coords, conn = _t(mesh.coords), _t(mesh.conn)
    ep, vp = gfem.mesh_order(coords, conn)
    c2, k2 = gfem.renumber(coords, conn, ep, vp)
    r_shuffled = gfem.Workspace(coords, conn).n_records()
    r_ordered = gfem.Workspace(c2, k2).n_records()
    assert r_ordered < 0.5 * r_shuffled, (r_ordered, r_shuffled)


def test_order_edge_cases(gfem):
    from paper_1103_0066_gb300 import _native as nat
    mesh = _meshes()["tet"]
    conn = mesh.conn.copy()
    conn[3, 2] = mesh.n_vert + 5  # an out-of-range vertex: code 0, kept as is by the renumbering
    coords_t, conn_t = _t(mesh.coords), _t(conn)
    ep, vp = gfem.mesh_order(coords_t, conn_t)
    assert np.array_equal(np.sort(ep.cpu().numpy()), np.arange(mesh.n_elem))
    assert np.array_equal(np.sort(vp.cpu().numpy()), np.arange(mesh.n_vert))
    _, k2 = gfem.renumber(coords_t, conn_t, ep, vp)
    pos = int(np.flatnonzero(ep.cpu().numpy() == 3)[0])
    assert int(k2[pos, 2]) == mesh.n_vert + 5
    # FP64 coordinates are refused
    with pytest.raises(nat.FemError) as ei:
        gfem.mesh_order(coords_t.double(), conn_t)
    assert ei.value.status == nat.FEM_ERR_UNSUPPORTED
    # a mesh packed into one grid cell: refused before the sort
    flat = torch.zeros((2000, 3), device=DEV)
    tets = torch.arange(2000, device=DEV, dtype=torch.int32)[:1996].view(-1, 4).contiguous()
    with pytest.raises(nat.FemError) as ei:
        gfem.mesh_order(flat, tets)
    assert ei.value.status == nat.FEM_ERR_UNSUPPORTED
