"""Parity on unstructured meshes (-m gpu).

Every other parity test integrates structured meshes in cell-major order,
where a 32-element tile touches about 30 distinct vertices.  A mesh from an
unstructured generator comes in no such order: here the elements of the
jittered sliver cube are put in a seeded random order and its vertices are
renumbered at random (``meshgen.shuffled``).  The element matrices and
gradients are the same mathematics -- element order and vertex numbering
carry no meaning in Eq. 6 -- but the kernels take other branches:

* the adjoint's record tiles have up to 128 records, which do not fit the
  aligned 256-position stage on tets, so every such tile packs its runs back
  to back (asserted from the built workspace);
* the assembly's tiles have more distinct vertices than its dense 36 x 36
  tile holds, so they take the per-record scan (asserted from the
  connectivity, which decides the branch);
* the coordinate gather has no locality to speak of.

Tolerances are those of the structured tests: 1e-5 per element relative to
max |A_e| for FP32, 1e-5 of max |g| for gradients; the deterministic and
batched paths must match their per-mesh counterparts bit for bit."""
import numpy as np
import pytest
import torch

from paper_1103_0066_gb300 import meshgen as mg
from conftest import rel_err_per_element

pytestmark = pytest.mark.gpu
LP1, LP2, EP1, LP1W, LP2W = 0, 1, 2, 3, 4
TOL = 1e-5
DEV = "cuda:0"


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _mesh(dim, n=None, seed=101):
    if dim == 2:
        base = mg.square_tri_mesh(n or 13, 0.2, mg.rng_for(seed), np.float32)
    else:
        base = mg.cube_tet_mesh(n or 7, 0.15, mg.rng_for(seed), 0.05, np.float32)
    return mg.shuffled(base, mg.rng_for(seed + 1))[0]


def _rel(a, b):
    return float(np.abs(np.asarray(a, np.float64) - b).max() / np.abs(b).max())


def _tile_layout(ws, mesh):
    """(tile_rec [T+1], record spans [R]) read from a built adjoint workspace."""
    E, NV, TS = mesh.n_elem, mesh.dim + 1, 32
    T = (E + TS - 1) // TS
    al = lambda x: ((x + 255) // 256) * 256
    raw = ws.buf.cpu().numpy()
    tile_rec = raw[: 4 * (T + 1)].view(np.int32)
    o_rank = al(4 * (T + 1))
    o_span = al(o_rank + 4 * T * TS)
    R = int(tile_rec[T])
    span = raw[o_span: o_span + 2 * R].view(np.uint16).astype(np.int64)
    return tile_rec, span


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("form", [LP1, LP2, EP1])
def test_forward_unstructured(gfem, orc, dim, form):
    mesh = _mesh(dim)
    coef = mg.lognormal_coef(mg.rng_for(102), mesh.n_elem)
    Ar, fl = orc.integrate(dim, form, mesh.conn, mesh.coords, coef)
    assert not fl.any()
    contracts = [gfem.CONTRACT_F32] + ([gfem.CONTRACT_BF16X3] if form != LP1 else [])
    for contract in contracts:
        A = gfem.integrate_fwd(_t(mesh.coords), _t(mesh.conn), form, _t(coef), contract=contract)
        err = rel_err_per_element(A.cpu().numpy(), Ar)
        assert err.max() <= TOL, (contract, err.max())
    if dim == 3:
        assert mesh.sliver.any() and err[mesh.sliver].max() <= TOL


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("form", [LP1, LP2, EP1])
def test_adjoint_unstructured(gfem, orc, dim, form):
    """Both reductions and the saved-det adjoint against the oracle's reverse
    mode; the deterministic result is bitwise reproducible and equal with and
    without the saved det; on tets the record stage packs its runs."""
    mesh = _mesh(dim)
    n = mg.form_n(form, dim)
    coef = mg.lognormal_coef(mg.rng_for(103), mesh.n_elem)
    dA = mg.upstream(mg.rng_for(104), mesh.n_elem, n)
    coords, conn = _t(mesh.coords), _t(mesh.conn)
    gx, gw = orc.integrate_vjp(dim, form, mesh.conn, mesh.coords, dA, coef)
    ws = gfem.Workspace(coords, conn, form)
    det = torch.empty(mesh.n_elem, device=DEV)
    gfem.integrate_fwd(coords, conn, form, _t(coef), det_out=det)
    det_x = None
    for reduce in (0, 1):
        dx, dw = gfem.integrate_bwd(coords, conn, form, _t(dA), _t(coef), ws=ws, reduce=reduce)
        assert _rel(dx.cpu().numpy(), gx) <= TOL
        assert _rel(dw.cpu().numpy(), gw) <= TOL
        sx, sw = gfem.integrate_bwd(coords, conn, form, _t(dA), _t(coef), ws=ws, reduce=reduce, det=det)
        assert torch.equal(sw, dw)
        if reduce == 0:
            assert torch.equal(sx, dx)
            again, _ = gfem.integrate_bwd(coords, conn, form, _t(dA), _t(coef), ws=gfem.Workspace(coords, conn),
                                          need_dcoef=False, warps_per_cta=4, ctas_per_sm=1)
            assert torch.equal(again, dx)
            det_x = dx
    tile_rec, span = _tile_layout(ws, mesh)
    T = len(tile_rec) - 1
    packed = 0
    for t in range(T):
        rb, re = tile_rec[t], tile_rec[t + 1]
        beg, ln = span[rb:re] & 0xFF, span[rb:re] >> 8
        if np.array_equal(beg, np.concatenate([[0], np.cumsum(ln)[:-1]])):
            packed += 1
    assert tile_rec[T] > 0.6 * (dim + 1) * mesh.n_elem  # most slots are records of their own
    if dim == 3:
        assert packed > T // 2                       # the packed stage is the common case here
    assert det_x is not None


@pytest.mark.parametrize("dim", [2, 3])
def test_tile_order_records_parity(gfem, orc, dim):
    """A shuffled mesh large enough that the vertex-major record rows would
    scatter (12^3 tets, 60^2 triangles): the build keeps the records in tile
    order (rec_dest is the identity) and the reduction gathers them.  Both
    reductions and the saved-det adjoint against the oracle; the deterministic
    result is reproducible."""
    mesh = _mesh(dim, 12 if dim == 3 else 60)
    coef = mg.lognormal_coef(mg.rng_for(116), mesh.n_elem)
    dA = mg.upstream(mg.rng_for(117), mesh.n_elem, dim + 1)
    coords, conn = _t(mesh.coords), _t(mesh.conn)
    ws = gfem.Workspace(coords, conn)
    assert ws.record_layout() == gfem.nat.RECORDS_TILE_ORDER
    E, NV = mesh.n_elem, dim + 1
    T = (E + 31) // 32
    al = lambda x: ((x + 255) // 256) * 256
    raw = ws.buf.cpu().numpy()
    o_dest = al(al(al(4 * (T + 1)) + 4 * T * 32) + 2 * NV * E)
    R = ws.n_records()
    assert np.array_equal(raw[o_dest: o_dest + 4 * R].view(np.int32), np.arange(R))
    gx, gw = orc.integrate_vjp(dim, LP1, mesh.conn, mesh.coords, dA, coef)
    det = torch.empty(E, device=DEV)
    gfem.integrate_fwd(coords, conn, LP1, _t(coef), det_out=det)
    dx, dw = gfem.integrate_bwd(coords, conn, LP1, _t(dA), _t(coef), ws=ws)
    assert _rel(dx.cpu().numpy(), gx) <= TOL and _rel(dw.cpu().numpy(), gw) <= TOL
    sx, _ = gfem.integrate_bwd(coords, conn, LP1, _t(dA), _t(coef), ws=ws, det=det)
    ax, _ = gfem.integrate_bwd(coords, conn, LP1, _t(dA), _t(coef), reduce=1)
    again, _ = gfem.integrate_bwd(coords, conn, LP1, _t(dA), _t(coef), ws=gfem.Workspace(coords, conn))
    assert torch.equal(sx, dx) and torch.equal(again, dx)
    assert _rel(ax.cpu().numpy(), gx) <= TOL


def test_record_layouts_give_the_same_bits(gfem):
    """The same mesh, once with cell-major elements and vertices (vertex-major
    records) and once with only its vertices renumbered at random (tile-order
    records: the record tiles are the same, but their vertex-major rows
    scatter): dcoords, mapped back to the original vertex numbers, is equal
    bit for bit, because both layouts sum each vertex's records in increasing
    record order."""
    base = mg.cube_tet_mesh(9, 0.15, mg.rng_for(113), 0.05, np.float32)
    renum, _ = mg.shuffled(base, mg.rng_for(114), elements=False, vertices=True)
    dA = _t(mg.upstream(mg.rng_for(115), base.n_elem, 4))
    out = []
    for m in (base, renum):
        coords, conn = _t(m.coords), _t(m.conn)
        ws = gfem.Workspace(coords, conn)
        dx, _ = gfem.integrate_bwd(coords, conn, LP1, dA, ws=ws, need_dcoef=False)
        out.append((dx.cpu().numpy(), ws.record_layout()))
    assert out[0][1] == gfem.nat.RECORDS_VERTEX_MAJOR and out[1][1] == gfem.nat.RECORDS_TILE_ORDER
    # vertex v of base is vertex new_id[v] of renum; recover new_id from the coordinates
    key = {tuple(x): i for i, x in enumerate(renum.coords.tolist())}
    new_id = np.array([key[tuple(x)] for x in base.coords.tolist()])
    assert np.array_equal(out[1][0][new_id], out[0][0])


def test_deferred_reduction_and_sharded_slices_unstructured(gfem, orc):
    mesh = _mesh(3, 8)
    coords, conn = _t(mesh.coords), _t(mesh.conn)
    dA = _t(mg.upstream(mg.rng_for(105), mesh.n_elem, 4))
    ws = gfem.Workspace(coords, conn)
    ref, _ = gfem.integrate_bwd(coords, conn, LP1, dA, ws=ws, need_dcoef=False)
    dx = torch.full_like(ref, float("nan"))
    gfem.integrate_bwd(coords, conn, LP1, dA, ws=ws, reduce=gfem.REDUCE_DEFERRED, dcoords=dx, need_dcoef=False)
    gfem.adjoint_reduce(coords, conn, ws, dx)
    assert torch.equal(dx, ref)
    from paper_1103_0066_gb300.shard import element_range
    gx, _ = orc.integrate_vjp(3, LP1, mesh.conn, mesh.coords, dA.cpu().numpy())
    acc = np.zeros((mesh.n_vert, 3))
    for r in range(3):
        e0, e1 = element_range(mesh.n_elem, 3, r)
        px, _ = gfem.integrate_bwd(coords, conn[e0:e1].contiguous(), LP1, dA[e0:e1].contiguous(), need_dcoef=False)
        acc += px.double().cpu().numpy()
    assert _rel(acc, gx) <= TOL


@pytest.mark.parametrize("mode", ["single", "grouped", "concurrent", "per_item", "per_item_concurrent", "phased"])
def test_batch_unstructured(gfem, orc, mode):
    modes = {"single": gfem.BATCH_SINGLE, "grouped": gfem.BATCH_GROUPED,
             "concurrent": gfem.BATCH_GROUPED_CONCURRENT, "per_item": gfem.BATCH_PER_ITEM,
             "per_item_concurrent": gfem.BATCH_PER_ITEM_CONCURRENT, "phased": gfem.BATCH_PHASED}
    src = mg.mixed_batch(n_meshes=24, scale=0.003, shuffle=True)
    items = []
    for b in src:
        m = b.mesh
        n = mg.form_n(b.form, m.dim)
        items.append({"coords": _t(m.coords), "conn": _t(m.conn), "form": b.form, "coef": _t(b.coef), "src": b,
                      "A": torch.full((m.n_elem, n, n), float("nan"), device=DEV), "dA": _t(b.dA),
                      "dcoords": torch.full((m.n_vert, m.dim), float("nan"), device=DEV),
                      "dcoef": torch.full((m.n_elem,), float("nan"), device=DEV)})
    batch = gfem.Batch(items)
    batch.set_config(2, 1, modes[mode])
    batch.run()
    torch.cuda.synchronize()
    assert batch.errors() == 0
    for k, it in enumerate(items):
        A_ref = gfem.integrate_fwd(it["coords"], it["conn"], it["form"], it["coef"])
        dx_ref, dw_ref = gfem.integrate_bwd(it["coords"], it["conn"], it["form"], it["dA"], it["coef"])
        assert torch.equal(it["A"], A_ref), k
        assert torch.equal(it["dcoords"], dx_ref), k
        assert torch.equal(it["dcoef"], dw_ref), k
        if mode == "single" and k % 5 == 0:
            b = it["src"]
            Ar, _ = orc.integrate(b.mesh.dim, b.form, b.mesh.conn, b.mesh.coords, b.coef)
            assert rel_err_per_element(it["A"].cpu().numpy(), Ar).max() <= TOL
            gx, gw = orc.integrate_vjp(b.mesh.dim, b.form, b.mesh.conn, b.mesh.coords, b.dA, b.coef)
            assert _rel(it["dcoords"].cpu().numpy(), gx) <= TOL and _rel(it["dcoef"].cpu().numpy(), gw) <= TOL


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("form", [LP1, EP1, LP1W])
def test_assembly_unstructured(gfem, orc, dim, form):
    """CSR / BSR assembly on a shuffled mesh: bitwise the library's fixed-order
    sums (per 32-element tile in element order, then in tile order; blocks in
    element order), and the FP64 oracle within the per-row bound.  On tets the
    scalar forms' tiles exceed the 36 distinct vertices of the dense tile, so
    the per-record scan runs."""
    mesh = _mesh(dim, 6 if dim == 3 else 11)
    coords, conn = _t(mesh.coords), _t(mesh.conn)
    coef = (mg.lognormal_coef(mg.rng_for(106), mesh.n_vert) if form == LP1W
            else mg.lognormal_coef(mg.rng_for(107), mesh.n_elem))
    A = gfem.integrate_fwd(coords, conn, form, _t(coef))
    asm = gfem.Assembly(coords, conn, form)
    vals = asm.assemble(A)
    torch.cuda.synchronize()
    b = dim if form == EP1 else 1
    rp, ci = asm.row_ptr.cpu().numpy(), asm.col_idx.cpu().numpy()
    P = orc.assemble(dim, LP1, mesh.conn, mesh.n_vert, np.ones((mesh.n_elem, dim + 1, dim + 1)))
    assert np.array_equal(rp, P.indptr) and np.array_equal(ci, P.indices)
    Ah = A.cpu().numpy()
    if form == EP1:
        g = (mesh.conn[:, None, :].astype(np.int64) * dim + np.arange(dim)[None, :, None]).reshape(mesh.n_elem, -1)
    else:
        g = mesh.conn.astype(np.int64)
    pos = {}
    for v in range(mesh.n_vert):
        for k in range(rp[v], rp[v + 1]):
            pos[(v, ci[k])] = k
    vi, vj = g[:, :, None] // b, g[:, None, :] // b
    slot = np.vectorize(lambda x, y: pos[(x, y)])(np.broadcast_to(vi, (mesh.n_elem, g.shape[1], g.shape[1])),
                                                  np.broadcast_to(vj, (mesh.n_elem, g.shape[1], g.shape[1])))
    slot = slot * b * b + (g[:, :, None] % b) * b + (g[:, None, :] % b)
    ref32 = np.zeros(asm.nnz * b * b, np.float32)
    n = g.shape[1]
    if b == 1:
        tiles = np.arange(mesh.n_elem) // 32
        nr = np.array([np.unique(mesh.conn[32 * t: 32 * t + 32]).size for t in range((mesh.n_elem + 31) // 32)])
        if dim == 3:
            assert (nr > 36).sum() > len(nr) // 2         # the dense tile's capacity is exceeded
        ent = slot.reshape(-1)
        tile = np.repeat(tiles, n * n)
        keys, inv = np.unique(tile * ref32.size + ent, return_inverse=True)
        part = np.zeros(keys.size, np.float32)
        np.add.at(part, inv, Ah.reshape(-1))
        np.add.at(ref32, keys % ref32.size, part)
        assert asm.n_records == keys.size
    else:
        np.add.at(ref32, slot.ravel(), Ah.reshape(-1))
    got = vals.cpu().numpy().reshape(-1)
    assert np.array_equal(got, ref32)
    if form == LP1W:
        Ar, _ = orc.integrate_w1(dim, LP1, mesh.conn, mesh.coords, coef)
        Mr = orc.assemble(dim, LP1, mesh.conn, mesh.n_vert, Ar)
    else:
        Ar, _ = orc.integrate(dim, form, mesh.conn, mesh.coords, coef)
        Mr = orc.assemble(dim, form, mesh.conn, mesh.n_vert, Ar)
    Mr = Mr.toarray()
    D = np.zeros((mesh.n_vert * b, mesh.n_vert * b))
    gv = got.astype(np.float64).reshape(-1, b, b)
    for v in range(mesh.n_vert):
        for k in range(rp[v], rp[v + 1]):
            D[v * b:(v + 1) * b, ci[k] * b:(ci[k] + 1) * b] = gv[k]
    elmax = np.abs(Ar).reshape(mesh.n_elem, -1).max(1)
    bound = np.zeros(mesh.n_vert)
    for i in range(dim + 1):
        np.add.at(bound, mesh.conn[:, i], elmax)
    bound = np.repeat(bound, b)
    err = np.abs(D - Mr).max(1)
    assert np.all(err <= TOL * bound + 1e-300)


@pytest.mark.parametrize("dim", [2, 3])
def test_p1_coefficient_and_non_affine_unstructured(gfem, orc, dim):
    """The P1-coefficient forms (Eqs. 20-23; P2 also on the tensor cores) and
    the non-affine forms (Eqs. 16-19; P2 also on the tensor cores) on a
    shuffled mesh, against the oracle."""
    mesh = _mesh(dim)
    coords, conn = _t(mesh.coords), _t(mesh.conn)
    wv = mg.lognormal_coef(mg.rng_for(108), mesh.n_vert)
    for form, contract in ((LP1W, 0), (LP2W, 0), (LP2W, 1)):
        A = gfem.integrate_fwd(coords, conn, form, _t(wv), contract=contract)
        Ar, _ = orc.integrate_w1(dim, form - 3, mesh.conn, mesh.coords, wv)
        assert rel_err_per_element(A.cpu().numpy(), Ar).max() <= TOL, (form, contract)
    base = mg.cube_tet_mesh(6, 0.15, mg.rng_for(109), 0.0, np.float32) if dim == 3 else \
        mg.square_tri_mesh(12, 0.2, mg.rng_for(109), np.float32)
    curved, mid = mg.curved_mesh(base)
    sh, order = mg.shuffled(curved, mg.rng_for(110))
    mid = np.ascontiguousarray(mid[order])
    for form, contract in ((gfem.LAPLACE_P1_ISO, 0), (gfem.LAPLACE_P2_ISO, 0), (gfem.LAPLACE_P2_ISO, 1)):
        A = gfem.integrate_fwd_iso(_t(sh.coords), _t(sh.conn), _t(mid), form, contract=contract)
        Ar, _ = orc.integrate_iso(dim, form - 5, sh.conn, sh.coords, mid)
        assert rel_err_per_element(A.cpu().numpy(), Ar).max() <= TOL, (form, contract)


def test_full_size_unstructured_step_sampled(gfem, orc):
    """The benchmark step on the shuffled 128^3 sliver cube (12,582,912 tets in
    random order, vertices renumbered): forward saving det J, deterministic
    adjoint with it, in the bench's launch configuration.  dcoords at sampled
    vertices against the oracle's reverse mode over all their incident
    elements; A on a stratified element sample."""
    mesh = mg.workload_tet_shuffled(128)
    E, V = mesh.n_elem, mesh.n_vert
    dA_h = mg.upstream(mg.rng_for(111), E, 4)
    coords, conn, dA = _t(mesh.coords), _t(mesh.conn), _t(dA_h)
    det = torch.empty(E, device=DEV)
    A = gfem.integrate_fwd(coords, conn, LP1, det_out=det)
    ws = gfem.Workspace(coords, conn)
    dx, _ = gfem.integrate_bwd(coords, conn, LP1, dA, ws=ws, reduce=gfem.REDUCE_DEFERRED, need_dcoef=False,
                               det=det)
    gfem.adjoint_reduce(coords, conn, ws, dx)
    torch.cuda.synchronize()
    rng = np.random.default_rng(112)
    verts = rng.choice(V, 2000, replace=False)
    hit = np.zeros(V, bool)
    hit[verts] = True
    el = np.where(hit[mesh.conn].any(1))[0]
    gx, _ = orc.integrate_vjp(3, LP1, mesh.conn[el], mesh.coords, dA_h[el])
    got = dx.cpu().numpy()[verts].astype(np.float64)
    assert np.abs(got - gx[verts]).max() <= TOL * np.abs(gx[verts]).max()
    idx = np.unique(np.concatenate([rng.choice(np.where(mesh.sliver)[0], 5000, replace=False),
                                    rng.choice(E, 5000, replace=False), np.arange(E - 40, E)]))
    Ar, _ = orc.integrate(3, LP1, mesh.conn[idx], mesh.coords)
    Ag = A[torch.from_numpy(idx).to(DEV)].double().cpu().numpy()
    assert rel_err_per_element(Ag, Ar).max() <= TOL
