"""GPU parity of the adjoint against the oracle's reverse mode (-m gpu).

Tolerance: max_v |g_gpu - g_ref| <= 1e-5 max_v |g_ref| for the coordinate
gradient and the same, relative to max |dcoef_ref|, for the coefficient
gradient.  The deterministic reduction must be bitwise reproducible; the
atomic variant differs from it only by FP32 summation order."""
import numpy as np
import pytest
import torch

from paper_1103_0066_gb300 import meshgen as mg
from conftest import rel_err_per_element

pytestmark = pytest.mark.gpu
LP1, LP2, EP1 = 0, 1, 2
TOL = 1e-5
DEV = "cuda:0"


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _mesh(dim, n=None):
    if dim == 2:
        return mg.square_tri_mesh(n or 11, 0.2, mg.rng_for(41), np.float32)
    return mg.cube_tet_mesh(n or 6, 0.15, mg.rng_for(41), 0.05, np.float32)


def _rel(a, b):
    return float(np.abs(np.asarray(a, np.float64) - b).max() / np.abs(b).max())


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("form", [LP1, LP2, EP1])
@pytest.mark.parametrize("reduce", [0, 1])
def test_adjoint_matches_oracle(gfem, orc, dim, form, reduce):
    mesh = _mesh(dim)
    n = mg.form_n(form, dim)
    coef = mg.lognormal_coef(mg.rng_for(42), mesh.n_elem)
    dA = mg.upstream(mg.rng_for(43), mesh.n_elem, n)
    dx, dw = gfem.integrate_bwd(_t(mesh.coords), _t(mesh.conn), form, _t(dA), _t(coef), reduce=reduce)
    gx, gw = orc.integrate_vjp(dim, form, mesh.conn, mesh.coords, dA, coef)
    assert _rel(dx.cpu().numpy(), gx) <= TOL
    assert _rel(dw.cpu().numpy(), gw) <= TOL


def test_deterministic_is_bitwise_reproducible(gfem):
    mesh = _mesh(3, 10)
    dA = _t(mg.upstream(mg.rng_for(44), mesh.n_elem, 4))
    coords, conn = _t(mesh.coords), _t(mesh.conn)
    ws = gfem.Workspace(coords, conn)
    a, _ = gfem.integrate_bwd(coords, conn, LP1, dA, ws=ws, need_dcoef=False)
    b, _ = gfem.integrate_bwd(coords, conn, LP1, dA, ws=ws, need_dcoef=False, warps_per_cta=8, ctas_per_sm=1)
    ws2 = gfem.Workspace(coords, conn)  # rebuilt incidence: same sorted order
    c, _ = gfem.integrate_bwd(coords, conn, LP1, dA, ws=ws2, need_dcoef=False)
    assert torch.equal(a, b) and torch.equal(a, c)
    d, _ = gfem.integrate_bwd(coords, conn, LP1, dA, reduce=1, need_dcoef=False)
    assert _rel(d.cpu().numpy(), a.cpu().numpy().astype(np.float64)) <= 1e-6


def test_tile_records_structure(gfem):
    """Workspace of the deterministic reduction: each 32-element record tile has
    one record per distinct vertex, in vertex order; each record's span (start,
    length) in the tile's slot stage holds exactly the slots of its vertex, in
    increasing slot order (the slot's rank is its stage position); the spans
    are disjoint and ordered; on tets a padded tile starts record r at a
    position congruent to 3r mod 8 (a packed one back to back); absent slots sit
    past the last run; and rec_dest places the records of every vertex, in
    record order, in that vertex's run [voff[v], voff[v+1]) of the
    vertex-major array."""
    for dim, n, cut in ((3, 5, 0), (3, 6, 37), (2, 9, 11)):
        mesh = _mesh(dim, n)
        if cut:  # a ragged last tile
            mesh.conn = mesh.conn[: mesh.n_elem - cut]
        coords, conn = _t(mesh.coords), _t(mesh.conn)
        ws = gfem.Workspace(coords, conn)
        E, NV, TS = mesh.n_elem, dim + 1, 32
        cap = 256 if dim == 3 else TS * NV
        T = (E + TS - 1) // TS
        al = lambda x: ((x + 255) // 256) * 256
        raw = ws.buf.cpu().numpy()
        tile_rec = raw[: 4 * (T + 1)].view(np.int32)
        o_rank = al(4 * (T + 1))
        rank = raw[o_rank: o_rank + 4 * T * TS].reshape(T * TS, 4)
        o_span = al(o_rank + 4 * T * TS)
        R = int(tile_rec[T])
        span = raw[o_span: o_span + 2 * R].view(np.uint16).astype(np.int64)
        o_dest = al(o_span + 2 * NV * E)
        rec_dest = raw[o_dest: o_dest + 4 * R].view(np.int32)
        o_voff = al(al(o_dest + 4 * NV * E) + 4 * NV * E)
        voff = raw[o_voff: o_voff + 4 * (mesh.n_vert + 1)].view(np.int32)
        flat = mesh.conn.ravel()
        assert tile_rec[0] == 0
        assert np.array_equal(np.sort(rec_dest), np.arange(R))      # a permutation of the records
        rec_vtx = np.empty(R, np.int64)
        n_padded = 0
        for t in range(T):
            slots = np.arange(t * TS * NV, min((t + 1) * TS * NV, NV * E))
            verts = flat[slots]
            local = slots - t * TS * NV
            order = local[np.lexsort((local, verts))]              # slots in (vertex, slot) order
            u, counts = np.unique(verts, return_counts=True)
            rb, rn = tile_rec[t], tile_rec[t + 1] - tile_rec[t]
            assert rn == len(u)
            beg, ln = span[rb: rb + rn] & 0xFF, span[rb: rb + rn] >> 8
            assert np.array_equal(ln, counts)
            assert np.all(beg[1:] >= beg[:-1] + ln[:-1])              # disjoint, in record order
            padded = not np.array_equal(beg, np.concatenate([[0], np.cumsum(counts)[:-1]]))
            if padded:
                assert dim == 3 and np.all(beg % 8 == (3 * np.arange(rn)) % 8)
                n_padded += 1
            pos = np.concatenate([b + np.arange(c) for b, c in zip(beg, ln)])
            got = rank[t * TS + order // NV, order % NV].astype(np.int64)
            assert np.array_equal(got, pos)                          # slot order within each run
            absent = np.arange(len(slots), TS * NV)                  # slots past the last element
            if len(absent):
                ra = rank[t * TS + absent // NV, absent % NV].astype(np.int64)
                end = beg[-1] + ln[-1]
                assert np.array_equal(np.sort(ra), end + np.arange(len(absent))) and ra.max() < cap
            assert pos.max() < cap
            rec_vtx[rb: rb + rn] = u
        assert (n_padded > 0) == (dim == 3)
        assert np.array_equal(np.diff(voff), np.bincount(rec_vtx, minlength=mesh.n_vert))
        n_rec, layout = gfem.nat.fem_incidence_info(ws.m, ws.buf.data_ptr(), ws.bytes, 0)
        assert n_rec == R and layout == gfem.nat.RECORDS_VERTEX_MAJOR   # cell-major meshes keep their locality
        order = np.argsort(rec_dest)                                 # record stored at each row
        assert np.array_equal(rec_vtx[order], np.repeat(np.arange(mesh.n_vert), np.diff(voff)))
        for v in range(mesh.n_vert):                                  # record order within a vertex
            assert np.all(np.diff(order[voff[v]: voff[v + 1]]) > 0)


def test_coefficient_only_and_coords_only(gfem, orc):
    mesh = _mesh(3)
    coef = mg.lognormal_coef(mg.rng_for(45), mesh.n_elem)
    dA = mg.upstream(mg.rng_for(46), mesh.n_elem, 4)
    gx, gw = orc.integrate_vjp(3, LP1, mesh.conn, mesh.coords, dA, coef)
    dx, dw = gfem.integrate_bwd(_t(mesh.coords), _t(mesh.conn), LP1, _t(dA), _t(coef), need_dcoords=False)
    assert dx is None and _rel(dw.cpu().numpy(), gw) <= TOL
    dx, dw = gfem.integrate_bwd(_t(mesh.coords), _t(mesh.conn), LP1, _t(dA), _t(coef), need_dcoef=False)
    assert dw is None and _rel(dx.cpu().numpy(), gx) <= TOL


def test_autograd_function(gfem, orc):
    mesh = _mesh(3)
    coef0 = mg.lognormal_coef(mg.rng_for(47), mesh.n_elem)
    dA = mg.upstream(mg.rng_for(48), mesh.n_elem, 12)
    x = _t(mesh.coords).requires_grad_(True)
    w = _t(coef0).requires_grad_(True)
    A = gfem.Mesh(x, _t(mesh.conn)).integrate(EP1, w)
    (A * _t(dA)).sum().backward()
    gx, gw = orc.integrate_vjp(3, EP1, mesh.conn, mesh.coords, dA, coef0)
    assert _rel(x.grad.cpu().numpy(), gx) <= TOL
    assert _rel(w.grad.cpu().numpy(), gw) <= TOL


def test_autograd_tensor_core_forward(gfem, orc):
    """fem.integrate(..., contract=BF16X3): the forward on the tensor cores within
    the FP32 tolerance of the oracle; the adjoint is the FP32 one, so the
    deterministic gradients equal the FP32-contract ones bit for bit."""
    mesh = _mesh(3)
    coef0 = mg.lognormal_coef(mg.rng_for(47), mesh.n_elem)
    dA = _t(mg.upstream(mg.rng_for(48), mesh.n_elem, 12))
    grads = {}
    for contract in (gfem.CONTRACT_F32, gfem.CONTRACT_BF16X3):
        x = _t(mesh.coords).requires_grad_(True)
        w = _t(coef0).requires_grad_(True)
        A = gfem.integrate(x, _t(mesh.conn), EP1, w, contract=contract)
        (A * dA).sum().backward()
        grads[contract] = (A.detach(), x.grad, w.grad)
    Ar, _ = orc.integrate(3, EP1, mesh.conn, mesh.coords, coef0)
    assert rel_err_per_element(grads[gfem.CONTRACT_BF16X3][0].cpu().numpy(), Ar).max() <= TOL
    assert torch.equal(grads[gfem.CONTRACT_F32][1], grads[gfem.CONTRACT_BF16X3][1])
    assert torch.equal(grads[gfem.CONTRACT_F32][2], grads[gfem.CONTRACT_BF16X3][2])


def test_sharded_slices_sum_to_the_whole_adjoint(gfem, orc):
    """One mesh split by elements as N ranks would split it (here one after
    another on one GPU, no collective): the slices' partial vertex gradients
    from the kernels add up to the whole mesh's gradient within the FP32
    tolerance, and their coefficient gradients are its rows bit for bit.  On
    one rank (no process group) ShardedMesh is integrate_bwd itself."""
    from paper_1103_0066_gb300.shard import ShardedMesh, element_range
    mesh = _mesh(3)
    coords, conn = _t(mesh.coords), _t(mesh.conn)
    coef = _t(mg.lognormal_coef(mg.rng_for(91), mesh.n_elem))
    dA = _t(mg.upstream(mg.rng_for(92), mesh.n_elem, 4))
    dx, dw = gfem.integrate_bwd(coords, conn, LP1, dA, coef)
    gx, _ = orc.integrate_vjp(3, LP1, mesh.conn, mesh.coords, dA.cpu().numpy(), coef.cpu().numpy())
    for world in (2, 3):
        acc = np.zeros((mesh.n_vert, 3))
        for r in range(world):
            e0, e1 = element_range(mesh.n_elem, world, r)
            px, pw = gfem.integrate_bwd(coords, conn[e0:e1].contiguous(), LP1, dA[e0:e1].contiguous(), coef[e0:e1])
            acc += px.double().cpu().numpy()
            assert torch.equal(pw, dw[e0:e1])
        assert _rel(acc, gx) <= TOL
    sm = ShardedMesh(coords, conn, LP1)
    assert (sm.world, sm.e0, sm.e1) == (1, 0, mesh.n_elem)
    sx, sw = sm.integrate_bwd(dA, coef)
    torch.cuda.synchronize()
    assert torch.equal(sx, dx) and torch.equal(sw, dw)
    assert torch.equal(sm.integrate_fwd(coef), gfem.integrate_fwd(coords, conn, LP1, coef))


def test_adjoint_against_fp64_finite_differences(gfem, orc):
    """4^3 mesh with slivers: the GPU gradient against FP64 central differences of
    the oracle's forward, per-vertex step 1e-4 x the smallest incident height."""
    mesh = mg.cube_tet_mesh(4, 0.15, mg.rng_for(4), 0.05, np.float32)
    X = mesh.coords.astype(np.float64)
    dA = mg.upstream(mg.rng_for(49), mesh.n_elem, 4).astype(np.float64)
    dx, _ = gfem.integrate_bwd(_t(mesh.coords), _t(mesh.conn), LP1, _t(dA.astype(np.float32)),
                               need_dcoef=False)
    g = dx.cpu().numpy().astype(np.float64)
    P = X[mesh.conn]
    vol = np.abs(np.linalg.det(P[:, 1:] - P[:, :1]))
    fd = np.zeros_like(X)
    for v in range(X.shape[0]):
        inc = np.where((mesh.conn == v).any(1))[0]
        if inc.size == 0:
            continue
        sub = mesh.conn[inc]
        h = np.inf
        for e in inc:
            for k in range(4):
                f = np.delete(P[e], k, axis=0)
                area = np.linalg.norm(np.cross(f[1] - f[0], f[2] - f[0]))
                h = min(h, vol[e] / area)
        d = 1e-4 * h
        for a in range(3):
            Xp, Xm = X.copy(), X.copy()
            Xp[v, a] += d
            Xm[v, a] -= d
            Ap, _ = orc.integrate(3, LP1, sub, Xp)
            Am, _ = orc.integrate(3, LP1, sub, Xm)
            fd[v, a] = (np.sum(dA[inc] * Ap) - np.sum(dA[inc] * Am)) / (2 * d)
    assert np.abs(g - fd).max() / np.abs(fd).max() <= TOL


def test_full_adjoint_64_cube(gfem, orc):
    """64^3 Kuhn cube with 5% slivers (1,572,864 tets), lognormal coefficient,
    dA ~ N(0,1): the whole gradient against the oracle, both reductions."""
    mesh = mg.workload_tet_slivers(64, k=4)
    coef = mg.lognormal_coef(mg.rng_for(50), mesh.n_elem)
    dA = mg.upstream(mg.rng_for(51), mesh.n_elem, 4)
    gx, gw = orc.integrate_vjp(3, LP1, mesh.conn, mesh.coords, dA, coef)
    coords, conn = _t(mesh.coords), _t(mesh.conn)
    ws = gfem.Workspace(coords, conn)
    for reduce in (0, 1):
        dx, dw = gfem.integrate_bwd(coords, conn, LP1, _t(dA), _t(coef), ws=ws, reduce=reduce)
        assert _rel(dx.cpu().numpy(), gx) <= TOL
        assert _rel(dw.cpu().numpy(), gw) <= TOL


@pytest.mark.parametrize("dim,form", [(3, LP1), (3, EP1), (2, LP1), (3, LP2)])
def test_saved_det_is_bitwise_the_same(gfem, dim, form):
    """fem_integrate_fwd_save returns the same A plus det J; the adjoint with
    that det (fem_integrate_bwd_saved) equals fem_integrate_bwd bit for bit
    (dcoef always; dcoords with the deterministic reduction, and to rounding
    with the atomic one, whose order varies from run to run), and det J is
    the compensated determinant of the geometry hook (its double-float value)
    to within one FP32 rounding."""
    mesh = _mesh(dim)
    n = {LP1: dim + 1, LP2: (dim + 1) * (dim + 2) // 2, EP1: dim * (dim + 1)}[form]
    coef = _t(mg.lognormal_coef(mg.rng_for(61), mesh.n_elem))
    dA = _t(mg.upstream(mg.rng_for(62), mesh.n_elem, n))
    coords, conn = _t(mesh.coords), _t(mesh.conn)
    det = torch.empty(mesh.n_elem, device="cuda")
    A0 = gfem.integrate_fwd(coords, conn, form, coef)
    A1 = gfem.integrate_fwd(coords, conn, form, coef, det_out=det)
    assert torch.equal(A0, A1)
    dref, _ = gfem.geometry(coords, conn)
    assert torch.all((det.double() - dref).abs() <= 2.0 ** -23 * dref.abs())
    ws = gfem.Workspace(coords, conn)
    for reduce in (0, 1):
        a = gfem.integrate_bwd(coords, conn, form, dA, coef, ws=ws, reduce=reduce)
        b = gfem.integrate_bwd(coords, conn, form, dA, coef, ws=ws, reduce=reduce, det=det)
        assert torch.equal(a[1], b[1])
        if reduce == 0:
            assert torch.equal(a[0], b[0])
        else:
            assert _rel(b[0].cpu().numpy(), a[0].cpu().numpy().astype(np.float64)) <= 1e-6
    with pytest.raises(ValueError):
        gfem.integrate_bwd(coords, conn, form, dA, coef, det=det[:-1])


@pytest.mark.parametrize("reduce", [0, 1])
def test_adjoint_device_errors(gfem, orc, reduce):
    """An element with an out-of-range vertex (FEM_DEVERR_CONN) and one with a
    repeated vertex (det J = 0, FEM_DEVERR_DEGENERATE) contribute nothing:
    dcoef is 0 there, and dcoords equals the oracle's reverse mode over the
    other elements, for both reductions."""
    mesh = _mesh(3)
    conn = mesh.conn.copy()
    conn[5, 2] = mesh.n_vert + 3
    conn[9, 1] = conn[9, 0]
    coef = mg.lognormal_coef(mg.rng_for(63), mesh.n_elem)
    dA = mg.upstream(mg.rng_for(64), mesh.n_elem, 4)
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    dx, dw = gfem.integrate_bwd(_t(mesh.coords), _t(conn), LP1, _t(dA), _t(coef), reduce=reduce, dev_err=err)
    assert int(err.item()) == gfem.DEVERR_CONN | gfem.DEVERR_DEGENERATE
    keep = np.setdiff1d(np.arange(mesh.n_elem), [5, 9])
    gx, gw = orc.integrate_vjp(3, LP1, mesh.conn[keep], mesh.coords, dA[keep], coef[keep])
    assert _rel(dx.cpu().numpy(), gx) <= TOL
    dwh = dw.cpu().numpy()
    assert dwh[5] == 0 and dwh[9] == 0 and _rel(dwh[keep], gw) <= TOL


@pytest.mark.parametrize("dim,form,out", [(2, 3, torch.float32), (3, 4, torch.float32), (3, LP1, torch.float64),
                                          (2, LP2, torch.float32)])
def test_fwd_save_other_paths(gfem, dim, form, out):
    """det J is written by every forward path fem_integrate_fwd_save serves (the
    P1-coefficient forms, FP64 output, triangles) and A is unchanged."""
    mesh = _mesh(dim)
    coords, conn = _t(mesh.coords), _t(mesh.conn)
    w1 = form in (3, 4)
    coef = _t(mg.lognormal_coef(mg.rng_for(65), mesh.n_vert if w1 else mesh.n_elem))
    det = torch.full((mesh.n_elem,), float("nan"), device="cuda")
    A0 = gfem.integrate_fwd(coords, conn, form, coef, out_dtype=out)
    A1 = gfem.integrate_fwd(coords, conn, form, coef, out_dtype=out, det_out=det)
    assert torch.equal(A0, A1)
    jac = gfem.JAC_F64 if out == torch.float64 else gfem.JAC_AUTO
    dref, _ = gfem.geometry(coords, conn, jac=jac)
    assert torch.all((det.double() - dref).abs() <= 2.0 ** -23 * dref.abs())


def test_full_size_step_sampled(gfem, orc):
    """The benchmark step at full size: 128^3 Kuhn cube with 5% slivers
    (12,582,912 tets), forward saving det J, deterministic adjoint with it, in
    the bench's launch configuration.  dcoords is checked at a random sample of
    vertices, each against the oracle's reverse mode over all of its incident
    elements; A on a stratified element sample."""
    mesh = mg.workload_tet_slivers(128)
    E, V = mesh.n_elem, mesh.n_vert
    dA_h = mg.upstream(mg.rng_for(66), E, 4)
    coords, conn, dA = _t(mesh.coords), _t(mesh.conn), _t(dA_h)
    det = torch.empty(E, device="cuda")
    A = gfem.integrate_fwd(coords, conn, LP1, det_out=det)
    ws = gfem.Workspace(coords, conn)
    dx, _ = gfem.integrate_bwd(coords, conn, LP1, dA, ws=ws, reduce=gfem.REDUCE_DEFERRED, need_dcoef=False,
                               det=det)
    gfem.adjoint_reduce(coords, conn, ws, dx)
    torch.cuda.synchronize()
    rng = np.random.default_rng(67)
    verts = rng.choice(V, 3000, replace=False)
    hit = np.zeros(V, bool)
    hit[verts] = True
    el = np.where(hit[mesh.conn].any(1))[0]                    # every element incident to a sampled vertex
    gx, _ = orc.integrate_vjp(3, LP1, mesh.conn[el], mesh.coords, dA_h[el])
    got = dx.cpu().numpy()[verts].astype(np.float64)
    ref = gx[verts]
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() <= TOL * scale
    idx = np.unique(np.concatenate([rng.choice(np.where(mesh.sliver)[0], 5000, replace=False),
                                    rng.choice(E, 5000, replace=False), np.arange(E - 40, E)]))
    Ar, _ = orc.integrate(3, LP1, mesh.conn[idx], mesh.coords)
    Ag = A[torch.from_numpy(idx).to("cuda")].double().cpu().numpy()
    assert (np.abs(Ag - Ar).reshape(len(idx), -1).max(1) / np.abs(Ar).reshape(len(idx), -1).max(1)).max() <= TOL
