"""GPU parity of the non-affine adjoint (fem_integrate_bwd_iso, Eqs. 16-19)
against the FP64 oracle's reverse mode (-m gpu).

The gradients of L = sum dA : A with respect to the vertices (dcoords, summed
over the elements at each vertex), the edge nodes (dmid, per element) and the
per-element coefficient are compared element by element and vertex by vertex:
  dcoords: per vertex, |g - g_ref| <= TOL * (the largest node gradient of the
           elements at the vertex, edge nodes included).  A vertex's gradient
           combines its elements' Jacobian adjoints with coefficients that sum
           to zero; on nearly straight elements those adjoints are nearly
           equal, so the P1 vertex gradients come out about 400 times smaller
           than the edge-node gradients formed from the same FP32 terms, and
           the FP32 bound scales with the terms, not with their difference
  dmid:    max |dmid - dmid_ref| over an element <= TOL * max over the mesh of |dmid_ref|
  dcoef:   per element, |dw - dw_ref| <= TOL * sum_ij |dA_ij| |A_ij| / w, the
           error bound of dw = (dA : A) / w when every entry of A carries a
           relative error up to TOL (the sum cancels: |dw| itself can be far
           smaller than that scale)
TOL = 1e-5 (the forward's per-element bound, on curved non-sliver elements
whose Jacobian steps run in FP32).  The deterministic reduction is bitwise
reproducible and equals the deferred one; the atomic one agrees within TOL;
autograd returns the same bits; straight-sided elements reduce to the affine
adjoint; degenerate and invalid elements contribute zeros and set the error
bits."""
import numpy as np
import pytest
import torch

from paper_1103_0066_gb300 import meshgen as mg

pytestmark = pytest.mark.gpu
LP1, LP2, ISO1, ISO2 = 0, 1, 5, 6
DEV = "cuda:0"
TOL = 1e-5


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _curved(dim, eps=0.05, seed=51, n=None):
    base = (mg.square_tri_mesh(n or 13, 0.2, mg.rng_for(seed), np.float32) if dim == 2
            else mg.cube_tet_mesh(n or 6, 0.15, mg.rng_for(seed), 0.0, np.float32))
    return mg.curved_mesh(base, eps)


def node_scale(conn, rx, rm):
    """Per vertex: the largest node gradient (edge nodes, and the vertex's own
    sum) over the elements at the vertex."""
    s_e = np.abs(rm).reshape(len(rm), -1).max(1)
    scale = np.abs(rx).max(1)
    ok = (conn >= 0) & (conn < len(rx))
    np.maximum.at(scale, conn[ok], np.repeat(s_e[:, None], conn.shape[1], 1)[ok])
    return scale


def _errs(got, ref, A_ref=None, dA=None, coef=None, conn=None):
    dx, dm, dw = (None if g is None else g.cpu().numpy().astype(np.float64) for g in got)
    rx, rm, rw = ref
    out = {}
    if dx is not None:
        scale = node_scale(conn, rx, rm)
        out["dcoords"] = (np.abs(dx - rx).max(1) / np.where(scale > 0, scale, 1.0)).max()
    if dm is not None:
        out["dmid"] = np.abs(dm - rm).max() / np.abs(rm).max()
    if dw is not None:
        w = np.ones(len(rw)) if coef is None else np.asarray(coef, np.float64)
        scale = (np.abs(dA.astype(np.float64)) * np.abs(A_ref)).reshape(len(rw), -1).sum(1) / w
        out["dcoef"] = (np.abs(dw - rw) / np.where(scale > 0, scale, 1.0)).max()
    return out


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("form", [ISO1, ISO2])
def test_iso_adjoint_matches_oracle(gfem, orc, dim, form):
    mesh, mid = _curved(dim)
    E = mesh.n_elem
    n = gfem.form_info(form, dim)[0]
    coef = mg.lognormal_coef(mg.rng_for(52), E)
    dA = np.random.default_rng(53).standard_normal((E, n, n)).astype(np.float32)
    got = gfem.integrate_bwd_iso(_t(mesh.coords), _t(mesh.conn), _t(mid), form, _t(dA), _t(coef), need_dcoef=True)
    ref = orc.integrate_iso_vjp(dim, form - 5, mesh.conn, mesh.coords, mid, dA, coef)
    A_ref, _ = orc.integrate_iso(dim, form - 5, mesh.conn, mesh.coords, mid, coef)
    errs = _errs(got, ref, A_ref, dA, coef, mesh.conn)
    assert max(errs.values()) <= TOL, errs


@pytest.mark.parametrize("form", [ISO1, ISO2])
def test_iso_adjoint_reductions(gfem, orc, form):
    mesh, mid = _curved(3, seed=54)
    E = mesh.n_elem
    n = gfem.form_info(form, 3)[0]
    coords, conn, m = _t(mesh.coords), _t(mesh.conn), _t(mid)
    dA = _t(np.random.default_rng(55).standard_normal((E, n, n)).astype(np.float32))
    ws = gfem.Workspace(coords, conn, form)
    a, am, _ = gfem.integrate_bwd_iso(coords, conn, m, form, dA, ws=ws)
    b, bm, _ = gfem.integrate_bwd_iso(coords, conn, m, form, dA, ws=ws)
    assert torch.equal(a, b) and torch.equal(am, bm)                      # reproducible bits
    d = torch.empty_like(a)
    gfem.integrate_bwd_iso(coords, conn, m, form, dA, ws=ws, reduce=gfem.REDUCE_DEFERRED, dcoords=d,
                           need_dmid=False)
    gfem.adjoint_reduce(coords, conn, ws, d)
    assert torch.equal(a, d)                                              # deferred = deterministic
    c, cm, _ = gfem.integrate_bwd_iso(coords, conn, m, form, dA, reduce=gfem.REDUCE_ATOMIC)
    assert torch.equal(cm, am)
    assert float((c - a).abs().max()) <= TOL * float(a.abs().max())      # atomic: another summation order
    # outputs asked for separately give the same bits
    only_m = gfem.integrate_bwd_iso(coords, conn, m, form, dA, need_dcoords=False)[1]
    assert torch.equal(only_m, am)


@pytest.mark.parametrize("dim", [2, 3])
def test_iso_autograd(gfem, dim):
    mesh, mid = _curved(dim, seed=56)
    E = mesh.n_elem
    coef = _t(mg.lognormal_coef(mg.rng_for(57), E))
    x = _t(mesh.coords).requires_grad_()
    m = _t(mid).requires_grad_()
    w = coef.clone().requires_grad_()
    conn = _t(mesh.conn)
    A = gfem.integrate_iso(x, conn, m, ISO2, w)
    W = torch.randn_like(A)
    (A * W).sum().backward()
    dx, dm, dw = gfem.integrate_bwd_iso(x.detach(), conn, m.detach(), ISO2, W, coef, need_dcoef=True)
    assert torch.equal(x.grad, dx) and torch.equal(m.grad, dm) and torch.equal(w.grad, dw)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("form", [ISO1, ISO2])
def test_iso_adjoint_straight_sides_reduce_to_affine(gfem, dim, form):
    """mid at the edge midpoints: dx_affine = dx_iso + (1/2) sum over the edges at v of dmid."""
    mesh, _ = _curved(dim, eps=0.0, seed=58)
    E, V = mesh.n_elem, mesh.n_vert
    pairs = mg.edge_pairs(dim)
    mid = np.stack([0.5 * (mesh.coords[mesh.conn[:, a]] + mesh.coords[mesh.conn[:, b]]) for a, b in pairs],
                   axis=1).astype(np.float32)
    n = gfem.form_info(form, dim)[0]
    dA = np.random.default_rng(59).standard_normal((E, n, n)).astype(np.float32)
    coords, conn = _t(mesh.coords), _t(mesh.conn)
    dx, dm, _ = gfem.integrate_bwd_iso(coords, conn, _t(mid), form, _t(dA))
    dxa, _ = gfem.integrate_bwd(coords, conn, form - 5, _t(dA), need_dcoef=False)
    moved = dx.cpu().numpy().astype(np.float64)
    dmn = dm.cpu().numpy().astype(np.float64)
    for q, (a, b) in enumerate(pairs):
        np.add.at(moved, mesh.conn[:, a], 0.5 * dmn[:, q])
        np.add.at(moved, mesh.conn[:, b], 0.5 * dmn[:, q])
    ref = dxa.cpu().numpy().astype(np.float64)
    # the sum combines edge-node gradients far larger than the vertex ones (see above)
    assert np.abs(moved - ref).max() <= TOL * max(np.abs(ref).max(), np.abs(dmn).max())


@pytest.mark.parametrize("E", [1, 31, 33, 257])
def test_iso_adjoint_ragged_tails_and_flags(gfem, orc, E):
    mesh, mid = _curved(3, seed=60)
    conn = mesh.conn[:E].copy()
    m = mid[:E].copy()
    if E > 5:
        conn[5, 1] = mesh.n_vert + 7                                     # invalid vertex
    if E > 9:
        conn[9, :] = conn[9, 0]                                          # every node on one point:
        m[9] = mesh.coords[conn[9, 0]]                                   # J = 0 everywhere
    n = 10
    dA = np.random.default_rng(61).standard_normal((E, n, n)).astype(np.float32)
    err = torch.zeros(1, dtype=torch.int32, device=DEV)
    got = gfem.integrate_bwd_iso(_t(mesh.coords), _t(conn), _t(m), ISO2, _t(dA), need_dcoef=True, dev_err=err)
    ref = orc.integrate_iso_vjp(3, LP2, conn, mesh.coords, m, dA)
    A_ref, fl = orc.integrate_iso(3, LP2, conn, mesh.coords, m)
    errs = _errs(got, ref, A_ref, dA, conn=conn)
    assert max(errs.values()) <= TOL, errs
    if E > 5:
        assert fl[5] == 1 and int(err.item()) & 1
        assert torch.all(got[1][5] == 0) and float(got[2][5]) == 0.0
    if E > 9:
        assert fl[9] == 2 and int(err.item()) & 2 and torch.all(got[1][9] == 0)


def test_iso_adjoint_argument_errors(gfem):
    mesh, mid = _curved(2)
    coords, conn, m = _t(mesh.coords), _t(mesh.conn), _t(mid)
    dA = torch.zeros((mesh.n_elem, 3, 3), device=DEV)
    with pytest.raises(gfem.FemError):
        gfem.integrate_bwd(coords, conn, ISO1, dA)                        # the iso entry point serves them
    with pytest.raises(gfem.FemError):
        gfem.integrate_bwd_iso(coords, conn, m, LP1, dA)                   # not a non-affine form
    with pytest.raises(ValueError):
        gfem.integrate_bwd_iso(coords, conn, m[:, :2].contiguous(), ISO1, dA)


def test_iso_adjoint_full_size_sample(gfem, orc):
    """The warped 96^3 cube (5.3M curved tets): dmid and dcoef on a stratified
    sample of elements, dcoords on vertices whose incident elements are all
    evaluated by the oracle."""
    mesh, mid = mg.workload_curved_tets(96)
    E, V = mesh.n_elem, mesh.n_vert
    rng = np.random.default_rng(62)
    dA = mg.upstream(mg.rng_for(63), E, 10)
    coords, conn = _t(mesh.coords), _t(mesh.conn)
    dx, dm, dw = gfem.integrate_bwd_iso(coords, conn, _t(mid), ISO2, _t(dA), need_dcoef=True)
    torch.cuda.synchronize()
    verts = rng.choice(V, 40, replace=False)
    inc = np.isin(mesh.conn, verts).any(1)
    els = np.unique(np.concatenate([np.flatnonzero(inc), rng.choice(E, 2000, replace=False), [0, E - 1]]))
    sub_conn = mesh.conn[els]
    rx, rm, rw = orc.integrate_iso_vjp(3, LP2, sub_conn, mesh.coords, mid[els], dA[els], np.ones(len(els)))
    dmn = dm[_t(els.astype(np.int64))].cpu().numpy()
    dwn = dw[_t(els.astype(np.int64))].cpu().numpy()
    A_ref, _ = orc.integrate_iso(3, LP2, sub_conn, mesh.coords, mid[els])
    assert np.abs(dmn - rm).max() <= TOL * np.abs(rm).max()
    scale = (np.abs(dA[els].astype(np.float64)) * np.abs(A_ref)).reshape(len(els), -1).sum(1)
    assert (np.abs(dwn - rw) / scale).max() <= TOL
    gx = dx.cpu().numpy()[verts]
    scale = node_scale(sub_conn, rx, rm)[verts]
    assert (np.abs(gx - rx[verts]).max(1) / scale).max() <= TOL


@pytest.mark.parametrize("E", [None, 1, 129, 300])
def test_iso_adjoint_tensor_cores(gfem, orc, E):
    """The curved P2 adjoint with its contraction on the tensor cores (sym(dA)
    split into three BF16 terms, K' exact in BF16, FP32 accumulation): the same
    tolerances against the oracle's reverse mode, over ragged 128-element CTA
    tiles, an invalid vertex and a degenerate element flagged and zeroed;
    reproducible bits, deferred = deterministic, and within the tolerance of
    the FP32 adjoint."""
    mesh, mid = _curved(3, seed=64, n=7)
    conn, m = mesh.conn, mid
    if E is not None:
        conn, m = conn[:E].copy(), mid[:E].copy()
        if E > 5:
            conn[5, 1] = mesh.n_vert + 7
        if E > 9:
            conn[9, :] = conn[9, 0]
            m[9] = mesh.coords[conn[9, 0]]
    n_e = conn.shape[0]
    coef = mg.lognormal_coef(mg.rng_for(65), n_e)
    dA = np.random.default_rng(66).standard_normal((n_e, 10, 10)).astype(np.float32)
    coords, conn_t, m_t = _t(mesh.coords), _t(conn), _t(m)
    err = torch.zeros(1, dtype=torch.int32, device=DEV)
    ws = gfem.Workspace(coords, conn_t, ISO2)
    got = gfem.integrate_bwd_iso(coords, conn_t, m_t, ISO2, _t(dA), _t(coef), ws=ws, need_dcoef=True, dev_err=err,
                                 contract=gfem.CONTRACT_BF16X3)
    ref = orc.integrate_iso_vjp(3, LP2, conn, mesh.coords, m, dA, coef)
    A_ref, fl = orc.integrate_iso(3, LP2, conn, mesh.coords, m, coef)
    errs = _errs(got, ref, A_ref, dA, coef, conn)
    assert max(errs.values()) <= TOL, errs
    assert int(err.item()) == (int(np.bitwise_or.reduce(fl)) if fl.any() else 0)
    if E is not None and E > 5:
        assert torch.all(got[1][5] == 0) and float(got[2][5]) == 0.0
    again = gfem.integrate_bwd_iso(coords, conn_t, m_t, ISO2, _t(dA), _t(coef), ws=ws, need_dcoef=True,
                                   contract=gfem.CONTRACT_BF16X3)
    assert all(torch.equal(a, b) for a, b in zip(got, again))
    d = torch.empty_like(got[0])
    gfem.integrate_bwd_iso(coords, conn_t, m_t, ISO2, _t(dA), _t(coef), ws=ws, reduce=gfem.REDUCE_DEFERRED,
                           dcoords=d, need_dmid=False, contract=gfem.CONTRACT_BF16X3)
    gfem.adjoint_reduce(coords, conn_t, ws, d)
    assert torch.equal(d, got[0])
    f32 = gfem.integrate_bwd_iso(coords, conn_t, m_t, ISO2, _t(dA), _t(coef), ws=ws, need_dcoef=True)
    assert float((got[1] - f32[1]).abs().max()) <= TOL * float(f32[1].abs().max())


def test_iso_adjoint_tensor_core_refusals(gfem):
    from paper_1103_0066_gb300 import _native as nat
    for dim, form, reduce in ((2, ISO2, gfem.REDUCE_DETERMINISTIC), (3, ISO1, gfem.REDUCE_DETERMINISTIC),
                              (3, ISO2, gfem.REDUCE_ATOMIC)):
        mesh, mid = _curved(dim)
        n = gfem.form_info(form, dim)[0]
        dA = torch.zeros((mesh.n_elem, n, n), device=DEV)
        with pytest.raises(nat.FemError) as ei:
            gfem.integrate_bwd_iso(_t(mesh.coords), _t(mesh.conn), _t(mid), form, dA, reduce=reduce,
                                   contract=gfem.CONTRACT_BF16X3)
        assert ei.value.status == nat.FEM_ERR_UNSUPPORTED
