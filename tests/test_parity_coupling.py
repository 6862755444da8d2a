"""GPU parity of the coupling blocks int w q div v (-m gpu).

The off-diagonal block of a multiphysics pair (Sec. 6: coupled systems broken
into blocks), B_{i,(c,j)} = int_T w phi_i d psi_j / d x_c with phi the P1
basis and psi the P1 (DIV_P1P1) or P2 (DIV_P2P1) basis of each component of a
vector field.  The CUDA path contracts G^{mu c} = w sgn(det J) adj(J)_{mu c}
with K^{ij}_mu = int_ref lambda_i d_mu psi_j as immediates; the oracle
integrates by quadrature.  Tolerances as for the square forms: 1e-5 per
element relative to max |B_e| (every element, slivers included), 1e-5 of the
largest gradient entry for the adjoint; the deterministic and batched paths
match their per-form counterparts bit for bit."""
import numpy as np
import pytest
import torch

from paper_1103_0066_gb300 import meshgen as mg
from conftest import rel_err_per_element

pytestmark = pytest.mark.gpu
TOL = 1e-5
DEV = "cuda:0"
DIV = {1: 7, 2: 8}  # vdeg -> form id


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _mesh(dim, n=None, seed=121):
    if dim == 2:
        return mg.square_tri_mesh(n or 13, 0.2, mg.rng_for(seed), np.float32)
    return mg.cube_tet_mesh(n or 7, 0.15, mg.rng_for(seed), 0.05, np.float32)


def _rel(a, b):
    return float(np.abs(np.asarray(a, np.float64) - b).max() / np.abs(b).max())


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("vdeg", [1, 2])
@pytest.mark.parametrize("shuffle", [False, True])
def test_coupling_forward_matches_oracle(gfem, orc, dim, vdeg, shuffle):
    mesh = _mesh(dim)
    if shuffle:
        mesh = mg.shuffled(mesh, mg.rng_for(122))[0]
    coef = mg.lognormal_coef(mg.rng_for(123), mesh.n_elem)
    form = DIV[vdeg]
    rows, cols = gfem.form_shape(form, dim)
    B = gfem.integrate_fwd(_t(mesh.coords), _t(mesh.conn), form, _t(coef))
    assert tuple(B.shape) == (mesh.n_elem, rows, cols) == (mesh.n_elem,) + orc.div_shape(dim, vdeg)
    Br, fl = orc.integrate_div(dim, vdeg, mesh.conn, mesh.coords, coef)
    assert not fl.any()
    err = rel_err_per_element(B.cpu().numpy(), Br)
    assert err.max() <= TOL, err.max()
    if dim == 3:
        assert err[mesh.sliver].max() <= TOL


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("vdeg", [1, 2])
def test_coupling_adjoint_matches_oracle(gfem, orc, dim, vdeg):
    """Both reductions and the saved-det adjoint against the oracle's reverse
    mode; the deterministic result is reproducible and equal with and without
    the saved det J."""
    mesh = _mesh(dim)
    form = DIV[vdeg]
    coef = mg.lognormal_coef(mg.rng_for(124), mesh.n_elem)
    rows, cols = gfem.form_shape(form, dim)
    dB = np.random.default_rng(125).standard_normal((mesh.n_elem, rows, cols)).astype(np.float32)
    coords, conn = _t(mesh.coords), _t(mesh.conn)
    gx, gw = orc.integrate_div_vjp(dim, vdeg, mesh.conn, mesh.coords, dB, coef)
    ws = gfem.Workspace(coords, conn, form)
    det = torch.empty(mesh.n_elem, device=DEV)
    B0 = gfem.integrate_fwd(coords, conn, form, _t(coef))
    B1 = gfem.integrate_fwd(coords, conn, form, _t(coef), det_out=det)
    assert torch.equal(B0, B1)
    ref = None
    for reduce in (0, 1):
        dx, dw = gfem.integrate_bwd(coords, conn, form, _t(dB), _t(coef), ws=ws, reduce=reduce)
        assert _rel(dx.cpu().numpy(), gx) <= TOL, reduce
        assert _rel(dw.cpu().numpy(), gw) <= TOL, reduce
        sx, sw = gfem.integrate_bwd(coords, conn, form, _t(dB), _t(coef), ws=ws, reduce=reduce, det=det)
        assert torch.equal(sw, dw)
        if reduce == 0:
            assert torch.equal(sx, dx)
            ref = dx
    again, _ = gfem.integrate_bwd(coords, conn, form, _t(dB), _t(coef), ws=gfem.Workspace(coords, conn))
    assert torch.equal(again, ref)


def test_coupling_adjoint_against_fp64_finite_differences(gfem, orc):
    """4^3 cube with slivers, Taylor-Hood block: the GPU coordinate gradient
    against FP64 central differences of the oracle's forward."""
    mesh = mg.cube_tet_mesh(4, 0.15, mg.rng_for(126), 0.05, np.float32)
    X = mesh.coords.astype(np.float64)
    dB = np.random.default_rng(127).standard_normal((mesh.n_elem, 4, 30))
    dx, _ = gfem.integrate_bwd(_t(mesh.coords), _t(mesh.conn), 8, _t(dB.astype(np.float32)), need_dcoef=False)
    g = dx.cpu().numpy().astype(np.float64)
    fd = np.zeros_like(X)
    for v in range(X.shape[0]):
        inc = np.where((mesh.conn == v).any(1))[0]
        if inc.size == 0:
            continue
        h = 1e-6 * np.abs(X).max()
        for a in range(3):
            Xp, Xm = X.copy(), X.copy()
            Xp[v, a] += h
            Xm[v, a] -= h
            Bp, _ = orc.integrate_div(3, 2, mesh.conn[inc], Xp)
            Bm, _ = orc.integrate_div(3, 2, mesh.conn[inc], Xm)
            fd[v, a] = (np.sum(dB[inc] * Bp) - np.sum(dB[inc] * Bm)) / (2 * h)
    assert np.abs(g - fd).max() <= TOL * np.abs(fd).max()


def test_coupling_autograd(gfem, orc):
    mesh = _mesh(3)
    coef0 = mg.lognormal_coef(mg.rng_for(128), mesh.n_elem)
    dB = np.random.default_rng(129).standard_normal((mesh.n_elem, 4, 12)).astype(np.float32)
    x = _t(mesh.coords).requires_grad_(True)
    w = _t(coef0).requires_grad_(True)
    B = gfem.Mesh(x, _t(mesh.conn)).integrate(gfem.DIV_P1P1, w)
    (B * _t(dB)).sum().backward()
    gx, gw = orc.integrate_div_vjp(3, 1, mesh.conn, mesh.coords, dB, coef0)
    assert _rel(x.grad.cpu().numpy(), gx) <= TOL and _rel(w.grad.cpu().numpy(), gw) <= TOL


def test_coupling_device_errors_and_refusals(gfem, orc):
    mesh = _mesh(3)
    conn = mesh.conn.copy()
    conn[5, 2] = mesh.n_vert + 3
    conn[9, 1] = conn[9, 0]
    err = torch.zeros(1, dtype=torch.int32, device=DEV)
    B = gfem.integrate_fwd(_t(mesh.coords), _t(conn), 8, dev_err=err).cpu().numpy()
    assert int(err.item()) == gfem.DEVERR_CONN | gfem.DEVERR_DEGENERATE
    assert not B[5].any() and not B[9].any()
    keep = np.setdiff1d(np.arange(mesh.n_elem), [5, 9])
    Br, _ = orc.integrate_div(3, 2, mesh.conn[keep], mesh.coords)
    assert rel_err_per_element(B[keep], Br).max() <= TOL
    with pytest.raises(gfem.FemError):  # FP64 output is not served
        gfem.integrate_fwd(_t(mesh.coords), _t(mesh.conn), 7, out_dtype=torch.float64)
    with pytest.raises(gfem.FemError):  # nor the tensor-core contraction
        gfem.integrate_fwd(_t(mesh.coords), _t(mesh.conn), 7, contract=gfem.CONTRACT_BF16X3)


def test_coupling_in_the_multiphysics_batch(gfem):
    """The blocks of a thermo-elastic pair on one mesh in one batch: P1
    elasticity (displacement), the P1 Laplacian (temperature) and the coupling
    block int T div v -- plus the P2 Laplacian and a Taylor-Hood block.  The
    batch runs the per-item modes (the persistent kernels serve the square
    kinds and refuse it); every block equals its per-form call bit for bit."""
    mesh = mg.cube_tet_mesh(6, 0.15, mg.rng_for(130), 0.05, np.float32)
    coords, conn = _t(mesh.coords), _t(mesh.conn)
    coef = _t(mg.lognormal_coef(mg.rng_for(131), mesh.n_elem))
    items = []
    for k, form in enumerate((2, 0, 7, 1, 8)):
        rows, cols = gfem.form_shape(form, 3)
        items.append({"coords": coords, "conn": conn, "form": form, "coef": coef,
                      "A": torch.full((mesh.n_elem, rows, cols), float("nan"), device=DEV),
                      "dA": _t(np.random.default_rng(132 + k).standard_normal((mesh.n_elem, rows, cols))
                               .astype(np.float32)),
                      "dcoords": torch.empty((mesh.n_vert, 3), device=DEV),
                      "dcoef": torch.empty(mesh.n_elem, device=DEV)})
    batch = gfem.Batch(items)
    assert batch.config()[2] in (gfem.BATCH_PER_ITEM, gfem.BATCH_PER_ITEM_CONCURRENT)
    with pytest.raises(gfem.FemError):
        batch.set_config(2, 1, gfem.BATCH_SINGLE)
    for mode in (gfem.BATCH_PER_ITEM, gfem.BATCH_PER_ITEM_CONCURRENT):
        batch.set_config(1, 1, mode)
        batch.run()
        torch.cuda.synchronize()
        assert batch.errors() == 0
        for it in items:
            A_ref = gfem.integrate_fwd(coords, conn, it["form"], coef)
            dx_ref, dw_ref = gfem.integrate_bwd(coords, conn, it["form"], it["dA"], coef)
            assert torch.equal(it["A"], A_ref) and torch.equal(it["dcoords"], dx_ref)
            assert torch.equal(it["dcoef"], dw_ref)
    assert batch.tune()[2] in (gfem.BATCH_PER_ITEM, gfem.BATCH_PER_ITEM_CONCURRENT)


def test_coupling_full_size_sampled(gfem, orc):
    """The Taylor-Hood block on the 128^3 sliver cube (12,582,912 tets, 4 x 30
    FP32 blocks, 6 GB) in the bench's launch configuration: a stratified
    element sample against the oracle, and the patch identity at any size --
    for the linear field v = x, every row sums B applied to the nodal values
    to d * int_T phi_i = d |T| / (d+1)."""
    mesh = mg.workload_tet_slivers(128)
    E = mesh.n_elem
    coords, conn = _t(mesh.coords), _t(mesh.conn)
    B = gfem.integrate_fwd(coords, conn, 8)
    rng = np.random.default_rng(133)
    idx = np.unique(np.concatenate([rng.choice(np.where(mesh.sliver)[0], 4000, replace=False),
                                    rng.choice(E, 4000, replace=False), np.arange(E - 40, E)]))
    Br, _ = orc.integrate_div(3, 2, mesh.conn[idx], mesh.coords)
    Bg = B[torch.from_numpy(idx).to(DEV)].double().cpu().numpy()
    assert rel_err_per_element(Bg, Br).max() <= TOL
    # patch identity on every element: nodal values of v = x (P2 nodes: vertices, then edge midpoints)
    P = coords[conn.long()]                                           # [E][4][3]
    mids = [0.5 * (P[:, a] + P[:, b]) for a in range(4) for b in range(a + 1, 4)]
    nodes = torch.cat([P, torch.stack(mids, 1)], 1)                   # [E][10][3]
    u = nodes.transpose(1, 2).reshape(E, 30)                          # component-major
    Bu = torch.bmm(B, u.unsqueeze(2)).squeeze(2)                      # [E][4]
    vol = torch.linalg.det((P[:, 1:] - P[:, :1]).double()).abs() / 6
    expect = (3 * vol / 4).unsqueeze(1)
    scale = B.abs().amax((1, 2)).double() * nodes.abs().amax((1, 2)).double()
    assert float(((Bu.double() - expect).abs().amax(1) / scale).max()) < 1e-5
