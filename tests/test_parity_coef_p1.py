"""GPU parity of the Laplacian with a P1 coefficient (Eqs. 20-23) against the
FP64 oracle (-m gpu).  The coefficient is given by its vertex values; the
library contracts w_k G^{mu nu} with the arity-3 reference tensor.

Tolerance as for the other forms: per element, every element, slivers
included, max_ij |A_gpu - A_ref| <= tol * max_ij |A_ref| with tol = 1e-5 for
FP32 output and 1e-12 for the FP64 path."""
import numpy as np
import pytest
import torch

from paper_1103_0066_gb300 import meshgen as mg
from conftest import rel_err_per_element

pytestmark = pytest.mark.gpu
LP1, LP2, LP1W, LP2W = 0, 1, 3, 4
TOL32, TOL64 = 1e-5, 1e-12
DEV = "cuda:0"


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _mesh(dim, seed=31):
    if dim == 2:
        return mg.square_tri_mesh(13, 0.2, mg.rng_for(seed), np.float32)
    return mg.cube_tet_mesh(7, 0.15, mg.rng_for(seed), 0.05, np.float32)


def _wvert(n, seed=32):
    return mg.lognormal_coef(mg.rng_for(seed), n)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("form", [LP1W, LP2W])
@pytest.mark.parametrize("jac", [0, 1])
def test_coef_p1_matches_oracle(gfem, orc, dim, form, jac):
    mesh = _mesh(dim)
    w = _wvert(mesh.n_vert)
    A = gfem.integrate_fwd(_t(mesh.coords), _t(mesh.conn), form, _t(w), jac=jac)
    torch.cuda.synchronize()
    Ar, fl = orc.integrate_w1(dim, form - 3, mesh.conn, mesh.coords, w)
    assert not fl.any()
    err = rel_err_per_element(A.cpu().numpy(), Ar)
    assert err.max() <= TOL32, (err.max(), int(err.argmax()))
    if dim == 3:
        assert err[mesh.sliver].max() <= TOL32


def test_coef_p1_fp64_path(gfem, orc):
    mesh = mg.workload_tri_p1_fp64()
    w = _wvert(mesh.n_vert, 33).astype(np.float32)
    for form in (LP1W, LP2W):
        A = gfem.integrate_fwd(_t(mesh.coords), _t(mesh.conn), form, _t(w), out_dtype=torch.float64)
        Ar, _ = orc.integrate_w1(2, form - 3, mesh.conn, mesh.coords, w)
        assert rel_err_per_element(A.cpu().numpy(), Ar).max() <= TOL64


@pytest.mark.parametrize("E", [1, 31, 33, 1000])
def test_coef_p1_ragged_and_reductions(gfem, orc, E):
    """Ragged element counts; constant vertex values equal the per-element
    coefficient path, and the P1 form equals it with the vertex mean."""
    full = mg.cube_tet_mesh(6, 0.15, mg.rng_for(34), 0.05, np.float32)
    conn = full.conn[:E]
    coords, c = _t(full.coords), _t(conn)
    w = _wvert(full.n_vert, 35)
    A = gfem.integrate_fwd(coords, c, LP2W, _t(w))
    Ar, _ = orc.integrate_w1(3, LP2, conn, full.coords, w)
    assert rel_err_per_element(A.cpu().numpy(), Ar).max() <= TOL32
    const = np.full(full.n_vert, 1.7, np.float32)
    A1 = gfem.integrate_fwd(coords, c, LP2W, _t(const))
    A0 = gfem.integrate_fwd(coords, c, LP2, _t(np.full(E, 1.7, np.float32)))
    assert rel_err_per_element(A1.cpu().numpy(), A0.cpu().numpy().astype(np.float64)).max() <= 1e-6
    mean = w[conn].mean(1).astype(np.float32)
    B1 = gfem.integrate_fwd(coords, c, LP1W, _t(w))
    B0 = gfem.integrate_fwd(coords, c, LP1, _t(mean))
    assert rel_err_per_element(B1.cpu().numpy(), B0.cpu().numpy().astype(np.float64)).max() <= 1e-6


def test_coef_p1_bad_connectivity_and_no_coefficient(gfem, orc):
    mesh = _mesh(3)
    conn = mesh.conn.copy()
    conn[5, 2] = mesh.n_vert + 3
    err = torch.zeros(1, dtype=torch.int32, device=DEV)
    A = gfem.integrate_fwd(_t(mesh.coords), _t(conn), LP2W, _t(_wvert(mesh.n_vert)), dev_err=err)
    assert int(err.item()) & 1 and torch.all(A[5] == 0)
    # no coefficient: w = 1, the plain P2 Laplacian
    A1 = gfem.integrate_fwd(_t(mesh.coords), _t(mesh.conn), LP2W)
    A0 = gfem.integrate_fwd(_t(mesh.coords), _t(mesh.conn), LP2)
    assert rel_err_per_element(A1.cpu().numpy(), A0.cpu().numpy().astype(np.float64)).max() <= 1e-6


@pytest.mark.parametrize("dim", [2, 3])
def test_coef_p1_tensor_cores(gfem, orc, dim):
    """P2 with a P1 coefficient contracted on the tensor cores: the arity-3 K
    times DEN is exact in BF16 and G = w_k G_g is split into three BF16 terms
    (at most 2^-24 |G| left per entry), so the FP32 tolerance holds on every
    element, slivers included."""
    mesh = _mesh(dim)
    w = _wvert(mesh.n_vert)
    err = torch.zeros(1, dtype=torch.int32, device=DEV)
    A = gfem.integrate_fwd(_t(mesh.coords), _t(mesh.conn), LP2W, _t(w), contract=gfem.CONTRACT_BF16X3,
                           dev_err=err)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    Ar, fl = orc.integrate_w1(dim, LP2, mesh.conn, mesh.coords, w)
    assert not fl.any()
    e = rel_err_per_element(A.cpu().numpy(), Ar)
    assert e.max() <= TOL32, (e.max(), int(e.argmax()))
    if dim == 3:
        assert e[mesh.sliver].max() <= TOL32


@pytest.mark.parametrize("E", [1, 127, 129, 1000])
def test_coef_p1_tensor_cores_ragged_and_no_coefficient(gfem, orc, E):
    mesh = _mesh(3, seed=35)
    conn = mesh.conn[:E]
    w = _wvert(mesh.n_vert, 36)
    Ar, _ = orc.integrate_w1(3, LP2, conn, mesh.coords, w)
    A = gfem.integrate_fwd(_t(mesh.coords), _t(conn), LP2W, _t(w), contract=gfem.CONTRACT_BF16X3)
    assert rel_err_per_element(A.cpu().numpy(), Ar).max() <= TOL32
    # no coefficient: w = 1, the P2 Laplacian
    Ar1, _ = orc.integrate(3, LP2, conn, mesh.coords)
    A1 = gfem.integrate_fwd(_t(mesh.coords), _t(conn), LP2W, None, contract=gfem.CONTRACT_BF16X3)
    assert rel_err_per_element(A1.cpu().numpy(), Ar1).max() <= TOL32


def test_coef_p1_unsupported_paths(gfem):
    mesh = _mesh(3)
    coords, conn = _t(mesh.coords), _t(mesh.conn)
    w = _t(_wvert(mesh.n_vert))
    with pytest.raises(gfem.FemError):  # no batched path for the P1-coefficient forms
        gfem.Batch([{"coords": coords, "conn": conn, "form": LP2W,
                     "A": torch.empty(mesh.n_elem, 10, 10, device=DEV)}])
    with pytest.raises(gfem.FemError):
        gfem.integrate_fwd(coords, conn, LP1W, w, contract=gfem.CONTRACT_BF16X3)  # P1: no tensor-core path
    with pytest.raises(ValueError):
        gfem.integrate_fwd(coords, conn, LP2W, _t(np.ones(mesh.n_elem, np.float32)))  # [E], not [V]


def _rel(a, b):
    return float(np.abs(np.asarray(a, np.float64) - b).max() / np.abs(b).max())


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("form", [LP1W, LP2W])
@pytest.mark.parametrize("shuffle", [False, True])
def test_coef_p1_adjoint_matches_oracle(gfem, orc, dim, form, shuffle):
    """The adjoint of the P1-coefficient Laplacian: the coordinate gradient and
    the gradient of the coefficient's vertex values against the oracle's
    reverse mode (1e-5 of the largest entry), both reductions; the
    deterministic results are reproducible and equal with and without the
    saved det J, and a dcoef-only call gives the same dcoef bits."""
    mesh = _mesh(dim)
    if shuffle:
        mesh = mg.shuffled(mesh, mg.rng_for(33))[0]
    w = _wvert(mesh.n_vert)
    n = mg.form_n(form - 3, dim)
    dA = mg.upstream(mg.rng_for(34), mesh.n_elem, n)
    coords, conn, wt, dAt = _t(mesh.coords), _t(mesh.conn), _t(w), _t(dA)
    gx, gw = orc.integrate_w1_vjp(dim, form - 3, mesh.conn, mesh.coords, w, dA)
    ws = gfem.Workspace(coords, conn, form)
    det = torch.empty(mesh.n_elem, device=DEV)
    gfem.integrate_fwd(coords, conn, form, wt, det_out=det)
    for reduce in (0, 1):
        dx, dw = gfem.integrate_bwd(coords, conn, form, dAt, wt, ws=ws, reduce=reduce)
        assert dw.shape == (mesh.n_vert,)
        assert _rel(dx.cpu().numpy(), gx) <= TOL32, reduce
        assert _rel(dw.cpu().numpy(), gw) <= TOL32, reduce
        sx, sw = gfem.integrate_bwd(coords, conn, form, dAt, wt, ws=ws, reduce=reduce, det=det)
        if reduce == 0:
            assert torch.equal(sx, dx) and torch.equal(sw, dw)
            _, ow = gfem.integrate_bwd(coords, conn, form, dAt, wt, ws=ws, need_dcoords=False)
            assert torch.equal(ow, dw)
            again = gfem.integrate_bwd(coords, conn, form, dAt, wt, ws=gfem.Workspace(coords, conn, form))
            assert torch.equal(again[0], dx) and torch.equal(again[1], dw)


def test_coef_p1_adjoint_autograd_and_identities(gfem, orc):
    """Through the autograd function: gradients of a scalar loss with respect
    to the coordinates and the coefficient's vertex values; the coefficient
    gradient satisfies the linearity identity sum_v w_v dL/dw_v = L."""
    mesh = _mesh(3)
    w0 = _wvert(mesh.n_vert)
    dA = mg.upstream(mg.rng_for(35), mesh.n_elem, 10)
    x = _t(mesh.coords).requires_grad_(True)
    w = _t(w0).requires_grad_(True)
    A = gfem.Mesh(x, _t(mesh.conn)).integrate(LP2W, w)
    L = (A * _t(dA)).sum()
    L.backward()
    gx, gw = orc.integrate_w1_vjp(3, LP2, mesh.conn, mesh.coords, w0, dA)
    assert _rel(x.grad.cpu().numpy(), gx) <= TOL32 and _rel(w.grad.cpu().numpy(), gw) <= TOL32
    lin = float(torch.dot(w.detach().double(), w.grad.double()))
    assert abs(lin - float(L.detach())) <= 1e-5 * float((A.detach() * _t(dA)).abs().sum())


def test_coef_p1_adjoint_device_errors_and_refusals(gfem, orc):
    mesh = _mesh(3)
    conn = mesh.conn.copy()
    conn[5, 2] = mesh.n_vert + 3
    conn[9, 1] = conn[9, 0]
    w = _wvert(mesh.n_vert)
    dA = mg.upstream(mg.rng_for(36), mesh.n_elem, 4)
    err = torch.zeros(1, dtype=torch.int32, device=DEV)
    for reduce in (0, 1):
        err.zero_()
        dx, dw = gfem.integrate_bwd(_t(mesh.coords), _t(conn), LP1W, _t(dA), _t(w), reduce=reduce, dev_err=err)
        assert int(err.item()) == gfem.DEVERR_CONN | gfem.DEVERR_DEGENERATE
        keep = np.setdiff1d(np.arange(mesh.n_elem), [5, 9])
        gx, gw = orc.integrate_w1_vjp(3, LP1, mesh.conn[keep], mesh.coords, w, dA[keep])
        assert _rel(dx.cpu().numpy(), gx) <= TOL32 and _rel(dw.cpu().numpy(), gw) <= TOL32
    coords, c2 = _t(mesh.coords), _t(mesh.conn)
    with pytest.raises(gfem.FemError):
        gfem.integrate_bwd(coords, c2, LP1W, _t(dA), _t(w), jac=gfem.JAC_F64)
    with pytest.raises(gfem.FemError):
        gfem.integrate_bwd(coords, c2, LP1W, _t(dA), _t(w), reduce=gfem.REDUCE_DEFERRED)


def test_coef_p1_adjoint_full_size_sampled(gfem, orc):
    """The P2 Laplacian with a P1 coefficient on the 128^3 sliver cube
    (12,582,912 tets): the coordinate and coefficient gradients at sampled
    vertices against the oracle's reverse mode over all their incident
    elements, and the linearity identity over the whole mesh."""
    mesh = mg.workload_tet_slivers(128)
    E, V = mesh.n_elem, mesh.n_vert
    w = mg.lognormal_coef(mg.rng_for(37), V)
    coords, conn, wt = _t(mesh.coords), _t(mesh.conn), _t(w)
    dA = torch.randn((E, 10, 10), device=DEV, generator=torch.Generator(device=DEV).manual_seed(38))
    det = torch.empty(E, device=DEV)
    A = gfem.integrate_fwd(coords, conn, LP2W, wt, det_out=det)
    dx, dw = gfem.integrate_bwd(coords, conn, LP2W, dA, wt, det=det)
    torch.cuda.synchronize()
    rng = np.random.default_rng(39)
    verts = rng.choice(V, 600, replace=False)
    hit = np.zeros(V, bool)
    hit[verts] = True
    el = np.where(hit[mesh.conn].any(1))[0]
    gx, gw = orc.integrate_w1_vjp(3, LP2, mesh.conn[el], mesh.coords, w, dA[torch.from_numpy(el).to(DEV)].cpu().numpy())
    assert np.abs(dx.cpu().numpy()[verts] - gx[verts]).max() <= TOL32 * np.abs(gx[verts]).max()
    assert np.abs(dw.cpu().numpy()[verts] - gw[verts]).max() <= TOL32 * np.abs(gw[verts]).max()
    L = float((A.double() * dA.double()).sum())
    lin = float(torch.dot(wt.double(), dw.double()))
    assert abs(lin - L) <= 1e-5 * float((A.double() * dA.double()).abs().sum())
