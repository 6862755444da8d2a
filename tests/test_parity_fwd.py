"""GPU parity of the forward integration against the FP64 oracle (-m gpu).

Tolerance (per element, every element, slivers included):
max_ij |A_gpu - A_ref| <= tol * max_ij |A_ref| with tol = 1e-5 for FP32 output
and 1e-12 for the FP64 path."""
import numpy as np
import pytest
import torch

from paper_1103_0066_gb300 import meshgen as mg
from conftest import rel_err_per_element

pytestmark = pytest.mark.gpu
LP1, LP2, EP1 = 0, 1, 2
TOL32, TOL64 = 1e-5, 1e-12
DEV = "cuda:0"


def _small_mesh(dim, slivers=True, n=None, seed=21):
    if dim == 2:
        return mg.square_tri_mesh(n or 13, 0.2, mg.rng_for(seed), np.float32)   # 338 tris
    return mg.cube_tet_mesh(n or 7, 0.15, mg.rng_for(seed), 0.05 if slivers else 0.0, np.float32)  # 2058 tets


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("form", [LP1, LP2, EP1])
@pytest.mark.parametrize("jac", [0, 1])
def test_forward_matches_oracle(gfem, orc, dim, form, jac):
    mesh = _small_mesh(dim)
    coef = mg.lognormal_coef(mg.rng_for(30), mesh.n_elem)
    A = gfem.integrate_fwd(_t(mesh.coords), _t(mesh.conn), form, _t(coef), jac=jac)
    torch.cuda.synchronize()
    Ar, fl = orc.integrate(dim, form, mesh.conn, mesh.coords, coef)
    assert not fl.any()
    err = rel_err_per_element(A.cpu().numpy(), Ar)
    assert err.max() <= TOL32, (err.max(), int(err.argmax()))
    if dim == 3:
        assert mesh.sliver.any() and err[mesh.sliver].max() <= TOL32


def test_fp64_path_triangles(gfem, orc):
    """64x64 jittered square, FP64 coordinates and FP64 3x3 output."""
    mesh = mg.workload_tri_p1_fp64()
    A = gfem.integrate_fwd(_t(mesh.coords), _t(mesh.conn), LP1, out_dtype=torch.float64)
    Ar, fl = orc.integrate(2, LP1, mesh.conn, mesh.coords)
    err = rel_err_per_element(A.cpu().numpy(), Ar)
    assert err.max() <= TOL64, err.max()
    for form in (LP2, EP1):
        A = gfem.integrate_fwd(_t(mesh.coords), _t(mesh.conn), form, out_dtype=torch.float64)
        Ar, _ = orc.integrate(2, form, mesh.conn, mesh.coords)
        assert rel_err_per_element(A.cpu().numpy(), Ar).max() <= TOL64


def test_fp64_output_from_fp32_coords(gfem, orc):
    mesh = _small_mesh(3)
    A = gfem.integrate_fwd(_t(mesh.coords), _t(mesh.conn), LP1, out_dtype=torch.float64)
    Ar, _ = orc.integrate(3, LP1, mesh.conn, mesh.coords)
    assert rel_err_per_element(A.cpu().numpy(), Ar).max() <= 1e-11


def test_plain_fp32_jacobian_fails_on_slivers_only(gfem, orc):
    """The error study the compensated Jacobian exists for: plain FP32 is fine on
    regular elements and loses accuracy on slivers."""
    mesh = _small_mesh(3)
    A = gfem.integrate_fwd(_t(mesh.coords), _t(mesh.conn), LP1, jac=gfem.JAC_F32)
    Ar, _ = orc.integrate(3, LP1, mesh.conn, mesh.coords)
    err = rel_err_per_element(A.cpu().numpy(), Ar)
    assert err[~mesh.sliver].max() <= TOL32
    assert err[mesh.sliver].max() > TOL32


@pytest.mark.parametrize("E", [1, 31, 32, 33, 97])
@pytest.mark.parametrize("form", [LP1, EP1])
def test_ragged_tails_and_launch_shapes(gfem, orc, E, form):
    mesh = _small_mesh(3)
    conn = mesh.conn[:E]
    ref, _ = orc.integrate(3, form, conn, mesh.coords)
    base = None
    for warps, cps in ((0, 0), (1, 0), (8, 0), (2, 1), (16, 2)):
        A = gfem.integrate_fwd(_t(mesh.coords), _t(conn), form, warps_per_cta=warps, ctas_per_sm=cps)
        a = A.cpu().numpy()
        assert rel_err_per_element(a, ref).max() <= TOL32
        if base is None:
            base = a
        assert np.array_equal(a, base)  # launch shape never changes the bits


def test_unaligned_pointers_take_scalar_paths(gfem, orc):
    mesh = _small_mesh(3)
    E = 77
    n = 4
    buf = torch.empty(E * n * n + 1, dtype=torch.float32, device=DEV)
    out = buf[1:].view(E, n, n)                         # 4-byte offset: no 16-byte stores
    cbuf = torch.empty(E * 4 + 1, dtype=torch.int32, device=DEV)
    cbuf[1:] = _t(mesh.conn[:E].ravel())
    conn = cbuf[1:].view(E, 4)                           # 4-byte offset: no int4 loads
    gfem.integrate_fwd(_t(mesh.coords), conn, LP1, out=out)
    ref, _ = orc.integrate(3, LP1, mesh.conn[:E], mesh.coords)
    assert rel_err_per_element(out.cpu().numpy(), ref).max() <= TOL32


def test_degenerate_and_bad_connectivity(gfem):
    X = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=np.float32)
    conn = np.array([[0, 1, 2, 3], [0, 1, 1, 3], [0, 1, 2, 9], [0, -1, 2, 3]] * 10, dtype=np.int32)
    err = torch.zeros(1, dtype=torch.int32, device=DEV)
    A = gfem.integrate_fwd(_t(X), _t(conn), LP1, dev_err=err).cpu().numpy()
    assert int(err.item()) == gfem.DEVERR_CONN | gfem.DEVERR_DEGENERATE
    assert np.all(A[1::4] == 0) and np.all(A[2::4] == 0) and np.all(A[3::4] == 0)
    assert np.allclose(A[0] * 6, [[3, -1, -1, -1], [-1, 1, 0, 0], [-1, 0, 1, 0], [-1, 0, 0, 1]], atol=1e-6)
    err.zero_()
    gfem.integrate_fwd(_t(X), _t(conn[:1]), LP1, dev_err=err)
    assert int(err.item()) == 0


def test_empty_mesh_is_noop(gfem):
    X = torch.zeros((4, 3), device=DEV)
    conn = torch.zeros((0, 4), dtype=torch.int32, device=DEV)
    A = gfem.integrate_fwd(X, conn, LP1)
    assert A.shape == (0, 4, 4)


@pytest.mark.parametrize("jac,tol_det", [(2, 1e-9), (1, 1e-12)])
def test_geometry_hook(gfem, orc, jac, tol_det):
    """det J (compensated: <= 1e-9 relative; FP64: 1e-12 plus the FP64
    evaluation bound of the oracle's own det) and G against G = d! A[1:,1:] of
    the oracle's P1 matrix (A_ij = G_{i-1,j-1}/d! for i, j >= 1 on P1, Eqs. 6-7)."""
    mesh = _small_mesh(3)
    coef = mg.lognormal_coef(mg.rng_for(31), mesh.n_elem)
    det, G = gfem.geometry(_t(mesh.coords), _t(mesh.conn), _t(coef), jac=jac)
    Ar, fl, detr = orc.integrate(3, LP1, mesh.conn, mesh.coords, coef, return_det=True)
    P = mesh.coords[mesh.conn].astype(np.float64)
    J = P[:, 1:] - P[:, :1]
    prod_scale = np.abs(J).max(axis=(1, 2)) ** 3 * 6
    bound = tol_det * np.abs(detr) + 64 * 2.0 ** -53 * prod_scale
    assert np.all(np.abs(det.cpu().numpy() - detr) <= bound)
    Gr = 6.0 * Ar[:, 1:, 1:]
    Gr = np.stack([Gr[:, m, k] for m in range(3) for k in range(m, 3)], axis=1)
    Gg = G.cpu().numpy().astype(np.float64)
    gerr = np.abs(Gg - Gr).max(1) / np.abs(Gr).max(1)
    assert gerr.max() <= 2e-6, gerr.max()


def test_full_size_sliver_cube_sampled(gfem, orc):
    """128^3 Kuhn cube with 5% slivers (12,582,912 tets) in the benchmark's
    launch configuration; a stratified sample (every sliver class plus random
    regular elements and the ragged last tile) is checked element by element."""
    mesh = mg.workload_tet_slivers(128)
    coords, conn = _t(mesh.coords), _t(mesh.conn)
    A = gfem.integrate_fwd(coords, conn, LP1)
    torch.cuda.synchronize()
    rng = np.random.default_rng(5)
    sl = np.where(mesh.sliver)[0]
    idx = np.unique(np.concatenate([rng.choice(sl, 20000, replace=False),
                                    rng.choice(mesh.n_elem, 20000, replace=False),
                                    np.arange(mesh.n_elem - 40, mesh.n_elem)]))
    Ag = A[torch.from_numpy(idx).to(DEV)].cpu().numpy()
    Ar, fl = orc.integrate(3, LP1, mesh.conn[idx], mesh.coords)
    assert not fl.any()
    err = rel_err_per_element(Ag, Ar)
    assert err.max() <= TOL32, err.max()
    # symmetric, zero row sums on the whole output (property at any size)
    Af = A.view(mesh.n_elem, 16)
    Am = A
    assert torch.equal(Am, Am.transpose(1, 2))
    rs = Am.sum(2).abs().max(1).values / Am.abs().amax((1, 2))
    assert float(rs.max()) < 1e-5
    del Af
