"""GPU parity of the Laplacian on non-affine (quadratic-geometry) elements,
Eqs. 16-19, against the FP64 oracle (-m gpu).  Per element, every element:
max_ij |A_gpu - A_ref| <= 1e-5 max_ij |A_ref| (FP32 Jacobian steps on curved,
non-sliver elements)."""
import numpy as np
import pytest
import torch

from paper_1103_0066_gb300 import meshgen as mg
from conftest import rel_err_per_element

pytestmark = pytest.mark.gpu
LP1, LP2, ISO1, ISO2 = 0, 1, 5, 6
DEV = "cuda:0"
TOL = 1e-5


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _curved(dim, eps=0.05, seed=41):
    base = (mg.square_tri_mesh(13, 0.2, mg.rng_for(seed), np.float32) if dim == 2
            else mg.cube_tet_mesh(7, 0.15, mg.rng_for(seed), 0.0, np.float32))
    return mg.curved_mesh(base, eps)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("form", [ISO1, ISO2])
def test_iso_matches_oracle(gfem, orc, dim, form):
    mesh, mid = _curved(dim)
    coef = mg.lognormal_coef(mg.rng_for(42), mesh.n_elem)
    A = gfem.integrate_fwd_iso(_t(mesh.coords), _t(mesh.conn), _t(mid), form, _t(coef))
    torch.cuda.synchronize()
    Ar, fl = orc.integrate_iso(dim, form - 5, mesh.conn, mesh.coords, mid, coef)
    assert not fl.any()
    err = rel_err_per_element(A.cpu().numpy(), Ar)
    assert err.max() <= TOL, (err.max(), int(err.argmax()))


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("form", [ISO1, ISO2])
def test_iso_straight_sides_give_affine(gfem, orc, dim, form):
    mesh, _ = _curved(dim, eps=0.0)
    mid = np.stack([0.5 * (mesh.coords[mesh.conn[:, a]] + mesh.coords[mesh.conn[:, b]])
                    for a, b in mg.edge_pairs(dim)], axis=1).astype(np.float32)
    A = gfem.integrate_fwd_iso(_t(mesh.coords), _t(mesh.conn), _t(mid), form)
    Ar, _ = orc.integrate(dim, form - 5, mesh.conn, mesh.coords)
    assert rel_err_per_element(A.cpu().numpy(), Ar).max() <= TOL


@pytest.mark.parametrize("E", [1, 31, 33, 257])
def test_iso_ragged_tails_and_flags(gfem, orc, E):
    mesh, mid = _curved(3)
    conn = mesh.conn[:E].copy()
    m = mid[:E]
    err = torch.zeros(1, dtype=torch.int32, device=DEV)
    if E > 5:
        conn[5, 1] = mesh.n_vert + 7
    A = gfem.integrate_fwd_iso(_t(mesh.coords), _t(conn), _t(m), ISO2, dev_err=err)
    Ar, fl = orc.integrate_iso(3, LP2, conn, mesh.coords, m)
    assert rel_err_per_element(A.cpu().numpy(), Ar).max() <= TOL
    if E > 5:
        assert fl[5] == 1 and int(err.item()) & 1 and torch.all(A[5] == 0)


def test_iso_argument_errors(gfem):
    mesh, mid = _curved(2)
    coords, conn = _t(mesh.coords), _t(mesh.conn)
    with pytest.raises(gfem.FemError):
        gfem.integrate_fwd(coords, conn, ISO1)          # needs its edge nodes
    with pytest.raises(ValueError):
        gfem.integrate_fwd_iso(coords, conn, _t(mid[:, :2]), ISO1)
    with pytest.raises(gfem.FemError):
        gfem.integrate_fwd_iso(coords, conn, _t(mid), LP1)   # not a non-affine form


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("E", [None, 1, 129, 300])
def test_iso_p2_tensor_cores(gfem, orc, dim, E):
    """The P2 contraction on the tensor cores (split-BF16 G, exact BF16 K, FP32
    accumulation): the same per-element tolerance against the FP64 oracle,
    ragged 128-element tiles, an invalid vertex flagged and zeroed."""
    mesh, mid = _curved(dim)
    conn, m = mesh.conn, mid
    if E is not None:
        conn, m = conn[:E].copy(), mid[:E]
        if E > 5:
            conn[5, 1] = mesh.n_vert + 7
    coef = mg.lognormal_coef(mg.rng_for(43), conn.shape[0])
    err = torch.zeros(1, dtype=torch.int32, device=DEV)
    A = gfem.integrate_fwd_iso(_t(mesh.coords), _t(conn), _t(m), ISO2, _t(coef), dev_err=err,
                               contract=gfem.CONTRACT_BF16X3)
    Ar, fl = orc.integrate_iso(dim, LP2, conn, mesh.coords, m, coef)
    assert rel_err_per_element(A.cpu().numpy(), Ar).max() <= TOL
    assert int(err.item()) == (1 if fl.any() else 0)
    if fl.any():
        assert torch.all(A[5] == 0)


@pytest.mark.parametrize("E", [None, 129, 300])
def test_iso_tensor_core_kernels_agree(gfem, E):
    """Curved tetrahedra on the tensor cores take the kernel with two threads
    per element when the output is 16-byte aligned (tensor stores), and the
    one-thread-per-element kernel otherwise: both form every G entry by the
    same operations, so their outputs are the same bits (an invalid vertex
    flagged and zeroed in both)."""
    mesh, mid = _curved(3)
    conn, m = mesh.conn, mid
    if E is not None:
        conn, m = conn[:E].copy(), mid[:E]
        conn[5, 1] = mesh.n_vert + 7
    n = conn.shape[0]
    coef = _t(mg.lognormal_coef(mg.rng_for(44), n))
    args = (_t(mesh.coords), _t(conn), _t(m), ISO2, coef)
    err_a = torch.zeros(1, dtype=torch.int32, device=DEV)
    A = gfem.integrate_fwd_iso(*args, dev_err=err_a, contract=gfem.CONTRACT_BF16X3)
    buf = torch.full((n * 100 + 1,), float("nan"), device=DEV)
    B = buf[1:].view(n, 10, 10)  # 4-byte offset: no tensor map, the one-thread kernel
    assert B.data_ptr() % 16 != 0
    err_b = torch.zeros(1, dtype=torch.int32, device=DEV)
    gfem.integrate_fwd_iso(*args, out=B, dev_err=err_b, contract=gfem.CONTRACT_BF16X3)
    assert torch.equal(A, B)
    assert int(err_a.item()) == int(err_b.item())


def test_iso_tensor_cores_only_for_p2(gfem):
    mesh, mid = _curved(3)
    with pytest.raises(gfem.FemError):
        gfem.integrate_fwd_iso(_t(mesh.coords), _t(mesh.conn), _t(mid), ISO1, contract=gfem.CONTRACT_BF16X3)
