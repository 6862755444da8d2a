"""Split-BF16 tensor-core contraction (tcgen05) against the FP64 oracle (-m gpu).

Each rounding to bf16's 8-bit significand leaves at most 2^-8 of what it
rounds, so the three-term split of G leaves at most 2^-24 |G| per entry (FP32's
own unit roundoff), and K is exact in bf16: the per-element tolerance is the
FP32 one, 1e-5 relative to max |A_e|, on every element including slivers."""
import numpy as np
import pytest
import torch

from paper_1103_0066_gb300 import meshgen as mg
from conftest import rel_err_per_element

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
TOL = 1e-5
LP2, EP1 = 1, 2


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@pytest.mark.parametrize("dim,form", [(3, EP1), (3, LP2), (2, EP1), (2, LP2)])
def test_tensor_core_matches_oracle(gfem, orc, dim, form):
    if dim == 3:
        mesh = mg.cube_tet_mesh(7, 0.15, mg.rng_for(71), 0.05, np.float32)   # 2,058 tets incl. slivers
    else:
        mesh = mg.square_tri_mesh(23, 0.2, mg.rng_for(71), np.float32)       # 1,058 triangles
    coef = mg.lognormal_coef(mg.rng_for(72), mesh.n_elem)
    err = torch.zeros(1, dtype=torch.int32, device=DEV)
    A = gfem.integrate_fwd(_t(mesh.coords), _t(mesh.conn), form, _t(coef), contract=gfem.CONTRACT_BF16X3,
                           dev_err=err)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    Ar, fl = orc.integrate(dim, form, mesh.conn, mesh.coords, coef)
    e = rel_err_per_element(A.cpu().numpy(), Ar)
    assert e.max() <= TOL, e.max()
    A32 = gfem.integrate_fwd(_t(mesh.coords), _t(mesh.conn), form, _t(coef))
    assert rel_err_per_element(A.cpu().numpy(), A32.double().cpu().numpy()).max() <= TOL


@pytest.mark.parametrize("E", [1, 127, 128, 129, 300])
def test_tensor_core_tails_and_grids(gfem, orc, E):
    mesh = mg.cube_tet_mesh(4, 0.15, mg.rng_for(73), 0.05, np.float32)
    conn = mesh.conn[:E]
    ref, _ = orc.integrate(3, EP1, conn, mesh.coords)
    for cps in (0, 1):
        A = gfem.integrate_fwd(_t(mesh.coords), _t(conn), EP1, contract=gfem.CONTRACT_BF16X3, ctas_per_sm=cps)
        assert rel_err_per_element(A.cpu().numpy(), ref).max() <= TOL


def test_tensor_core_degenerate_and_conn_errors(gfem):
    X = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=np.float32)
    conn = np.array([[0, 1, 2, 3], [0, 1, 1, 3], [0, 1, 2, 9]] * 50, dtype=np.int32)
    err = torch.zeros(1, dtype=torch.int32, device=DEV)
    A = gfem.integrate_fwd(_t(X), _t(conn), EP1, contract=gfem.CONTRACT_BF16X3, dev_err=err).cpu().numpy()
    assert int(err.item()) == gfem.DEVERR_CONN | gfem.DEVERR_DEGENERATE
    assert np.all(A[1::3] == 0) and np.all(A[2::3] == 0) and np.abs(A[0]).max() > 0


def test_full_size_elasticity_sampled(gfem, orc):
    """128^3 sliver cube (12,582,912 tets), P1 elasticity with a lognormal
    coefficient: the FP32 and the tensor-core paths at full size, each on a
    stratified sample of elements (slivers, regular, the ragged last tiles)."""
    mesh = mg.workload_tet_slivers(128)
    E = mesh.n_elem
    coef_h = mg.lognormal_coef(mg.rng_for(68), E)
    coords, conn, coef = _t(mesh.coords), _t(mesh.conn), _t(coef_h)
    rng = np.random.default_rng(69)
    idx = np.unique(np.concatenate([rng.choice(np.where(mesh.sliver)[0], 5000, replace=False),
                                    rng.choice(E, 5000, replace=False), np.arange(E - 200, E)]))
    Ar, fl = orc.integrate(3, EP1, mesh.conn[idx], mesh.coords, coef_h[idx])
    assert not fl.any()
    sel = torch.from_numpy(idx).to(DEV)
    for contract in (gfem.CONTRACT_F32, gfem.CONTRACT_BF16X3):
        A = gfem.integrate_fwd(coords, conn, EP1, coef, contract=contract)
        Ag = A[sel].cpu().numpy()
        del A
        assert rel_err_per_element(Ag, Ar).max() <= TOL


@pytest.mark.parametrize("dim,form", [(3, EP1), (2, LP2)])
def test_tensor_core_unaligned_output_same_bits(gfem, dim, form):
    """An output 4 bytes off a 16-byte boundary has no tensor map: the kernel
    takes its plain stage and scalar stores. Only the epilogue's data movement
    differs, so the bits equal the TMA path's."""
    if dim == 3:
        mesh = mg.cube_tet_mesh(5, 0.15, mg.rng_for(75), 0.05, np.float32)
    else:
        mesh = mg.square_tri_mesh(17, 0.2, mg.rng_for(75), np.float32)
    n = (dim + 1) * dim if form == EP1 else (dim + 1) * (dim + 2) // 2
    coords, conn = _t(mesh.coords), _t(mesh.conn)
    A = gfem.integrate_fwd(coords, conn, form, contract=gfem.CONTRACT_BF16X3)
    buf = torch.full((mesh.n_elem * n * n + 1,), float("nan"), device=DEV)
    out = buf[1:].view(mesh.n_elem, n, n)
    assert out.data_ptr() % 16 == 4
    B = gfem.integrate_fwd(coords, conn, form, contract=gfem.CONTRACT_BF16X3, out=out)
    torch.cuda.synchronize()
    assert B.data_ptr() == out.data_ptr() and torch.equal(A, B)
