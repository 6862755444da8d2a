"""HostStep / fem_host_step_* (-m gpu): forward + adjoint from pinned host
buffers with the copies overlapped.  Its outputs equal the device path's bit
for bit, for slices that split the mesh raggedly and for one slice, on the
run that builds the incidence and on the runs that reuse it (slice-wise
adjoint); a rebuild takes a new connectivity; pageable or misshapen buffers
are rejected."""
import numpy as np
import pytest
import torch

from paper_1103_0066_gb300 import meshgen as mg

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _pinned(a):
    return torch.from_numpy(np.ascontiguousarray(a)).pin_memory()


@pytest.mark.parametrize("chunk,form", [(1000, 0), (1 << 20, 0), (700, 2)])
def test_host_step_equals_device_path(gfem, chunk, form):
    mesh = mg.cube_tet_mesh(9, 0.15, mg.rng_for(91), 0.05, np.float32)
    E, V = mesh.n_elem, mesh.n_vert
    n = 4 if form == 0 else 12
    dA = np.random.default_rng(92).standard_normal((E, n, n)).astype(np.float32)
    coords, conn = torch.from_numpy(mesh.coords).to(DEV), torch.from_numpy(mesh.conn).to(DEV)
    A_ref = gfem.integrate_fwd(coords, conn, form)
    dx_ref, _ = gfem.integrate_bwd(coords, conn, form, torch.from_numpy(dA).to(DEV), need_dcoef=False)
    hs = gfem.HostStep(V, E, 3, form, chunk=chunk, device=DEV)
    A_h = torch.empty((E, n, n)).pin_memory()
    dx_h = torch.empty((V, 3)).pin_memory()
    for _ in range(3):  # the later runs reuse the incidence
        A_h.zero_()
        dx_h.zero_()
        hs.run(_pinned(mesh.coords), _pinned(mesh.conn), _pinned(dA), A_h, dx_h)
        torch.cuda.synchronize()
        assert torch.equal(A_h, A_ref.cpu()) and torch.equal(dx_h, dx_ref.cpu())


def test_host_step_rejects_bad_buffers(gfem):
    mesh = mg.cube_tet_mesh(3, 0.1, mg.rng_for(93), 0.0, np.float32)
    E, V = mesh.n_elem, mesh.n_vert
    hs = gfem.HostStep(V, E, 3, device=DEV)
    A_h, dx_h = torch.empty((E, 4, 4)).pin_memory(), torch.empty((V, 3)).pin_memory()
    dA = _pinned(np.zeros((E, 4, 4), np.float32))
    with pytest.raises(ValueError):  # pageable coordinates
        hs.run(torch.from_numpy(mesh.coords), _pinned(mesh.conn), dA, A_h, dx_h)
    with pytest.raises(ValueError):  # wrong shape
        hs.run(_pinned(mesh.coords), _pinned(mesh.conn), dA, torch.empty((E, 3, 3)).pin_memory(), dx_h)
    with pytest.raises(ValueError):
        gfem.HostStep(V, E, 3, gfem.LAPLACE_P1_W1, device=DEV)


def test_host_step_rebuild_takes_new_connectivity(gfem):
    m1 = mg.cube_tet_mesh(6, 0.15, mg.rng_for(94), 0.05, np.float32)
    m2, _ = mg.shuffled(m1, mg.rng_for(95))  # same sizes, another connectivity
    E, V = m1.n_elem, m1.n_vert
    dA = np.random.default_rng(96).standard_normal((E, 4, 4)).astype(np.float32)
    hs = gfem.HostStep(V, E, 3, chunk=480, device=DEV)
    A_h, dx_h = torch.empty((E, 4, 4)).pin_memory(), torch.empty((V, 3)).pin_memory()
    for mesh, rebuild in ((m1, False), (m2, True), (m2, False)):
        coords, conn = torch.from_numpy(mesh.coords).to(DEV), torch.from_numpy(mesh.conn).to(DEV)
        dx_ref, _ = gfem.integrate_bwd(coords, conn, 0, torch.from_numpy(dA).to(DEV), need_dcoef=False)
        hs.run(_pinned(mesh.coords), _pinned(mesh.conn), _pinned(dA), A_h, dx_h, rebuild=rebuild)
        torch.cuda.synchronize()
        assert torch.equal(A_h, gfem.integrate_fwd(coords, conn, 0).cpu())
        assert torch.equal(dx_h, dx_ref.cpu())


def test_host_step_reuse_does_not_read_the_connectivity(gfem):
    """A run without rebuild keeps the connectivity of the last building run
    on the device: a connectivity buffer of zeros passed then changes nothing."""
    mesh = mg.cube_tet_mesh(5, 0.15, mg.rng_for(97), 0.05, np.float32)
    E, V = mesh.n_elem, mesh.n_vert
    dA = np.random.default_rng(98).standard_normal((E, 4, 4)).astype(np.float32)
    coords, conn = torch.from_numpy(mesh.coords).to(DEV), torch.from_numpy(mesh.conn).to(DEV)
    A_ref = gfem.integrate_fwd(coords, conn, 0).cpu()
    dx_ref, _ = gfem.integrate_bwd(coords, conn, 0, torch.from_numpy(dA).to(DEV), need_dcoef=False)
    hs = gfem.HostStep(V, E, 3, chunk=256, device=DEV)
    A_h, dx_h = torch.empty((E, 4, 4)).pin_memory(), torch.empty((V, 3)).pin_memory()
    hs.run(_pinned(mesh.coords), _pinned(mesh.conn), _pinned(dA), A_h, dx_h)
    zeros = _pinned(np.zeros_like(mesh.conn))
    for _ in range(2):
        A_h.zero_()
        dx_h.zero_()
        hs.run(_pinned(mesh.coords), zeros, _pinned(dA), A_h, dx_h)
        torch.cuda.synchronize()
        assert torch.equal(A_h, A_ref) and torch.equal(dx_h, dx_ref.cpu())


def test_host_step_abi_refusals(gfem):
    from paper_1103_0066_gb300 import _native as nat
    with pytest.raises(nat.FemError) as ei:
        nat.fem_host_step_create(gfem.DIV_P1P1, 3, 10, 10, 0)
    assert ei.value.status == nat.FEM_ERR_UNSUPPORTED
    with pytest.raises(nat.FemError) as ei:
        nat.fem_host_step_create(0, 3, 0, 10, 0)
    assert ei.value.status == nat.FEM_ERR_ARG
    h = nat.fem_host_step_create(0, 3, 64, 64, 0)
    try:
        pageable = np.zeros(64 * 16, np.float32)
        pinned = torch.zeros(64 * 16).pin_memory()
        p = pinned.data_ptr()
        with pytest.raises(nat.FemError) as ei:  # pageable host memory is refused before any copy
            nat.fem_host_step_run(h, pageable.ctypes.data, p, p, p, p, False, 0)
        assert ei.value.status == nat.FEM_ERR_ARG
        dev = torch.zeros(16, device=DEV)
        with pytest.raises(nat.FemError):  # so is device memory
            nat.fem_host_step_run(h, dev.data_ptr(), p, p, p, p, False, 0)
    finally:
        nat.fem_host_step_destroy(h)
