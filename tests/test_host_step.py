"""HostStep (-m gpu): forward + adjoint from pinned host buffers with the
copies overlapped.  Its outputs equal the device path's bit for bit, for
slices that split the mesh raggedly and for one slice; it rejects pageable or
misshapen buffers."""
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
    for _ in range(2):  # the second run reuses the incidence
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
