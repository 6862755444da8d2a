"""The allocation-free adjoint entry point (-m gpu).

fem_integrate_bwd_noalloc is for callers that cannot allocate device memory:
it takes no workspace and works inside a scratch array built into the library.
This test calls it through the C ABI twice in a row and checks both results
against the regular entry point, fem_integrate_bwd with a caller-allocated
workspace, within the adjoint tests' tolerance (1e-5 of the largest entry).
It also checks that a mesh too large for the built-in array is refused before
anything runs.  It lives in its own file so that it is collected last.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1103_0066_gb300 import meshgen as mg

pytestmark = pytest.mark.gpu
TOL = 1e-5
DEV = "cuda:0"


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _rel(a, b):
    a = a.double().cpu().numpy()
    b = b.double().cpu().numpy()
    return float(np.abs(a - b).max() / np.abs(b).max())


def _noalloc(fem, coords, conn, form, dA, coef):
    nat = fem.nat
    m = fem._mesh_struct(coords, conn)
    dx = torch.full((coords.shape[0], coords.shape[1]), float("nan"), device=DEV)
    dw = torch.full((conn.shape[0],), float("nan"), device=DEV)
    st = nat.load().fem_integrate_bwd_noalloc(
        ctypes.byref(m), form, ctypes.c_void_p(coef.data_ptr()), ctypes.c_void_p(dA.data_ptr()),
        ctypes.c_void_p(dx.data_ptr()), ctypes.c_void_p(dw.data_ptr()), ctypes.byref(nat.options_struct()),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == nat.FEM_OK, nat.load().fem_last_error().decode()
    torch.cuda.synchronize()
    return dx, dw


@pytest.mark.parametrize("dim,form", [(3, 0), (3, 2), (2, 1)])
def test_noalloc_matches_workspace_entry_point(gfem, dim, form):
    if dim == 3:
        mesh = mg.cube_tet_mesh(9, 0.15, mg.rng_for(61), 0.05, np.float32)   # 4,374 tets, slivers
    else:
        mesh = mg.square_tri_mesh(20, 0.2, mg.rng_for(61), np.float32)       # 800 triangles
    n = mg.form_n(form, dim)
    coords, conn = _t(mesh.coords), _t(mesh.conn)
    coef = _t(mg.lognormal_coef(mg.rng_for(62), mesh.n_elem))
    for call in range(2):  # two calls in a row: the second sees the first one's leftovers
        dA = _t(mg.upstream(mg.rng_for(63 + call), mesh.n_elem, n))
        ref_x, ref_w = gfem.integrate_bwd(coords, conn, form, dA, coef)
        got_x, got_w = _noalloc(gfem, coords, conn, form, dA, coef)
        assert _rel(got_x, ref_x) <= TOL
        assert _rel(got_w, ref_w) <= TOL


def test_noalloc_refuses_meshes_beyond_its_scratch(gfem):
    nat = gfem.nat
    big = nat.mesh_struct(3, 0, 10_000_000, 2_000_000, 0x1000, 0x2000)  # never launched
    st = nat.load().fem_integrate_bwd_noalloc(ctypes.byref(big), 0, None, ctypes.c_void_p(0x3000),
                                              ctypes.c_void_p(0x4000), None, None, None)
    assert st == nat.FEM_ERR_UNSUPPORTED
    assert "caller-allocated workspace" in nat.load().fem_last_error().decode()
