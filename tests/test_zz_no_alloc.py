"""The allocation-free adjoint entry point (-m gpu).

fem_integrate_bwd_noalloc is for callers that cannot allocate device memory:
it takes no workspace and works inside a scratch array built into the library.
These tests call it through the C ABI twice in a row and compare each result
with the regular entry point, fem_integrate_bwd with a caller-allocated
workspace.  Both run the same incidence build, element pass and
deterministic reduction on the same inputs, so the results must be equal bit
for bit; any stale scratch left by an earlier call would break that.  A large
mesh followed by a smaller one, a coefficient-gradient-only call and calls
refused before anything runs are covered too.  The file is collected last.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1103_0066_gb300 import meshgen as mg

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _noalloc(fem, coords, conn, form, dA, coef, want_dcoords=True):
    nat = fem.nat
    m = fem._mesh_struct(coords, conn)
    dx = torch.full((coords.shape[0], coords.shape[1]), float("nan"), device=DEV) if want_dcoords else None
    dw = torch.full((conn.shape[0],), float("nan"), device=DEV)
    st = nat.load().fem_integrate_bwd_noalloc(
        ctypes.byref(m), form, ctypes.c_void_p(coef.data_ptr()), ctypes.c_void_p(dA.data_ptr()),
        ctypes.c_void_p(dx.data_ptr() if dx is not None else 0), ctypes.c_void_p(dw.data_ptr()),
        ctypes.byref(nat.options_struct()), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == nat.FEM_OK, nat.load().fem_last_error().decode()
    torch.cuda.synchronize()
    return dx, dw


def _case(dim, n, seed):
    if dim == 3:
        return mg.cube_tet_mesh(n, 0.15, mg.rng_for(seed), 0.05, np.float32)
    return mg.square_tri_mesh(n, 0.2, mg.rng_for(seed), np.float32)


@pytest.mark.parametrize("dim,form", [(3, 0), (3, 2), (2, 1)])
def test_noalloc_matches_workspace_entry_point(gfem, dim, form):
    mesh = _case(dim, 9 if dim == 3 else 20, 61)   # 4,374 tets with slivers / 800 triangles
    n = mg.form_n(form, dim)
    coords, conn = _t(mesh.coords), _t(mesh.conn)
    coef = _t(mg.lognormal_coef(mg.rng_for(62), mesh.n_elem))
    for call in range(2):  # two calls in a row: the second sees the first one's leftovers
        dA = _t(mg.upstream(mg.rng_for(63 + call), mesh.n_elem, n))
        ref_x, ref_w = gfem.integrate_bwd(coords, conn, form, dA, coef)
        got_x, got_w = _noalloc(gfem, coords, conn, form, dA, coef)
        assert torch.equal(got_x, ref_x)
        assert torch.equal(got_w, ref_w)


def test_noalloc_larger_then_smaller_mesh(gfem):
    """A large mesh fills much of the scratch array; a smaller one right after
    must not read anything the large one left behind."""
    big, small = _case(3, 28, 64), _case(3, 5, 65)        # 131,712 and 750 tets (+ slivers)
    for mesh in (big, small, big):
        coords, conn = _t(mesh.coords), _t(mesh.conn)
        coef = _t(mg.lognormal_coef(mg.rng_for(66), mesh.n_elem))
        dA = _t(mg.upstream(mg.rng_for(67), mesh.n_elem, 4))
        ref_x, ref_w = gfem.integrate_bwd(coords, conn, 0, dA, coef)
        got_x, got_w = _noalloc(gfem, coords, conn, 0, dA, coef)
        assert torch.equal(got_x, ref_x) and torch.equal(got_w, ref_w)


def test_noalloc_coefficient_gradient_only(gfem):
    mesh = _case(3, 6, 68)
    coords, conn = _t(mesh.coords), _t(mesh.conn)
    coef = _t(mg.lognormal_coef(mg.rng_for(69), mesh.n_elem))
    dA = _t(mg.upstream(mg.rng_for(70), mesh.n_elem, 4))
    _, ref_w = gfem.integrate_bwd(coords, conn, 0, dA, coef, need_dcoords=False)
    got_x, got_w = _noalloc(gfem, coords, conn, 0, dA, coef, want_dcoords=False)
    assert got_x is None and torch.equal(got_w, ref_w)


def test_noalloc_refusals_launch_nothing(gfem):
    """Refused calls return before the scratch array is touched: a mesh too
    large for it, FP64 coordinates and a tensor-core contraction (the adjoint is
    FP32 only).  The pointers of the first case are never dereferenced.  A
    valid call afterwards still matches the workspace entry point bit for bit."""
    nat = gfem.nat
    lib = nat.load()
    big = nat.mesh_struct(3, 0, 10_000_000, 2_000_000, 0x1000, 0x2000)  # never launched
    st = lib.fem_integrate_bwd_noalloc(ctypes.byref(big), 0, None, ctypes.c_void_p(0x3000),
                                       ctypes.c_void_p(0x4000), None, None, None)
    assert st == nat.FEM_ERR_UNSUPPORTED
    assert "caller-allocated workspace" in lib.fem_last_error().decode()
    mesh = _case(3, 5, 71)
    coords64, conn = _t(mesh.coords.astype(np.float64)), _t(mesh.conn)
    dA = _t(mg.upstream(mg.rng_for(72), mesh.n_elem, 4))
    dx = torch.zeros((mesh.n_vert, 3), device=DEV)
    m64 = gfem._mesh_struct(coords64, conn)
    st = lib.fem_integrate_bwd_noalloc(ctypes.byref(m64), 0, None, ctypes.c_void_p(dA.data_ptr()),
                                       ctypes.c_void_p(dx.data_ptr()), None, None, None)
    assert st == nat.FEM_ERR_UNSUPPORTED and "FP32 coordinates" in lib.fem_last_error().decode()
    coords = _t(mesh.coords)
    m32 = gfem._mesh_struct(coords, conn)
    tc = nat.options_struct(contract=nat.CONTRACT_BF16X3)
    st = lib.fem_integrate_bwd_noalloc(ctypes.byref(m32), 0, None, ctypes.c_void_p(dA.data_ptr()),
                                       ctypes.c_void_p(dx.data_ptr()), None, ctypes.byref(tc), None)
    assert st == nat.FEM_ERR_UNSUPPORTED and "FP32" in lib.fem_last_error().decode()
    torch.cuda.synchronize()
    assert torch.count_nonzero(dx) == 0  # nothing was written
    coef = _t(mg.lognormal_coef(mg.rng_for(73), mesh.n_elem))
    ref_x, ref_w = gfem.integrate_bwd(coords, conn, 0, dA, coef)
    got_x, got_w = _noalloc(gfem, coords, conn, 0, dA, coef)
    assert torch.equal(got_x, ref_x) and torch.equal(got_w, ref_w)


def test_noalloc_p1_coefficient_gradient(gfem):
    """The P1-coefficient Laplacian, whose coefficient gradient is summed over
    the vertices through the scratch records even without dcoords."""
    mesh = _case(3, 8, 74)
    coords, conn = _t(mesh.coords), _t(mesh.conn)
    wv = _t(mg.lognormal_coef(mg.rng_for(75), mesh.n_vert))
    dA = _t(mg.upstream(mg.rng_for(76), mesh.n_elem, 10))
    ref_x, ref_w = gfem.integrate_bwd(coords, conn, 4, dA, wv)
    nat = gfem.nat
    m = gfem._mesh_struct(coords, conn)
    for want_x in (True, False):
        dx = torch.full((mesh.n_vert, 3), float("nan"), device=DEV) if want_x else None
        dw = torch.full((mesh.n_vert,), float("nan"), device=DEV)
        st = nat.load().fem_integrate_bwd_noalloc(
            ctypes.byref(m), 4, ctypes.c_void_p(wv.data_ptr()), ctypes.c_void_p(dA.data_ptr()),
            ctypes.c_void_p(dx.data_ptr() if dx is not None else 0), ctypes.c_void_p(dw.data_ptr()),
            ctypes.byref(nat.options_struct()), None)
        assert st == nat.FEM_OK, nat.load().fem_last_error().decode()
        torch.cuda.synchronize()
        assert torch.equal(dw, ref_w) and (dx is None or torch.equal(dx, ref_x))
