"""Batched mixed-mesh launch (-m gpu): one persistent kernel over many meshes
of mixed forms must reproduce the per-mesh entry points and the oracle, be
capturable in a CUDA graph, and survive autotuning."""
import numpy as np
import pytest
import torch

from paper_1103_0066_gb300 import meshgen as mg
from conftest import rel_err_per_element

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
TOL = 1e-5


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _items(scale, n_meshes=96, with_fwd=True, with_bwd=True):
    batch = mg.mixed_batch(n_meshes=n_meshes, scale=scale)
    items = []
    for b in batch:
        m = b.mesh
        n = mg.form_n(b.form, m.dim)
        it = {"coords": _t(m.coords), "conn": _t(m.conn), "form": b.form, "coef": _t(b.coef), "src": b}
        if with_fwd:
            it["A"] = torch.full((m.n_elem, n, n), float("nan"), device=DEV)
        if with_bwd:
            it["dA"] = _t(b.dA)
            it["dcoords"] = torch.full((m.n_vert, m.dim), float("nan"), device=DEV)
            it["dcoef"] = torch.full((m.n_elem,), float("nan"), device=DEV)
        items.append(it)
    return items


def _rel(a, b):
    a = a.double().cpu().numpy()
    b = np.asarray(b, np.float64)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def test_batch_matches_per_mesh_and_oracle(gfem, orc):
    items = _items(scale=0.003)  # 96 meshes of ~3 to ~6,000 elements, all six kinds
    batch = gfem.Batch(items)
    batch.run(gfem.PHASE_FWD | gfem.PHASE_BWD)
    torch.cuda.synchronize()
    assert batch.errors() == 0
    for k, it in enumerate(items):
        src = it["src"]
        dim = src.mesh.dim
        A_ref = gfem.integrate_fwd(it["coords"], it["conn"], it["form"], it["coef"])
        dx_ref, dw_ref = gfem.integrate_bwd(it["coords"], it["conn"], it["form"], it["dA"], it["coef"])
        assert torch.equal(it["A"], A_ref), k             # same per-tile code, same bits
        assert torch.equal(it["dcoords"], dx_ref), k      # same records, same order
        assert torch.equal(it["dcoef"], dw_ref), k
        if k % 8 == 0:  # oracle parity on a spread of meshes and kinds
            Ar, fl = orc.integrate(dim, it["form"], src.mesh.conn, src.mesh.coords, src.coef)
            assert rel_err_per_element(it["A"].cpu().numpy(), Ar).max() <= TOL
            gx, gw = orc.integrate_vjp(dim, it["form"], src.mesh.conn, src.mesh.coords, src.dA, src.coef)
            assert _rel(it["dcoords"], gx) <= TOL and _rel(it["dcoef"], gw) <= TOL


def test_batch_phases_separately(gfem):
    items = _items(scale=0.002, n_meshes=24)
    batch = gfem.Batch(items)
    batch.run(gfem.PHASE_FWD)
    torch.cuda.synchronize()
    for it in items:
        assert not torch.isnan(it["A"]).any()
        assert torch.isnan(it["dcoords"]).all()  # adjoint not run
    batch.run(gfem.PHASE_BWD)
    torch.cuda.synchronize()
    for it in items:
        assert not torch.isnan(it["dcoords"]).any() and not torch.isnan(it["dcoef"]).any()


def test_batch_graph_capture_and_tuning(gfem):
    items = _items(scale=0.002, n_meshes=48)
    batch = gfem.Batch(items)
    batch.run()
    torch.cuda.synchronize()
    ref = [(it["A"].clone(), it["dcoords"].clone()) for it in items]
    cfg = batch.tune()
    assert cfg[0] >= 1 and cfg[1] >= 1
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        batch.run(stream=s)  # warm-up outside capture
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=s):
            batch.run(stream=s)
    for it in items:
        it["A"].fill_(float("nan"))
        it["dcoords"].fill_(float("nan"))
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    assert batch.errors() == 0
    for it, (A0, x0) in zip(items, ref):
        assert torch.equal(it["A"], A0) and torch.equal(it["dcoords"], x0)


def test_batch_argument_errors(gfem):
    import ctypes
    nat = gfem.nat
    arr = (nat.FemBatchItem * 1)()
    arr[0] = nat.FemBatchItem(nat.mesh_struct(4, 0, 10, 10, 0x1000, 0x2000), 0, 0, None, None, None, None, None)
    b = ctypes.c_size_t()
    assert nat.load().fem_batch_workspace_size(arr, 1, ctypes.byref(b)) == nat.FEM_ERR_ARG
    assert nat.load().fem_batch_run(None, 3, None) == nat.FEM_ERR_ARG
