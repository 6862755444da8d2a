"""Batched mixed-mesh launch (-m gpu): the persistent kernel over many meshes
of mixed forms, in each mode (one kernel for all kinds; one kind-specialised
kernel per kind, serial or forked onto side streams), must reproduce the
per-mesh entry points bit for bit and the oracle, be capturable in a CUDA
graph, and survive autotuning."""
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


MODES = ["single", "grouped", "concurrent", "per_item", "per_item_concurrent", "phased"]


def _mode(gfem, name):
    return {"single": gfem.BATCH_SINGLE, "grouped": gfem.BATCH_GROUPED,
            "concurrent": gfem.BATCH_GROUPED_CONCURRENT, "per_item": gfem.BATCH_PER_ITEM,
            "per_item_concurrent": gfem.BATCH_PER_ITEM_CONCURRENT, "phased": gfem.BATCH_PHASED}[name]


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("chunk", [1, 3])
def test_batch_matches_per_mesh_and_oracle(gfem, orc, mode, chunk):
    items = _items(scale=0.003)  # 96 meshes of ~3 to ~6,000 elements, all six kinds
    batch = gfem.Batch(items)
    batch.set_config(batch.config()[0], chunk, _mode(gfem, mode))
    assert batch.config()[1:] == (chunk, _mode(gfem, mode))
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
        if k % 8 == 0 and mode == "grouped" and chunk == 1:  # oracle parity on a spread of meshes and kinds
            Ar, fl = orc.integrate(dim, it["form"], src.mesh.conn, src.mesh.coords, src.coef)
            assert rel_err_per_element(it["A"].cpu().numpy(), Ar).max() <= TOL
            gx, gw = orc.integrate_vjp(dim, it["form"], src.mesh.conn, src.mesh.coords, src.dA, src.coef)
            assert _rel(it["dcoords"], gx) <= TOL and _rel(it["dcoef"], gw) <= TOL


@pytest.mark.parametrize("mode", MODES)
def test_batch_phases_separately(gfem, mode):
    items = _items(scale=0.002, n_meshes=24)
    batch = gfem.Batch(items)
    batch.set_config(1, 2, _mode(gfem, mode))
    batch.run(gfem.PHASE_FWD)
    torch.cuda.synchronize()
    for it in items:
        assert not torch.isnan(it["A"]).any()
        assert torch.isnan(it["dcoords"]).all()  # adjoint not run
    batch.run(gfem.PHASE_BWD)
    torch.cuda.synchronize()
    for it in items:
        assert not torch.isnan(it["dcoords"]).any() and not torch.isnan(it["dcoef"]).any()


@pytest.mark.parametrize("mode", ["tuned", "concurrent", "phased"])
def test_batch_graph_capture_and_tuning(gfem, mode):
    items = _items(scale=0.002, n_meshes=48)
    batch = gfem.Batch(items)
    batch.run()
    torch.cuda.synchronize()
    ref = [(it["A"].clone(), it["dcoords"].clone()) for it in items]
    cfg = batch.tune()
    assert cfg[0] >= 1 and cfg[1] >= 1 and cfg[2] in (gfem.BATCH_SINGLE, gfem.BATCH_GROUPED,
                                                       gfem.BATCH_GROUPED_CONCURRENT, gfem.BATCH_PER_ITEM,
                                                       gfem.BATCH_PER_ITEM_CONCURRENT, gfem.BATCH_PHASED)
    if mode == "concurrent":  # fork/join side streams inside the capture
        batch.set_config(cfg[0], cfg[1], gfem.BATCH_GROUPED_CONCURRENT)
    if mode == "per_item_concurrent":
        batch.set_config(1, 1, gfem.BATCH_PER_ITEM_CONCURRENT)
    if mode == "phased":  # per-kind multi-mesh launches forked onto side streams inside the capture
        batch.set_config(1, 1, gfem.BATCH_PHASED)
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


def test_batch_empty_meshes_and_single_kind(gfem):
    """Meshes without elements, and a batch of one kind (one group, so the
    concurrent mode has nothing to fork), in every mode."""
    big = _items(scale=0.002, n_meshes=6)
    keep = [it for it in big if it["form"] == 0 and it["src"].mesh.dim == 3][:1] or big[:1]
    empty = {"coords": keep[0]["coords"], "conn": keep[0]["conn"][:0], "form": keep[0]["form"],
             "coef": keep[0]["coef"][:0], "A": keep[0]["A"][:0], "dA": keep[0]["dA"][:0],
             "dcoords": torch.zeros_like(keep[0]["dcoords"]), "dcoef": keep[0]["dcoef"][:0]}
    items = [empty] + keep + [dict(empty, dcoords=torch.zeros_like(keep[0]["dcoords"]))]
    it = keep[0]
    A_ref = gfem.integrate_fwd(it["coords"], it["conn"], it["form"], it["coef"])
    dx_ref, _ = gfem.integrate_bwd(it["coords"], it["conn"], it["form"], it["dA"], it["coef"])
    for mode in MODES:
        batch = gfem.Batch(items)
        batch.set_config(2, 1, _mode(gfem, mode))
        it["A"].fill_(float("nan"))
        batch.run()
        torch.cuda.synchronize()
        assert batch.errors() == 0
        assert torch.equal(it["A"], A_ref) and torch.equal(it["dcoords"], dx_ref)
        assert (items[0]["dcoords"] == 0).all() and (items[2]["dcoords"] == 0).all()  # no tiles: sum of nothing


def test_multiphysics_blocks_share_one_mesh(gfem):
    """Diagonal blocks of a coupled system on one mesh (P1 elasticity for the
    displacement, P1 and P2 Laplacians for two scalar fields) in one batched
    launch: the items share the coordinate and connectivity tensors, and each
    block equals its per-form call bit for bit."""
    mesh = mg.cube_tet_mesh(6, 0.15, mg.rng_for(81), 0.05, np.float32)
    coords, conn = _t(mesh.coords), _t(mesh.conn)
    coef = _t(mg.lognormal_coef(mg.rng_for(82), mesh.n_elem))
    items = []
    for form in (2, 0, 1):
        n = mg.form_n(form, 3)
        items.append({"coords": coords, "conn": conn, "form": form, "coef": coef,
                      "A": torch.full((mesh.n_elem, n, n), float("nan"), device=DEV),
                      "dA": _t(mg.upstream(mg.rng_for(83 + form), mesh.n_elem, n)),
                      "dcoords": torch.empty((mesh.n_vert, 3), device=DEV),
                      "dcoef": torch.empty(mesh.n_elem, device=DEV)})
    batch = gfem.Batch(items)
    batch.tune()
    batch.run()
    torch.cuda.synchronize()
    assert batch.errors() == 0
    for it in items:
        A_ref = gfem.integrate_fwd(coords, conn, it["form"], coef)
        dx_ref, dw_ref = gfem.integrate_bwd(coords, conn, it["form"], it["dA"], coef)
        assert torch.equal(it["A"], A_ref) and torch.equal(it["dcoords"], dx_ref) and torch.equal(it["dcoef"], dw_ref)


@pytest.mark.parametrize("mode", ["single", "grouped", "concurrent"])
def test_bounded_wait_expires_and_the_next_run_is_correct(gfem, mode):
    """Failure detection without a GPU fault.  On the host, one mesh's
    descriptor is rewritten so that its reduction items wait for one tile more
    than the mesh has, and every wait is bounded at 2,000 polls (about 0.1 ms).
    The run completes, reports FEM_DEVERR_TIMEOUT, leaves that mesh's dcoords
    unwritten and every other output as in a normal run.  After the injection
    is lifted, the next run on the same GPU is correct again."""
    items = _items(scale=0.002, n_meshes=12)
    batch = gfem.Batch(items)
    batch.set_config(2, 1, _mode(gfem, mode))
    batch.run()
    torch.cuda.synchronize()
    assert batch.errors() == 0
    ref = [(it["A"].clone(), it["dcoords"].clone(), it["dcoef"].clone()) for it in items]
    victim = max(range(len(items)), key=lambda k: items[k]["src"].mesh.n_elem)
    batch.inject_wait(victim, extra_tiles=1, spin_limit=2000)
    for it in items:
        it["dcoords"].fill_(float("nan"))
    batch.run()
    torch.cuda.synchronize()
    assert batch.errors() & gfem.nat.DEVERR_TIMEOUT
    for k, (it, (A0, x0, w0)) in enumerate(zip(items, ref)):
        assert torch.equal(it["A"], A0) and torch.equal(it["dcoef"], w0)
        if k == victim:
            assert torch.isnan(it["dcoords"]).all()       # its records were never summed
        else:
            assert torch.equal(it["dcoords"], x0)
    batch.inject_wait(victim, 0, 0)
    batch.run()
    torch.cuda.synchronize()
    assert batch.errors() == 0
    for it, (A0, x0, w0) in zip(items, ref):
        assert torch.equal(it["A"], A0) and torch.equal(it["dcoords"], x0) and torch.equal(it["dcoef"], w0)


def test_phased_many_meshes_per_kind_and_partial_outputs(gfem):
    """The phased mode splits a kind's meshes into launches of at most 32, and
    separates meshes whose adjoint takes det J from the forward from those
    that recompute it.  70 triangle P1 meshes: some want only A, some only the
    adjoint (no A, so no saved det J), some only dcoef (no records); every
    output equals its per-mesh call bit for bit."""
    src = [b for b in mg.mixed_batch(n_meshes=420, scale=0.002) if b.mesh.dim == 2 and b.form == 0][:70]
    assert len(src) == 70
    items = []
    for k, b in enumerate(src):
        m = b.mesh
        it = {"coords": _t(m.coords), "conn": _t(m.conn), "form": 0, "coef": _t(b.coef), "src": b}
        if k % 5 != 1:
            it["A"] = torch.full((m.n_elem, 3, 3), float("nan"), device=DEV)
        if k % 5 != 2:
            it["dA"] = _t(b.dA)
            it["dcoef"] = torch.full((m.n_elem,), float("nan"), device=DEV)
            if k % 5 != 3:
                it["dcoords"] = torch.full((m.n_vert, 2), float("nan"), device=DEV)
        items.append(it)
    batch = gfem.Batch(items)
    batch.set_config(1, 1, gfem.BATCH_PHASED)
    batch.run()
    torch.cuda.synchronize()
    assert batch.errors() == 0
    for k, it in enumerate(items):
        if "A" in it:
            assert torch.equal(it["A"], gfem.integrate_fwd(it["coords"], it["conn"], 0, it["coef"])), k
        if "dA" in it:
            dx_ref, dw_ref = gfem.integrate_bwd(it["coords"], it["conn"], 0, it["dA"], it["coef"])
            assert torch.equal(it["dcoef"], dw_ref), k
            if "dcoords" in it:
                assert torch.equal(it["dcoords"], dx_ref), k
