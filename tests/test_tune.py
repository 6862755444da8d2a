"""Launch-shape autotuner of the single-mesh kernels (fem_tune_fwd /
fem_tune_bwd) and its JSON cache.  CPU: the cache's keys and persistence, and
the host refusal.  GPU: the chosen shape is a candidate, the outputs the
tuner leaves are bitwise the default shape's (elements are independent and
the deterministic reduction's order does not depend on the launch shape), and
the cache tunes once per key."""
import ctypes

import numpy as np
import pytest
import torch

from paper_1103_0066_gb300 import meshgen as mg

DEV = "cuda:0"
WARPS, CTAS = {0, 1, 2, 4, 8}, {0, 2, 4, 8, 16, 24, 32}


@pytest.fixture(scope="module")
def fem():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1103_0066_gb300 as fem
    return fem


def test_cache_keys_and_persistence(fem, tmp_path):
    path = tmp_path / "tune.json"
    c = fem.TuneCache(str(path))
    assert c.entries == {}
    k1 = c.key("fwd", 0, 3, 0, 12_582_912, "NVIDIA GB300")
    assert k1 == "NVIDIA_GB300/fwd/0/3/0/23"
    # same power-of-two bucket, same key; the next bucket, another key
    assert c.key("fwd", 0, 3, 0, (1 << 23) + 1, "NVIDIA GB300") == k1
    assert c.key("fwd", 0, 3, 0, 1 << 24, "NVIDIA GB300") != k1
    assert c.key("bwd", 0, 3, 0, 12_582_912, "NVIDIA GB300") != k1
    c.entries[k1] = {"warps_per_cta": 0, "ctas_per_sm": 16, "ms": 0.18, "n_elem": 12_582_912}
    c._save()
    assert fem.TuneCache(str(path)).entries == c.entries


def test_tune_refuses_null_options(fem):
    nat = fem.nat
    lib = nat.load()
    ms = ctypes.c_float()
    assert lib.fem_tune_fwd(None, 0, None, None, 0, None, None, ctypes.byref(ms), None) == nat.FEM_ERR_ARG
    assert lib.fem_tune_bwd(None, 0, None, None, None, None, None, None, 0, None, ctypes.byref(ms),
                            None) == nat.FEM_ERR_ARG


@pytest.mark.gpu
@pytest.mark.parametrize("form", [0, 1, 2])
def test_tuned_shape_gives_default_bits(gfem, form):
    mesh = mg.cube_tet_mesh(10, 0.15, mg.rng_for(97), 0.05, np.float32)
    E, V = mesh.n_elem, mesh.n_vert
    n = gfem.form_info(form, 3)[0]
    coords, conn = torch.from_numpy(mesh.coords).to(DEV), torch.from_numpy(mesh.conn).to(DEV)
    dA = torch.from_numpy(np.random.default_rng(98).standard_normal((E, n, n)).astype(np.float32)).to(DEV)
    det_ref = torch.empty(E, device=DEV)
    A_ref = gfem.integrate_fwd(coords, conn, form, det_out=det_ref)
    ws = gfem.Workspace(coords, conn, form)
    dx_ref, _ = gfem.integrate_bwd(coords, conn, form, dA, ws=ws, need_dcoef=False, det=det_ref)
    out, det = torch.empty_like(A_ref), torch.empty(E, device=DEV)
    w, c, ms = gfem.tune_fwd(coords, conn, form, out=out, det_out=det)
    assert w in WARPS and c in CTAS and ms > 0
    assert torch.equal(out, A_ref) and torch.equal(det, det_ref)
    A2 = gfem.integrate_fwd(coords, conn, form, warps_per_cta=w, ctas_per_sm=c)
    assert torch.equal(A2, A_ref)
    dx = torch.empty_like(dx_ref)
    w, c, ms = gfem.tune_bwd(coords, conn, form, dA, ws=ws, det=det_ref, dcoords=dx)
    assert w in WARPS and c in CTAS and ms > 0
    assert torch.equal(dx, dx_ref)
    dx2, _ = gfem.integrate_bwd(coords, conn, form, dA, ws=ws, need_dcoef=False, det=det_ref, warps_per_cta=w,
                                ctas_per_sm=c)
    assert torch.equal(dx2, dx_ref)


@pytest.mark.gpu
def test_cache_tunes_once_per_key(gfem, tmp_path):
    mesh = mg.cube_tet_mesh(8, 0.15, mg.rng_for(99), 0.0, np.float32)
    coords, conn = torch.from_numpy(mesh.coords).to(DEV), torch.from_numpy(mesh.conn).to(DEV)
    cache = gfem.TuneCache(str(tmp_path / "t.json"))
    shape = cache.fwd(coords, conn, 0)
    assert len(cache.entries) == 1
    entry = dict(next(iter(cache.entries.values())))
    assert cache.fwd(coords, conn, 0) == shape  # a hit: no second tuning
    assert next(iter(cache.entries.values())) == entry
    assert gfem.TuneCache(str(tmp_path / "t.json")).entries == cache.entries
