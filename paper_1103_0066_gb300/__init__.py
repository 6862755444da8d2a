"""GB300-native finite element integration by tensor contraction.

Knepley & Terrel, "Finite Element Integration on GPUs": element matrices
A_e = G_e : K (Eq. 1, Eq. 6) for the P1/P2 Laplacian and P1 symmetric-gradient
elasticity on triangles and tetrahedra, their adjoint, and batched launches.
The computation runs in ``libfem_gb300.so`` (CUDA, sm_103a) behind the C ABI of
``include/fem.h``; this package marshals torch tensors (device memory and
streams) into that ABI.  There is no CPU fallback: without the built library
every call raises.

Quick use::

    import paper_1103_0066_gb300 as fem
    mesh = fem.Mesh(coords, conn)              # CUDA tensors: [V][d] float32, [E][d+1] int32
    A = mesh.integrate(fem.LAPLACE_P1)         # [E][n][n]; differentiable in coords / coef
"""
from __future__ import annotations

import torch

from . import _native as nat
from ._native import (CONTRACT_BF16X3, CONTRACT_F32, DEVERR_CONN, DEVERR_DEGENERATE, ELASTIC_P1, F32,
                      F64, JAC_AUTO, JAC_COMP_F32, JAC_F32, JAC_F64, LAPLACE_P1, LAPLACE_P2, LAPLACE_P1_W1, LAPLACE_P2_W1,
                      LAPLACE_P1_ISO, LAPLACE_P2_ISO, DIV_P1P1, DIV_P2P1,
                      REDUCE_ATOMIC, REDUCE_DEFERRED, REDUCE_DETERMINISTIC, PHASE_BWD, PHASE_FWD, FemError,
                      BATCH_SINGLE, BATCH_GROUPED, BATCH_GROUPED_CONCURRENT, BATCH_PER_ITEM,
                      BATCH_PER_ITEM_CONCURRENT, BATCH_PHASED)

__all__ = ["Mesh", "Batch", "Assembly", "HostStep", "PHASE_FWD", "PHASE_BWD", "BATCH_SINGLE", "BATCH_GROUPED", "BATCH_GROUPED_CONCURRENT",
           "BATCH_PER_ITEM", "BATCH_PER_ITEM_CONCURRENT", "BATCH_PHASED", "mesh_order", "renumber", "integrate", "integrate_fwd", "integrate_bwd", "geometry", "form_info",
           "reference_tensor", "FemError", "LAPLACE_P1", "LAPLACE_P2", "ELASTIC_P1", "LAPLACE_P1_W1",
           "LAPLACE_P2_W1", "LAPLACE_P1_ISO", "LAPLACE_P2_ISO", "DIV_P1P1", "DIV_P2P1", "form_shape",
           "integrate_fwd_iso", "JAC_AUTO",
           "JAC_F64", "JAC_COMP_F32", "JAC_F32", "CONTRACT_F32", "CONTRACT_BF16X3",
           "REDUCE_DETERMINISTIC", "REDUCE_ATOMIC", "REDUCE_DEFERRED", "adjoint_reduce", "DEVERR_CONN", "DEVERR_DEGENERATE", "F32", "F64"]


def form_info(form: int, dim: int):
    """(n, n_geom, den): rows of A_e, folded G entries, integer scale of K."""
    return nat.fem_form_info(form, dim)


def form_shape(form: int, dim: int):
    """(rows, cols) of the form's element blocks: (n, n), or (d+1, d * nbv) for
    the coupling forms DIV_P1P1 / DIV_P2P1."""
    return nat.fem_form_shape(form, dim)


def reference_tensor(form: int, dim: int):
    """Folded reference tensor K' * den as an int32 CPU tensor [n_geom][rows][cols] (host call)."""
    _, ng, den = form_info(form, dim)
    rows, cols = form_shape(form, dim)
    K = torch.empty((ng, rows, cols), dtype=torch.int32)
    nat.fem_reference_tensor(form, dim, K.data_ptr(), K.numel())
    return K, den


def _stream_ptr(stream) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _mesh_struct(coords: torch.Tensor, conn: torch.Tensor) -> nat.FemMesh:
    if not (coords.is_cuda and conn.is_cuda):
        raise ValueError("coords and conn must be CUDA tensors")
    if conn.dtype != torch.int32 or conn.dim() != 2 or not conn.is_contiguous():
        raise ValueError("conn must be a contiguous int32 tensor [E][d+1]")
    if coords.dim() != 2 or not coords.is_contiguous() or coords.dtype not in (torch.float32, torch.float64):
        raise ValueError("coords must be a contiguous float32/float64 tensor [V][d]")
    dim = coords.shape[1]
    if conn.shape[1] != dim + 1:
        raise ValueError("conn must have d+1 columns")
    return nat.mesh_struct(dim, F64 if coords.dtype == torch.float64 else F32, coords.shape[0],
                           conn.shape[0], conn.data_ptr(), coords.data_ptr())


def _coef_ptr(coef, E, what="[E]"):
    if coef is None:
        return 0
    if coef.dtype != torch.float32 or not coef.is_contiguous() or coef.numel() != E or not coef.is_cuda:
        raise ValueError(f"coef must be a contiguous CUDA float32 tensor {what}")
    return coef.data_ptr()


def integrate_fwd(coords, conn, form, coef=None, out=None, out_dtype=torch.float32, jac=JAC_AUTO,
                  contract=CONTRACT_F32, warps_per_cta=0, ctas_per_sm=0, dev_err=None, stream=None, det_out=None):
    """fem_integrate_fwd: element matrices [E][n][n] (not differentiable; see integrate).
    coef: [E] per-element values, or [V] vertex values for LAPLACE_P1_W1 / LAPLACE_P2_W1.
    det_out: optional float32 [E] tensor that receives det J for integrate_bwd(det=...)
    (fem_integrate_fwd_save)."""
    m = _mesh_struct(coords, conn)
    rows, cols = form_shape(form, m.dim)
    E = conn.shape[0]
    w1 = form in (LAPLACE_P1_W1, LAPLACE_P2_W1)
    if out is None:
        out = torch.empty((E, rows, cols), dtype=out_dtype, device=coords.device)
    elif out.shape != (E, rows, cols) or not out.is_contiguous():
        raise ValueError(f"out must be a contiguous [E][{rows}][{cols}] tensor")
    od = F64 if out.dtype == torch.float64 else F32
    opts = nat.options_struct(jac, contract, 0, warps_per_cta, ctas_per_sm,
                              dev_err.data_ptr() if dev_err is not None else 0)
    cp = _coef_ptr(coef, coords.shape[0], "[V]") if w1 else _coef_ptr(coef, E)
    if det_out is not None:
        _check_det(det_out, E)
        nat.fem_integrate_fwd_save(m, form, cp, out.data_ptr(), od, det_out.data_ptr(), opts, _stream_ptr(stream))
    else:
        nat.fem_integrate_fwd(m, form, cp, out.data_ptr(), od, opts, _stream_ptr(stream))
    return out


def _check_det(det, E):
    if not (det.is_cuda and det.dtype == torch.float32 and det.is_contiguous() and det.numel() == E):
        raise ValueError("det must be a contiguous CUDA float32 tensor [E]")


def integrate_fwd_iso(coords, conn, mid, form=LAPLACE_P1_ISO, coef=None, out=None, dev_err=None, stream=None,
                      contract=CONTRACT_F32, ctas_per_sm=0):
    """fem_integrate_fwd_iso: element matrices [E][n][n] of the Laplacian on
    non-affine elements with edge-midpoint nodes mid [E][d(d+1)/2][d] (FP32).
    contract=CONTRACT_BF16X3 runs the P2 contraction on the tensor cores."""
    m = _mesh_struct(coords, conn)
    n, _, _ = form_info(form, m.dim)
    E = conn.shape[0]
    ne = m.dim * (m.dim + 1) // 2
    if mid.dtype != torch.float32 or not mid.is_contiguous() or tuple(mid.shape) != (E, ne, m.dim) or not mid.is_cuda:
        raise ValueError(f"mid must be a contiguous CUDA float32 tensor [E][{ne}][{m.dim}]")
    if out is None:
        out = torch.empty((E, n, n), dtype=torch.float32, device=coords.device)
    elif out.shape != (E, n, n) or not out.is_contiguous() or out.dtype != torch.float32:
        raise ValueError("out must be a contiguous float32 [E][n][n] tensor")
    opts = nat.options_struct(JAC_AUTO, contract, 0, 0, ctas_per_sm, dev_err.data_ptr() if dev_err is not None else 0)
    nat.fem_integrate_fwd_iso(m, form, mid.data_ptr(), _coef_ptr(coef, E), out.data_ptr(), opts, _stream_ptr(stream))
    return out


def geometry(coords, conn, coef=None, jac=JAC_AUTO, dev_err=None, stream=None):
    """fem_geometry test hook: (detJ [E] float64, G [E][d(d+1)/2] float32)."""
    m = _mesh_struct(coords, conn)
    E = conn.shape[0]
    det = torch.empty(E, dtype=torch.float64, device=coords.device)
    G = torch.empty((E, m.dim * (m.dim + 1) // 2), dtype=torch.float32, device=coords.device)
    opts = nat.options_struct(jac, 0, 0, 0, 0, dev_err.data_ptr() if dev_err is not None else 0)
    nat.fem_geometry(m, _coef_ptr(coef, E), opts, det.data_ptr(), G.data_ptr(), _stream_ptr(stream))
    return det, G


class Workspace:
    """Device workspace of the adjoint for one connectivity (incidence CSR + scratch)."""

    def __init__(self, coords, conn, form=LAPLACE_P1, stream=None):
        self.m = _mesh_struct(coords, conn)
        opts = nat.options_struct()
        self.bytes = nat.fem_bwd_workspace_size(self.m, form, opts)
        self.buf = torch.empty(max(self.bytes, 1), dtype=torch.uint8, device=coords.device)
        self.stream = stream
        nat.fem_incidence_build(self.m, self.buf.data_ptr(), self.bytes, _stream_ptr(stream))

    def n_records(self) -> int:
        """Records of the deterministic reduction (fem_incidence_info; synchronizes)."""
        return nat.fem_incidence_info(self.m, self.buf.data_ptr(), self.bytes, _stream_ptr(self.stream))[0]

    def record_layout(self) -> int:
        """nat.RECORDS_VERTEX_MAJOR or nat.RECORDS_TILE_ORDER, as the build chose it."""
        return nat.fem_incidence_info(self.m, self.buf.data_ptr(), self.bytes, _stream_ptr(self.stream))[1]


def mesh_order(coords, conn, stream=None):
    """fem_mesh_order: a locality numbering of an unstructured mesh (Z-order of
    vertex positions and element centroids).  Returns (elem_perm, vert_perm),
    int32 CUDA tensors mapping new position -> old number."""
    m = _mesh_struct(coords, conn)
    ws_bytes = nat.fem_mesh_order_workspace_size(m)
    ws = torch.empty(max(ws_bytes, 256), dtype=torch.uint8, device=coords.device)
    elem_perm = torch.empty(conn.shape[0], dtype=torch.int32, device=coords.device)
    vert_perm = torch.empty(coords.shape[0], dtype=torch.int32, device=coords.device)
    nat.fem_mesh_order(m, ws.data_ptr(), ws_bytes, elem_perm.data_ptr(), vert_perm.data_ptr(), _stream_ptr(stream))
    return elem_perm, vert_perm


def renumber(coords, conn, elem_perm, vert_perm, stream=None):
    """fem_mesh_renumber: the mesh in the new numbering, (coords[vert_perm],
    new numbers of conn[elem_perm]); element matrices keep their values."""
    m = _mesh_struct(coords, conn)
    for t, n in ((elem_perm, conn.shape[0]), (vert_perm, coords.shape[0])):
        if t.dtype != torch.int32 or not t.is_cuda or not t.is_contiguous() or t.numel() != n:
            raise ValueError("permutations must be contiguous CUDA int32 tensors of n_elem / n_vert entries")
    ws_bytes = nat.fem_mesh_order_workspace_size(m)
    ws = torch.empty(max(ws_bytes, 256), dtype=torch.uint8, device=coords.device)
    coords_out = torch.empty_like(coords)
    conn_out = torch.empty_like(conn)
    nat.fem_mesh_renumber(m, elem_perm.data_ptr(), vert_perm.data_ptr(), ws.data_ptr(), ws_bytes,
                          coords_out.data_ptr(), conn_out.data_ptr(), _stream_ptr(stream))
    return coords_out, conn_out


class Assembly:
    """Global sparse assembly (fem_assembly_*) of the element matrices of one
    connectivity: CSR for the scalar forms, BSR with d x d blocks for
    ELASTIC_P1 (node-major unknowns v*d + c).  The P2 forms' unknowns are the
    vertices, then the edges in increasing (lower, higher) vertex order:
    n_rows of them, dofs [E][n] each element's (device, int32).

    row_ptr [n_rows+1] and col_idx [nnz] (int32, device) describe the pattern;
    assemble(A) returns the values [nnz] (or [nnz][d][d]) of sum_e P_e^T A_e P_e,
    each entry summed in a fixed order."""

    def __init__(self, coords, conn, form=LAPLACE_P1, stream=None):
        self.m = _mesh_struct(coords, conn)
        self.form = form
        self.block = self.m.dim if form == ELASTIC_P1 else 1
        self.bytes = nat.fem_assembly_workspace_size(self.m, form)
        self.buf = torch.empty(max(self.bytes, 256), dtype=torch.uint8, device=coords.device)
        self._keep = (coords, conn)
        self.nnz, self.n_records = nat.fem_assembly_build(self.m, form, self.buf.data_ptr(), self.bytes,
                                                          _stream_ptr(stream))
        rp, ci = nat.fem_assembly_pattern(self.m, form, self.buf.data_ptr(), self.bytes)
        self.n_rows, dp = nat.fem_assembly_unknowns(self.m, form, self.buf.data_ptr(), self.bytes)
        base = self.buf.data_ptr()
        self.row_ptr = self.buf[rp - base: rp - base + 4 * (self.n_rows + 1)].view(torch.int32)
        self.col_idx = self.buf[ci - base: ci - base + 4 * self.nnz].view(torch.int32)
        E, n = conn.shape[0], form_info(form, self.m.dim)[0] // self.block
        self.dofs = (self.buf[dp - base: dp - base + 4 * E * n].view(torch.int32).view(E, n)
                     if base <= dp < base + self.buf.numel() else conn)

    def assemble(self, A, out=None, stream=None):
        b = self.block
        shape = (self.nnz,) if b == 1 else (self.nnz, b, b)
        if out is None:
            out = torch.empty(shape, dtype=torch.float32, device=A.device)
        if A.dtype != torch.float32 or not A.is_contiguous() or out.shape != shape or not out.is_contiguous():
            raise ValueError("A must be contiguous float32 [E][n][n]; out float32 " + str(shape))
        nat.fem_assemble(self.m, self.form, A.data_ptr(), self.buf.data_ptr(), self.bytes, out.data_ptr(),
                         _stream_ptr(stream))
        return out


def integrate_bwd(coords, conn, form, dA, coef=None, ws: Workspace | None = None,
                  reduce=REDUCE_DETERMINISTIC, need_dcoords=True, need_dcoef=True, jac=JAC_AUTO,
                  warps_per_cta=0, ctas_per_sm=0, dcoords=None, dcoef=None, dev_err=None, stream=None, det=None):
    """fem_integrate_bwd: (dcoords [V][d] or None, dcoef or None) for the upstream dA.
    dcoef is [E] for a per-element coefficient, [V] (the gradient of the
    coefficient's vertex values) for LAPLACE_P1_W1 / LAPLACE_P2_W1.
    det: det J saved by integrate_fwd(det_out=...) (fem_integrate_bwd_saved)."""
    m = _mesh_struct(coords, conn)
    E, V = conn.shape[0], coords.shape[0]
    w1 = form in (LAPLACE_P1_W1, LAPLACE_P2_W1)
    if dA.dtype != torch.float32 or not dA.is_contiguous() or tuple(dA.shape) != (E,) + form_shape(form, m.dim):
        raise ValueError("dA must be a contiguous float32 tensor shaped like the forward's output")
    if need_dcoords and dcoords is None:
        dcoords = torch.empty((V, m.dim), dtype=torch.float32, device=coords.device)
    if need_dcoef and dcoef is None:
        dcoef = torch.empty(V if w1 else E, dtype=torch.float32, device=coords.device)
    if not need_dcoords:
        dcoords = None
    if not need_dcoef:
        dcoef = None
    ws_ptr, ws_bytes = 0, 0
    if reduce in (REDUCE_DETERMINISTIC, REDUCE_DEFERRED) and (dcoords is not None or (w1 and dcoef is not None)):
        if ws is None:
            ws = Workspace(coords, conn, form, stream)
        ws_ptr, ws_bytes = ws.buf.data_ptr(), ws.bytes
    opts = nat.options_struct(jac, 0, reduce, warps_per_cta, ctas_per_sm,
                              dev_err.data_ptr() if dev_err is not None else 0)
    dx_ptr = dcoords.data_ptr() if dcoords is not None else 0
    dw_ptr = dcoef.data_ptr() if dcoef is not None else 0
    cp = _coef_ptr(coef, V, "[V]") if w1 else _coef_ptr(coef, E)
    if det is not None:
        _check_det(det, E)
        nat.fem_integrate_bwd_saved(m, form, cp, dA.data_ptr(), det.data_ptr(), dx_ptr, dw_ptr,
                                    ws_ptr, ws_bytes, opts, _stream_ptr(stream))
    else:
        nat.fem_integrate_bwd(m, form, cp, dA.data_ptr(), dx_ptr, dw_ptr, ws_ptr, ws_bytes, opts,
                              _stream_ptr(stream))
    return dcoords, dcoef


def integrate_bwd_iso(coords, conn, mid, form, dA, coef=None, ws: Workspace | None = None,
                      reduce=REDUCE_DETERMINISTIC, need_dcoords=True, need_dmid=True, need_dcoef=False,
                      dcoords=None, dmid=None, dcoef=None, dev_err=None, stream=None, contract=CONTRACT_F32):
    """fem_integrate_bwd_iso: (dcoords [V][d], dmid [E][d(d+1)/2][d], dcoef [E]),
    each None when not asked for, for the upstream dA of integrate_fwd_iso.
    contract=CONTRACT_BF16X3 runs the P2 contraction's adjoint on the tensor
    cores (tetrahedra, deterministic or deferred reduction)."""
    m = _mesh_struct(coords, conn)
    E, V, d = conn.shape[0], coords.shape[0], m.dim
    ne = d * (d + 1) // 2
    if mid.dtype != torch.float32 or not mid.is_contiguous() or tuple(mid.shape) != (E, ne, d) or not mid.is_cuda:
        raise ValueError(f"mid must be a contiguous CUDA float32 tensor [E][{ne}][{d}]")
    n, _, _ = form_info(form, d)
    if dA.dtype != torch.float32 or not dA.is_contiguous() or tuple(dA.shape) != (E, n, n):
        raise ValueError(f"dA must be a contiguous float32 tensor [E][{n}][{n}]")
    dev = coords.device
    dcoords = (dcoords if dcoords is not None else torch.empty((V, d), dtype=torch.float32, device=dev)) \
        if need_dcoords else None
    dmid = (dmid if dmid is not None else torch.empty_like(mid)) if need_dmid else None
    dcoef = (dcoef if dcoef is not None else torch.empty(E, dtype=torch.float32, device=dev)) if need_dcoef else None
    ws_ptr, ws_bytes = 0, 0
    if dcoords is not None and reduce != REDUCE_ATOMIC:
        if ws is None:
            ws = Workspace(coords, conn, form, stream)
        ws_ptr, ws_bytes = ws.buf.data_ptr(), ws.bytes
    opts = nat.options_struct(JAC_AUTO, contract, reduce, 0, 0, dev_err.data_ptr() if dev_err is not None else 0)
    nat.fem_integrate_bwd_iso(m, form, mid.data_ptr(), _coef_ptr(coef, E), dA.data_ptr(),
                              dcoords.data_ptr() if dcoords is not None else 0,
                              dmid.data_ptr() if dmid is not None else 0,
                              dcoef.data_ptr() if dcoef is not None else 0, ws_ptr, ws_bytes, opts,
                              _stream_ptr(stream))
    return dcoords, dmid, dcoef


def adjoint_reduce(coords, conn, ws: Workspace, dcoords, stream=None):
    """fem_adjoint_reduce: completes a REDUCE_DEFERRED adjoint into dcoords."""
    m = _mesh_struct(coords, conn)
    nat.fem_adjoint_reduce(m, ws.buf.data_ptr(), ws.bytes, dcoords.data_ptr(), _stream_ptr(stream))
    return dcoords


def tune_fwd(coords, conn, form, coef=None, out=None, jac=JAC_AUTO, det_out=None, stream=None):
    """fem_tune_fwd: the fastest (warps_per_cta, ctas_per_sm) of integrate_fwd
    for this mesh and form, and its time per call in ms.  `out` (allocated if
    None) and `det_out` receive the values of one call."""
    m = _mesh_struct(coords, conn)
    rows, cols = form_shape(form, m.dim)
    E = conn.shape[0]
    if out is None:
        out = torch.empty((E, rows, cols), dtype=torch.float32, device=coords.device)
    w1 = form in (LAPLACE_P1_W1, LAPLACE_P2_W1)
    cp = _coef_ptr(coef, coords.shape[0], "[V]") if w1 else _coef_ptr(coef, E)
    if det_out is not None:
        _check_det(det_out, E)
    opts = nat.options_struct(jac, 0, 0, 0, 0, 0)
    ms = nat.fem_tune_fwd(m, form, cp, out.data_ptr(), F64 if out.dtype == torch.float64 else F32,
                          det_out.data_ptr() if det_out is not None else 0, opts, _stream_ptr(stream))
    return opts.warps_per_cta, opts.ctas_per_sm, ms


def tune_bwd(coords, conn, form, dA, coef=None, ws: Workspace | None = None, reduce=REDUCE_DETERMINISTIC,
             need_dcoef=False, jac=JAC_AUTO, det=None, dcoords=None, stream=None):
    """fem_tune_bwd: the fastest (warps_per_cta, ctas_per_sm) of integrate_bwd
    (dcoords, and dcoef if need_dcoef) for this mesh and form, and its time
    per call in ms."""
    m = _mesh_struct(coords, conn)
    E, V = conn.shape[0], coords.shape[0]
    w1 = form in (LAPLACE_P1_W1, LAPLACE_P2_W1)
    if dcoords is None:
        dcoords = torch.empty((V, m.dim), dtype=torch.float32, device=coords.device)
    dcoef = torch.empty(V if w1 else E, dtype=torch.float32, device=coords.device) if need_dcoef else None
    if ws is None and reduce != REDUCE_ATOMIC:
        ws = Workspace(coords, conn, form, stream)
    ws_ptr, ws_bytes = (ws.buf.data_ptr(), ws.bytes) if ws is not None else (0, 0)
    cp = _coef_ptr(coef, V, "[V]") if w1 else _coef_ptr(coef, E)
    if det is not None:
        _check_det(det, E)
    opts = nat.options_struct(jac, 0, reduce, 0, 0, 0)
    ms = nat.fem_tune_bwd(m, form, cp, dA.data_ptr(), det.data_ptr() if det is not None else 0, dcoords.data_ptr(),
                          dcoef.data_ptr() if dcoef is not None else 0, ws_ptr, ws_bytes, opts, _stream_ptr(stream))
    return opts.warps_per_cta, opts.ctas_per_sm, ms


class TuneCache:
    """Launch shapes chosen by tune_fwd / tune_bwd, kept in a JSON file: one
    entry per (GPU name, phase, form, dim, Jacobian mode, floor(log2 E)), so
    a mesh of another size in the same power-of-two bucket reuses the shape
    without tuning.  The file is `path`, else $FEM_TUNE_CACHE, else
    ~/.cache/paper_1103_0066_gb300/tune.json."""

    def __init__(self, path=None):
        import os
        self.path = path or os.environ.get("FEM_TUNE_CACHE") or os.path.join(
            os.path.expanduser("~"), ".cache", "paper_1103_0066_gb300", "tune.json")
        self.entries = {}
        try:
            import json
            with open(self.path) as f:
                self.entries = json.load(f)
        except (OSError, ValueError):
            self.entries = {}

    @staticmethod
    def key(phase, form, dim, jac, n_elem, gpu_name):
        name = gpu_name.replace(" ", "_")
        return f"{name}/{phase}/{form}/{dim}/{jac}/{max(int(n_elem), 1).bit_length() - 1}"

    def _save(self):
        import json
        import os
        os.makedirs(os.path.dirname(self.path) or ".", exist_ok=True)
        tmp = self.path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(self.entries, f, indent=1, sort_keys=True)
        os.replace(tmp, self.path)

    def fwd(self, coords, conn, form, jac=JAC_AUTO, **kw):
        """(warps_per_cta, ctas_per_sm) for integrate_fwd, tuned on a miss."""
        k = self.key("fwd", form, conn.shape[1] - 1, jac, conn.shape[0], torch.cuda.get_device_name(coords.device))
        if k not in self.entries:
            w, c, ms = tune_fwd(coords, conn, form, jac=jac, **kw)
            self.entries[k] = {"warps_per_cta": w, "ctas_per_sm": c, "ms": ms, "n_elem": int(conn.shape[0])}
            self._save()
        e = self.entries[k]
        return e["warps_per_cta"], e["ctas_per_sm"]

    def bwd(self, coords, conn, form, dA, jac=JAC_AUTO, **kw):
        """(warps_per_cta, ctas_per_sm) for integrate_bwd, tuned on a miss."""
        k = self.key("bwd", form, conn.shape[1] - 1, jac, conn.shape[0], torch.cuda.get_device_name(coords.device))
        if k not in self.entries:
            w, c, ms = tune_bwd(coords, conn, form, dA, jac=jac, **kw)
            self.entries[k] = {"warps_per_cta": w, "ctas_per_sm": c, "ms": ms, "n_elem": int(conn.shape[0])}
            self._save()
        e = self.entries[k]
        return e["warps_per_cta"], e["ctas_per_sm"]


class HostStep:
    """Forward and adjoint of one mesh whose inputs and outputs live in pinned
    host memory (the C ABI's fem_host_step_*).

    run() copies coords, conn and dA in, integrates A = G:K (Eq. 6) saving
    det J, runs the deterministic adjoint taking it, and copies A and dcoords
    out.  The library splits the elements in slices of `chunk` elements: a
    copy-in stream sends the coordinates, then each slice's connectivity and
    dA; the caller's stream runs each slice's forward as soon as its
    connectivity has arrived and, once the incidence is built, its adjoint
    element pass as soon as its dA has; a copy-out stream returns each slice's
    A as soon as it is written, and dcoords after the reduction.  The results
    equal the device path's bit for bit.  The caller's stream waits for the
    copies out, so an event recorded on it after run() marks the step's end."""

    def __init__(self, n_vert, n_elem, dim=3, form=LAPLACE_P1, chunk=1 << 20, device="cuda"):
        if form not in (LAPLACE_P1, LAPLACE_P2, ELASTIC_P1):
            raise ValueError("HostStep takes LAPLACE_P1, LAPLACE_P2 or ELASTIC_P1")
        self.device = torch.device(device)
        n, _, _ = form_info(form, dim)
        self.form, self.dim, self.n = form, dim, n
        self.n_vert, self.n_elem = int(n_vert), int(n_elem)
        self.chunk = max(32, (int(chunk) + 31) // 32 * 32)
        with torch.cuda.device(self.device):
            self._h = _native.fem_host_step_create(form, dim, self.n_vert, self.n_elem, self.chunk)
        self._built = False

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            torch.cuda.synchronize(self.device)
            _native.fem_host_step_destroy(h)
            self._h = None

    @staticmethod
    def _check(t, shape, dtype, name):
        if t.is_cuda or not t.is_pinned() or tuple(t.shape) != shape or t.dtype != dtype or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous pinned host tensor {shape} {dtype}")

    def run(self, coords_h, conn_h, dA_h, A_h, dcoords_h, rebuild=False):
        """One step; rebuild=True copies conn in and rebuilds the adjoint's
        incidence (a new connectivity).  Runs with rebuild=False keep the
        connectivity of the last building run on the device (conn_h is not
        read); the first run always builds."""
        V, E, d, n = self.n_vert, self.n_elem, self.dim, self.n
        for t, shape, dtype, name in ((coords_h, (V, d), torch.float32, "coords"),
                                      (conn_h, (E, d + 1), torch.int32, "conn"),
                                      (dA_h, (E, n, n), torch.float32, "dA"), (A_h, (E, n, n), torch.float32, "A"),
                                      (dcoords_h, (V, d), torch.float32, "dcoords")):
            self._check(t, shape, dtype, name)
        stream = torch.cuda.current_stream(self.device)
        with torch.cuda.device(self.device):
            _native.fem_host_step_run(self._h, coords_h.data_ptr(), conn_h.data_ptr(), dA_h.data_ptr(),
                                      A_h.data_ptr(), dcoords_h.data_ptr(), rebuild, stream.cuda_stream)
        return A_h, dcoords_h


class _IntegrateFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, coords, coef, mesh, form, jac, reduce, contract):
        # det J is kept for the adjoint when it can take it (FP32 coordinates, affine
        # form, FP32 contraction)
        keep = (coords.dtype == torch.float32
                and form in (LAPLACE_P1, LAPLACE_P2, ELASTIC_P1, DIV_P1P1, DIV_P2P1, LAPLACE_P1_W1, LAPLACE_P2_W1)
                and jac in (JAC_AUTO, JAC_COMP_F32) and contract == CONTRACT_F32)
        det = torch.empty(mesh.conn.shape[0], dtype=torch.float32, device=coords.device) if keep else None
        A = integrate_fwd(coords, mesh.conn, form, coef, jac=jac, contract=contract, det_out=det)
        ctx.det = det
        ctx.save_for_backward(coords, coef if coef is not None else torch.empty(0))
        ctx.mesh, ctx.form, ctx.jac, ctx.reduce = mesh, form, jac, reduce
        ctx.has_coef = coef is not None
        return A

    @staticmethod
    def backward(ctx, dA):
        coords, coef = ctx.saved_tensors
        coef = coef if ctx.has_coef else None
        need_x = ctx.needs_input_grad[0]
        need_w = ctx.has_coef and ctx.needs_input_grad[1]
        w1 = ctx.form in (LAPLACE_P1_W1, LAPLACE_P2_W1)
        ws = (ctx.mesh.workspace(ctx.form) if ((need_x or (w1 and need_w)) and ctx.reduce == REDUCE_DETERMINISTIC)
              else None)
        dx, dw = integrate_bwd(coords.detach(), ctx.mesh.conn, ctx.form, dA.contiguous().float(), coef,
                               ws=ws, reduce=ctx.reduce, need_dcoords=need_x, need_dcoef=need_w,
                               jac=ctx.jac, det=ctx.det)
        return dx, dw, None, None, None, None, None


class _IntegrateIsoFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, coords, mid, coef, mesh, form, reduce):
        A = integrate_fwd_iso(coords, mesh.conn, mid, form, coef)
        ctx.save_for_backward(coords, mid, coef if coef is not None else torch.empty(0))
        ctx.mesh, ctx.form, ctx.reduce, ctx.has_coef = mesh, form, reduce, coef is not None
        return A

    @staticmethod
    def backward(ctx, dA):
        coords, mid, coef = ctx.saved_tensors
        coef = coef if ctx.has_coef else None
        need_x, need_m = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        need_w = ctx.has_coef and ctx.needs_input_grad[2]
        ws = ctx.mesh.workspace(ctx.form) if (need_x and ctx.reduce != REDUCE_ATOMIC) else None
        dx, dm, dw = integrate_bwd_iso(coords.detach(), ctx.mesh.conn, mid.detach(), ctx.form,
                                       dA.contiguous().float(), coef, ws=ws, reduce=ctx.reduce,
                                       need_dcoords=need_x, need_dmid=need_m, need_dcoef=need_w)
        return dx, dm, dw, None, None, None


def integrate_iso(coords, conn, mid, form=LAPLACE_P1_ISO, coef=None, reduce=REDUCE_DETERMINISTIC, mesh=None):
    """Element matrices of the non-affine Laplacian (Eqs. 16-19), differentiable
    with respect to coords, mid (the edge nodes) and coef.  Pass a Mesh built
    on (coords, conn) to reuse its adjoint workspace across calls."""
    if coords.dtype != torch.float32 or mid.dtype != torch.float32:
        raise ValueError("non-affine elements take float32 coordinates and edge nodes")
    mesh = mesh if mesh is not None else Mesh(coords.detach(), conn)
    return _IntegrateIsoFn.apply(coords, mid, coef, mesh, form, reduce)


class Mesh:
    """A simplex mesh on the GPU: coords [V][d] (float32/float64), conn [E][d+1] int32."""

    def __init__(self, coords: torch.Tensor, conn: torch.Tensor):
        self.coords = coords
        self.conn = conn.contiguous()
        self._ws = {}

    @property
    def dim(self):
        return self.conn.shape[1] - 1

    def workspace(self, form=LAPLACE_P1) -> Workspace:
        # the P1-coefficient forms' records carry one more component: a larger workspace
        key = "w1" if form in (LAPLACE_P1_W1, LAPLACE_P2_W1) else "ws"
        if key not in self._ws:
            self._ws[key] = Workspace(self.coords.detach(), self.conn, form)
        return self._ws[key]

    def integrate(self, form, coef=None, jac=JAC_AUTO, reduce=REDUCE_DETERMINISTIC, coords=None,
                  contract=CONTRACT_F32):
        """Element matrices, differentiable with respect to coords and coef.

        contract=CONTRACT_BF16X3 contracts the forward on the tensor cores (P2 and
        elasticity); the adjoint is the FP32 one either way."""
        x = self.coords if coords is None else coords
        if x.dtype != torch.float32 and (x.requires_grad or (coef is not None and coef.requires_grad)):
            raise ValueError("the adjoint takes float32 coordinates")
        return _IntegrateFn.apply(x, coef, self, form, jac, reduce, contract)


def integrate(coords, conn, form, coef=None, jac=JAC_AUTO, reduce=REDUCE_DETERMINISTIC, contract=CONTRACT_F32):
    """Differentiable element matrices for a one-off mesh (builds the incidence on first backward)."""
    return Mesh(coords, conn).integrate(form, coef, jac, reduce, contract=contract)


class Batch:
    """Many meshes of mixed forms integrated by one persistent launch (fem_batch_*).

    items: sequence of dicts with CUDA tensors ``coords`` [V][d] float32, ``conn``
    [E][d+1] int32, ``form``, and optional ``coef``, ``A`` (forward output),
    ``dA``, ``dcoords``, ``dcoef`` (adjoint).  The tensors must outlive the batch.
    """

    def __init__(self, items, stream=None):
        self._keep = []
        arr = (nat.FemBatchItem * len(items))()
        for k, it in enumerate(items):
            m = _mesh_struct(it["coords"], it["conn"])
            if m.coord_dtype != F32:
                raise ValueError("batched meshes take float32 coordinates")
            E = it["conn"].shape[0]
            ptr = {}
            for name in ("coef", "A", "dA", "dcoords", "dcoef"):
                t = it.get(name)
                if t is not None:
                    if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
                        raise ValueError(f"item {k}: {name} must be a contiguous CUDA float32 tensor")
                    self._keep.append(t)
                ptr[name] = t.data_ptr() if t is not None else None
            if ptr["coef"] is not None and it["coef"].numel() != E:
                raise ValueError(f"item {k}: coef must have n_elem entries")
            self._keep += [it["coords"], it["conn"]]
            arr[k] = nat.FemBatchItem(m, it["form"], 0, ptr["coef"], ptr["A"], ptr["dA"], ptr["dcoords"],
                                      ptr["dcoef"])
        self._items = arr
        self.ws_bytes = nat.fem_batch_workspace_size(arr)
        dev = items[0]["coords"].device
        self.ws = torch.empty(max(self.ws_bytes, 256), dtype=torch.uint8, device=dev)
        self.handle = nat.fem_batch_create(arr, self.ws.data_ptr(), self.ws_bytes, _stream_ptr(stream))

    def tune(self, phases=PHASE_FWD | PHASE_BWD, stream=None):
        nat.fem_batch_tune(self.handle, phases, _stream_ptr(stream))
        return self.config()

    def config(self):
        """(CTAs per SM, work-chunk size, mode) used by run(); mode is one of
        BATCH_SINGLE, BATCH_GROUPED, BATCH_GROUPED_CONCURRENT, BATCH_PER_ITEM,
        BATCH_PER_ITEM_CONCURRENT, BATCH_PHASED."""
        return nat.fem_batch_config(self.handle)

    def set_config(self, ctas_per_sm, chunk, mode):
        nat.fem_batch_set_config(self.handle, ctas_per_sm, chunk, mode)

    def run(self, phases=PHASE_FWD | PHASE_BWD, stream=None):
        nat.fem_batch_run(self.handle, phases, _stream_ptr(stream))

    def errors(self, stream=None) -> int:
        return nat.fem_batch_errors(self.handle, _stream_ptr(stream))

    def inject_wait(self, item, extra_tiles, spin_limit=0, stream=None):
        """Test hook (fem_batch_inject_wait): item's reduction waits for
        extra_tiles more tiles than exist, each wait bounded by spin_limit
        polls; inject_wait(item, 0) restores normal runs."""
        nat.fem_batch_inject_wait(self.handle, item, extra_tiles, spin_limit, _stream_ptr(stream))

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            nat.fem_batch_destroy(h)
            self.handle = None
