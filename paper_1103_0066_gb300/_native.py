"""ctypes binding of libfem_gb300 (the C ABI in include/fem.h).

Argument marshalling only: every computation runs in the library's CUDA
kernels.  If the library is missing this module raises; there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libfem_gb300.so")

FEM_OK, FEM_ERR_ARG, FEM_ERR_UNSUPPORTED, FEM_ERR_WORKSPACE, FEM_ERR_CUDA = range(5)
LAPLACE_P1, LAPLACE_P2, ELASTIC_P1, LAPLACE_P1_W1, LAPLACE_P2_W1, LAPLACE_P1_ISO, LAPLACE_P2_ISO = range(7)
DIV_P1P1, DIV_P2P1 = 7, 8
F32, F64 = 0, 1
JAC_AUTO, JAC_F64, JAC_COMP_F32, JAC_F32 = 0, 1, 2, 3
CONTRACT_F32, CONTRACT_BF16X3 = 0, 1
REDUCE_DETERMINISTIC, REDUCE_ATOMIC, REDUCE_DEFERRED = 0, 1, 2
DEVERR_CONN, DEVERR_DEGENERATE = 1, 2

# every symbol include/fem.h declares
EXPORTS = ("fem_version", "fem_status_string", "fem_last_error", "fem_form_info", "fem_form_shape",
           "fem_reference_tensor", "fem_integrate_fwd", "fem_geometry", "fem_bwd_workspace_size",
           "fem_incidence_build", "fem_incidence_info", "fem_integrate_bwd", "fem_adjoint_reduce", "fem_integrate_bwd_noalloc",
           "fem_batch_workspace_size", "fem_batch_create", "fem_batch_tune", "fem_batch_config", "fem_batch_set_config", "fem_batch_run",
           "fem_batch_errors", "fem_batch_inject_wait", "fem_batch_destroy", "fem_assembly_workspace_size", "fem_assembly_build",
           "fem_assembly_pattern", "fem_assemble", "fem_integrate_fwd_iso", "fem_integrate_fwd_save",
           "fem_integrate_bwd_saved", "fem_host_step_create", "fem_host_step_run", "fem_host_step_destroy", "fem_tune_fwd",
           "fem_tune_bwd", "fem_integrate_bwd_iso", "fem_assembly_unknowns", "fem_mesh_order_workspace_size",
           "fem_mesh_order", "fem_mesh_renumber")
PHASE_FWD, PHASE_BWD = 1, 2
BATCH_SINGLE, BATCH_GROUPED, BATCH_GROUPED_CONCURRENT, BATCH_PER_ITEM, BATCH_PER_ITEM_CONCURRENT = 0, 1, 2, 3, 4
BATCH_PHASED = 5
DEVERR_TIMEOUT = 4
RECORDS_VERTEX_MAJOR, RECORDS_TILE_ORDER = 0, 1
NOALLOC_SCRATCH_BYTES = 32 << 20


class FemError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_status_name(status)}: {msg}")
        self.status = status


class FemMesh(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("coord_dtype", ctypes.c_int32),
                ("n_vert", ctypes.c_int64), ("n_elem", ctypes.c_int64),
                ("conn", ctypes.c_void_p), ("coords", ctypes.c_void_p)]


class FemOptions(ctypes.Structure):
    _fields_ = [("jac", ctypes.c_int32), ("contract", ctypes.c_int32), ("reduce", ctypes.c_int32),
                ("warps_per_cta", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("dev_err", ctypes.c_void_p)]


class FemBatchItem(ctypes.Structure):
    _fields_ = [("mesh", FemMesh), ("form", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("coef", ctypes.c_void_p), ("A", ctypes.c_void_p), ("dA", ctypes.c_void_p),
                ("dcoords", ctypes.c_void_p), ("dcoef", ctypes.c_void_p)]


_lock = threading.Lock()
_lib = None


def load():
    """Loads the library (it must have been built, e.g. by __graft_entry__.build())."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libfem_gb300.so is not built ({LIB_PATH}); run "
                               "`python -m paper_1103_0066_gb300.build`")
        lib = ctypes.CDLL(LIB_PATH)
        P, I32, I64, SZ = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
        MP, OP = ctypes.POINTER(FemMesh), ctypes.POINTER(FemOptions)
        sig = {
            "fem_version": ([], ctypes.c_char_p),
            "fem_status_string": ([ctypes.c_int], ctypes.c_char_p),
            "fem_last_error": ([], ctypes.c_char_p),
            "fem_form_info": ([I32, I32, P, P, P], ctypes.c_int),
            "fem_form_shape": ([I32, I32, P, P], ctypes.c_int),
            "fem_reference_tensor": ([I32, I32, P, SZ], ctypes.c_int),
            "fem_integrate_fwd": ([MP, I32, P, P, I32, OP, P], ctypes.c_int),
            "fem_integrate_fwd_iso": ([MP, I32, P, P, P, OP, P], ctypes.c_int),
            "fem_integrate_fwd_save": ([MP, I32, P, P, I32, P, OP, P], ctypes.c_int),
            "fem_integrate_bwd_saved": ([MP, I32, P, P, P, P, P, P, SZ, OP, P], ctypes.c_int),
            "fem_integrate_bwd_iso": ([MP, I32, P, P, P, P, P, P, P, SZ, OP, P], ctypes.c_int),
            "fem_geometry": ([MP, P, OP, P, P, P], ctypes.c_int),
            "fem_bwd_workspace_size": ([MP, I32, OP, ctypes.POINTER(SZ)], ctypes.c_int),
            "fem_incidence_build": ([MP, P, SZ, P], ctypes.c_int),
            "fem_incidence_info": ([MP, P, SZ, ctypes.POINTER(I64), ctypes.POINTER(I32), P], ctypes.c_int),
            "fem_integrate_bwd": ([MP, I32, P, P, P, P, P, SZ, OP, P], ctypes.c_int),
            "fem_adjoint_reduce": ([MP, P, SZ, P, P], ctypes.c_int),
            "fem_integrate_bwd_noalloc": ([MP, I32, P, P, P, P, OP, P], ctypes.c_int),
            "fem_batch_workspace_size": ([ctypes.POINTER(FemBatchItem), I32, ctypes.POINTER(SZ)], ctypes.c_int),
            "fem_batch_create": ([ctypes.POINTER(FemBatchItem), I32, P, SZ, ctypes.POINTER(P), P], ctypes.c_int),
            "fem_batch_tune": ([P, I32, P], ctypes.c_int),
            "fem_batch_config": ([P, ctypes.POINTER(I32), ctypes.POINTER(I32), ctypes.POINTER(I32)], ctypes.c_int),
            "fem_batch_set_config": ([P, I32, I32, I32], ctypes.c_int),
            "fem_batch_run": ([P, I32, P], ctypes.c_int),
            "fem_batch_errors": ([P, ctypes.POINTER(I32), P], ctypes.c_int),
            "fem_batch_inject_wait": ([P, I32, I64, ctypes.c_uint32, P], ctypes.c_int),
            "fem_batch_destroy": ([P], None),
            "fem_assembly_workspace_size": ([MP, I32, ctypes.POINTER(SZ)], ctypes.c_int),
            "fem_assembly_build": ([MP, I32, P, SZ, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64), P],
                                   ctypes.c_int),
            "fem_assembly_pattern": ([MP, I32, P, SZ, ctypes.POINTER(P), ctypes.POINTER(P)], ctypes.c_int),
            "fem_assemble": ([MP, I32, P, P, SZ, P, P], ctypes.c_int),
            "fem_assembly_unknowns": ([MP, I32, P, SZ, ctypes.POINTER(I64), ctypes.POINTER(P)], ctypes.c_int),
            "fem_mesh_order_workspace_size": ([MP, ctypes.POINTER(SZ)], ctypes.c_int),
            "fem_mesh_order": ([MP, P, SZ, P, P, P], ctypes.c_int),
            "fem_mesh_renumber": ([MP, P, P, P, SZ, P, P, P], ctypes.c_int),
            "fem_host_step_create": ([I32, I32, I64, I64, I64, ctypes.POINTER(P)], ctypes.c_int),
            "fem_host_step_run": ([P, P, P, P, P, P, I32, P], ctypes.c_int),
            "fem_host_step_destroy": ([P], None),
            "fem_tune_fwd": ([MP, I32, P, P, I32, P, OP, ctypes.POINTER(ctypes.c_float), P], ctypes.c_int),
            "fem_tune_bwd": ([MP, I32, P, P, P, P, P, P, SZ, OP, ctypes.POINTER(ctypes.c_float), P], ctypes.c_int),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def _status_name(s: int) -> str:
    try:
        return load().fem_status_string(s).decode()
    except Exception:  # noqa: BLE001 - used while formatting another error
        return f"status {s}"


def check(status: int) -> None:
    if status != FEM_OK:
        raise FemError(status, load().fem_last_error().decode())


def mesh_struct(dim: int, coord_dtype: int, n_vert: int, n_elem: int, conn_ptr: int,
                coords_ptr: int) -> FemMesh:
    return FemMesh(dim, coord_dtype, n_vert, n_elem, conn_ptr or None, coords_ptr or None)


def options_struct(jac=JAC_AUTO, contract=CONTRACT_F32, reduce=REDUCE_DETERMINISTIC, warps_per_cta=0,
                   ctas_per_sm=0, dev_err_ptr=0) -> FemOptions:
    return FemOptions(jac, contract, reduce, warps_per_cta, ctas_per_sm, 0, dev_err_ptr or None)


def version() -> str:
    return load().fem_version().decode()


def fem_form_info(form: int, dim: int):
    n, ng, den = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    check(load().fem_form_info(form, dim, ctypes.byref(n), ctypes.byref(ng), ctypes.byref(den)))
    return n.value, ng.value, den.value


def fem_form_shape(form: int, dim: int):
    r, c = ctypes.c_int32(), ctypes.c_int32()
    check(load().fem_form_shape(form, dim, ctypes.byref(r), ctypes.byref(c)))
    return r.value, c.value


def fem_reference_tensor(form: int, dim: int, out_ptr: int, cap: int) -> None:
    check(load().fem_reference_tensor(form, dim, out_ptr, cap))


def fem_integrate_fwd(mesh: FemMesh, form: int, coef_ptr: int, A_ptr: int, out_dtype: int,
                      opts: FemOptions, stream: int) -> None:
    check(load().fem_integrate_fwd(ctypes.byref(mesh), form, coef_ptr or None, A_ptr or None,
                                   out_dtype, ctypes.byref(opts), stream or None))


def fem_integrate_fwd_save(mesh: FemMesh, form: int, coef_ptr: int, A_ptr: int, out_dtype: int, det_ptr: int,
                           opts: FemOptions, stream: int) -> None:
    check(load().fem_integrate_fwd_save(ctypes.byref(mesh), form, coef_ptr or None, A_ptr or None, out_dtype,
                                        det_ptr or None, ctypes.byref(opts), stream or None))


def fem_integrate_fwd_iso(mesh: FemMesh, form: int, mid_ptr: int, coef_ptr: int, A_ptr: int, opts: FemOptions,
                          stream: int) -> None:
    check(load().fem_integrate_fwd_iso(ctypes.byref(mesh), form, mid_ptr or None, coef_ptr or None, A_ptr or None,
                                       ctypes.byref(opts), stream or None))


def fem_geometry(mesh: FemMesh, coef_ptr: int, opts: FemOptions, det_ptr: int, G_ptr: int,
                 stream: int) -> None:
    check(load().fem_geometry(ctypes.byref(mesh), coef_ptr or None, ctypes.byref(opts),
                              det_ptr or None, G_ptr or None, stream or None))


def fem_bwd_workspace_size(mesh: FemMesh, form: int, opts: FemOptions) -> int:
    b = ctypes.c_size_t()
    check(load().fem_bwd_workspace_size(ctypes.byref(mesh), form, ctypes.byref(opts), ctypes.byref(b)))
    return b.value


def fem_incidence_build(mesh: FemMesh, ws_ptr: int, ws_bytes: int, stream: int) -> None:
    check(load().fem_incidence_build(ctypes.byref(mesh), ws_ptr or None, ws_bytes, stream or None))


def fem_incidence_info(mesh: FemMesh, ws_ptr: int, ws_bytes: int, stream: int):
    n, lay = ctypes.c_int64(), ctypes.c_int32()
    check(load().fem_incidence_info(ctypes.byref(mesh), ws_ptr or None, ws_bytes, ctypes.byref(n), ctypes.byref(lay),
                                    stream or None))
    return n.value, lay.value


def fem_integrate_bwd(mesh: FemMesh, form: int, coef_ptr: int, dA_ptr: int, dcoords_ptr: int,
                      dcoef_ptr: int, ws_ptr: int, ws_bytes: int, opts: FemOptions, stream: int) -> None:
    check(load().fem_integrate_bwd(ctypes.byref(mesh), form, coef_ptr or None, dA_ptr or None,
                                   dcoords_ptr or None, dcoef_ptr or None, ws_ptr or None, ws_bytes,
                                   ctypes.byref(opts), stream or None))


def fem_adjoint_reduce(mesh: FemMesh, ws_ptr: int, ws_bytes: int, dcoords_ptr: int, stream: int) -> None:
    check(load().fem_adjoint_reduce(ctypes.byref(mesh), ws_ptr or None, ws_bytes, dcoords_ptr or None,
                                    stream or None))


def fem_integrate_bwd_saved(mesh: FemMesh, form: int, coef_ptr: int, dA_ptr: int, det_ptr: int, dcoords_ptr: int,
                            dcoef_ptr: int, ws_ptr: int, ws_bytes: int, opts: FemOptions, stream: int) -> None:
    check(load().fem_integrate_bwd_saved(ctypes.byref(mesh), form, coef_ptr or None, dA_ptr or None, det_ptr or None,
                                         dcoords_ptr or None, dcoef_ptr or None, ws_ptr or None, ws_bytes,
                                         ctypes.byref(opts), stream or None))


def fem_integrate_bwd_noalloc(mesh: FemMesh, form: int, coef_ptr: int, dA_ptr: int, dcoords_ptr: int,
                              dcoef_ptr: int, opts: FemOptions, stream: int) -> None:
    check(load().fem_integrate_bwd_noalloc(ctypes.byref(mesh), form, coef_ptr or None, dA_ptr or None,
                                           dcoords_ptr or None, dcoef_ptr or None, ctypes.byref(opts),
                                           stream or None))


def fem_batch_workspace_size(items) -> int:
    b = ctypes.c_size_t()
    check(load().fem_batch_workspace_size(items, len(items), ctypes.byref(b)))
    return b.value


def fem_batch_create(items, ws_ptr: int, ws_bytes: int, stream: int) -> int:
    h = ctypes.c_void_p()
    check(load().fem_batch_create(items, len(items), ws_ptr, ws_bytes, ctypes.byref(h), stream or None))
    return h.value


def fem_batch_tune(handle: int, phases: int, stream: int) -> None:
    check(load().fem_batch_tune(handle, phases, stream or None))


def fem_batch_config(handle: int):
    c, k, m = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    check(load().fem_batch_config(handle, ctypes.byref(c), ctypes.byref(k), ctypes.byref(m)))
    return c.value, k.value, m.value


def fem_batch_set_config(handle: int, ctas_per_sm: int, chunk: int, mode: int) -> None:
    check(load().fem_batch_set_config(handle, ctas_per_sm, chunk, mode))


def fem_batch_run(handle: int, phases: int, stream: int) -> None:
    check(load().fem_batch_run(handle, phases, stream or None))


def fem_batch_errors(handle: int, stream: int) -> int:
    e = ctypes.c_int32()
    check(load().fem_batch_errors(handle, ctypes.byref(e), stream or None))
    return e.value


def fem_batch_inject_wait(handle: int, item: int, extra_tiles: int, spin_limit: int, stream: int) -> None:
    check(load().fem_batch_inject_wait(handle, item, extra_tiles, spin_limit, stream or None))


def fem_batch_destroy(handle: int) -> None:
    load().fem_batch_destroy(handle)


def fem_assembly_workspace_size(mesh: FemMesh, form: int) -> int:
    b = ctypes.c_size_t()
    check(load().fem_assembly_workspace_size(ctypes.byref(mesh), form, ctypes.byref(b)))
    return b.value


def fem_assembly_build(mesh: FemMesh, form: int, ws_ptr: int, ws_bytes: int, stream: int):
    nnz, nrec = ctypes.c_int64(), ctypes.c_int64()
    check(load().fem_assembly_build(ctypes.byref(mesh), form, ws_ptr, ws_bytes, ctypes.byref(nnz), ctypes.byref(nrec),
                                    stream or None))
    return nnz.value, nrec.value


def fem_assembly_pattern(mesh: FemMesh, form: int, ws_ptr: int, ws_bytes: int):
    rp, ci = ctypes.c_void_p(), ctypes.c_void_p()
    check(load().fem_assembly_pattern(ctypes.byref(mesh), form, ws_ptr, ws_bytes, ctypes.byref(rp), ctypes.byref(ci)))
    return rp.value or 0, ci.value or 0


def fem_assemble(mesh: FemMesh, form: int, A_ptr: int, ws_ptr: int, ws_bytes: int, values_ptr: int,
                 stream: int) -> None:
    check(load().fem_assemble(ctypes.byref(mesh), form, A_ptr or None, ws_ptr, ws_bytes, values_ptr or None,
                              stream or None))


def fem_host_step_create(form: int, dim: int, n_vert: int, n_elem: int, chunk: int) -> int:
    h = ctypes.c_void_p()
    check(load().fem_host_step_create(form, dim, n_vert, n_elem, chunk, ctypes.byref(h)))
    return h.value


def fem_host_step_run(handle: int, coords_ptr: int, conn_ptr: int, dA_ptr: int, A_ptr: int, dcoords_ptr: int,
                      rebuild: bool, stream: int) -> None:
    check(load().fem_host_step_run(handle, coords_ptr or None, conn_ptr or None, dA_ptr or None, A_ptr or None,
                                   dcoords_ptr or None, 1 if rebuild else 0, stream or None))


def fem_host_step_destroy(handle: int) -> None:
    load().fem_host_step_destroy(handle)


def fem_tune_fwd(mesh: FemMesh, form: int, coef_ptr: int, A_ptr: int, out_dtype: int, det_ptr: int,
                 opts: FemOptions, stream: int) -> float:
    ms = ctypes.c_float()
    check(load().fem_tune_fwd(ctypes.byref(mesh), form, coef_ptr or None, A_ptr or None, out_dtype, det_ptr or None,
                              ctypes.byref(opts), ctypes.byref(ms), stream or None))
    return ms.value


def fem_tune_bwd(mesh: FemMesh, form: int, coef_ptr: int, dA_ptr: int, det_ptr: int, dcoords_ptr: int,
                 dcoef_ptr: int, ws_ptr: int, ws_bytes: int, opts: FemOptions, stream: int) -> float:
    ms = ctypes.c_float()
    check(load().fem_tune_bwd(ctypes.byref(mesh), form, coef_ptr or None, dA_ptr or None, det_ptr or None,
                              dcoords_ptr or None, dcoef_ptr or None, ws_ptr or None, ws_bytes, ctypes.byref(opts),
                              ctypes.byref(ms), stream or None))
    return ms.value


def fem_integrate_bwd_iso(mesh: FemMesh, form: int, mid_ptr: int, coef_ptr: int, dA_ptr: int, dcoords_ptr: int,
                          dmid_ptr: int, dcoef_ptr: int, ws_ptr: int, ws_bytes: int, opts: FemOptions,
                          stream: int) -> None:
    check(load().fem_integrate_bwd_iso(ctypes.byref(mesh), form, mid_ptr or None, coef_ptr or None, dA_ptr or None,
                                       dcoords_ptr or None, dmid_ptr or None, dcoef_ptr or None, ws_ptr or None,
                                       ws_bytes, ctypes.byref(opts), stream or None))


def fem_mesh_order_workspace_size(mesh: FemMesh) -> int:
    b = ctypes.c_size_t()
    check(load().fem_mesh_order_workspace_size(ctypes.byref(mesh), ctypes.byref(b)))
    return b.value


def fem_mesh_order(mesh: FemMesh, ws_ptr: int, ws_bytes: int, elem_perm: int, vert_perm: int, stream: int):
    check(load().fem_mesh_order(ctypes.byref(mesh), ws_ptr, ws_bytes, elem_perm, vert_perm, stream))


def fem_mesh_renumber(mesh: FemMesh, elem_perm: int, vert_perm: int, ws_ptr: int, ws_bytes: int, coords_out: int,
                      conn_out: int, stream: int):
    check(load().fem_mesh_renumber(ctypes.byref(mesh), elem_perm, vert_perm, ws_ptr, ws_bytes, coords_out, conn_out,
                                   stream))


def fem_assembly_unknowns(mesh: FemMesh, form: int, ws_ptr: int, ws_bytes: int):
    n, d = ctypes.c_int64(), ctypes.c_void_p()
    check(load().fem_assembly_unknowns(ctypes.byref(mesh), form, ws_ptr, ws_bytes, ctypes.byref(n), ctypes.byref(d)))
    return n.value, d.value or 0
