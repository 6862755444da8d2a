"""FP64 CPU oracle for finite element integration by direct quadrature.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product library
never imports this package, and this package imports nothing from it.

The arithmetic lives in ``fem_oracle.c`` (plain C, FP64, OpenMP over elements);
this module compiles it with gcc and marshals numpy arrays through ctypes.

What it computes (Knepley & Terrel, Sec. 3):
  * ``integrate``: element matrices by quadrature of Eqs. 3-5 (Laplacian) and of
    Eq. 10 scaled by the 1/4 of Eq. 14 / Eq. 24 (elasticity eps:eps), times a
    per-element constant coefficient (piecewise-constant case of Eq. 20).
  * ``integrate_vjp``: the hand-derived reverse mode of the same steps;
    ``integrate_w1_vjp`` that of the P1-coefficient Laplacian (Eqs. 20-23),
    with the gradient of the coefficient's vertex values.
  * ``integrate_div`` / ``integrate_div_vjp``: the coupling block of a
    multiphysics pair, B = int q div v with q in P1 and v in [P1]^d or
    [P2]^d (Sec. 6's blocks of coupled systems; Eq. 1 with one derivative in
    K), by the same quadrature, and its reverse mode.
  * ``simplex_rule`` / ``basis`` / ``element_matrix``: the building blocks,
    exposed so the tests can pin each one separately.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

LAPLACE_P1, LAPLACE_P2, ELASTIC_P1 = 0, 1, 2
FLAG_CONN, FLAG_DEGENERATE = 1, 2

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fem_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libfem_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``fem_oracle.c`` into ``libfem_oracle.so`` next to it (gcc, -O2, OpenMP)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True)  # no OpenMP runtime: single-threaded oracle
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P, I, I64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
        D = ctypes.c_double
        lib.orc_max_threads.restype = I
        lib.orc_gauss_legendre01.argtypes = [I, P, P]
        lib.orc_simplex_rule.argtypes = [I, I, P, P]
        lib.orc_basis.argtypes = [I, I, P, P, P]
        lib.orc_n_basis.argtypes = [I, I]
        lib.orc_form_n.argtypes = [I, I]
        lib.orc_element_matrix.argtypes = [I, I, P, D, I, P, P]
        lib.orc_element_vjp.argtypes = [I, I, P, D, I, P, P, P]
        lib.orc_integrate.argtypes = [I, I, I64, I64, P, P, P, I, P, P, P, I]
        lib.orc_integrate_vjp.argtypes = [I, I, I64, I64, P, P, P, I, P, P, P, I]
        lib.orc_element_matrix_w1.argtypes = [I, I, P, P, I, P, P]
        lib.orc_integrate_w1.argtypes = [I, I, I64, I64, P, P, P, I, P, P, I]
        lib.orc_element_matrix_iso.argtypes = [I, I, P, P, D, I, P, P]
        lib.orc_integrate_iso.argtypes = [I, I, I64, I64, P, P, P, P, I, P, P, I]
        lib.orc_element_vjp_w1.argtypes = [I, I, P, P, I, P, P, P]
        lib.orc_integrate_w1_vjp.argtypes = [I, I, I64, I64, P, P, P, I, P, P, P, I]
        lib.orc_element_matrix_div.argtypes = [I, I, P, D, I, P, P]
        lib.orc_element_vjp_div.argtypes = [I, I, P, D, I, P, P, P]
        lib.orc_integrate_div.argtypes = [I, I, I64, I64, P, P, P, I, P, P, I]
        lib.orc_integrate_div_vjp.argtypes = [I, I, I64, I64, P, P, P, I, P, P, P, I]
        lib.orc_element_vjp_iso.argtypes = [I, I, P, P, D, I, P, P, P, P]
        lib.orc_integrate_iso_vjp.argtypes = [I, I, I64, I64, P, P, P, P, I, P, P, P, P, I]
        for name in ("orc_element_vjp_iso", "orc_integrate_iso_vjp", "orc_element_vjp_w1", "orc_integrate_w1_vjp", "orc_element_matrix_div", "orc_element_vjp_div",
                     "orc_integrate_div",
                     "orc_integrate_div_vjp", "orc_gauss_legendre01", "orc_simplex_rule", "orc_basis", "orc_n_basis",
                     "orc_form_n", "orc_element_matrix", "orc_element_vjp", "orc_integrate",
                     "orc_integrate_vjp", "orc_element_matrix_w1", "orc_integrate_w1",
                     "orc_element_matrix_iso", "orc_integrate_iso"):
            getattr(lib, name).restype = I
        _lib = lib
        return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def max_threads() -> int:
    return _load().orc_max_threads()


def form_n(form: int, dim: int) -> int:
    """Rows of the element matrix: basis functions times components."""
    return _load().orc_form_n(form, dim)


def gauss_legendre01(q: int):
    x = np.zeros(q)
    w = np.zeros(q)
    if _load().orc_gauss_legendre01(q, _ptr(x), _ptr(w)) != 0:
        raise ValueError("q out of range")
    return x, w


def simplex_rule(dim: int, q: int):
    """Duffy-collapsed Gauss rule on the reference simplex: (points [np][dim], weights [np])."""
    pts = np.zeros((q ** dim, dim))
    wts = np.zeros(q ** dim)
    n = _load().orc_simplex_rule(dim, q, _ptr(pts), _ptr(wts))
    if n < 0:
        raise ValueError("bad rule request")
    return pts[:n], wts[:n]


def basis(dim: int, degree: int, xi):
    """Values [nb] and reference gradients [nb][dim] of the P1/P2 basis at xi."""
    xi = _f64(xi)
    nb = _load().orc_n_basis(dim, degree)
    phi = np.zeros(nb)
    grad = np.zeros((nb, dim))
    _load().orc_basis(dim, degree, _ptr(xi), _ptr(phi), _ptr(grad))
    return phi, grad


def element_matrix(dim: int, form: int, X, coef: float = 1.0, q: int = 3):
    """Element matrix of one element with vertex coordinates X [dim+1][dim]."""
    X = _f64(X)
    n = form_n(form, dim)
    A = np.zeros((n, n))
    det = np.zeros(1)
    rc = _load().orc_element_matrix(dim, form, _ptr(X), float(coef), q, _ptr(A), _ptr(det))
    if rc < 0:
        raise ValueError("bad element request")
    return A, float(det[0]), rc


def element_matrix_w1(dim: int, form: int, X, wv, q: int = 3):
    """Element matrix of a Laplacian form (LAPLACE_P1 or LAPLACE_P2) with the P1
    coefficient of vertex values wv [dim+1] (Eqs. 20-23)."""
    X = _f64(X)
    wv = _f64(wv)
    n = form_n(form, dim)
    A = np.zeros((n, n))
    det = np.zeros(1)
    rc = _load().orc_element_matrix_w1(dim, form, _ptr(X), _ptr(wv), q, _ptr(A), _ptr(det))
    if rc < 0:
        raise ValueError("bad element request")
    return A, float(det[0]), rc


def integrate_w1(dim: int, form: int, conn, coords, wvert, q: int = 3, nthreads: int | None = None):
    """Element matrices [E][n][n] (FP64) and flags of a Laplacian form with the P1
    coefficient whose values at the mesh vertices are wvert [V]."""
    conn = np.ascontiguousarray(conn, dtype=np.int32)
    coords = _f64(coords)
    wvert = _f64(wvert)
    E, V = conn.shape[0], coords.shape[0]
    if wvert.shape != (V,):
        raise ValueError("wvert must have one value per vertex")
    n = form_n(form, dim)
    A = np.zeros((E, n, n))
    flags = np.zeros(E, dtype=np.int32)
    nt = max_threads() if nthreads is None else nthreads
    rc = _load().orc_integrate_w1(dim, form, E, V, _ptr(conn), _ptr(coords), _ptr(wvert), q, _ptr(A),
                                  _ptr(flags), nt)
    if rc < 0:
        raise ValueError("bad integrate request")
    return A, flags


def element_vjp_w1(dim: int, form: int, X, wv, Abar, q: int = 3):
    """Reverse mode of element_matrix_w1: (Xbar [dim+1][dim], wbar [dim+1])."""
    X = _f64(X)
    wv = _f64(wv)
    Abar = _f64(Abar)
    Xbar = np.zeros_like(X)
    wbar = np.zeros(dim + 1)
    rc = _load().orc_element_vjp_w1(dim, form, _ptr(X), _ptr(wv), q, _ptr(Abar), _ptr(Xbar), _ptr(wbar))
    if rc < 0:
        raise ValueError("bad element request")
    return Xbar, wbar


def integrate_w1_vjp(dim: int, form: int, conn, coords, wvert, dA, q: int = 3, nthreads: int | None = None):
    """Reverse mode of integrate_w1: (dcoords [V][dim], dwvert [V]) for dA [E][n][n]."""
    conn = np.ascontiguousarray(conn, dtype=np.int32)
    coords = _f64(coords)
    wvert = _f64(wvert)
    dA = _f64(dA)
    E, V = conn.shape[0], coords.shape[0]
    dcoords = np.zeros((V, dim))
    dw = np.zeros(V)
    nt = max_threads() if nthreads is None else nthreads
    rc = _load().orc_integrate_w1_vjp(dim, form, E, V, _ptr(conn), _ptr(coords), _ptr(wvert), q, _ptr(dA),
                                      _ptr(dcoords), _ptr(dw), nt)
    if rc < 0:
        raise ValueError("bad vjp request")
    return dcoords, dw


def element_matrix_iso(dim: int, form: int, X, mid, coef: float = 1.0, q: int = 4):
    """Element matrix of a Laplacian form on a non-affine element (Eqs. 16-19):
    X [dim+1][dim] vertices, mid [n_edges][dim] edge-midpoint nodes (P2 edge
    order).  Returns (A, det J at the centroid, flags)."""
    X = _f64(X)
    mid = _f64(mid)
    n = form_n(form, dim)
    A = np.zeros((n, n))
    det = np.zeros(1)
    rc = _load().orc_element_matrix_iso(dim, form, _ptr(X), _ptr(mid), float(coef), q, _ptr(A), _ptr(det))
    if rc < 0:
        raise ValueError("bad element request")
    return A, float(det[0]), rc


def integrate_iso(dim: int, form: int, conn, coords, mid, coef=None, q: int = 4, nthreads: int | None = None):
    """Element matrices [E][n][n] (FP64) and flags of a Laplacian form on
    non-affine elements whose edge-midpoint nodes are mid [E][n_edges][dim]."""
    conn = np.ascontiguousarray(conn, dtype=np.int32)
    coords = _f64(coords)
    mid = _f64(mid)
    E, V = conn.shape[0], coords.shape[0]
    ne = 3 if dim == 2 else 6
    if mid.shape != (E, ne, dim):
        raise ValueError("mid must be [E][n_edges][dim]")
    n = form_n(form, dim)
    cf = None if coef is None else _f64(coef)
    A = np.zeros((E, n, n))
    flags = np.zeros(E, dtype=np.int32)
    nt = max_threads() if nthreads is None else nthreads
    rc = _load().orc_integrate_iso(dim, form, E, V, _ptr(conn), _ptr(coords), _ptr(mid), _ptr(cf), q, _ptr(A),
                                   _ptr(flags), nt)
    if rc < 0:
        raise ValueError("bad integrate request")
    return A, flags


def element_vjp_iso(dim: int, form: int, X, mid, Abar, coef: float = 1.0, q: int = 4):
    """Reverse mode of element_matrix_iso: (Xbar [dim+1][dim], midbar
    [n_edges][dim], coefbar, flags) for Abar = dL/dA [n][n]."""
    X = _f64(X)
    mid = _f64(mid)
    Abar = _f64(Abar)
    Xbar = np.zeros_like(X)
    midbar = np.zeros_like(mid)
    cbar = np.zeros(1)
    rc = _load().orc_element_vjp_iso(dim, form, _ptr(X), _ptr(mid), float(coef), q, _ptr(Abar), _ptr(Xbar),
                                     _ptr(midbar), _ptr(cbar))
    if rc < 0:
        raise ValueError("bad vjp request")
    return Xbar, midbar, float(cbar[0]), rc


def integrate_iso_vjp(dim: int, form: int, conn, coords, mid, dA, coef=None, q: int = 4,
                      nthreads: int | None = None):
    """Reverse mode of integrate_iso: (dcoords [V][dim], dmid [E][n_edges][dim],
    dcoef [E]) for dA [E][n][n]."""
    conn = np.ascontiguousarray(conn, dtype=np.int32)
    coords = _f64(coords)
    mid = _f64(mid)
    dA = _f64(dA)
    E, V = conn.shape[0], coords.shape[0]
    cf = None if coef is None else _f64(coef)
    dcoords = np.zeros((V, dim))
    dmid = np.zeros_like(mid)
    dcoef = np.zeros(E)
    nt = max_threads() if nthreads is None else nthreads
    rc = _load().orc_integrate_iso_vjp(dim, form, E, V, _ptr(conn), _ptr(coords), _ptr(mid), _ptr(cf), q, _ptr(dA),
                                       _ptr(dcoords), _ptr(dmid), _ptr(dcoef), nt)
    if rc < 0:
        raise ValueError("bad vjp request")
    return dcoords, dmid, dcoef


def element_vjp(dim: int, form: int, X, Abar, coef: float = 1.0, q: int = 3):
    X = _f64(X)
    Abar = _f64(Abar)
    Xbar = np.zeros_like(X)
    cbar = np.zeros(1)
    rc = _load().orc_element_vjp(dim, form, _ptr(X), float(coef), q, _ptr(Abar), _ptr(Xbar),
                                 _ptr(cbar))
    if rc < 0:
        raise ValueError("bad element request")
    return Xbar, float(cbar[0])


def integrate(dim: int, form: int, conn, coords, coef=None, q: int = 3, nthreads: int | None = None,
              return_det: bool = False):
    """Element matrices A [E][n][n] (FP64) and per-element flags [E] (int32).

    coords are taken exactly as FP64 whatever their storage type."""
    conn = np.ascontiguousarray(conn, dtype=np.int32)
    coords = _f64(coords)
    E = conn.shape[0]
    V = coords.shape[0]
    n = form_n(form, dim)
    cf = None if coef is None else _f64(coef)
    A = np.zeros((E, n, n))
    flags = np.zeros(E, dtype=np.int32)
    det = np.zeros(E)
    nt = max_threads() if nthreads is None else nthreads
    rc = _load().orc_integrate(dim, form, E, V, _ptr(conn), _ptr(coords), _ptr(cf), q, _ptr(A),
                               _ptr(flags), _ptr(det), nt)
    if rc < 0:
        raise ValueError("bad integrate request")
    if return_det:
        return A, flags, det
    return A, flags


def integrate_vjp(dim: int, form: int, conn, coords, dA, coef=None, q: int = 3,
                  nthreads: int | None = None):
    """Reverse mode: (dcoords [V][dim], dcoef [E]) for the upstream dA [E][n][n]."""
    conn = np.ascontiguousarray(conn, dtype=np.int32)
    coords = _f64(coords)
    dA = _f64(dA)
    E = conn.shape[0]
    V = coords.shape[0]
    cf = None if coef is None else _f64(coef)
    dcoords = np.zeros((V, dim))
    dcoef = np.zeros(E)
    nt = max_threads() if nthreads is None else nthreads
    rc = _load().orc_integrate_vjp(dim, form, E, V, _ptr(conn), _ptr(coords), _ptr(cf), q,
                                   _ptr(dA), _ptr(dcoords), _ptr(dcoef), nt)
    if rc < 0:
        raise ValueError("bad vjp request")
    return dcoords, dcoef


def div_shape(dim: int, vdeg: int):
    """(rows, columns) of the coupling block: d+1 P1 rows, d * n_basis(vdeg) columns."""
    return dim + 1, dim * _load().orc_n_basis(dim, vdeg)


def element_matrix_div(dim: int, vdeg: int, X, coef: float = 1.0, q: int = 3):
    """Coupling block B [d+1][d * nbv] of one element: B_{i,(c,j)} = int coef
    phi_i d psi_j / d x_c (phi P1, psi P`vdeg`, column c * nbv + j).  Returns
    (B, det J, flags)."""
    X = _f64(X)
    B = np.zeros(div_shape(dim, vdeg))
    det = np.zeros(1)
    rc = _load().orc_element_matrix_div(dim, vdeg, _ptr(X), float(coef), q, _ptr(B), _ptr(det))
    if rc < 0:
        raise ValueError("bad element request")
    return B, float(det[0]), rc


def element_vjp_div(dim: int, vdeg: int, X, Bbar, coef: float = 1.0, q: int = 3):
    X = _f64(X)
    Bbar = _f64(Bbar)
    Xbar = np.zeros_like(X)
    cbar = np.zeros(1)
    rc = _load().orc_element_vjp_div(dim, vdeg, _ptr(X), float(coef), q, _ptr(Bbar), _ptr(Xbar), _ptr(cbar))
    if rc < 0:
        raise ValueError("bad element request")
    return Xbar, float(cbar[0])


def integrate_div(dim: int, vdeg: int, conn, coords, coef=None, q: int = 3, nthreads: int | None = None):
    """Coupling blocks B [E][d+1][d * nbv] (FP64) and per-element flags."""
    conn = np.ascontiguousarray(conn, dtype=np.int32)
    coords = _f64(coords)
    E, V = conn.shape[0], coords.shape[0]
    cf = None if coef is None else _f64(coef)
    B = np.zeros((E,) + div_shape(dim, vdeg))
    flags = np.zeros(E, dtype=np.int32)
    nt = max_threads() if nthreads is None else nthreads
    rc = _load().orc_integrate_div(dim, vdeg, E, V, _ptr(conn), _ptr(coords), _ptr(cf), q, _ptr(B), _ptr(flags), nt)
    if rc < 0:
        raise ValueError("bad integrate request")
    return B, flags


def integrate_div_vjp(dim: int, vdeg: int, conn, coords, dB, coef=None, q: int = 3, nthreads: int | None = None):
    """Reverse mode of integrate_div: (dcoords [V][dim], dcoef [E]) for dB [E][d+1][d * nbv]."""
    conn = np.ascontiguousarray(conn, dtype=np.int32)
    coords = _f64(coords)
    dB = _f64(dB)
    E, V = conn.shape[0], coords.shape[0]
    if dB.shape != (E,) + div_shape(dim, vdeg):
        raise ValueError("dB must be [E][d+1][d * nbv]")
    cf = None if coef is None else _f64(coef)
    dcoords = np.zeros((V, dim))
    dcoef = np.zeros(E)
    nt = max_threads() if nthreads is None else nthreads
    rc = _load().orc_integrate_div_vjp(dim, vdeg, E, V, _ptr(conn), _ptr(coords), _ptr(cf), q, _ptr(dB),
                                       _ptr(dcoords), _ptr(dcoef), nt)
    if rc < 0:
        raise ValueError("bad vjp request")
    return dcoords, dcoef


def p2_dofs(dim: int, conn, n_vert: int):
    """Global unknowns of the P2 basis over a mesh: the vertices 0 .. V-1,
    then one per edge, V + k for the k-th distinct edge in increasing
    (lower vertex, higher vertex) order.  Returns (dofs [E][n], n_unknowns)
    with the element's unknowns in the local P2 order (vertices, then edges
    (0,1),(0,2),...)."""
    conn = np.asarray(conn, dtype=np.int64)
    pairs = [(a, b) for a in range(dim + 1) for b in range(a + 1, dim + 1)]
    lo = np.stack([np.minimum(conn[:, a], conn[:, b]) for a, b in pairs], axis=1)
    hi = np.stack([np.maximum(conn[:, a], conn[:, b]) for a, b in pairs], axis=1)
    uniq, inv = np.unique((lo * int(n_vert) + hi).ravel(), return_inverse=True)
    return np.concatenate([conn, int(n_vert) + inv.reshape(lo.shape)], axis=1), int(n_vert) + len(uniq)


def assemble(dim: int, form: int, conn, n_vert: int, A):
    """Global matrix sum_e P_e^T A_e P_e of the element matrices A [E][n][n]
    (FP64 scipy CSR over scalar unknowns): every element entry is placed at its
    global (row, column) and duplicates are summed (scipy's COO -> CSR
    conversion).  Unknown v for the P1 Laplacian; for P1 elasticity the
    node-major unknown v*dim + c of the local unknown (c, i) = row
    c*(dim+1) + i of A_e; for the P2 Laplacian the unknowns of p2_dofs."""
    import scipy.sparse as sps
    conn = np.asarray(conn, dtype=np.int64)
    A = np.asarray(A, dtype=np.float64)
    E, nv = conn.shape
    if form == ELASTIC_P1:
        g = (conn[:, None, :] * dim + np.arange(dim)[None, :, None]).reshape(E, dim * nv)
        N = n_vert * dim
    elif form == LAPLACE_P1:
        g = conn
        N = n_vert
    elif form == LAPLACE_P2:
        g, N = p2_dofs(dim, conn, n_vert)
    else:
        raise ValueError("assembly of the Laplacian (P1, P2) and P1 elasticity")
    n = g.shape[1]
    if A.shape != (E, n, n):
        raise ValueError("A must be [E][n][n]")
    rows = np.repeat(g, n, axis=1).ravel()
    cols = np.tile(g, (1, n)).ravel()
    M = sps.coo_matrix((A.reshape(-1), (rows, cols)), shape=(N, N)).tocsr()
    M.sum_duplicates()
    M.sort_indices()
    return M
