"""C-ABI checks that need no GPU: the library loads, exports every symbol the
header declares, its host-side reference tensor K reproduces the oracle's
direct quadrature through Eq. 6, and host-detectable errors return status
codes before any launch."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LP1, LP2, EP1 = 0, 1, 2


@pytest.fixture(scope="module")
def fem():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1103_0066_gb300 as fem
    return fem


def _declared_symbols():
    src = open(os.path.join(ROOT, "include", "fem.h")).read()
    return sorted(set(re.findall(r"FEM_API\s+[\w\s\*]+?\b(fem_\w+)\s*\(", src)))


def test_exports_every_declared_symbol(fem):
    lib = fem.nat.load()
    declared = _declared_symbols()
    assert len(declared) >= 10
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(fem.nat.EXPORTS) == declared
    assert "sm_103a" in fem.nat.version()


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("form", [3, 4])
def test_reference_tensor_p1_coefficient(fem, orc, dim, form):
    """Eq. 22: A = sum_k w_k G : K^{.. k} with the library's arity-3 K equals the
    oracle's direct quadrature with the P1 coefficient of vertex values w_k."""
    K, den = fem.reference_tensor(form, dim)
    K = K.numpy().astype(np.float64)
    n, ng, _ = fem.form_info(form, dim)
    ngb = dim * (dim + 1) // 2
    assert ng == (dim + 1) * ngb and K.shape == (ng, n, n) and den == (120 if dim == 2 else 720)
    rng = np.random.default_rng(13)
    for trial in range(8):
        X = rng.standard_normal((dim + 1, dim)) if trial else np.vstack([np.zeros(dim), np.eye(dim)])
        if abs(np.linalg.det(X[1:] - X[0])) < 0.05:
            continue
        wv = np.exp(rng.standard_normal(dim + 1))
        G = np.concatenate([wv[k] * _G_true(LP1, X) for k in range(dim + 1)])
        A = np.einsum("g,gij->ij", G, K) / den
        Ar, _, _ = orc.element_matrix_w1(dim, form - 3, X, wv)
        assert np.abs(A - Ar).max() < 1e-12 * np.abs(Ar).max()


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("form", [5, 6])
def test_reference_tensor_non_affine(fem, orc, dim, form):
    """Eqs. 18-19: A = G^{(k mu),(l nu)} K^{ij}_{(k mu),(l nu)} with the library's
    K and G = |det J(centroid)| J^{-1}_k J^{-1}_l^T built here from the quadratic
    geometry map equals the oracle's quadrature on curved elements."""
    K, den = fem.reference_tensor(form, dim)
    K = K.numpy().astype(np.float64)
    n, ng, _ = fem.form_info(form, dim)
    npair = (dim + 1) * dim
    assert ng == npair * (npair + 1) // 2 and den == (720 if dim == 2 else 5040)
    rng = np.random.default_rng(14)
    edges = [(a, b) for a in range(dim + 1) for b in range(a + 1, dim + 1)]
    for _ in range(6):
        X = np.vstack([np.zeros(dim), np.eye(dim)]) + 0.1 * rng.standard_normal((dim + 1, dim))
        M = np.array([0.5 * (X[a] + X[b]) for a, b in edges]) + 0.05 * rng.standard_normal((len(edges), dim))
        nodes = np.vstack([X, M])

        def jac(xi):  # J[alpha][mu] of the quadratic map
            _, g = orc.basis(dim, 2, xi)
            return nodes.T @ g

        verts = [np.zeros(dim)] + [np.eye(dim)[k] for k in range(dim)]
        Ji = [np.linalg.inv(jac(v)) for v in verts]            # Ji[k][mu][alpha]
        detc = abs(np.linalg.det(jac(np.full(dim, 1.0 / (dim + 1)))))
        slots = [(k, mu) for k in range(dim + 1) for mu in range(dim)]
        G = [detc * Ji[slots[p][0]][slots[p][1]] @ Ji[slots[q][0]][slots[q][1]]
             for p in range(npair) for q in range(p, npair)]
        A = np.einsum("g,gij->ij", np.array(G), K) / den
        Ar, _, _ = orc.element_matrix_iso(dim, form - 5, X, M)
        assert np.abs(A - Ar).max() < 1e-12 * np.abs(Ar).max()


@pytest.mark.parametrize("dim", [2, 3])
def test_form_info(fem, dim):
    assert fem.form_info(LP1, dim) == (dim + 1, dim * (dim + 1) // 2, 24 if dim == 2 else 120)
    nb2 = (dim + 1) * (dim + 2) // 2
    assert fem.form_info(LP2, dim)[0] == nb2
    n, ng, den = fem.form_info(EP1, dim)
    assert n == dim * (dim + 1) and ng == dim * dim * (dim * dim + 1) // 2 and den == 2 * (24 if dim == 2 else 120)


def _G_true(form, X):
    """Folded geometric tensor of Eq. 8 (and its symmetric-gradient analogue),
    written out with numpy for one element: |J| Jinv Jinv^T."""
    dim = X.shape[1]
    J = (X[1:] - X[0]).T            # J[a][mu]
    B = np.linalg.inv(J)            # B[mu][a] = d xi_mu / d x_a
    s = abs(np.linalg.det(J))
    if form != EP1:
        M = s * B @ B.T
        return np.array([M[m, n] for m in range(dim) for n in range(m, dim)])
    b = B.ravel()                   # p = mu*d + a
    M = s * np.outer(b, b)
    npp = dim * dim
    return np.array([M[p, q] for p in range(npp) for q in range(p, npp)])


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("form", [LP1, LP2, EP1])
def test_reference_tensor_reproduces_quadrature(fem, orc, dim, form):
    """Eq. 6: A = G : K with the library's K equals the oracle's direct quadrature."""
    K, den = fem.reference_tensor(form, dim)
    K = K.numpy().astype(np.float64)
    n = K.shape[1]
    assert np.array_equal(K, np.transpose(K, (0, 2, 1)))   # folded K' symmetric in (i, j)
    rng = np.random.default_rng(12)
    for trial in range(10):
        X = rng.standard_normal((dim + 1, dim)) if trial else np.vstack([np.zeros(dim), np.eye(dim)])
        if abs(np.linalg.det(X[1:] - X[0])) < 0.05:
            continue
        A = np.einsum("g,gij->ij", _G_true(form, X), K) / den
        Ar, _, _ = orc.element_matrix(dim, form, X)
        assert np.abs(A - Ar).max() < 1e-12 * np.abs(Ar).max()
    if dim == 3 and form == EP1:
        assert int((K != 0).sum()) == 513


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("vdeg", [1, 2])
def test_coupling_shape_and_reference_tensor(fem, orc, dim, vdeg):
    """The coupling blocks int q div v: fem_form_shape gives (d+1, d * nbv), and
    B = sum_g G_g K_g / den with G_{mu c} = |J| J^{-1}_{mu c} (numpy) and the
    library's K equals the oracle's direct quadrature."""
    form = 6 + vdeg
    nbv = dim + 1 if vdeg == 1 else (dim + 1) * (dim + 2) // 2
    assert fem.form_shape(form, dim) == (dim + 1, dim * nbv) == orc.div_shape(dim, vdeg)
    assert fem.form_shape(LP2, dim) == (fem.form_info(LP2, dim)[0],) * 2
    n, ng, den = fem.form_info(form, dim)
    assert (n, ng, den) == (dim + 1, dim * dim, 24 if dim == 2 else 120)
    K, den = fem.reference_tensor(form, dim)
    K = K.numpy().astype(np.float64)
    assert K.shape == (dim * dim, dim + 1, dim * nbv)
    rng = np.random.default_rng(13)
    for trial in range(8):
        X = rng.standard_normal((dim + 1, dim)) if trial else np.vstack([np.zeros(dim), np.eye(dim)])
        J = (X[1:] - X[0]).T
        if abs(np.linalg.det(J)) < 0.05:
            continue
        G = (abs(np.linalg.det(J)) * np.linalg.inv(J)).ravel()      # g = mu * d + c
        B = np.einsum("g,gij->ij", G, K) / den
        Br, _, _ = orc.element_matrix_div(dim, vdeg, X)
        assert np.abs(B - Br).max() < 1e-12 * np.abs(Br).max()


def _mesh(fem, dim=3, dtype=0, n_elem=10, conn=0x1000, coords=0x2000):
    return fem.nat.mesh_struct(dim, dtype, 100, n_elem, conn, coords)


def test_host_detected_errors(fem):
    nat = fem.nat
    lib = nat.load()
    opts = nat.options_struct()
    A = ctypes.c_void_p(0x3000)
    # NULL mesh
    assert lib.fem_integrate_fwd(None, LP1, None, A, 0, ctypes.byref(opts), None) == nat.FEM_ERR_ARG
    assert "mesh" in lib.fem_last_error().decode()
    # bad dim / form / dtype
    m = _mesh(fem, dim=4)
    assert lib.fem_integrate_fwd(ctypes.byref(m), LP1, None, A, 0, ctypes.byref(opts), None) == nat.FEM_ERR_ARG
    m = _mesh(fem)
    assert lib.fem_integrate_fwd(ctypes.byref(m), 9, None, A, 0, ctypes.byref(opts), None) == nat.FEM_ERR_ARG
    assert lib.fem_integrate_fwd(ctypes.byref(m), LP1, None, A, 5, ctypes.byref(opts), None) == nat.FEM_ERR_ARG
    # NULL output / NULL conn with elements
    assert lib.fem_integrate_fwd(ctypes.byref(m), LP1, None, None, 0, ctypes.byref(opts), None) == nat.FEM_ERR_ARG
    m0 = _mesh(fem, conn=0)
    assert lib.fem_integrate_fwd(ctypes.byref(m0), LP1, None, A, 0, ctypes.byref(opts), None) == nat.FEM_ERR_ARG
    # options out of range
    for bad in (nat.options_struct(jac=9), nat.options_struct(warps_per_cta=17),
                nat.options_struct(reduce=3), nat.FemOptions(0, 0, 0, 0, 0, 1, None)):
        assert lib.fem_integrate_fwd(ctypes.byref(m), LP1, None, A, 0, ctypes.byref(bad), None) == nat.FEM_ERR_ARG
    # FP64 coordinates with a FP32 Jacobian mode: unsupported combination
    m64 = _mesh(fem, dtype=1)
    o = nat.options_struct(jac=nat.JAC_COMP_F32)
    assert lib.fem_integrate_fwd(ctypes.byref(m64), LP1, None, A, 0, ctypes.byref(o), None) == nat.FEM_ERR_UNSUPPORTED
    # empty mesh: a no-op that launches nothing
    me = _mesh(fem, n_elem=0)
    assert lib.fem_integrate_fwd(ctypes.byref(me), LP1, None, None, 0, None, None) == nat.FEM_OK
    # adjoint: FP64 coordinates unsupported, workspace checks
    assert lib.fem_integrate_bwd(ctypes.byref(m64), LP1, None, A, A, None, None, 0, None, None) == nat.FEM_ERR_UNSUPPORTED
    assert lib.fem_integrate_bwd(ctypes.byref(m), LP1, None, A, A, None, None, 0, None, None) == nat.FEM_ERR_WORKSPACE
    big = fem.nat.mesh_struct(3, 0, 100, 2 ** 30, 0x1000, 0x2000)
    b = ctypes.c_size_t()
    assert lib.fem_bwd_workspace_size(ctypes.byref(big), LP1, None, ctypes.byref(b)) == nat.FEM_ERR_UNSUPPORTED
    assert lib.fem_bwd_workspace_size(ctypes.byref(m), LP1, None, ctypes.byref(b)) == nat.FEM_OK
    assert b.value >= 4 * (101 + 40) + 4 * 10 * 4 * 3
    with pytest.raises(fem.FemError):
        fem.nat.fem_form_info(9, 3)


def test_tensor_core_combinations_rejected_on_host(fem):
    nat = fem.nat
    lib = nat.load()
    A = ctypes.c_void_p(0x3000)
    m = _mesh(fem)
    tc = nat.options_struct(contract=nat.CONTRACT_BF16X3)
    # P1 Laplacian has no tensor-core path; FP64 output neither; nor a plain-FP32 Jacobian
    assert lib.fem_integrate_fwd(ctypes.byref(m), LP1, None, A, 0, ctypes.byref(tc), None) == nat.FEM_ERR_UNSUPPORTED
    assert lib.fem_integrate_fwd(ctypes.byref(m), EP1, None, A, 1, ctypes.byref(tc), None) == nat.FEM_ERR_UNSUPPORTED
    tc32 = nat.options_struct(jac=nat.JAC_F32, contract=nat.CONTRACT_BF16X3)
    assert lib.fem_integrate_fwd(ctypes.byref(m), EP1, None, A, 0, ctypes.byref(tc32), None) == nat.FEM_ERR_UNSUPPORTED
    # P1 with a P1 coefficient has none either (P2 with one has)
    assert lib.fem_integrate_fwd(ctypes.byref(m), 3, None, A, 0, ctypes.byref(tc), None) == nat.FEM_ERR_UNSUPPORTED


def test_saved_det_and_iso_contract_errors_on_host(fem):
    """fem_integrate_fwd_save / fem_integrate_bwd_saved refuse a NULL det and
    the tensor-core contraction; fem_integrate_fwd_iso takes BF16X3 only for
    the P2 form.  All detected on the host, before any launch."""
    nat = fem.nat
    lib = nat.load()
    A = ctypes.c_void_p(0x3000)
    m = _mesh(fem)
    opts = nat.options_struct()
    assert lib.fem_integrate_fwd_save(ctypes.byref(m), LP1, None, A, 0, None, ctypes.byref(opts), None) == nat.FEM_ERR_ARG
    tc = nat.options_struct(contract=nat.CONTRACT_BF16X3)
    assert lib.fem_integrate_fwd_save(ctypes.byref(m), EP1, None, A, 0, A, ctypes.byref(tc), None) == nat.FEM_ERR_UNSUPPORTED
    assert lib.fem_integrate_bwd_saved(ctypes.byref(m), LP1, None, A, None, A, None, None, 0, None, None) == nat.FEM_ERR_ARG
    assert lib.fem_integrate_bwd_saved(ctypes.byref(m), 5, None, A, A, A, None, None, 0, None, None) == nat.FEM_ERR_UNSUPPORTED
    # the P1-coefficient adjoint reduces dcoef through the workspace: missing workspace
    assert lib.fem_integrate_bwd_saved(ctypes.byref(m), 3, None, A, A, A, None, None, 0, None, None) == nat.FEM_ERR_WORKSPACE
    b = ctypes.c_size_t()
    assert lib.fem_bwd_workspace_size(ctypes.byref(m), 3, None, ctypes.byref(b)) == nat.FEM_OK
    b0 = ctypes.c_size_t()
    assert lib.fem_bwd_workspace_size(ctypes.byref(m), LP1, None, ctypes.byref(b0)) == nat.FEM_OK
    assert b.value > b0.value  # records of d + 1 components
    me = _mesh(fem, n_elem=0)
    assert lib.fem_integrate_fwd_save(ctypes.byref(me), LP1, None, None, 0, None, None, None) == nat.FEM_OK
    assert lib.fem_integrate_fwd_iso(ctypes.byref(m), 5, A, None, A, ctypes.byref(tc), None) == nat.FEM_ERR_UNSUPPORTED


def test_host_step_refusals_on_host(fem):
    """fem_host_step_*: every argument refusal comes before any CUDA call."""
    nat = fem.nat
    lib = nat.load()
    h = ctypes.c_void_p()
    assert lib.fem_host_step_create(nat.DIV_P1P1, 3, 10, 10, 0, ctypes.byref(h)) == nat.FEM_ERR_UNSUPPORTED
    assert lib.fem_host_step_create(LP1, 3, 10, 10, 0, None) == nat.FEM_ERR_ARG
    assert lib.fem_host_step_create(LP1, 4, 10, 10, 0, ctypes.byref(h)) == nat.FEM_ERR_ARG
    assert lib.fem_host_step_create(LP1, 3, 0, 10, 0, ctypes.byref(h)) == nat.FEM_ERR_ARG
    assert lib.fem_host_step_create(LP1, 3, 10, 10, -1, ctypes.byref(h)) == nat.FEM_ERR_ARG
    assert lib.fem_host_step_create(LP1, 3, 10, 1 << 30, 0, ctypes.byref(h)) == nat.FEM_ERR_UNSUPPORTED
    assert not h.value
    p = ctypes.c_void_p(0x3000)
    assert lib.fem_host_step_run(None, p, p, p, p, p, 0, None) == nat.FEM_ERR_ARG
    lib.fem_host_step_destroy(None)  # no-op


def test_mesh_order_refusals_on_host(fem):
    """fem_mesh_order / fem_mesh_renumber: argument refusals come before any
    CUDA call, and the workspace size is a host computation."""
    nat = fem.nat
    lib = nat.load()
    p = ctypes.c_void_p(0x3000)
    b = ctypes.c_size_t()
    m = _mesh(fem)
    assert lib.fem_mesh_order_workspace_size(ctypes.byref(m), ctypes.byref(b)) == nat.FEM_OK and b.value > 0
    assert lib.fem_mesh_order_workspace_size(None, ctypes.byref(b)) == nat.FEM_ERR_ARG
    assert lib.fem_mesh_order_workspace_size(ctypes.byref(m), None) == nat.FEM_ERR_ARG
    m64 = _mesh(fem, dtype=1)
    assert lib.fem_mesh_order_workspace_size(ctypes.byref(m64), ctypes.byref(b)) == nat.FEM_ERR_UNSUPPORTED
    m4 = _mesh(fem, dim=4)
    assert lib.fem_mesh_order(ctypes.byref(m4), p, 1 << 30, p, p, None) == nat.FEM_ERR_ARG
    assert lib.fem_mesh_order(ctypes.byref(m), p, 1 << 30, None, p, None) == nat.FEM_ERR_ARG
    assert lib.fem_mesh_order(ctypes.byref(m), None, 0, p, p, None) == nat.FEM_ERR_WORKSPACE
    assert lib.fem_mesh_renumber(ctypes.byref(m), p, p, p, 1 << 30, None, p, None) == nat.FEM_ERR_ARG
    assert lib.fem_mesh_renumber(ctypes.byref(m), p, p, None, 0, p, p, None) == nat.FEM_ERR_WORKSPACE


def test_iso_adjoint_contract_refusals_on_host(fem):
    """fem_integrate_bwd_iso takes FEM_CONTRACT_BF16X3 for the P2 form on
    tetrahedra with the deterministic or deferred reduction only."""
    nat = fem.nat
    lib = nat.load()
    A = ctypes.c_void_p(0x3000)
    tc = nat.options_struct(contract=nat.CONTRACT_BF16X3)
    tca = nat.options_struct(contract=nat.CONTRACT_BF16X3, reduce=nat.REDUCE_ATOMIC)
    m3, m2 = _mesh(fem), _mesh(fem, dim=2)
    for mesh, form, opts in ((m3, nat.LAPLACE_P1_ISO, tc), (m2, nat.LAPLACE_P2_ISO, tc),
                             (m3, nat.LAPLACE_P2_ISO, tca)):
        assert lib.fem_integrate_bwd_iso(ctypes.byref(mesh), form, A, None, A, A, None, None, None, 0,
                                         ctypes.byref(opts), None) == nat.FEM_ERR_UNSUPPORTED
