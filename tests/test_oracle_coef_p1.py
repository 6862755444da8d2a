"""Pins for the oracle's Laplacian with a P1 coefficient (Eqs. 20-23), no GPU.

The coefficient is w = sum_k w_k lambda_k, given by its vertex values, and
A_ij = int_T w grad(phi_i).grad(phi_j).  Every check comes from mathematics:
exact barycentric integrals of cubic integrands, symbolic reference tensors
K^{ij k} = int_ref lambda_k grad(phi_i).grad(phi_j) (Eq. 21), the special cases
w constant and P1 elements, and independence of the quadrature rule.
"""
import itertools
import math

import numpy as np
import pytest

LP1, LP2 = 0, 1


def _ref(dim):
    return np.vstack([np.zeros(dim), np.eye(dim)])


def _rand_simplex(rng, dim, scale=1.0):
    while True:
        X = rng.standard_normal((dim + 1, dim)) * scale
        if abs(np.linalg.det(X[1:] - X[0])) > 0.05 * scale ** dim:
            return X


def _volume(X):
    d = X.shape[1]
    return abs(np.linalg.det(X[1:] - X[0])) / math.factorial(d)


def _p2_nodes(X):
    dim = X.shape[1]
    nodes = [X[i] for i in range(dim + 1)]
    for i in range(dim + 1):
        for j in range(i + 1, dim + 1):
            nodes.append(0.5 * (X[i] + X[j]))
    return np.array(nodes)


def _exact_weighted_energy(X, wv, gradfun):
    """int_T w |grad u|^2 for w = sum_m wv[m] lambda_m and a quadratic u whose
    gradient is the linear field gradfun (grad u = sum_k c_k lambda_k with
    c_k = grad u(x_k)).  Barycentric identity: int_T lambda^a = |T| d! a! / (|a| + d)!,
    so for three factors the multiplicity is 6 (all equal), 2 (two equal), 1."""
    d = X.shape[1]
    c = np.array([gradfun(x) for x in X])
    G = c @ c.T
    tot = 0.0
    for m, k, l in itertools.product(range(d + 1), repeat=3):
        mult = 6 if m == k == l else (2 if (m == k or m == l or k == l) else 1)
        tot += wv[m] * G[k, l] * mult
    return _volume(X) * math.factorial(d) / math.factorial(d + 3) * tot


@pytest.mark.parametrize("dim", [2, 3])
def test_w1_exact_energy_of_quadratics(orc, dim):
    rng = np.random.default_rng(21)
    for _ in range(20):
        X = _rand_simplex(rng, dim)
        wv = np.exp(rng.standard_normal(dim + 1))
        M = rng.standard_normal((dim, dim))
        M = M + M.T
        b = rng.standard_normal(dim)
        nodes = _p2_nodes(X)
        u = np.einsum("ni,ij,nj->n", nodes, M, nodes) + nodes @ b
        A, _, rc = orc.element_matrix_w1(dim, LP2, X, wv)
        assert rc == 0
        ex = _exact_weighted_energy(X, wv, lambda x: 2 * M @ x + b)
        assert abs(u @ A @ u - ex) < 1e-11 * abs(ex)
        # a linear u in P1: grad u = b is constant, so u^T A u = |b|^2 |T| mean(w)
        u1 = X @ b - 0.4
        A1, _, _ = orc.element_matrix_w1(dim, LP1, X, wv)
        assert abs(u1 @ A1 @ u1 - b @ b * _volume(X) * wv.mean()) < 1e-12 * (b @ b) * _volume(X) * wv.max()


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("form", [LP1, LP2])
def test_w1_constant_coefficient_is_p0(orc, dim, form):
    rng = np.random.default_rng(22)
    for _ in range(10):
        X = _rand_simplex(rng, dim)
        c = float(np.exp(rng.standard_normal()))
        A, _, _ = orc.element_matrix_w1(dim, form, X, np.full(dim + 1, c))
        B, _, _ = orc.element_matrix(dim, form, X, coef=c)
        assert np.abs(A - B).max() <= 1e-13 * np.abs(B).max()


@pytest.mark.parametrize("dim", [2, 3])
def test_w1_p1_elements_see_the_mean(orc, dim):
    """P1 gradients are constant and int_T lambda_k = |T|/(d+1), so the P1
    Laplacian with a P1 coefficient is the per-element one with w = mean(w_k)."""
    rng = np.random.default_rng(23)
    for _ in range(10):
        X = _rand_simplex(rng, dim)
        wv = np.exp(rng.standard_normal(dim + 1))
        A, _, _ = orc.element_matrix_w1(dim, LP1, X, wv)
        B, _, _ = orc.element_matrix(dim, LP1, X, coef=float(wv.mean()))
        assert np.abs(A - B).max() <= 1e-13 * np.abs(B).max()


def test_w1_symbolic_reference_tensors(orc):
    """K^{ij k} = int_ref lambda_k grad(phi_i).grad(phi_j) (Eq. 21) by exact
    symbolic integration, against the oracle on the reference simplex with
    the coefficient lambda_k (vertex values e_k)."""
    sp = pytest.importorskip("sympy")
    for dim in (2, 3):
        xi = sp.symbols(f"x0:{dim}")
        lam = [1 - sum(xi)] + list(xi)
        p2 = [l * (2 * l - 1) for l in lam] + [4 * lam[i] * lam[j] for i in range(dim + 1)
                                             for j in range(i + 1, dim + 1)]

        def integ(f):
            expr = sp.expand(f)
            for k in range(dim - 1, -1, -1):
                expr = sp.integrate(expr, (xi[k], 0, 1 - sum(xi[:k])))
            return expr

        for form, basis in ((LP1, lam), (LP2, p2)):
            grads = [[sp.diff(b, v) for v in xi] for b in basis]
            n = len(basis)
            for k in range(dim + 1):
                S = np.array([[float(integ(lam[k] * sum(grads[i][m] * grads[j][m] for m in range(dim))))
                               for j in range(n)] for i in range(n)])
                A, _, _ = orc.element_matrix_w1(dim, form, _ref(dim), np.eye(dim + 1)[k])
                assert np.abs(A - S).max() < 1e-14 * np.abs(S).max(), (dim, form, k)


@pytest.mark.parametrize("dim", [2, 3])
def test_w1_rule_independence_and_linearity(orc, dim):
    rng = np.random.default_rng(24)
    for _ in range(5):
        X = _rand_simplex(rng, dim)
        w1, w2 = np.exp(rng.standard_normal((2, dim + 1)))
        A3, _, _ = orc.element_matrix_w1(dim, LP2, X, w1, q=3)
        A5, _, _ = orc.element_matrix_w1(dim, LP2, X, w1, q=5)
        assert np.abs(A3 - A5).max() <= 1e-14 * np.abs(A5).max()
        B, _, _ = orc.element_matrix_w1(dim, LP2, X, w2)
        C, _, _ = orc.element_matrix_w1(dim, LP2, X, 0.5 * w1 - 2.0 * w2)
        assert np.abs(C - (0.5 * A3 - 2.0 * B)).max() <= 1e-13 * np.abs(C).max()


def test_w1_mesh_driver_gathers_vertex_values(orc):
    """orc.integrate_w1 over a mesh equals the element routine fed each element's
    own vertex values; bad connectivity is flagged and zeroed."""
    from paper_1103_0066_gb300 import meshgen as mg
    mesh = mg.cube_tet_mesh(2, 0.15, mg.rng_for(25), 0.0, np.float64)
    rng = np.random.default_rng(26)
    wvert = np.exp(rng.standard_normal(mesh.n_vert))
    conn = mesh.conn.copy()
    conn[3, 1] = mesh.n_vert + 5
    A, flags = orc.integrate_w1(3, LP2, conn, mesh.coords, wvert)
    assert flags[3] == 1 and np.all(A[3] == 0)
    for e in (0, 7, mesh.n_elem - 1):
        Ae, _, _ = orc.element_matrix_w1(3, LP2, mesh.coords[conn[e]], wvert[conn[e]])
        assert np.array_equal(A[e], Ae)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("form", [0, 1])
def test_w1_vjp_pins(orc, dim, form):
    """Reverse mode of the P1-coefficient Laplacian (Eqs. 20-23): the
    coordinate and coefficient gradients against FP64 central differences of
    the forward, and identities that hold exactly -- translation invariance,
    homogeneity sum_k x_k . xbar_k = (d-2) L, and linearity in w:
    sum_k w_k wbar_k = L."""
    rng = np.random.default_rng(20 + dim + 3 * form)
    X = np.vstack([np.zeros(dim), np.eye(dim)]) + 0.25 * rng.standard_normal((dim + 1, dim))
    if np.linalg.det(X[1:] - X[0]) < 0:
        X[[1, 2]] = X[[2, 1]]
    wv = np.exp(rng.standard_normal(dim + 1))
    n = orc.form_n(form, dim)
    Abar = rng.standard_normal((n, n))
    Xbar, wbar = orc.element_vjp_w1(dim, form, X, wv, Abar)
    L = np.sum(Abar * orc.element_matrix_w1(dim, form, X, wv)[0])
    h = 1e-6
    fdx = np.zeros_like(X)
    for k in range(dim + 1):
        for a in range(dim):
            Xp, Xm = X.copy(), X.copy()
            Xp[k, a] += h
            Xm[k, a] -= h
            fdx[k, a] = (np.sum(Abar * orc.element_matrix_w1(dim, form, Xp, wv)[0])
                         - np.sum(Abar * orc.element_matrix_w1(dim, form, Xm, wv)[0])) / (2 * h)
    fdw = np.zeros(dim + 1)
    hw = 0.5  # L is linear in w: a large step is exact and keeps roundoff out
    for k in range(dim + 1):
        wp, wm = wv.copy(), wv.copy()
        wp[k] += hw
        wm[k] -= hw
        fdw[k] = (np.sum(Abar * orc.element_matrix_w1(dim, form, X, wp)[0])
                  - np.sum(Abar * orc.element_matrix_w1(dim, form, X, wm)[0])) / (2 * hw)
    assert np.abs(Xbar - fdx).max() <= 1e-7 * np.abs(fdx).max()
    assert np.abs(wbar - fdw).max() <= 1e-7 * np.abs(fdw).max()
    assert np.abs(Xbar.sum(0)).max() <= 1e-12 * np.abs(Xbar).max()
    assert abs(np.sum(X * Xbar) - (dim - 2) * L) <= 1e-12 * max(1.0, abs(L))
    assert abs(np.dot(wv, wbar) - L) <= 1e-12 * max(1.0, abs(L))
    # constant coefficient: the coordinate gradient is the per-element-coefficient one
    Xc, _ = orc.element_vjp_w1(dim, form, X, np.full(dim + 1, 1.7), Abar)
    Xr, _ = orc.element_vjp(dim, form, X, Abar, coef=1.7)
    assert np.abs(Xc - Xr).max() <= 1e-12 * np.abs(Xr).max()


def test_w1_vjp_mesh_driver(orc):
    from paper_1103_0066_gb300 import meshgen as mg
    m = mg.cube_tet_mesh(3, 0.15, mg.rng_for(24), 0.05, np.float32)
    wv = mg.lognormal_coef(mg.rng_for(25), m.n_vert).astype(np.float64)
    dA = np.random.default_rng(26).standard_normal((m.n_elem, 10, 10))
    gx, gw = orc.integrate_w1_vjp(3, 1, m.conn, m.coords, wv, dA)
    rx, rw = np.zeros_like(gx), np.zeros_like(gw)
    for e in range(m.n_elem):
        xb, wb = orc.element_vjp_w1(3, 1, m.coords[m.conn[e]].astype(np.float64), wv[m.conn[e]], dA[e])
        np.add.at(rx, m.conn[e], xb)
        np.add.at(rw, m.conn[e], wb)
    assert np.allclose(gx, rx, rtol=1e-12, atol=1e-14 * np.abs(rx).max())
    assert np.allclose(gw, rw, rtol=1e-12, atol=1e-14 * np.abs(rw).max())
    A, _ = orc.integrate_w1(3, 1, m.conn, m.coords, wv)
    assert abs(np.dot(wv, gw) - np.sum(dA * A)) <= 1e-11 * np.abs(dA * A).sum()
