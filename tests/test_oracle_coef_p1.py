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
