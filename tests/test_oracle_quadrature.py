"""Pins for the oracle's quadrature and basis (no GPU).

The oracle integrates the weak forms of Eqs. 3-5 and Eq. 10 by quadrature on
the reference simplex; these tests pin the rule and the basis against exact
mathematics, independently of the element-matrix code.
"""
import math

import numpy as np
import pytest


@pytest.mark.parametrize("q", [1, 2, 3, 4, 5, 6])
def test_gauss_legendre_exact_monomials(orc, q):
    x, w = orc.gauss_legendre01(q)
    assert np.all((x > 0) & (x < 1))
    for k in range(2 * q):  # exact up to degree 2q-1
        assert abs(np.dot(w, x ** k) - 1.0 / (k + 1)) < 1e-14


def _simplex_monomial(a):
    """Integral of xi^a over the reference simplex: a! / (|a| + d)!."""
    d = len(a)
    return math.prod(math.factorial(k) for k in a) / math.factorial(sum(a) + d)


@pytest.mark.parametrize("dim,q", [(2, 2), (2, 3), (2, 4), (3, 2), (3, 3), (3, 4)])
def test_simplex_rule_exact(orc, dim, q):
    pts, wts = orc.simplex_rule(dim, q)
    assert pts.shape == (q ** dim, dim)
    assert np.all(pts >= 0) and np.all(pts.sum(1) <= 1 + 1e-15)
    pmax = 2 * q - 1 - (dim - 1)  # collapsed direction carries (1-u)^(d-1)
    for deg in range(pmax + 1):
        for a in np.ndindex(*(deg + 1,) * dim):
            if sum(a) != deg:
                continue
            got = np.sum(wts * np.prod(pts ** np.array(a), axis=1))
            assert abs(got - _simplex_monomial(a)) < 1e-15, (a, got)


def _nodes(dim, degree):
    verts = [np.zeros(dim)] + [np.eye(dim)[k] for k in range(dim)]
    nodes = list(verts)
    if degree == 2:
        for i in range(dim + 1):
            for j in range(i + 1, dim + 1):
                nodes.append(0.5 * (verts[i] + verts[j]))
    return nodes


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("degree", [1, 2])
def test_basis_nodal_and_partition(orc, dim, degree):
    nodes = _nodes(dim, degree)
    for k, xi in enumerate(nodes):
        phi, grad = orc.basis(dim, degree, xi)
        assert np.allclose(phi, np.eye(len(nodes))[k], atol=1e-15)  # Lagrange property
    rng = np.random.default_rng(0)
    for _ in range(20):
        xi = rng.dirichlet(np.ones(dim + 1))[1:]
        phi, grad = orc.basis(dim, degree, xi)
        assert abs(phi.sum() - 1) < 1e-14
        assert np.allclose(grad.sum(0), 0, atol=1e-13)
        # gradients against central differences of the values
        h = 1e-6
        for mu in range(dim):
            e = np.zeros(dim)
            e[mu] = h
            fd = (orc.basis(dim, degree, xi + e)[0] - orc.basis(dim, degree, xi - e)[0]) / (2 * h)
            assert np.allclose(fd, grad[:, mu], atol=1e-8)
