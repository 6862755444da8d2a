"""Pins for the oracle's non-affine (isoparametric) element matrices, Eqs.
16-19 (no GPU).

The element has quadratic geometry (vertices and edge-midpoint nodes); J^{-1}
is projected onto P1 by its vertex values and |J| is |det J| at the centroid.
Checks: affine elements reduce exactly to the standard matrices; on curved
elements the result is symmetric, annihilates constants and is positive
semidefinite; it equals an exact symbolic evaluation of the same formula on
elements with rational nodes; and it does not depend on the quadrature rule."""
import numpy as np
import pytest

from paper_1103_0066_gb300 import meshgen as mg

LP1, LP2 = 0, 1


def _ref(dim):
    return np.vstack([np.zeros(dim), np.eye(dim)])


def _mids(X):
    return np.array([0.5 * (X[a] + X[b]) for a, b in mg.edge_pairs(X.shape[1])])


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("form", [LP1, LP2])
def test_iso_affine_elements_are_standard(orc, dim, form):
    rng = np.random.default_rng(31)
    for _ in range(8):
        X = rng.standard_normal((dim + 1, dim))
        if abs(np.linalg.det(X[1:] - X[0])) < 0.05:
            continue
        c = float(np.exp(rng.standard_normal()))
        A, _, rc = orc.element_matrix_iso(dim, form, X, _mids(X), coef=c)
        B, _, _ = orc.element_matrix(dim, form, X, coef=c)
        assert rc == 0 and np.abs(A - B).max() <= 1e-13 * np.abs(B).max()


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("form", [LP1, LP2])
def test_iso_curved_structure_and_rule(orc, dim, form):
    rng = np.random.default_rng(32)
    for _ in range(8):
        X = _ref(dim) + 0.1 * rng.standard_normal((dim + 1, dim))
        M = _mids(X) + 0.06 * rng.standard_normal((dim * (dim + 1) // 2, dim))
        A, _, rc = orc.element_matrix_iso(dim, form, X, M)
        assert rc == 0
        s = np.abs(A).max()
        assert np.abs(A - A.T).max() <= 1e-14 * s
        assert np.abs(A.sum(1)).max() <= 1e-13 * s             # constants: zero gradient
        assert np.linalg.eigvalsh(A).min() >= -1e-12 * s        # |J_c| >= 0, integrand a square
        A6, _, _ = orc.element_matrix_iso(dim, form, X, M, q=6)
        assert np.abs(A - A6).max() <= 1e-13 * s                # degree-4 integrand, exact at q = 4


def _symbolic_iso(dim, deg, X, M):
    """Exact evaluation of |J_c| int_ref (Jinv(xi)^T grad phi_i).(Jinv(xi)^T grad phi_j),
    Jinv(xi) = sum_k lambda_k Jinv(vertex k), with the quadratic geometry map."""
    import sympy as sp
    xi = sp.symbols(f"x0:{dim}")
    lam = [1 - sum(xi)] + list(xi)
    p2 = [l * (2 * l - 1) for l in lam] + [4 * lam[a] * lam[b] for a, b in mg.edge_pairs(dim)]
    nodes = [list(map(sp.Rational, r)) for r in list(X) + list(M)]
    x = [sum(nodes[a][al] * p2[a] for a in range(len(p2))) for al in range(dim)]
    J = sp.Matrix(dim, dim, lambda al, mu: sp.diff(x[al], xi[mu]))
    verts = [dict(zip(xi, [0] * dim))] + [dict(zip(xi, [1 if m == k else 0 for m in range(dim)])) for k in range(dim)]
    Jinv = [J.subs(v).inv() for v in verts]
    Ji = sum((lam[k] * Jinv[k] for k in range(dim + 1)), sp.zeros(dim, dim))
    detc = abs(J.subs(dict(zip(xi, [sp.Rational(1, dim + 1)] * dim))).det())
    basis = lam if deg == 1 else p2
    grads = [sp.Matrix([sp.diff(b, v) for v in xi]) for b in basis]
    phys = [Ji.T * g for g in grads]

    def integ(f):
        expr = sp.expand(f)
        for k in range(dim - 1, -1, -1):
            expr = sp.integrate(expr, (xi[k], 0, 1 - sum(xi[:k])))
        return expr

    n = len(basis)
    return np.array([[float(detc * integ((phys[i].T * phys[j])[0])) for j in range(n)] for i in range(n)])


@pytest.mark.parametrize("dim,form", [(2, LP2), (3, LP1)])
def test_iso_symbolic_on_rational_curved_elements(orc, dim, form):
    pytest.importorskip("sympy")
    from fractions import Fraction
    X = [[Fraction(0), Fraction(0)], [Fraction(1), Fraction(1, 10)], [Fraction(1, 5), Fraction(9, 10)]] if dim == 2 \
        else [[0, 0, 0], [1, Fraction(1, 10), 0], [Fraction(1, 10), 1, Fraction(1, 20)], [0, Fraction(1, 10), 1]]
    X = [[Fraction(v) for v in r] for r in X]
    bumps = [[Fraction(1, 20), Fraction(-1, 25), Fraction(1, 30)], [Fraction(-1, 40), Fraction(1, 50), 0],
             [0, Fraction(1, 25), Fraction(-1, 20)], [Fraction(1, 30), 0, Fraction(1, 40)],
             [Fraction(-1, 50), Fraction(1, 40), 0], [0, 0, Fraction(1, 25)]]
    M = []
    for e, (a, b) in enumerate(mg.edge_pairs(dim)):
        M.append([(X[a][m] + X[b][m]) / 2 + bumps[e][m] for m in range(dim)])
    S = _symbolic_iso(dim, 2 if form == LP2 else 1, X, M)
    A, _, rc = orc.element_matrix_iso(dim, form, np.array(X, float), np.array(M, float))
    assert rc == 0 and np.abs(A - S).max() <= 1e-13 * np.abs(S).max()


def test_iso_mesh_driver_and_flags(orc):
    mesh, mid = mg.curved_mesh(mg.cube_tet_mesh(2, 0.15, mg.rng_for(33), 0.0, np.float64), 0.05, np.float64)
    conn = mesh.conn.copy()
    conn[5, 2] = mesh.n_vert + 1
    A, flags = orc.integrate_iso(3, LP2, conn, mesh.coords, mid)
    assert flags[5] == 1 and np.all(A[5] == 0)
    for e in (0, 9, mesh.n_elem - 1):
        Ae, _, _ = orc.element_matrix_iso(3, LP2, mesh.coords[conn[e]], mid[e])
        assert np.array_equal(A[e], Ae)
    # the warp keeps a shared edge's node equal in both elements
    key = {}
    for e in range(mesh.n_elem):
        for m, (a, b) in enumerate(mg.edge_pairs(3)):
            k = tuple(sorted((mesh.conn[e, a], mesh.conn[e, b])))
            if k in key:
                assert np.array_equal(key[k], mid[e, m])
            key[k] = mid[e, m]
