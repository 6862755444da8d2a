"""Pins for the oracle's element matrices (no GPU).

Every check here comes from mathematics the paper fixes, not from the oracle
itself: closed-form reference matrices (Eq. 6 with J = I), the cotangent
formulas, null spaces (rigid modes for eps:eps, Eq. 24), exact energies of
interpolated polynomials, transformation laws, exact symbolic integrals, and
brute-force patch tests on tiny assembled meshes.
"""
import itertools
import os

import numpy as np
import pytest

from paper_1103_0066_gb300 import meshgen as mg

LP1, LP2, EP1 = 0, 1, 2
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _ref(dim):
    return np.vstack([np.zeros(dim), np.eye(dim)])


def _rand_simplex(rng, dim, scale=1.0):
    while True:
        X = rng.standard_normal((dim + 1, dim)) * scale
        if abs(np.linalg.det(X[1:] - X[0])) > 0.05 * scale ** dim:
            return X


def _golden_p1():
    out, lines = {}, [l for l in open(os.path.join(GOLDEN, "reference_p1_laplace.txt"))
                      if l.strip() and not l.startswith("#")]
    i = 0
    while i < len(lines):
        d = int(lines[i])
        out[d] = np.array([[float(t) for t in lines[i + 1 + r].split()] for r in range(d + 1)])
        i += d + 2
    return out


@pytest.mark.parametrize("dim", [2, 3])
def test_reference_p1_golden(orc, dim):
    A, det, rc = orc.element_matrix(dim, LP1, _ref(dim))
    assert rc == 0 and det == 1.0
    assert np.allclose(A, _golden_p1()[dim], rtol=0, atol=1e-15)


def _angle_cot(p, a, b):
    u, v = a - p, b - p
    return np.dot(u, v) / abs(u[0] * v[1] - u[1] * v[0])


def test_triangle_cotangent_formula(orc):
    rng = np.random.default_rng(1)
    for _ in range(50):
        X = _rand_simplex(rng, 2)
        A, _, _ = orc.element_matrix(2, LP1, X)
        for i, j in itertools.combinations(range(3), 2):
            k = 3 - i - j
            assert abs(A[i, j] - (-0.5 * _angle_cot(X[k], X[i], X[j]))) < 1e-12 * np.abs(A).max()


def test_tet_cotangent_formula(orc):
    rng = np.random.default_rng(2)
    for _ in range(50):
        X = _rand_simplex(rng, 3)
        A, _, _ = orc.element_matrix(3, LP1, X)
        for i, j in itertools.combinations(range(4), 2):
            k, l = [m for m in range(4) if m not in (i, j)]
            e = X[l] - X[k]
            ell = np.linalg.norm(e)
            eh = e / ell
            u = (X[i] - X[k]) - np.dot(X[i] - X[k], eh) * eh
            v = (X[j] - X[k]) - np.dot(X[j] - X[k], eh) * eh
            cot = np.dot(u, v) / np.linalg.norm(np.cross(u, v))
            assert abs(A[i, j] + ell * cot / 6.0) < 1e-12 * np.abs(A).max()


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("form", [LP1, LP2])
def test_laplacian_structure(orc, dim, form):
    rng = np.random.default_rng(3)
    for _ in range(20):
        X = _rand_simplex(rng, dim)
        A, _, _ = orc.element_matrix(dim, form, X, coef=2.5)
        n = A.shape[0]
        assert np.allclose(A, A.T, atol=1e-13 * np.abs(A).max())
        assert np.allclose(A.sum(1), 0, atol=1e-12 * np.abs(A).max())
        ev = np.linalg.eigvalsh(A)
        assert ev.min() > -1e-12 * ev.max()
        assert np.linalg.matrix_rank(A, tol=1e-9 * ev.max()) == n - 1


def _rigid_modes(X, dim):
    """Rigid displacements sampled at the P1 nodes, component-major DOFs."""
    nb = dim + 1
    modes = []
    for c in range(dim):                 # translations
        u = np.zeros((dim, nb))
        u[c] = 1.0
        modes.append(u.ravel())
    gens = [np.array([[0, -1], [1, 0]])] if dim == 2 else [
        np.array([[0, -1, 0], [1, 0, 0], [0, 0, 0]]), np.array([[0, 0, 1], [0, 0, 0], [-1, 0, 0]]),
        np.array([[0, 0, 0], [0, 0, -1], [0, 1, 0]])]
    for W in gens:                       # infinitesimal rotations u = W x
        modes.append((X @ W.T).T.ravel())
    return np.array(modes)


@pytest.mark.parametrize("dim", [2, 3])
def test_elasticity_rigid_null_space(orc, dim):
    """eps(u) vanishes exactly for rigid motions (reading of Eqs. 9-15 with the
    symmetric gradient; the vector-Laplacian reading of Eq. 14 as printed would
    not annihilate rotations)."""
    rng = np.random.default_rng(4)
    for _ in range(20):
        X = _rand_simplex(rng, dim)
        A, _, _ = orc.element_matrix(dim, EP1, X, coef=0.7)
        n = A.shape[0]
        assert n == dim * (dim + 1)
        assert np.allclose(A, A.T, atol=1e-13 * np.abs(A).max())
        R = _rigid_modes(X, dim)
        assert np.abs(A @ R.T).max() < 1e-12 * np.abs(A).max()
        ev = np.linalg.eigvalsh(A)
        assert ev.min() > -1e-12 * ev.max()
        assert np.linalg.matrix_rank(A, tol=1e-9 * ev.max()) == n - dim * (dim + 1) // 2
        # the printed vector Laplacian would give a rotation energy > 0
        L, _, _ = orc.element_matrix(dim, LP1, X, coef=0.7)
        VL = np.kron(np.eye(dim), L)
        assert np.abs(VL @ R[dim:].T).max() > 1e-3 * np.abs(VL).max()


def _p2_nodes(X):
    dim = X.shape[1]
    nodes = [X[i] for i in range(dim + 1)]
    for i in range(dim + 1):
        for j in range(i + 1, dim + 1):
            nodes.append(0.5 * (X[i] + X[j]))
    return np.array(nodes)


def _simplex_volume(X):
    d = X.shape[1]
    return abs(np.linalg.det(X[1:] - X[0])) / np.prod(range(1, d + 1))


def _exact_grad_energy(X, gradfun):
    """Integral over the simplex of |grad u|^2 for a quadratic u whose gradient
    is the linear field gradfun: with c_k = grad u(x_k), grad u = sum c_k lambda_k
    and the barycentric identity  int lambda_k lambda_l = |T| d! (1+delta_kl)/(d+2)!."""
    d = X.shape[1]
    c = np.array([gradfun(x) for x in X])
    fac = _simplex_volume(X) * np.prod(range(1, d + 1)) / np.prod(range(1, d + 3))
    G = c @ c.T
    return fac * (G.sum() + np.trace(G))


@pytest.mark.parametrize("dim", [2, 3])
def test_energy_of_interpolated_polynomials(orc, dim):
    rng = np.random.default_rng(5)
    for _ in range(20):
        X = _rand_simplex(rng, dim)
        w = float(np.exp(rng.standard_normal()))
        # P1, linear u = b.x + c0
        b = rng.standard_normal(dim)
        u = X @ b + 0.3
        A, _, _ = orc.element_matrix(dim, LP1, X, coef=w)
        assert abs(u @ A @ u - w * _simplex_volume(X) * b @ b) < 1e-12 * abs(w * b @ b)
        # P2, quadratic u = x^T M x + b.x
        M = rng.standard_normal((dim, dim))
        M = M + M.T
        nodes = _p2_nodes(X)
        u = np.einsum("ni,ij,nj->n", nodes, M, nodes) + nodes @ b
        A, _, _ = orc.element_matrix(dim, LP2, X, coef=w)
        ex = w * _exact_grad_energy(X, lambda x: 2 * M @ x + b)
        assert abs(u @ A @ u - ex) < 1e-11 * abs(ex)
        # elasticity, linear displacement u = B x + t: energy |T| |sym B|^2
        B = rng.standard_normal((dim, dim))
        U = (X @ B.T + rng.standard_normal(dim)).T.ravel()  # component-major
        A, _, _ = orc.element_matrix(dim, EP1, X, coef=w)
        S = 0.5 * (B + B.T)
        assert abs(U @ A @ U - w * _simplex_volume(X) * np.sum(S * S)) < 1e-11 * np.sum(S * S) * w


def _rot(dim, rng):
    Q, _ = np.linalg.qr(rng.standard_normal((dim, dim)))
    if np.linalg.det(Q) < 0:
        Q[:, 0] *= -1
    return Q


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("form", [LP1, LP2, EP1])
def test_transformation_laws(orc, dim, form):
    rng = np.random.default_rng(6)
    for _ in range(10):
        X = _rand_simplex(rng, dim)
        A, _, _ = orc.element_matrix(dim, form, X)
        s = 3.7
        As, _, _ = orc.element_matrix(dim, form, s * X)
        assert np.allclose(As, s ** (dim - 2) * A, rtol=0, atol=1e-12 * np.abs(A).max())
        At, _, _ = orc.element_matrix(dim, form, X + rng.standard_normal(dim))
        assert np.allclose(At, A, rtol=0, atol=1e-11 * np.abs(A).max())
        R = _rot(dim, rng)
        Ar, _, _ = orc.element_matrix(dim, form, X @ R.T)
        if form == EP1:
            nb = dim + 1
            P = np.kron(R, np.eye(nb))
            A = P @ A @ P.T
        assert np.allclose(Ar, A, rtol=0, atol=1e-11 * np.abs(A).max())
        # q-independence of the quadrature (the integrand is a polynomial of low degree)
        A5, _, _ = orc.element_matrix(dim, form, X, q=5)
        A3, _, _ = orc.element_matrix(dim, form, X, q=3)
        assert np.abs(A5 - A3).max() <= 1e-14 * np.abs(A3).max() * 10


@pytest.mark.parametrize("dim", [2, 3])
def test_vertex_permutation_permutes_p1(orc, dim):
    rng = np.random.default_rng(7)
    X = _rand_simplex(rng, dim)
    A, _, _ = orc.element_matrix(dim, LP1, X)
    for perm in itertools.permutations(range(dim + 1)):
        p = list(perm)
        Ap, _, _ = orc.element_matrix(dim, LP1, X[p])
        assert np.allclose(Ap, A[np.ix_(p, p)], atol=1e-13 * np.abs(A).max())


def test_symbolic_reference_matrices(orc):
    """Exact rational reference-element matrices by symbolic integration."""
    sp = pytest.importorskip("sympy")
    for dim in (2, 3):
        xi = sp.symbols(f"x0:{dim}")
        lam = [1 - sum(xi)] + list(xi)
        p1 = lam
        p2 = [l * (2 * l - 1) for l in lam] + [4 * lam[i] * lam[j] for i in range(dim + 1)
                                             for j in range(i + 1, dim + 1)]

        def integ(f):
            # nested integration over the reference simplex
            expr = f
            for k in range(dim - 1, -1, -1):
                upper = 1 - sum(xi[:k])
                expr = sp.integrate(expr, (xi[k], 0, upper))
            return expr

        for form, basis in ((LP1, p1), (LP2, p2)):
            grads = [[sp.diff(b, v) for v in xi] for b in basis]
            n = len(basis)
            S = np.array([[float(integ(sum(grads[i][m] * grads[j][m] for m in range(dim))))
                           for j in range(n)] for i in range(n)])
            A, _, _ = orc.element_matrix(dim, form, _ref(dim))
            assert np.abs(A - S).max() < 1e-14 * np.abs(S).max(), (dim, form)
        # elasticity eps:eps on the reference simplex
        nb = dim + 1
        grads = [[sp.diff(b, v) for v in xi] for b in p1]
        Ex = np.zeros((dim * nb, dim * nb))
        for I in range(dim * nb):
            cI, iI = divmod(I, nb)
            for K in range(dim * nb):
                cK, iK = divmod(K, nb)
                tot = 0
                for a in range(dim):
                    for b in range(dim):
                        eI = sp.Rational(1, 2) * ((a == cI) * grads[iI][b] + (b == cI) * grads[iI][a])
                        eK = sp.Rational(1, 2) * ((a == cK) * grads[iK][b] + (b == cK) * grads[iK][a])
                        tot += eI * eK
                Ex[I, K] = float(integ(tot))
        A, _, _ = orc.element_matrix(dim, EP1, _ref(dim))
        assert np.abs(A - Ex).max() < 1e-14 * np.abs(Ex).max()


# --------------------------------------------------------------- patch tests

def _edge_nodes(conn, coords):
    """Global P2 numbering: vertices, then one node per mesh edge (test-side assembly)."""
    V = coords.shape[0]
    dim = coords.shape[1]
    edge_id = {}
    extra = []
    loc = []
    for e in range(conn.shape[0]):
        ids = list(conn[e])
        for i in range(dim + 1):
            for j in range(i + 1, dim + 1):
                key = (min(ids[i], ids[j]), max(ids[i], ids[j]))
                if key not in edge_id:
                    edge_id[key] = V + len(extra)
                    extra.append(0.5 * (coords[key[0]] + coords[key[1]]))
                ids.append(edge_id[key])
        loc.append(ids)
    nodes = np.vstack([coords, np.array(extra)])
    return np.array(loc), nodes


def _on_boundary(P):
    return np.any((np.abs(P) < 1e-12) | (np.abs(P - 1) < 1e-12), axis=1)


@pytest.mark.parametrize("dim", [2, 3])
def test_patch_tests_assembled(orc, dim):
    if dim == 2:
        mesh = mg.square_tri_mesh(3, 0.2, np.random.default_rng(8), np.float64)
    else:
        mesh = mg.cube_tet_mesh(2, 0.15, np.random.default_rng(8), 0.0, np.float64)
    X, conn = mesh.coords.astype(np.float64), mesh.conn
    V = X.shape[0]
    # P1 Laplacian: linear u is discrete-harmonic at interior vertices
    A, fl = orc.integrate(dim, LP1, conn, X)
    assert not fl.any()
    K = np.zeros((V, V))
    for e in range(conn.shape[0]):
        K[np.ix_(conn[e], conn[e])] += A[e]
    b = np.arange(1, dim + 1) * 0.7
    u = X @ b
    inter = ~_on_boundary(X)
    assert inter.any()
    assert np.abs((K @ u)[inter]).max() < 1e-12 * np.abs(K).max()
    assert abs(u @ K @ u - b @ b) < 1e-12  # exact Dirichlet energy on the unit domain
    # P2 Laplacian: harmonic quadratic x^2 - y^2
    loc, nodes = _edge_nodes(conn, X)
    N = nodes.shape[0]
    A2, _ = orc.integrate(dim, LP2, conn, X)
    K2 = np.zeros((N, N))
    for e in range(conn.shape[0]):
        K2[np.ix_(loc[e], loc[e])] += A2[e]
    u2 = nodes[:, 0] ** 2 - nodes[:, 1] ** 2
    inter2 = ~_on_boundary(nodes)
    assert np.abs((K2 @ u2)[inter2]).max() < 1e-11 * np.abs(K2).max()
    assert abs(u2 @ K2 @ u2 - 8.0 / 3.0) < 1e-11
    # elasticity: a linear displacement is in equilibrium at interior vertices
    Ae, _ = orc.integrate(dim, EP1, conn, X)
    nb = dim + 1
    KE = np.zeros((dim * V, dim * V))
    for e in range(conn.shape[0]):
        g = np.concatenate([c * V + conn[e] for c in range(dim)])
        KE[np.ix_(g, g)] += Ae[e]
    Bm = np.arange(dim * dim).reshape(dim, dim) * 0.1 + np.eye(dim)
    U = (X @ Bm.T).T.ravel()
    rows = np.concatenate([c * V + np.where(inter)[0] for c in range(dim)])
    assert np.abs((KE @ U)[rows]).max() < 1e-12 * np.abs(KE).max()
    S = 0.5 * (Bm + Bm.T)
    assert abs(U @ KE @ U - np.sum(S * S)) < 1e-11


def test_flags_and_degenerate(orc):
    X = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 1]], dtype=np.float64)
    conn = np.array([[0, 1, 2, 3], [0, 1, 1, 3], [0, 1, 2, 7], [0, 1, 2, -1]], dtype=np.int32)
    A, fl = orc.integrate(3, LP1, conn, X)
    assert list(fl) == [0, 2, 1, 1]
    assert np.all(A[1:] == 0)
    assert np.abs(A[0]).max() > 0


def test_oracle_det_against_exact_rational(orc):
    """det J of sliver elements against exact rational arithmetic: the FP64
    oracle stays within the usual error bound of a 3x3 determinant."""
    from fractions import Fraction
    mesh = mg.cube_tet_mesh(4, 0.15, mg.rng_for(4), 0.05, np.float32)
    A, fl, det = orc.integrate(3, LP1, mesh.conn, mesh.coords, return_det=True)
    assert not fl.any()
    for e in np.where(mesh.sliver)[0][:20]:
        P = [[Fraction(float(c)) for c in mesh.coords[v]] for v in mesh.conn[e]]
        J = [[P[mu + 1][a] - P[0][a] for mu in range(3)] for a in range(3)]
        ex = (J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1])
              - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0])
              + J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]))
        Jf = np.array([[float(x) for x in r] for r in J])
        bound = 16 * 2.0 ** -53 * np.abs(Jf).max() ** 3 * 6
        assert abs(det[e] - float(ex)) <= bound
        assert float(ex) > 0
