"""Pins of the oracle's coupling block (no GPU).

The off-diagonal block of a multiphysics pair (Sec. 6: coupled systems broken
into blocks) is B_{i,(c,j)} = int_T w phi_i d psi_j / d x_c, with phi the P1
scalar basis and psi the P1 or P2 basis of each component of a vector field
(column c * nbv + j).  Its analytic tensor holds a basis function times a
basis-function derivative (Eq. 1; Sec. 3.1's closing remark on any member of
the jet space).  None of these checks re-types the oracle's formula:

* reference simplex: exact rational integrals by sympy;
* a patch test: for a field v the basis reproduces exactly (linear for P1,
  quadratic for P2), B applied to v's nodal values is int phi_i div v, which
  the test evaluates in closed form from barycentric monomial integrals;
* column sums: sum_i B_{i,(c,j)} = int_T d psi_j / d x_c in closed form from
  the barycentric gradients (numpy's inverse, not the oracle's LU solve);
* scaling (s^{d-1}), translation, rotation (the vector index rotates), and
  independence of the quadrature rule;
* the reverse mode: FP64 central differences, translation invariance,
  Euler homogeneity sum_k x_k . xbar_k = (d-1) L and dL/dw = L / w.
A transposed inverse Jacobian, a dropped |J| or a swapped component index
fails the patch test or the column sums."""
import math

import numpy as np
import pytest

import oracle


def _element(dim, seed):
    rng = np.random.default_rng(seed)
    X = np.vstack([np.zeros(dim), np.eye(dim)]) + 0.3 * rng.standard_normal((dim + 1, dim))
    if np.linalg.det(X[1:] - X[0]) < 0:
        X[[1, 2]] = X[[2, 1]]
    return X


def _bary_grads(X):
    """Physical gradients of lambda_0..lambda_d: rows of J^{-1} (numpy inverse)."""
    dim = X.shape[1]
    J = (X[1:] - X[0]).T                       # J[a][mu] = x_{mu+1,a} - x_{0,a}
    Ji = np.linalg.inv(J)                      # Ji[mu][a] = d xi_mu / d x_a
    G = np.zeros((dim + 1, dim))
    G[1:] = Ji
    G[0] = -Ji.sum(0)
    return G, abs(np.linalg.det(J)) / math.factorial(dim)


def _nodes(X, vdeg):
    dim = X.shape[1]
    if vdeg == 1:
        return X.copy()
    mids = [0.5 * (X[a] + X[b]) for a in range(dim + 1) for b in range(a + 1, dim + 1)]
    return np.vstack([X] + mids)


def _lam_int(exps, dim, vol):
    """int_T prod lambda_k^{a_k} = d! vol prod a_k! / (sum a + d)!."""
    num = math.factorial(dim) * vol
    for a in exps:
        num *= math.factorial(a)
    return num / math.factorial(sum(exps) + dim)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("vdeg", [1, 2])
def test_div_reference_symbolic(dim, vdeg):
    sp = pytest.importorskip("sympy")
    xi = sp.symbols(f"x0:{dim}")
    lam = [1 - sum(xi)] + list(xi)
    if vdeg == 1:
        psi = lam
    else:
        psi = [l * (2 * l - 1) for l in lam] + [4 * lam[a] * lam[b] for a in range(dim + 1)
                                                for b in range(a + 1, dim + 1)]

    def integ(f):
        f = sp.expand(f)
        if dim == 2:
            return sp.integrate(sp.integrate(f, (xi[1], 0, 1 - xi[0])), (xi[0], 0, 1))
        return sp.integrate(sp.integrate(sp.integrate(f, (xi[2], 0, 1 - xi[0] - xi[1])),
                                         (xi[1], 0, 1 - xi[0])), (xi[0], 0, 1))
    nbv = len(psi)
    ref = np.zeros((dim + 1, dim * nbv))
    for i in range(dim + 1):
        for c in range(dim):
            for j in range(nbv):
                ref[i, c * nbv + j] = float(integ(lam[i] * sp.diff(psi[j], xi[c])))
    X = np.vstack([np.zeros(dim), np.eye(dim)])
    B, det, rc = oracle.element_matrix_div(dim, vdeg, X)
    assert rc == 0 and det == 1.0
    assert np.abs(B - ref).max() <= 1e-15


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("vdeg", [1, 2])
def test_div_patch_test(dim, vdeg):
    """B applied to the nodal values of a field the basis reproduces is
    int_T phi_i div v: linear v for P1, quadratic v for P2 (div v then linear,
    so int lambda_i div v = sum_k div v(x_k) int lambda_i lambda_k)."""
    rng = np.random.default_rng(3 + dim + 10 * vdeg)
    for trial in range(4):
        X = _element(dim, 100 * dim + trial)
        M = rng.standard_normal((dim, dim))
        b = rng.standard_normal(dim)
        Q = rng.standard_normal((dim, dim, dim)) if vdeg == 2 else np.zeros((dim, dim, dim))
        Q = 0.5 * (Q + Q.transpose(0, 2, 1))   # v_c = x^T Q_c x + (M x)_c + b_c

        def v(x):
            return np.einsum("cab,a,b->c", Q, x, x) + M @ x + b

        def div(x):  # d/dx_c of x^T Q_c x is 2 (Q_c x)_c
            return np.trace(M) + 2 * sum(Q[c, c] @ x for c in range(dim))
        nodes = _nodes(X, vdeg)
        nbv = nodes.shape[0]
        vals = np.array([v(x) for x in nodes])          # [nbv][dim]
        u = vals.T.reshape(-1)                           # component-major: c * nbv + j
        w = 0.7 + trial
        B, _, rc = oracle.element_matrix_div(dim, vdeg, X, coef=w)
        assert rc == 0
        _, vol = _bary_grads(X)
        dv = np.array([div(x) for x in X])               # div v at the vertices
        expect = np.zeros(dim + 1)
        for i in range(dim + 1):
            for k in range(dim + 1):
                e = [0] * (dim + 1)
                e[i] += 1
                e[k] += 1
                expect[i] += dv[k] * _lam_int(e, dim, vol)
        assert np.allclose(B @ u, w * expect, rtol=0, atol=1e-13 * max(1.0, np.abs(expect).max()))


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("vdeg", [1, 2])
def test_div_column_sums(dim, vdeg):
    """sum_i B_{i,(c,j)} = int_T d psi_j / d x_c (sum_i lambda_i = 1): for P1
    vol * d lambda_j; for P2 vertex functions vol (4/(d+1) - 1) d lambda_j and
    edge functions 4 vol / (d+1) (d lambda_a + d lambda_b)."""
    X = _element(dim, 7 + dim)
    G, vol = _bary_grads(X)
    B, _, _ = oracle.element_matrix_div(dim, vdeg, X)
    nbv = B.shape[1] // dim
    colsum = B.sum(0).reshape(dim, nbv)                  # [c][j]
    ref = np.zeros((dim, nbv))
    for j in range(dim + 1):
        ref[:, j] = vol * G[j] * (1.0 if vdeg == 1 else 4.0 / (dim + 1) - 1.0)
    if vdeg == 2:
        t = dim + 1
        for a in range(dim + 1):
            for b in range(a + 1, dim + 1):
                ref[:, t] = 4.0 * vol / (dim + 1) * (G[a] + G[b])
                t += 1
    assert np.abs(colsum - ref).max() <= 1e-14 * np.abs(ref).max()


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("vdeg", [1, 2])
def test_div_transformation_laws_and_rule(dim, vdeg):
    X = _element(dim, 21 + dim)
    B, _, _ = oracle.element_matrix_div(dim, vdeg, X)
    s = 2.5
    Bs, _, _ = oracle.element_matrix_div(dim, vdeg, s * X)
    assert np.allclose(Bs, s ** (dim - 1) * B, rtol=1e-13, atol=1e-15)
    Bt, _, _ = oracle.element_matrix_div(dim, vdeg, X + np.arange(1, dim + 1))
    assert np.allclose(Bt, B, rtol=1e-12, atol=1e-14)
    rng = np.random.default_rng(5)
    R, _ = np.linalg.qr(rng.standard_normal((dim, dim)))
    if np.linalg.det(R) < 0:
        R[:, 0] *= -1
    Br, _, _ = oracle.element_matrix_div(dim, vdeg, X @ R.T)
    nbv = B.shape[1] // dim
    B3 = B.reshape(dim + 1, dim, nbv)
    rot = np.einsum("cd,idj->icj", R, B3).reshape(B.shape)   # the vector index rotates with x
    assert np.allclose(Br, rot, rtol=1e-12, atol=1e-14)
    B5, _, _ = oracle.element_matrix_div(dim, vdeg, X, q=5)
    assert np.abs(B5 - B).max() <= 1e-14 * np.abs(B).max()


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("vdeg", [1, 2])
def test_div_vjp_against_central_differences(dim, vdeg):
    X = _element(dim, 31 + dim)
    rng = np.random.default_rng(32)
    B0, _, _ = oracle.element_matrix_div(dim, vdeg, X)
    Bbar = rng.standard_normal(B0.shape)
    w = 1.7
    Xbar, cbar = oracle.element_vjp_div(dim, vdeg, X, Bbar, coef=w)
    h = 1e-6
    fd = np.zeros_like(X)
    for k in range(dim + 1):
        for a in range(dim):
            Xp, Xm = X.copy(), X.copy()
            Xp[k, a] += h
            Xm[k, a] -= h
            fd[k, a] = (np.sum(Bbar * oracle.element_matrix_div(dim, vdeg, Xp, coef=w)[0])
                        - np.sum(Bbar * oracle.element_matrix_div(dim, vdeg, Xm, coef=w)[0])) / (2 * h)
    assert np.abs(Xbar - fd).max() <= 1e-7 * np.abs(fd).max()
    L = np.sum(Bbar * oracle.element_matrix_div(dim, vdeg, X, coef=w)[0])
    assert abs(cbar - L / w) <= 1e-13 * abs(L / w)
    assert np.abs(Xbar.sum(0)).max() <= 1e-12 * np.abs(Xbar).max()          # translation
    assert abs(np.sum(X * Xbar) - (dim - 1) * L) <= 1e-12 * max(1.0, abs(L))  # homogeneity of degree d-1


def test_div_mesh_drivers_and_flags():
    from paper_1103_0066_gb300 import meshgen as mg
    m = mg.cube_tet_mesh(3, 0.15, mg.rng_for(5), 0.05, np.float32)
    coef = mg.lognormal_coef(mg.rng_for(6), m.n_elem)
    B, fl = oracle.integrate_div(3, 2, m.conn, m.coords, coef)
    assert not fl.any() and B.shape == (m.n_elem, 4, 30)
    for e in (0, 17, m.n_elem - 1):
        Be, _, _ = oracle.element_matrix_div(3, 2, m.coords[m.conn[e]].astype(np.float64), coef=coef[e])
        assert np.array_equal(B[e], Be)
    dB = np.random.default_rng(7).standard_normal(B.shape)
    gx, gw = oracle.integrate_div_vjp(3, 2, m.conn, m.coords, dB, coef)
    ref = np.zeros_like(gx)
    for e in range(m.n_elem):
        xb, cb = oracle.element_vjp_div(3, 2, m.coords[m.conn[e]].astype(np.float64), dB[e], coef=coef[e])
        np.add.at(ref, m.conn[e], xb)
        assert cb == gw[e]
    assert np.allclose(gx, ref, rtol=1e-12, atol=1e-14 * np.abs(ref).max())
    bad = m.conn.copy()
    bad[3, 1] = m.n_vert + 5
    bad[4, 2] = bad[4, 0]
    B2, fl2 = oracle.integrate_div(3, 1, bad, m.coords)
    assert fl2[3] == oracle.FLAG_CONN and fl2[4] == oracle.FLAG_DEGENERATE
    assert not B2[3].any() and not B2[4].any()
