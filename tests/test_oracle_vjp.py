"""Pins for the oracle's hand-derived reverse mode (no GPU).

The gradient of L(x, w) = sum_e <dA_e, A_e(x, w)> is checked against FP64
central finite differences, a Taylor-remainder test, and invariants that hold
exactly: translation (sum_v g_v = 0), rotation for the scalar Laplacian
(sum_v x_v x g_v = 0), Euler homogeneity (A(s x) = s^(d-2) A(x), so
sum_v x_v . g_v = (d-2) L) and linearity in the coefficient (dw_e = <dA_e, A_e>/w_e).
"""
import numpy as np
import pytest

from paper_1103_0066_gb300 import meshgen as mg

LP1, LP2, EP1 = 0, 1, 2


def _mesh(dim, slivers=True):
    if dim == 2:
        return mg.square_tri_mesh(4, 0.2, mg.rng_for(4), np.float64)
    return mg.cube_tet_mesh(4, 0.15, mg.rng_for(4), 0.05 if slivers else 0.0, np.float32)


def _loss(orc, dim, form, conn, X, dA, coef):
    A, fl = orc.integrate(dim, form, conn, X, coef)
    assert not fl.any()
    return float(np.sum(dA * A)), A


def _min_heights(X, conn):
    """Per-vertex minimum over incident elements of the smallest element height."""
    P = X[conn]
    dim = X.shape[1]
    vol = np.abs(np.linalg.det(P[:, 1:] - P[:, :1]))
    hmin = np.full(X.shape[0], np.inf)
    for k in range(dim + 1):
        face = np.delete(P, k, axis=1)
        if dim == 2:
            area = np.linalg.norm(face[:, 1] - face[:, 0], axis=1)
        else:
            area = np.linalg.norm(np.cross(face[:, 1] - face[:, 0], face[:, 2] - face[:, 0]), axis=1)
        h = vol / area
        for kk in range(dim + 1):
            np.minimum.at(hmin, conn[:, kk], h)
    return hmin


@pytest.mark.parametrize("dim,form", [(3, LP1), (2, LP1), (3, EP1), (2, LP2), (3, LP2)])
def test_vjp_central_differences(orc, dim, form):
    mesh = _mesh(dim)
    X = mesh.coords.astype(np.float64)
    conn = mesh.conn
    E = conn.shape[0]
    rng = np.random.default_rng(9)
    n = orc.form_n(form, dim)
    dA = rng.standard_normal((E, n, n))
    coef = np.exp(rng.standard_normal(E))
    g, dw = orc.integrate_vjp(dim, form, conn, X, dA, coef)
    hmin = _min_heights(X, conn)
    fd = np.zeros_like(X)
    for v in range(X.shape[0]):
        inc = np.where((conn == v).any(1))[0]
        if inc.size == 0:
            continue
        sub = conn[inc]
        for a in range(dim):
            d = 1e-4 * hmin[v]
            Xp = X.copy()
            Xp[v, a] += d
            Xm = X.copy()
            Xm[v, a] -= d
            lp, _ = _loss(orc, dim, form, sub, Xp, dA[inc], coef[inc])
            lm, _ = _loss(orc, dim, form, sub, Xm, dA[inc], coef[inc])
            fd[v, a] = (lp - lm) / (2 * d)
    err = np.abs(fd - g).max() / np.abs(g).max()
    assert err < 1e-6, err
    # coefficient gradient: A is linear in w
    L, A = _loss(orc, dim, form, conn, X, dA, coef)
    assert np.allclose(dw, np.einsum("eij,eij->e", dA, A) / coef, rtol=1e-12, atol=1e-300)


@pytest.mark.parametrize("dim,form", [(3, LP1), (3, EP1), (2, LP2)])
def test_vjp_taylor_remainder(orc, dim, form):
    mesh = _mesh(dim, slivers=False)
    X = mesh.coords.astype(np.float64)
    conn = mesh.conn
    rng = np.random.default_rng(10)
    n = orc.form_n(form, dim)
    dA = rng.standard_normal((conn.shape[0], n, n))
    g, _ = orc.integrate_vjp(dim, form, conn, X, dA)
    L0, _ = _loss(orc, dim, form, conn, X, dA, None)
    dirn = rng.standard_normal(X.shape) * 0.01 / 4
    rem = []
    for t in (1.0, 0.5, 0.25, 0.125):
        Lt, _ = _loss(orc, dim, form, conn, X + t * dirn, dA, None)
        rem.append(abs(Lt - L0 - t * np.sum(g * dirn)))
    ratios = [rem[i] / rem[i + 1] for i in range(3)]
    assert all(3.0 < r < 5.0 for r in ratios), ratios  # second order


@pytest.mark.parametrize("dim,form", [(2, LP1), (3, LP1), (2, LP2), (3, LP2), (2, EP1), (3, EP1)])
def test_vjp_invariants(orc, dim, form):
    mesh = _mesh(dim)
    X = mesh.coords.astype(np.float64)
    conn = mesh.conn
    rng = np.random.default_rng(11)
    n = orc.form_n(form, dim)
    dA = rng.standard_normal((conn.shape[0], n, n))
    coef = np.exp(rng.standard_normal(conn.shape[0]))
    g, dw = orc.integrate_vjp(dim, form, conn, X, dA, coef)
    L, A = _loss(orc, dim, form, conn, X, dA, coef)
    scale = np.abs(g).max() * np.abs(X).max() * X.shape[0]
    assert np.abs(g.sum(0)).max() < 1e-12 * np.abs(g).sum()            # translation
    assert abs(np.sum(X * g) - (dim - 2) * L) < 1e-11 * scale           # homogeneity
    if form != EP1:                                                     # rotation
        if dim == 3:
            tq = np.cross(X, g).sum(0)
        else:
            tq = np.array([np.sum(X[:, 0] * g[:, 1] - X[:, 1] * g[:, 0])])
        assert np.abs(tq).max() < 1e-11 * scale


def test_vjp_degenerate_contributes_nothing(orc):
    X = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 1]], dtype=np.float64)
    conn = np.array([[0, 1, 2, 3], [4, 1, 1, 3]], dtype=np.int32)
    dA = np.ones((2, 4, 4))
    g, dw = orc.integrate_vjp(3, LP1, conn, X, dA)
    g0, dw0 = orc.integrate_vjp(3, LP1, conn[:1], X, dA[:1])
    assert np.array_equal(g, g0) and dw[1] == 0.0 and dw[0] == dw0[0]
