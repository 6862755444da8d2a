"""Pins for the oracle's reverse mode on non-affine (isoparametric) elements,
Eqs. 16-19 (no GPU).

orc_element_vjp_iso / orc_integrate_iso_vjp give the gradients of
L = sum dA : A with respect to the vertices, the edge-midpoint nodes and the
per-element coefficient.  They are pinned by what the mathematics fixes, not by
re-deriving the same steps:
  * central differences of the (separately pinned) forward oracle, FP64,
    Richardson-extrapolated;
  * invariances of the Laplacian: a translation or a rotation of all nodes
    leaves A unchanged, so the node gradients sum to zero and their moment
    vanishes; a scaling by s multiplies A by s^(d-2) (Euler's relation);
  * the coefficient enters linearly: dL/dc = L / c;
  * straight-sided elements: with the edge nodes at the edge midpoints the
    element is affine, so moving a vertex of the affine element equals moving
    it and the midpoints of its edges by half as much -- the affine reverse
    mode (pinned elsewhere) must equal dx + (1/2) sum over its edges of dmid;
  * the mesh-level reverse mode sums the element ones in element order."""
import numpy as np
import pytest

from paper_1103_0066_gb300 import meshgen as mg

LP1, LP2 = 0, 1


def _ref(dim):
    return np.vstack([np.zeros(dim), np.eye(dim)])


def _mids(X):
    return np.array([0.5 * (X[a] + X[b]) for a, b in mg.edge_pairs(X.shape[1])])


def _min_vertex_det(orc, X, M):
    """Smallest |det J| of the quadratic geometry map over the vertices."""
    dim = X.shape[1]
    nodes = np.vstack([X, M])
    dets = []
    for k in range(dim + 1):
        xi = np.zeros(dim)
        if k:
            xi[k - 1] = 1.0
        _, g = orc.basis(dim, 2, xi)
        dets.append(abs(np.linalg.det(nodes.T @ g)))
    return min(dets)


def _curved(rng, dim, amp=0.06, orc=None):
    """A curved element whose Jacobian stays well away from singular at every
    vertex (central differences need a smooth neighbourhood)."""
    while True:
        X = _ref(dim) + 0.1 * rng.standard_normal((dim + 1, dim))
        M = _mids(X) + amp * rng.standard_normal((dim * (dim + 1) // 2, dim))
        if orc is None or _min_vertex_det(orc, X, M) > 0.4:
            return X, M


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("form", [LP1, LP2])
def test_iso_vjp_matches_central_differences(orc, dim, form):
    rng = np.random.default_rng(41)
    n = orc.form_n(form, dim)
    for _ in range(6):
        X, M = _curved(rng, dim, orc=orc)
        c = float(np.exp(0.3 * rng.standard_normal()))
        dA = rng.standard_normal((n, n))
        Xb, Mb, cb, rc = orc.element_vjp_iso(dim, form, X, M, dA, coef=c)
        assert rc == 0

        def L(X_, M_, c_):
            return float((orc.element_matrix_iso(dim, form, X_, M_, coef=c_)[0] * dA).sum())

        for _ in range(3):
            vX, vM, vc = rng.standard_normal(X.shape), rng.standard_normal(M.shape), float(rng.standard_normal())
            def cd(h):
                return (L(X + h * vX, M + h * vM, c + h * vc) - L(X - h * vX, M - h * vM, c - h * vc)) / (2 * h)

            fd = (4.0 * cd(5e-5) - cd(1e-4)) / 3.0  # Richardson: O(h^4)
            an = float((Xb * vX).sum() + (Mb * vM).sum() + cb * vc)
            scale = np.abs(Xb).sum() + np.abs(Mb).sum() + abs(cb)
            assert abs(fd - an) <= 1e-8 * scale


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("form", [LP1, LP2])
def test_iso_vjp_invariances(orc, dim, form):
    rng = np.random.default_rng(42)
    n = orc.form_n(form, dim)
    for _ in range(6):
        X, M = _curved(rng, dim)
        c = 1.7
        dA = rng.standard_normal((n, n))
        A, _, _ = orc.element_matrix_iso(dim, form, X, M, coef=c)
        Xb, Mb, cb, rc = orc.element_vjp_iso(dim, form, X, M, dA, coef=c)
        assert rc == 0
        nodes = np.vstack([X, M])
        grads = np.vstack([Xb, Mb])
        s = np.abs(grads).max() * np.abs(nodes).max()
        L = float((A * dA).sum())
        # translation
        assert np.abs(grads.sum(0)).max() <= 1e-12 * np.abs(grads).max()
        # rotation: the moment of the node gradients
        if dim == 3:
            mom = np.cross(nodes, grads).sum(0)
        else:
            mom = np.array([(nodes[:, 0] * grads[:, 1] - nodes[:, 1] * grads[:, 0]).sum()])
        assert np.abs(mom).max() <= 1e-12 * s
        # scaling: A(s x) = s^(d-2) A(x)
        assert abs((nodes * grads).sum() - (dim - 2) * L) <= 1e-12 * max(s, abs(L))
        # linear in the coefficient
        assert abs(cb - L / c) <= 1e-13 * max(abs(cb), 1.0)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("form", [LP1, LP2])
def test_iso_vjp_straight_sides_reduce_to_affine(orc, dim, form):
    rng = np.random.default_rng(43)
    n = orc.form_n(form, dim)
    pairs = mg.edge_pairs(dim)
    for _ in range(6):
        X = _ref(dim) + 0.15 * rng.standard_normal((dim + 1, dim))
        if abs(np.linalg.det(X[1:] - X[0])) < 0.05:
            continue
        c = 0.8
        dA = rng.standard_normal((n, n))
        Xb, Mb, cb, rc = orc.element_vjp_iso(dim, form, X, _mids(X), dA, coef=c)
        Xa, ca = orc.element_vjp(dim, form, X, dA, coef=c)
        assert rc == 0
        moved = Xb.copy()
        for q, (a, b) in enumerate(pairs):
            moved[a] += 0.5 * Mb[q]
            moved[b] += 0.5 * Mb[q]
        assert np.abs(moved - Xa).max() <= 1e-12 * np.abs(Xa).max()
        assert abs(cb - ca) <= 1e-12 * abs(ca)


def test_iso_vjp_mesh_sums_element_gradients(orc):
    """Mesh reverse mode = the element ones scattered to the vertices."""
    base = mg.cube_tet_mesh(2, 0.1, mg.rng_for(44), 0.0, np.float64)
    mesh, mid = mg.curved_mesh(base, 0.05, np.float64)
    E, V = mesh.n_elem, mesh.n_vert
    rng = np.random.default_rng(45)
    for form in (LP1, LP2):
        n = orc.form_n(form, 3)
        dA = rng.standard_normal((E, n, n))
        coef = np.exp(0.2 * rng.standard_normal(E))
        dx, dm, dc = orc.integrate_iso_vjp(3, form, mesh.conn, mesh.coords, mid, dA, coef)
        ref = np.zeros((V, 3))
        for e in range(E):
            X = mesh.coords[mesh.conn[e]]
            Xb, Mb, cb, rc = orc.element_vjp_iso(3, form, X, mid[e], dA[e], coef=coef[e])
            assert rc == 0
            np.add.at(ref, mesh.conn[e], Xb)
            assert np.abs(dm[e] - Mb).max() <= 1e-14 * max(np.abs(Mb).max(), 1e-300)
            assert dc[e] == cb
        assert np.abs(dx - ref).max() <= 1e-12 * np.abs(ref).max()
