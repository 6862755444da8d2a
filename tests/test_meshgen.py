"""Input-recipe checks for the seeded synthetic meshes (no GPU)."""
import numpy as np

from paper_1103_0066_gb300 import meshgen as mg


def test_tri_workload_shape_and_seed():
    m = mg.workload_tri_p1_fp64()
    assert (m.n_elem, m.n_vert) == (8192, 4225) and m.coords.dtype == np.float64
    mg.check_orientation(m)
    m2 = mg.workload_tri_p1_fp64()
    assert np.array_equal(m.coords, m2.coords) and np.array_equal(m.conn, m2.conn)
    # boundary vertices stay on the unit square
    b = (np.isclose(m.coords, 0) | np.isclose(m.coords, 1)).any(1)
    assert b.sum() == 4 * 64


def test_tet_mesh_slivers_recipe():
    m = mg.cube_tet_mesh(8, 0.15, mg.rng_for(2), 0.05, np.float32)
    E = 6 * 8 ** 3
    ns = int(round(0.05 * E))
    assert m.n_elem == E and m.n_vert == 9 ** 3 + ns and m.sliver.sum() == ns
    mg.check_orientation(m)
    # each sliver references exactly one appended private vertex
    assert np.all((m.conn[m.sliver] >= 9 ** 3).sum(1) == 1)
    assert np.all(m.conn[~m.sliver] < 9 ** 3)
    # height ratio of the moved vertex is within [5e-5, 2e-2] of a regular element's scale
    P = m.coords[m.conn].astype(np.float64)
    vol = np.abs(np.linalg.det(P[:, 1:] - P[:, :1])) / 6
    assert vol[m.sliver].max() < 0.05 * np.median(vol[~m.sliver])


def test_mixed_batch_recipe():
    items = mg.mixed_batch(scale=0.01)
    assert len(items) == 96
    kinds = [(it.mesh.dim, it.form) for it in items]
    for k in mg.BATCH_KINDS:
        assert kinds.count(k) == 16
    for it in items:
        assert it.coef.shape == (it.mesh.n_elem,)
        n = mg.form_n(it.form, it.mesh.dim)
        assert it.dA.shape == (it.mesh.n_elem, n, n)
        assert it.mesh.conn.max() < it.mesh.n_vert


def test_shuffled_mesh_is_a_relabelling():
    """Element k of the shuffled mesh is element order[k] of the original, with
    the same vertex positions in the same local order (so every element matrix
    is unchanged), and a shuffled tet mesh's 32-element tiles touch far more
    distinct vertices than the cell-major ones (more than the 36 of the
    assembly's dense tile in most tiles)."""
    m = mg.cube_tet_mesh(8, 0.15, mg.rng_for(2), 0.05, np.float32)
    s, order = mg.shuffled(m, mg.rng_for(12))
    assert s.n_elem == m.n_elem and s.n_vert == m.n_vert
    assert np.array_equal(s.coords[s.conn], m.coords[m.conn[order]])
    assert np.array_equal(s.sliver, m.sliver[order])
    assert sorted(map(tuple, np.sort(s.coords, 0))) == sorted(map(tuple, np.sort(m.coords, 0)))
    mg.check_orientation(s)

    def distinct_per_tile(mesh):
        T = mesh.n_elem // 32
        return np.array([np.unique(mesh.conn[32 * t:32 * t + 32]).size for t in range(T)])
    assert np.mean(distinct_per_tile(m) <= 36) > 0.95
    d = distinct_per_tile(s)
    assert np.mean(d > 36) > 0.9 and d.max() > 100
    b = mg.mixed_batch(n_meshes=6, scale=0.002, shuffle=True)
    b0 = mg.mixed_batch(n_meshes=6, scale=0.002)
    assert [x.mesh.n_elem for x in b] == [x.mesh.n_elem for x in b0]
