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
