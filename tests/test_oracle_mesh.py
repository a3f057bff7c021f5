"""Pins of the oracle mesh against what the paper and geometry fix (CPU only)."""
import os

import numpy as np
import pytest

from oracle.mesh import ShellMesh, icosahedron, diamond_corners, lateral_points, normalized_sum
from oracle.operators import pressure_mesh, prolongation, lateral_prolongation, _lateral_parents

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_icosahedron_is_regular():
    ico = icosahedron()
    V = np.vstack([ico["N"], ico["U"], ico["L"], ico["S"]])
    D = np.linalg.norm(V[:, None] - V[None], axis=2)
    # a regular icosahedron: each vertex has exactly 5 nearest neighbours, all at the same distance
    np.testing.assert_allclose(np.linalg.norm(V, axis=1), 1.0, atol=1e-15)
    edge = np.sort(D, axis=1)[:, 1]
    np.testing.assert_allclose(edge, edge[0], rtol=1e-14)
    assert np.all((np.abs(D - edge[0]) < 1e-12).sum(axis=1) == 5)
    # 30 edges, 20 faces
    assert (np.abs(D - edge[0]) < 1e-12).sum() == 60


def test_diamonds_are_pairs_of_faces():
    """Both triangles of every diamond are icosahedron faces (all sides are edges)."""
    c = diamond_corners()
    edge = np.linalg.norm(c[0, 0] - c[0, 1])
    for d in range(10):
        for tri in ((0, 1, 2), (3, 2, 1)):
            for a, b in ((0, 1), (1, 2), (2, 0)):
                assert abs(np.linalg.norm(c[d, tri[a]] - c[d, tri[b]]) - edge) < 1e-12
    # the 20 triangles are distinct and cover each icosahedron face once
    faces = set()
    for d in range(10):
        for tri in ((0, 1, 2), (3, 2, 1)):
            faces.add(tuple(sorted(tuple(np.round(c[d, t], 12)) for t in tri)))
    assert len(faces) == 20


@pytest.mark.parametrize("level", range(0, 6))
def test_node_counts(level):
    """N_lat = 10 * 4^l + 2 unique lateral points (Sec. 1 resolution estimate)."""
    m = ShellMesh(level, 3, 0.55, 1.0)
    assert m.n_lat == 10 * 4 ** level + 2
    assert m.n_nodes == (10 * 4 ** level + 2) * 3
    np.testing.assert_allclose(np.linalg.norm(m.lat_xyz, axis=1), 1.0, atol=4e-16)


@pytest.mark.parametrize("level", [1, 3, 4])
def test_lattice_multiplicities(level):
    """Poles are shared by 5 diamonds, the other 10 vertices by 3, edge points by 2."""
    m = ShellMesh(level, 2, 0.55, 1.0)
    N = m.N
    counts = np.bincount(m.lat_id.ravel())
    assert (counts == 5).sum() == 2
    assert (counts == 3).sum() == 10
    assert (counts == 2).sum() == 20 * (N - 1)
    assert (counts > 5).sum() == 0
    assert (counts == 1).sum() == 10 * (N - 1) ** 2


def test_mesh_nests_geometrically():
    """Each fine lattice point is the normalised midpoint of its coarse parents (or one of them)."""
    f, c = ShellMesh(4, 3, 0.55, 1.0), ShellMesh(3, 2, 0.55, 1.0)
    for d in range(10):
        for i in range(f.N + 1):
            for j in range(f.N + 1):
                par = _lateral_parents(i, j)
                pts = [c.lat_pts[d, I, J] for (I, J), _ in par]
                target = pts[0] if len(pts) == 1 else normalized_sum(pts[0], pts[1])
                assert np.array_equal(target, f.lat_pts[d, i, j])


def test_prolongation_partition_of_unity_and_radius():
    f = ShellMesh(3, 9, 0.55, 1.0)
    c = pressure_mesh(f)
    P = prolongation(f, c)
    np.testing.assert_allclose(P @ np.ones(c.n_nodes), 1.0, atol=1e-15)
    # interpolating the coarse node radius reproduces the fine radius (uniform spacing)
    rc = np.tile(c.radii, c.n_lat)
    rf = np.tile(f.radii, f.n_lat)
    np.testing.assert_allclose(P @ rc, rf, atol=1e-15)


def test_wedges_positively_oriented_and_volume_converges():
    """det J(q_c) > 0 everywhere; sum of V_e -> shell volume at second order."""
    from oracle.operators import wedge_geometry
    exact = 4.0 / 3.0 * np.pi * (1.0 - 0.55 ** 3)
    errs = []
    for level, n_r in ((2, 3), (3, 5), (4, 9)):
        m = ShellMesh(level, n_r, 0.55, 1.0)
        grad, V = wedge_geometry(m)
        nodes = m.wedge_nodes()
        from oracle.element import geometry
        _, detJ, _, _ = geometry(m.node_xyz(nodes.ravel()).reshape(-1, 6, 3))
        assert detJ.min() > 0
        errs.append(abs(V.sum() - exact))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert rates.min() > 1.8, (errs, rates)


def test_table1_dof_totals():
    """DoF totals of Table 1: 4 x fine nodes + coarse pressure nodes (MT = 2^l, MT/2 radial cells)."""
    rows = np.loadtxt(os.path.join(GOLDEN, "table1_dof_totals.txt"))
    for mt, printed in rows:
        mt = int(mt)
        level = int(round(np.log2(mt)))
        n_r = mt // 2 + 1
        fine = (10 * 4 ** level + 2) * n_r
        coarse = (10 * 4 ** (level - 1) + 2) * ((n_r - 1) // 2 + 1)
        total = 4 * fine + coarse
        # printed to 3 significant digits; two rows (MT128: 43.95 M printed 43.9 M, MT8192:
        # 11.34 T printed 11.4 T) differ from rounding by one unit in the last printed digit
        ulp = 10.0 ** (np.floor(np.log10(printed)) - 2)
        assert abs(total - printed) <= 1.0 * ulp, (mt, total, printed)
        exact_rows = {32, 64, 256, 512, 1024, 2048, 4096}
        if mt in exact_rows:
            assert abs(np.round(total / ulp) * ulp - printed) <= 1e-9 * printed, (mt, total, printed)
    # and the oracle's own de-duplicated count at MT32 agrees with the formula
    m = ShellMesh(5, 17, 0.55, 1.0)
    pm = pressure_mesh(m)
    assert 4 * m.n_nodes + pm.n_nodes == 4 * 10242 * 17 + 2562 * 9
