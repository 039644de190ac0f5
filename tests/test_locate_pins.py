"""Pins of the point-location oracle (oracle/locate.py, Sec. 2.5 source
positions placed in the mesh) against constructions that share nothing
with it: the Kuhn grid's own location rule (cube by floor, tet by sorting
the fractional coordinates), the reconstruction of the point from its
barycentric coordinates, and points outside the mesh."""
import numpy as np

from oracle import locate as LC, zi_oracle as O


def test_matches_the_kuhn_grid_rule_inside_cubes():
    mesh = O.mesh_from_grid(0.25, [1.0])
    rng = np.random.default_rng(3)
    d = rng.standard_normal((200, 3))
    pos = d / np.linalg.norm(d, axis=1, keepdims=True) * 0.7 * rng.uniform(0, 1, (200, 1)) ** (1 / 3)
    got = LC.locate_points(mesh["nodes"], mesh["tets"], pos)
    ref = O.locate_dipoles(mesh, pos)
    assert np.array_equal(got, ref)


def test_barycentric_coordinates_reconstruct_the_point():
    mesh = O.mesh_from_grid(0.3, [1.0])
    rng = np.random.default_rng(4)
    pos = rng.uniform(-0.5, 0.5, (30, 3))
    tet = LC.locate_points(mesh["nodes"], mesh["tets"], pos)
    for x, e in zip(pos, tet):
        lam = LC.barycentric(mesh["nodes"], mesh["tets"][e:e + 1], x)[0]
        assert abs(lam.sum() - 1.0) < 1e-12 and lam.min() >= -1e-12
        assert np.allclose(lam @ mesh["nodes"][mesh["tets"][e]], x, atol=1e-12)


def test_points_outside_the_mesh():
    mesh = O.mesh_from_grid(0.3, [1.0])
    pos = np.array([[0.0, 0.0, 3.0], [2.0, 2.0, 2.0], [0.0, 0.0, 0.1]])
    tet = LC.locate_points(mesh["nodes"], mesh["tets"], pos)
    assert tet[0] == -1 and tet[1] == -1 and tet[2] >= 0


def test_ties_go_to_the_lowest_index():
    # two tets sharing the face x = 0 of a tiny two-element mesh; a point on that face
    nodes = np.array([[0, 0, 0], [0, 1, 0], [0, 0, 1], [1, 0, 0], [-1, 0, 0]], dtype=float)
    tets = np.array([[0, 1, 2, 3], [0, 2, 1, 4]])
    x = np.array([[0.0, 0.25, 0.25]])
    assert LC.locate_points(nodes, tets, x)[0] == 0
    assert LC.locate_points(nodes, tets[::-1], x)[0] == 0
