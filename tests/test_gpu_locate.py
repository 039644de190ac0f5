"""GPU point location on any tetrahedral mesh (zi_locate_points, Sec. 2.5
source positions placed in the mesh) against the oracle's brute force, and
the lead field of dipoles given by position (zi_leadfield_at)."""
import numpy as np
import pytest

from oracle import locate as LC, zi_oracle as O
from paper_1811_07717_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1811_07717_gb300 import zi  # noqa: E402


def ball_points(n, r, seed):
    rng = np.random.default_rng(seed)
    d = rng.standard_normal((n, 3))
    return d / np.linalg.norm(d, axis=1, keepdims=True) * r * rng.uniform(0, 1, (n, 1)) ** (1 / 3)


def test_random_points_bit_exact_and_equal_to_the_grid_rule():
    mesh = O.mesh_from_grid(0.1, [1.0])
    pos = ball_points(300, 0.95, 5)
    got = zi.locate_points(mesh["nodes"], mesh["tets"], pos).cpu().numpy()
    assert np.array_equal(got, LC.locate_points(mesh["nodes"], mesh["tets"], pos))
    assert np.array_equal(got, zi.locate_dipoles_grid(0.1, [1.0], pos).cpu().numpy())


def test_points_on_faces_edges_and_vertices_get_a_holding_element():
    """Grid nodes and face centres lie in several elements: any holding one
    is valid (its smallest barycentric coordinate is ~0, the best there is)."""
    mesh = O.mesh_from_grid(0.25, [1.0])
    g = np.arange(-2, 3) * 0.25
    pts = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    pts = np.concatenate([pts, pts[:40] + [0.125, 0.125, 0.0]])
    got = zi.locate_points(mesh["nodes"], mesh["tets"], pts).cpu().numpy()
    for x, e in zip(pts, got):
        lam = LC.barycentric(mesh["nodes"], mesh["tets"][e:e + 1], x)[0]
        assert lam.min() >= -1e-12


def test_segmentation_mesh_and_outside_points():
    from oracle import segmesh as S
    surf = [W.icosphere(3, 0.97, (0.013, -0.007, 0.011))]
    ref = S.mesh_from_surfaces(0.15, surf, (1,))
    pos = ball_points(200, 0.8, 6)
    got = zi.locate_points(ref["nodes"], ref["tets"], pos).cpu().numpy()
    assert np.array_equal(got, LC.locate_points(ref["nodes"], ref["tets"], pos))
    with pytest.raises(zi.ZiError) as e:
        zi.locate_points(ref["nodes"], ref["tets"], np.array([[0.0, 0.0, 0.0], [0.0, 0.0, 1.5]]))
    assert e.value.status == zi.ZI_ERR_BAD_MESH
    with pytest.raises(zi.ZiError) as e:
        zi.locate_points(ref["nodes"], ref["tets"], np.array([[np.nan, 0.0, 0.0]]))
    assert e.value.status == zi.ZI_ERR_NONFINITE
    assert zi.locate_points(ref["nodes"], ref["tets"], np.zeros((0, 3))).numel() == 0


def test_lead_field_at_positions_equals_lead_field_at_tets():
    spec = W.three_shell(0.006, 16, 60, seed=7)
    mesh = zi.mesh_from_grid(spec.h, spec.radii)
    s6 = W.conductivity(spec, *(mesh[k].cpu().numpy() for k in ("nodes", "tets", "labels")))
    centres, z = W.electrode_inputs(spec)
    pos, _ = W.dipole_inputs(spec)
    gs = zi.System(mesh["nodes"], mesh["tets"], s6, mesh["bfaces"], centres, model="cem", z=z,
                   radius=spec.electrode_radius)
    opts = zi.SolverOpts(tol=1e-10)
    La = gs.leadfield_at(pos, opts).cpu().numpy()
    Lt = gs.leadfield(zi.locate_dipoles_grid(spec.h, spec.radii, pos), opts).cpu().numpy()
    assert np.array_equal(La, Lt)
    gs.close()
