"""GPU parity of the segmentation mesher (Sec. 2.5, mesh tool) and the source
interpolation through the C ABI: nodes, tets, labels and boundary faces
bit-exact against the oracle on surfaces kept off the grid nodes (so every
label is decided far from the winding number's threshold), the lead field of
the GPU mesh (from dipole positions) against the oracle's, nearest-DOF indices
bit-exact, empty inputs of the source and sensor calls, and the error paths the
kernels check."""
import numpy as np
import pytest

from oracle import segmesh as S, zi_oracle as O
from paper_1811_07717_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1811_07717_gb300 import zi  # noqa: E402

CENTRE = (0.013, -0.007, 0.011)


def clear_of_threshold(h, surfaces):
    """Every grid node's winding number is far from 1/2 for every surface."""
    R = max(float(np.max(np.abs(v))) for v, _ in surfaces)
    N = int(np.ceil(R / h)) + 1
    ax = (np.arange(2 * N + 1) - N) * h
    P = np.stack(np.meshgrid(ax, ax, ax, indexing="ij"), -1).reshape(-1, 3)
    return all(np.min(np.abs(S.winding_number(P, v, t) - 0.5)) > 1e-6 for v, t in surfaces)


CASES = [
    (0.2, [W.icosphere(2, r, CENTRE) for r in (0.8, 0.86, 1.0)], (3, 1, 2)),
    (0.2, [W.icosphere(2, r, CENTRE) for r in (0.8, 0.86, 1.0)], (1, 2, 3)),
    (0.15, [W.icosphere(3, 0.97, CENTRE)], (1,)),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_mesh_from_surfaces_bit_exact(case):
    h, surf, prio = CASES[case]
    assert clear_of_threshold(h, surf)
    ref = S.mesh_from_surfaces(h, surf, prio)
    got = zi.mesh_from_surfaces(h, surf, prio)
    assert np.array_equal(got["nodes"].cpu().numpy(), ref["nodes"])
    assert np.array_equal(got["tets"].cpu().numpy(), ref["tets"])
    assert np.array_equal(got["labels"].cpu().numpy(), ref["labels"])
    assert np.array_equal(got["bfaces"].cpu().numpy(), ref["bfaces"])


def test_lead_field_on_the_gpu_mesh_matches_the_oracle():
    h, surf, prio = CASES[2]
    ref = S.mesh_from_surfaces(h, surf, prio)
    got = zi.mesh_from_surfaces(h, surf, prio)
    spec = W.unit_sphere_point(h=h, n_electrodes=16, n_dipoles=30)
    s6 = W.conductivity(spec, ref["nodes"], ref["tets"], ref["labels"])
    centres, _ = W.electrode_inputs(spec)
    pos, _ = W.dipole_inputs(spec)
    # the oracle places the dipoles by brute-force point location; the GPU
    # build gets the positions only (zi_leadfield_at)
    from oracle import locate as LC
    dip = LC.locate_points(ref["nodes"], ref["tets"], pos)
    osys = O.System(ref, s6, centres, "point")
    Lo = O.leadfield(osys, O.source_matrix(osys.n, ref["nodes"], ref["tets"], dip))
    gsys = zi.System(got["nodes"], got["tets"], s6, got["bfaces"], centres, model="point")
    Lg = gsys.leadfield_at(pos, zi.SolverOpts(tol=1e-12)).cpu().numpy()
    assert np.linalg.norm(Lg - Lo) <= 1e-8 * np.linalg.norm(Lo)
    gsys.close()


def test_mesh_from_surfaces_errors():
    V, T = W.icosphere(1, 0.9, CENTRE)
    bad = T.copy()
    bad[3, 1] = V.shape[0]
    with pytest.raises(zi.ZiError) as e:
        zi.mesh_from_surfaces(0.3, [(V, bad)], (1,))
    assert e.value.status == zi.ZI_ERR_ARG
    Vn = V.copy()
    Vn[2, 0] = np.nan
    with pytest.raises(zi.ZiError) as e:
        zi.mesh_from_surfaces(0.3, [(Vn, T)], (1,))
    assert e.value.status == zi.ZI_ERR_NONFINITE
    with pytest.raises(ValueError):
        zi.mesh_from_surfaces(0.3, [(V, T)], (1, 2))


def test_nearest_source_bit_exact():
    """Source interpolation (nearest DOF, ties to the lowest index) against
    the oracle, with duplicated sources and points on a grid equidistant from
    several sources, across several shared-memory tiles of sources."""
    from oracle import interp as I
    rng = np.random.default_rng(12)
    S = rng.uniform(-1, 1, (700, 3))
    S[300:310] = S[10:20]                      # exact duplicates: ties
    S[600] = [0.0, 0.0, 0.0]
    S[601] = [0.5, 0.0, 0.0]
    X = np.concatenate([rng.uniform(-1.1, 1.1, (5000, 3)),
                        np.stack(np.meshgrid(*(np.arange(-2, 3) * 0.25,) * 3, indexing="ij"), -1).reshape(-1, 3)])
    ref = I.nearest_source(X, S)
    got = zi.nearest_source(X, S).cpu().numpy()
    assert np.array_equal(got, ref)
    # the mesh nodes of a segmentation mesh against its dipoles
    h, surf, prio = CASES[2]
    mesh = zi.mesh_from_surfaces(h, surf, prio)
    pos, _ = W.dipole_inputs(W.unit_sphere_point(h=h, n_electrodes=16, n_dipoles=300))
    ref = I.nearest_source(mesh["nodes"].cpu().numpy(), pos)
    assert np.array_equal(zi.nearest_source(mesh["nodes"], pos).cpu().numpy(), ref)
    Sn = S.copy()
    Sn[5, 1] = np.inf
    with pytest.raises(zi.ZiError) as e:
        zi.nearest_source(X, Sn)
    assert e.value.status == zi.ZI_ERR_NONFINITE


def test_empty_inputs_of_the_source_and_sensor_calls():
    """Zero sources, columns or points: the calls return empty results
    without launching work on empty arrays."""
    spec = W.unit_sphere_point(h=0.2, n_electrodes=8, n_dipoles=5)
    mesh = zi.mesh_from_grid(spec.h, spec.radii)
    s6 = W.conductivity(spec, *(mesh[k].cpu().numpy() for k in ("nodes", "tets", "labels")))
    centres, _ = W.electrode_inputs(spec)
    system = zi.System(mesh["nodes"], mesh["tets"], s6, mesh["bfaces"], centres, model="point")
    opts = zi.SolverOpts(tol=1e-10)
    no_pos = np.zeros((0, 3))
    no_tet = np.zeros(0, dtype=np.int32)
    Fn, Fw = system.source_stencil(no_pos, no_tet)
    assert Fn.shape == (0, zi.STENCIL_WIDTH) and Fw.shape == (0, zi.STENCIL_WIDTH)
    L = system.leadfield_sparse(np.zeros((0, 4), dtype=np.int32), np.zeros((0, 4)), opts)
    assert L.shape == (spec.n_electrodes - 1, 0)
    Fn, Fw = system.source_pi(no_tet)
    assert Fn.shape == (0, 4)
    sp_, sd = W.meg_sensors(4, 1.2)
    Tm, _, _ = system.meg_transfer(sp_, sd, opts)
    assert system.meg_leadfield(Tm, sp_, sd, no_pos, Fn, Fw).shape == (4, 0)
    assert zi.nearest_source(no_pos, np.ones((3, 3))).shape == (0,)
    system.close()


def test_source_apply_timing_reports_its_algorithmic_bytes():
    """zi_time_source_apply (the H(div) line's roofline): positive time, and
    bytes = F entries + distinct T rows per Cartesian source + the H^T write."""
    spec = W.unit_sphere_point(h=0.1, n_electrodes=16, n_dipoles=200)
    mesh = zi.mesh_from_grid(spec.h, spec.radii)
    s6 = W.conductivity(spec, *(mesh[k].cpu().numpy() for k in ("nodes", "tets", "labels")))
    centres, _ = W.electrode_inputs(spec)
    pos, _ = W.dipole_inputs(spec)
    system = zi.System(mesh["nodes"], mesh["tets"], s6, mesh["bfaces"], centres, model="point")
    system.transfer(zi.SolverOpts(tol=1e-10), want_T=False)
    dip = zi.locate_dipoles_grid(spec.h, spec.radii, pos)
    Fn, Fw = system.source_stencil(pos, dip, zi.SOURCE_PBO10)
    ms, b = system.time_source_apply(Fn, Fw, reps=3)
    fn = Fn.cpu().numpy()
    rows = sum(np.unique(fn[3 * p:3 * p + 3]).size for p in range(pos.shape[0]))
    ncol = spec.n_electrodes - 1
    assert ms > 0
    assert b == fn.size * 12.0 + rows * ncol * 8.0 + fn.shape[0] * ncol * 8.0
    system.close()
