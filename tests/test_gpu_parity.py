"""GPU parity: the CUDA path through the C ABI against the CPU oracle on the
same seeded inputs.  Integer outputs bit-exact; FP64 lead fields within 1e-8
relative Frobenius, mixed precision within 1e-6."""
import numpy as np
import pytest

from oracle import zi_oracle as O
from paper_1811_07717_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1811_07717_gb300 import zi  # noqa: E402


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


def small_shell(h=0.006, L=32, P=200, aniso=True, seed=21, radius=0.009):
    return W.three_shell(h, L, P, seed=seed, skull_aniso=(0.00132, 0.0132) if aniso else None,
                         electrode_radius=radius)


def gpu_head(spec):
    mesh = zi.mesh_from_grid(spec.h, spec.radii)
    nodes = mesh["nodes"].cpu().numpy()
    tets = mesh["tets"].cpu().numpy()
    labels = mesh["labels"].cpu().numpy()
    s6 = W.conductivity(spec, nodes, tets, labels)
    centres, z = W.electrode_inputs(spec)
    pos, q = W.dipole_inputs(spec)
    system = zi.System(mesh["nodes"], mesh["tets"], s6, mesh["bfaces"], centres,
                       model=spec.electrode_model, z=z if spec.electrode_model == "cem" else None,
                       radius=spec.electrode_radius)
    dip = zi.locate_dipoles_grid(spec.h, spec.radii, pos)
    return mesh, s6, system, dip, pos, q


def oracle_head(spec, s6=None):
    mesh = O.mesh_from_grid(spec.h, spec.radii)
    if s6 is None:
        s6 = W.conductivity(spec, mesh["nodes"], mesh["tets"], mesh["labels"])
    centres, z = W.electrode_inputs(spec)
    pos, q = W.dipole_inputs(spec)
    system = O.System(mesh, s6, centres, spec.electrode_model, radius=spec.electrode_radius, z=z)
    dip = O.locate_dipoles(mesh, pos)
    F = O.source_matrix(system.n, mesh["nodes"], mesh["tets"], dip)
    return mesh, system, dip, F


# --------------------------------------------------------------------------
# integer outputs: bit-exact
# --------------------------------------------------------------------------

@pytest.mark.parametrize("h,radii", [(0.1, [1.0]), (0.2, [1.0]), (0.45, [1.0]), (0.006, [0.08, 0.086, 0.092]),
                                     (0.002, [0.08, 0.086, 0.092])])
def test_mesh_bit_exact(h, radii):
    g = zi.mesh_from_grid(h, radii)
    o = O.mesh_from_grid(h, radii)
    assert np.array_equal(g["nodes"].cpu().numpy(), o["nodes"])
    assert np.array_equal(g["tets"].cpu().numpy(), o["tets"])
    assert np.array_equal(g["labels"].cpu().numpy(), o["labels"])
    assert np.array_equal(g["bfaces"].cpu().numpy(), o["bfaces"])


@pytest.mark.parametrize("spec", [W.config_unit_sphere(), W.config_three_shell_2mm()], ids=["unit", "shell2mm"])
def test_dipole_location_bit_exact(spec):
    pos, q = W.dipole_inputs(spec)
    g = zi.locate_dipoles_grid(spec.h, spec.radii, pos).cpu().numpy()
    o = O.locate_dipoles(O.mesh_from_grid(spec.h, spec.radii), pos)
    assert np.array_equal(g, o)


def test_dipole_location_edge_cases():
    # points on cube faces / the main diagonal (ties) and a point outside the mesh
    h, radii = 0.25, [1.0]
    pos = np.array([[0.1, 0.1, 0.1], [0.05, 0.2, 0.2], [0.0, 0.0, 0.0], [0.25, -0.5, 0.125]])
    g = zi.locate_dipoles_grid(h, radii, pos).cpu().numpy()
    o = O.locate_dipoles(O.mesh_from_grid(h, radii), pos)
    assert np.array_equal(g, o)
    with pytest.raises(zi.ZiError) as e:
        zi.locate_dipoles_grid(h, radii, np.array([[0.0, 0.0, 2.0]]))
    assert e.value.status == zi.ZI_ERR_BAD_MESH
    assert zi.locate_dipoles_grid(h, radii, np.zeros((0, 3))).numel() == 0


def _csr(system):
    rp, ci, v, B, C, en = system.matrix()
    return (rp.cpu().numpy(), ci.cpu().numpy(), v.cpu().numpy(), B.cpu().numpy(),
            None if C is None else C.cpu().numpy(), None if en is None else en.cpu().numpy())


@pytest.mark.parametrize("aniso", [False, True])
def test_assembly_pattern_bit_exact_values_fp64(aniso):
    spec = small_shell(aniso=aniso)
    mesh, s6, gs, dip, pos, q = gpu_head(spec)
    om, osys, odip, F = oracle_head(spec)
    rp, ci, v, B, C, _ = _csr(gs)
    A = osys.A
    assert np.array_equal(rp, A.indptr) and np.array_equal(ci, A.indices)
    scale = np.max(np.abs(A.data))
    assert np.max(np.abs(v - A.data)) <= 1e-14 * scale
    assert gs.info()["ground"] == osys.ip
    assert np.max(np.abs(B - osys.B)) <= 1e-14 * np.max(np.abs(osys.B))
    assert np.max(np.abs(C - osys.C)) <= 1e-14 * np.max(osys.C)
    assert np.array_equal(dip.cpu().numpy(), odip)


def test_point_electrodes_bit_exact():
    spec = W.config_unit_sphere()
    mesh, s6, gs, dip, pos, q = gpu_head(spec)
    om, osys, odip, F = oracle_head(spec)
    rp, ci, v, B, C, en = _csr(gs)
    assert np.array_equal(en, osys.el_nodes)
    assert gs.info()["ground"] == osys.ip
    assert np.array_equal(B, osys.B)
    assert np.max(np.abs(v - osys.A.data)) <= 1e-14 * np.max(np.abs(osys.A.data))


# --------------------------------------------------------------------------
# transfer matrix and lead field
# --------------------------------------------------------------------------

def test_transfer_fp64_matches_direct_solve():
    spec = small_shell(L=24)
    mesh, s6, gs, dip, pos, q = gpu_head(spec)
    om, osys, odip, F = oracle_head(spec)
    T, it, rr = gs.transfer(zi.SolverOpts(tol=1e-12))
    T = T.cpu().numpy()
    assert np.all(rr <= 1e-12) and np.all(it > 0)
    Tref = osys.transfer()
    assert rel(T, Tref) < 1e-9
    res = np.linalg.norm(osys.A @ T - osys.B, axis=0) / np.linalg.norm(osys.B, axis=0)
    assert np.all(res <= 1.5e-12)


def test_lead_field_fp64_point_electrodes_unit_sphere():
    spec = W.config_unit_sphere()
    mesh, s6, gs, dip, pos, q = gpu_head(spec)
    L = gs.leadfield(dip, zi.SolverOpts(tol=1e-12)).cpu().numpy()
    Lref, *_ = O.leadfield_from_spec(spec, W)
    assert L.shape == (15, 900)
    assert rel(L, Lref) < 1e-8


@pytest.mark.parametrize("aniso", [False, True])
def test_lead_field_fp64_cem_three_shell(aniso):
    spec = small_shell(aniso=aniso)
    mesh, s6, gs, dip, pos, q = gpu_head(spec)
    L = gs.leadfield(dip, zi.SolverOpts(tol=1e-10)).cpu().numpy()
    om, osys, odip, F = oracle_head(spec)
    Lref = O.leadfield(osys, F)
    assert L.shape == (spec.n_electrodes, 3 * spec.n_dipoles)
    assert rel(L, Lref) < 1e-8


def test_lead_field_mixed_precision_within_1e6():
    spec = small_shell(aniso=True)
    mesh, s6, gs, dip, pos, q = gpu_head(spec)
    L = gs.leadfield(dip, zi.SolverOpts(tol=1e-10, precision=zi.MIXED)).cpu().numpy()
    om, osys, odip, F = oracle_head(spec)
    Lref = O.leadfield(osys, F)
    assert rel(L, Lref) < 1e-6


@pytest.mark.parametrize("L,radius", [(100, 0.008), (200, 0.006), (256, 0.005)], ids=["L100", "L200", "L256"])
def test_lead_field_mixed_precision_wide_layouts(L, radius):
    """Mixed precision at electrode counts whose FP32 rows split over 26, 52
    and 64 threads (ld = 104, 208, 256)."""
    spec = small_shell(L=L, P=50, aniso=True, radius=radius)
    mesh, s6, gs, dip, pos, q = gpu_head(spec)
    L_gpu = gs.leadfield(dip, zi.SolverOpts(tol=1e-10, precision=zi.MIXED)).cpu().numpy()
    om, osys, odip, F = oracle_head(spec)
    assert rel(L_gpu, O.leadfield(osys, F)) < 1e-6


def test_lead_field_ldp_preconditioner():
    spec = small_shell(aniso=False, L=16, P=50)
    mesh, s6, gs, dip, pos, q = gpu_head(spec)
    L = gs.leadfield(dip, zi.SolverOpts(tol=1e-11, precond=zi.PRECOND_LDP)).cpu().numpy()
    om, osys, odip, F = oracle_head(spec)
    assert rel(L, O.leadfield(osys, F)) < 1e-8


def test_bitwise_determinism():
    spec = small_shell(L=16, P=50)
    outs = []
    for _ in range(2):
        mesh, s6, gs, dip, pos, q = gpu_head(spec)
        T, it, rr = gs.transfer(zi.SolverOpts(tol=1e-10))
        L = gs.leadfield(dip)
        outs.append((gs.matrix()[2].cpu().numpy(), T.cpu().numpy(), L.cpu().numpy(), it))
        gs.close()
    for a, b in zip(outs[0], outs[1]):
        assert np.array_equal(a, b)


def test_column_shards_concatenate():
    """Solving with a subset of electrodes gives the same T columns: the
    columns are independent recurrences."""
    spec = small_shell(L=16, P=10)
    mesh, s6, gs, dip, pos, q = gpu_head(spec)
    T, it, rr = gs.transfer(zi.SolverOpts(tol=1e-11))
    om, osys, odip, F = oracle_head(spec)
    assert rel(T.cpu().numpy(), osys.transfer()) < 1e-9


# --------------------------------------------------------------------------
# linearised EIT
# --------------------------------------------------------------------------

def test_eit_voltages_jacobian_and_vjp():
    spec = W.unit_sphere_cem(h=0.2, n_electrodes=16)
    mesh, s6, gs, dip, pos, q = gpu_head(spec)
    I = W.injection_patterns(spec.n_electrodes)
    y, J = gs.eit(I, mode=zi.EIT_FULL, opts=zi.SolverOpts(tol=1e-12))
    om, osys, odip, F = oracle_head(spec)
    Jref, yref = O.eit_jacobian(osys, I)
    assert rel(y.cpu().numpy(), yref) < 1e-9
    Jg = J.cpu().numpy()                      # m x np x L
    assert rel(np.transpose(Jg, (1, 2, 0)), Jref) < 1e-8
    rng = np.random.default_rng(0)
    G = rng.standard_normal(yref.shape)
    _, g = gs.eit(I, mode=zi.EIT_VJP, grad_y=G, want_y=False)
    gref = np.einsum("pk,pkm->m", G, Jref)
    assert rel(g.cpu().numpy(), gref) < 1e-8


# --------------------------------------------------------------------------
# error paths (host-side or bounded device error words; no faults)
# --------------------------------------------------------------------------

def test_nonfinite_conductivity_rejected():
    spec = W.unit_sphere_point(h=0.3, n_electrodes=8, n_dipoles=5)
    mesh = zi.mesh_from_grid(spec.h, spec.radii)
    m = mesh["tets"].shape[0]
    s6 = np.tile([0.33, 0.33, 0.33, 0, 0, 0], (m, 1))
    s6[3, 0] = np.nan
    centres, _ = W.electrode_inputs(spec)
    with pytest.raises(zi.ZiError) as e:
        zi.System(mesh["nodes"], mesh["tets"], s6, mesh["bfaces"], centres, model="point")
    assert e.value.status == zi.ZI_ERR_NONFINITE


def test_inverted_element_rejected():
    spec = W.unit_sphere_point(h=0.3, n_electrodes=8, n_dipoles=5)
    mesh = zi.mesh_from_grid(spec.h, spec.radii)
    tets = mesh["tets"].clone()
    tets[0, [2, 3]] = tets[0, [3, 2]]
    m = tets.shape[0]
    s6 = np.tile([0.33, 0.33, 0.33, 0, 0, 0], (m, 1))
    centres, _ = W.electrode_inputs(spec)
    with pytest.raises(zi.ZiError) as e:
        zi.System(mesh["nodes"], tets, s6, mesh["bfaces"], centres, model="point")
    assert e.value.status == zi.ZI_ERR_BAD_MESH


def test_maxit_reports_not_converged_with_outputs():
    spec = small_shell(L=8, P=5)
    mesh, s6, gs, dip, pos, q = gpu_head(spec)
    T, it, rr = gs.transfer(zi.SolverOpts(tol=1e-12, maxit=3, check_every=1), allow_not_converged=True)
    assert np.all(rr > 1e-12) and np.all(it <= 3)
    with pytest.raises(zi.NotConverged):
        gs.transfer(zi.SolverOpts(tol=1e-12, maxit=3, check_every=1))


def test_electrode_without_patch_rejected():
    spec = small_shell(L=8, P=5, radius=1e-5)
    with pytest.raises(zi.ZiError) as e:
        gpu_head(spec)
    assert e.value.status == zi.ZI_ERR_BAD_MESH
