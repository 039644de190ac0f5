"""GPU parity of the H(div) source model (Sec. 2.1) through the C ABI:
zi_source_stencil against the oracle's source matrix (node lists exact,
loads to rounding), zi_leadfield_sparse against the oracle lead field (FP64
within 1e-8, mixed within 1e-6), the sparse path reproducing the
partial-integration lead field, and the error paths the kernels check."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import hdiv as HD, zi_oracle as O
from paper_1811_07717_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1811_07717_gb300 import zi  # noqa: E402


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


def build(spec):
    """(oracle mesh, oracle system, GPU system, pos, dip_tet) on the same inputs."""
    mesh = O.mesh_from_grid(spec.h, spec.radii)
    s6 = W.conductivity(spec, mesh["nodes"], mesh["tets"], mesh["labels"])
    centres, z = W.electrode_inputs(spec)
    pos, _ = W.dipole_inputs(spec)
    osys = O.System(mesh, s6, centres, spec.electrode_model, radius=spec.electrode_radius, z=z)
    gsys = zi.System(mesh["nodes"], mesh["tets"], s6, mesh["bfaces"], centres, model=spec.electrode_model,
                     z=z if spec.electrode_model == "cem" else None, radius=spec.electrode_radius)
    dip = O.locate_dipoles(mesh, pos)
    return mesh, osys, gsys, pos, dip


def ell_to_sparse(Fn, Fw, n):
    Fn = Fn.cpu().numpy().astype(np.int64)
    Fw = Fw.cpu().numpy()
    cols = np.repeat(np.arange(Fn.shape[0]), Fn.shape[1])
    return sp.coo_matrix((Fw.ravel(), (Fn.ravel(), cols)), shape=(n, Fn.shape[0])).tocsc()


@pytest.mark.parametrize("model", [zi.SOURCE_WHITNEY4, zi.SOURCE_PBO10])
def test_stencil_matches_the_oracle(model):
    spec = W.unit_sphere_point(h=0.1, n_electrodes=16, n_dipoles=300)
    mesh, osys, gsys, pos, dip = build(spec)
    # add sources in tets with exactly one face on the boundary (three face sources)
    _, opp = HD.face_neighbours(mesh["tets"], np.arange(0, mesh["tets"].shape[0], 5))
    edge = 5 * np.nonzero(np.sum(opp < 0, axis=1) == 1)[0][:20]
    assert edge.size == 20
    pos = np.vstack([pos, mesh["nodes"][mesh["tets"][edge]].mean(axis=1)])
    dip = np.concatenate([dip, edge])
    Fn, Fw = gsys.source_stencil(pos, dip, model)
    n = mesh["nodes"].shape[0]
    Fo = HD.source_matrix_hdiv(mesh["nodes"], mesh["tets"], dip, pos, model).toarray()
    Fg = ell_to_sparse(Fn, Fw, n).toarray()
    assert np.max(np.abs(Fg - Fo)) <= 1e-12 * np.max(np.abs(Fo))
    # node lists: the tet's vertices, then the vertex across each face
    fn = Fn.cpu().numpy()
    tets = mesh["tets"]
    _, oppd = HD.face_neighbours(tets, dip)
    for p in range(dip.size):
        for j in range(3):
            assert np.array_equal(fn[3 * p + j, :4], tets[dip[p]])
            exp = np.where(oppd[p] >= 0, oppd[p], tets[dip[p]])
            assert np.array_equal(fn[3 * p + j, 4:], exp)
    gsys.close()


@pytest.mark.parametrize("model", [zi.SOURCE_WHITNEY4, zi.SOURCE_PBO10])
def test_hdiv_lead_field_fp64_point_electrodes(model):
    spec = W.unit_sphere_point(h=0.1, n_electrodes=16, n_dipoles=300)
    mesh, osys, gsys, pos, dip = build(spec)
    Lo = O.leadfield(osys, HD.source_matrix_hdiv(mesh["nodes"], mesh["tets"], dip, pos, model))
    Lg = gsys.leadfield_hdiv(pos, dip, model, opts=zi.SolverOpts(tol=1e-12)).cpu().numpy()
    assert Lg.shape == Lo.shape
    assert rel(Lg, Lo) <= 1e-8
    gsys.close()


def test_hdiv_lead_field_mixed_cem_anisotropic_head():
    spec = W.three_shell(0.006, 32, 200, seed=21, skull_aniso=(0.00132, 0.0132), electrode_radius=0.009)
    mesh, osys, gsys, pos, dip = build(spec)
    Lo = O.leadfield(osys, HD.source_matrix_hdiv(mesh["nodes"], mesh["tets"], dip, pos, HD.PBO10))
    Lg = gsys.leadfield_hdiv(pos, dip, zi.SOURCE_PBO10,
                             opts=zi.SolverOpts(tol=1e-10, precision=zi.MIXED)).cpu().numpy()
    assert rel(Lg, Lo) <= 1e-6
    gsys.close()


def test_sparse_path_reproduces_partial_integration():
    """The partial-integration F fed column by column (four entries each) gives
    the lead field of zi_leadfield."""
    spec = W.three_shell(0.006, 16, 120, seed=4)
    mesh, osys, gsys, pos, dip = build(spec)
    F = O.source_matrix(osys.n, mesh["nodes"], mesh["tets"], dip).tocsc()
    F.sort_indices()
    ncols = F.shape[1]
    assert np.all(np.diff(F.indptr) == 4)
    Fn = F.indices.reshape(ncols, 4).astype(np.int32)
    Fw = F.data.reshape(ncols, 4)
    opts = zi.SolverOpts(tol=1e-12)
    L_pi = gsys.leadfield(torch.from_numpy(dip.astype(np.int32)), opts).cpu().numpy()
    L_sp = gsys.leadfield_sparse(Fn, Fw, opts).cpu().numpy()
    assert rel(L_sp, L_pi) <= 1e-12
    gsys.close()


def test_errors_are_reported_not_faulted():
    spec = W.unit_sphere_point(h=0.2, n_electrodes=8, n_dipoles=10)
    mesh, osys, gsys, pos, dip = build(spec)
    gsys.transfer(zi.SolverOpts(tol=1e-10))
    # a node index outside the mesh: the apply kernel's bounds check
    Fn = np.zeros((3, 8), dtype=np.int32)
    Fn[1, 2] = mesh["nodes"].shape[0]
    with pytest.raises(zi.ZiError) as e:
        gsys.leadfield_sparse(Fn, np.ones((3, 8)))
    assert e.value.status == zi.ZI_ERR_ARG
    # a tet index outside the mesh
    bad = dip.copy()
    bad[3] = mesh["tets"].shape[0]
    with pytest.raises(zi.ZiError) as e:
        gsys.source_stencil(pos, bad)
    assert e.value.status == zi.ZI_ERR_BAD_MESH
    # a Whitney stencil with two boundary faces cannot carry all three orientations
    _, opp = HD.face_neighbours(mesh["tets"], np.arange(mesh["tets"].shape[0]))
    two = np.nonzero(np.sum(opp < 0, axis=1) >= 2)[0]
    if two.size:
        t = two[:1]
        with pytest.raises(zi.ZiError) as e:
            gsys.source_stencil(mesh["nodes"][mesh["tets"][t]].mean(axis=1), t, zi.SOURCE_WHITNEY4)
        assert e.value.status == zi.ZI_ERR_BAD_MESH
        # the 10-source stencil still can
        Fn, Fw = gsys.source_stencil(mesh["nodes"][mesh["tets"][t]].mean(axis=1), t, zi.SOURCE_PBO10)
        assert np.all(np.isfinite(Fw.cpu().numpy()))
    with pytest.raises(zi.ZiError):
        gsys.source_stencil(pos, dip, 7)
    gsys.close()
