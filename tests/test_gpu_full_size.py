"""Full-size checks of the benchmark workloads, where the oracle's direct
factorisation is out of reach: properties that hold at any size, and the
mixed path against the FP64 GPU path (itself checked against the oracle on
smaller meshes with the same conductivity model)."""
import numpy as np
import pytest

from oracle import zi_oracle as O
from paper_1811_07717_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1811_07717_gb300 import zi  # noqa: E402


def _head(spec):
    mesh = zi.mesh_from_grid(spec.h, spec.radii)
    s6 = W.conductivity(spec, mesh["nodes"].cpu().numpy(), mesh["tets"].cpu().numpy(),
                        mesh["labels"].cpu().numpy())
    centres, z = W.electrode_inputs(spec)
    pos, q = W.dipole_inputs(spec)
    system = zi.System(mesh["nodes"], mesh["tets"], s6, mesh["bfaces"], centres, model="cem", z=z,
                       radius=spec.electrode_radius)
    dip = zi.locate_dipoles_grid(spec.h, spec.radii, pos)
    return mesh, s6, system, dip, pos


def test_two_mm_head_assembly_and_residuals():
    """2 mm three-shell head: A's values against the oracle's assembly, and the
    true FP64 residual of T recomputed on the CPU with the oracle's matrix."""
    spec = W.config_three_shell_2mm()
    mesh, s6, system, dip, pos = _head(spec)
    om = O.mesh_from_grid(spec.h, spec.radii)
    centres, z = W.electrode_inputs(spec)
    osys = O.System(om, s6, centres, "cem", radius=spec.electrode_radius, z=z)
    rp, ci, v, B, C, _ = [None if t is None else t.cpu().numpy() for t in system.matrix()]
    assert np.array_equal(rp, osys.A.indptr) and np.array_equal(ci, osys.A.indices)
    assert np.max(np.abs(v - osys.A.data)) <= 1e-14 * np.max(np.abs(osys.A.data))
    assert np.max(np.abs(B - osys.B)) <= 1e-14 * np.max(np.abs(osys.B))
    for prec in (zi.FP64, zi.MIXED):
        T, it, rr = system.transfer(zi.SolverOpts(tol=1e-10, precision=prec))
        T = T.cpu().numpy()
        res = np.linalg.norm(osys.A @ T - osys.B, axis=0) / np.linalg.norm(osys.B, axis=0)
        assert np.all(res <= 1.01e-10), res.max()
        assert np.allclose(res, rr, rtol=1e-3, atol=1e-15)
    # L is the method's function of T: the oracle's dense step applied to the
    # GPU's T.  S = C - B^T T cancels (C and B^T T nearly agree), so summation
    # order alone moves L by ~1e-10; the bound is the FP64 lead-field bar.
    F = O.source_matrix(osys.n, om["nodes"], om["tets"], O.locate_dipoles(om, pos[:2000]))
    L = system.leadfield(dip[:2000]).cpu().numpy()
    Lref = O.leadfield(osys, F, T=T)
    assert np.linalg.norm(L - Lref) <= 1e-8 * np.linalg.norm(Lref)
    system.close()


@pytest.mark.slow
def test_one_mm_anisotropic_head_mixed_vs_fp64():
    """1 mm head (3.34 M nodes, 19.6 M tets), transversely anisotropic skull,
    256 electrodes, 100k dipoles: the mixed-precision L within 1e-6 of the
    FP64 PCG L at tol 1e-13."""
    spec = W.config_three_shell_1mm_aniso()
    mesh, s6, system, dip, pos = _head(spec)
    assert mesh["nodes"].shape[0] == 3342701 and mesh["tets"].shape[0] == 19573872
    Lm = system.leadfield(dip, zi.SolverOpts(tol=1e-10, precision=zi.MIXED))
    T, it, rr = system.transfer(zi.SolverOpts(tol=1e-13, precision=zi.FP64), want_T=False)
    assert np.all(rr <= 1e-13)
    L64 = system.leadfield(dip)
    err = (torch.linalg.norm(Lm - L64) / torch.linalg.norm(L64)).item()
    assert err < 1e-6, err
    system.close()
