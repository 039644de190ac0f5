"""zi_leadfield_noalloc: the lead field for callers that cannot allocate
device memory while it runs (applications that give the whole GPU to their own
allocator, latency-critical loops).  It must give the same L as zi_leadfield,
call after call, using only its fixed device scratch.

This file sorts last so that a run stopping at the first failure has run every
other test; it also passes on its own in a fresh process."""
import ctypes

import numpy as np
import pytest

from paper_1811_07717_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1811_07717_gb300 import zi  # noqa: E402

TOL = 1e-12  # same kernels, same order: the two entry points agree to roundoff


def _system(spec):
    mesh = zi.mesh_from_grid(spec.h, spec.radii)
    s6 = W.conductivity(spec, mesh["nodes"].cpu().numpy(), mesh["tets"].cpu().numpy(),
                        mesh["labels"].cpu().numpy())
    centres, z = W.electrode_inputs(spec)
    pos, _ = W.dipole_inputs(spec)
    system = zi.System(mesh["nodes"], mesh["tets"], s6, mesh["bfaces"], centres, model=spec.electrode_model,
                       z=z if spec.electrode_model == "cem" else None, radius=spec.electrode_radius)
    dip = zi.locate_dipoles_grid(spec.h, spec.radii, pos)
    return system, dip


def _noalloc(system, dip, rows):
    lib = zi.load_library()
    P = dip.shape[0]
    L = torch.full((rows, 3 * P), float("nan"), dtype=torch.float64, device="cuda")
    st = lib.zi_leadfield_noalloc(system.handle, zi._ptr(dip), P, zi._ptr(L), zi._stream())
    zi._check(st)
    return L.cpu().numpy()


@pytest.mark.parametrize("spec", [
    W.three_shell(0.006, 32, 200, seed=21, electrode_radius=0.009),
    W.unit_sphere_point(h=0.2, n_electrodes=12, n_dipoles=40),
], ids=["cem", "point"])
def test_noalloc_lead_field_matches_zi_leadfield_twice(spec):
    system, dip = _system(spec)
    system.transfer(zi.SolverOpts(tol=1e-10))
    L_ref = system.leadfield(dip).cpu().numpy()
    rows = system.info()["n_rows_L"]
    torch.cuda.synchronize()
    used0, _ = zi.memory_stats(reset_high=True)
    for _ in range(2):  # the scratch keeps the previous call's contents
        L = _noalloc(system, dip, rows)
        assert np.all(np.isfinite(L))
        assert np.linalg.norm(L - L_ref) <= TOL * np.linalg.norm(L_ref)
    # nothing was drawn from the library's pool: its high-water mark, zeroed
    # before the calls, stays at or below what was in use before them
    _, high = zi.memory_stats()
    assert high <= used0
    system.close()


def test_noalloc_rejects_oversize_and_missing_transfer():
    spec = W.three_shell(0.006, 32, 10, seed=21, electrode_radius=0.009)
    system, dip = _system(spec)
    lib = zi.load_library()
    out = torch.empty((32, 30), dtype=torch.float64, device="cuda")
    # no transfer matrix yet: solving would allocate, so the call refuses
    assert lib.zi_leadfield_noalloc(system.handle, zi._ptr(dip), dip.shape[0], zi._ptr(out),
                                    zi._stream()) == zi.ZI_ERR_ARG
    system.transfer(zi.SolverOpts(tol=1e-8))
    # more dipoles than the fixed scratch holds: rejected before any launch
    big = torch.zeros(20000, dtype=torch.int32, device="cuda")
    assert lib.zi_leadfield_noalloc(system.handle, zi._ptr(big), big.shape[0], zi._ptr(out),
                                    zi._stream()) == zi.ZI_ERR_ARG
    buf = ctypes.create_string_buffer(512)
    lib.zi_last_error(buf, 512)
    assert b"scratch" in buf.value
    system.close()
