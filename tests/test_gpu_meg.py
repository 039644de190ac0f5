"""GPU parity of the MEG lead field (App. A.2 by the Biot-Savart formula)
through the C ABI: Bm against the oracle (anisotropic conductivity, CEM
surface terms skipped, chunked sensor loop bitwise equal to one chunk),
T_meg and L against the oracle (FP64 within 1e-8, mixed within 1e-6) for
partial-integration and H(div) source columns."""
import os

import numpy as np
import pytest

from oracle import hdiv as HD, meg as M, zi_oracle as O
from paper_1811_07717_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1811_07717_gb300 import zi  # noqa: E402


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


def build(spec, Ns, radius):
    mesh = O.mesh_from_grid(spec.h, spec.radii)
    s6 = W.conductivity(spec, mesh["nodes"], mesh["tets"], mesh["labels"])
    centres, z = W.electrode_inputs(spec)
    pos, _ = W.dipole_inputs(spec)
    osys = O.System(mesh, s6, centres, spec.electrode_model, radius=spec.electrode_radius, z=z)
    gsys = zi.System(mesh["nodes"], mesh["tets"], s6, mesh["bfaces"], centres, model=spec.electrode_model,
                     z=z if spec.electrode_model == "cem" else None, radius=spec.electrode_radius)
    sp_, sd = W.meg_sensors(Ns, radius)
    return mesh, s6, osys, gsys, sp_, sd, pos, O.locate_dipoles(mesh, pos)


def head():
    spec = W.three_shell(0.006, 16, 60, seed=21, skull_aniso=(0.00132, 0.0132), electrode_radius=0.009)
    return build(spec, 40, 0.112)


def test_meg_rhs_matches_the_oracle_and_chunks_agree(monkeypatch):
    mesh, s6, osys, gsys, sp_, sd, pos, dip = head()
    Bo = M.meg_rhs(osys, s6, sp_, sd)
    Bg = gsys.meg_rhs(sp_, sd).cpu().numpy()
    assert np.max(np.abs(Bg - Bo)) <= 1e-12 * np.max(np.abs(Bo))
    assert np.all(Bg[osys.ip] == 0.0)
    monkeypatch.setenv("ZI_MEG_SENSORS_PER_CHUNK", "7")
    Bc = gsys.meg_rhs(sp_, sd).cpu().numpy()
    assert np.array_equal(Bc, Bg)
    gsys.close()


def test_source_pi_matches_the_oracle():
    mesh, s6, osys, gsys, sp_, sd, pos, dip = head()
    Fn, Fw = gsys.source_pi(dip)
    Fo = O.source_matrix(osys.n, mesh["nodes"], mesh["tets"], dip).toarray()
    fn, fw = Fn.cpu().numpy(), Fw.cpu().numpy()
    Fg = np.zeros_like(Fo)
    for c in range(fn.shape[0]):
        for j in range(4):
            Fg[fn[c, j], c] += fw[c, j]
    assert np.max(np.abs(Fg - Fo)) <= 1e-12 * np.max(np.abs(Fo))
    gsys.close()


@pytest.mark.parametrize("source", ["pi", "pbo10"])
def test_meg_lead_field_fp64(source):
    mesh, s6, osys, gsys, sp_, sd, pos, dip = head()
    Tg, it, rr = gsys.meg_transfer(sp_, sd, zi.SolverOpts(tol=1e-12))
    To = M.meg_transfer(osys, s6, sp_, sd)
    assert rel(Tg.cpu().numpy(), To) <= 1e-8
    assert rr.max() <= 1e-12
    if source == "pi":
        Fn, Fw = gsys.source_pi(dip)
        F = O.source_matrix(osys.n, mesh["nodes"], mesh["tets"], dip)
    else:
        Fn, Fw = gsys.source_stencil(pos, dip, zi.SOURCE_PBO10)
        F = HD.source_matrix_hdiv(mesh["nodes"], mesh["tets"], dip, pos, HD.PBO10)
    Lg = gsys.meg_leadfield(Tg, sp_, sd, pos, Fn, Fw).cpu().numpy()
    Lo = M.meg_leadfield(osys, s6, sp_, sd, pos, F, Tm=To)
    assert Lg.shape == (sp_.shape[0], 3 * pos.shape[0])
    assert rel(Lg, Lo) <= 1e-8
    gsys.close()


def test_meg_lead_field_mixed_unit_sphere():
    spec = W.unit_sphere_point(h=0.1, n_electrodes=16, n_dipoles=80)
    mesh, s6, osys, gsys, sp_, sd, pos, dip = build(spec, 24, 1.2)
    Tg, _, _ = gsys.meg_transfer(sp_, sd, zi.SolverOpts(tol=1e-10, precision=zi.MIXED))
    Fn, Fw = gsys.source_pi(dip)
    Lg = gsys.meg_leadfield(Tg, sp_, sd, pos, Fn, Fw).cpu().numpy()
    F = O.source_matrix(osys.n, mesh["nodes"], mesh["tets"], dip)
    Lo = M.meg_leadfield(osys, s6, sp_, sd, pos, F)
    assert rel(Lg, Lo) <= 1e-6
    # the EEG transfer matrix of the handle is untouched by the MEG solve
    T, _, _ = gsys.transfer(zi.SolverOpts(tol=1e-12))
    assert rel(T.cpu().numpy(), osys.transfer()) <= 1e-8
    gsys.close()
