"""Batched transfer solve: many heads of different sizes and electrode counts,
in the autotuned schedule and with every head in the persistent launch,
against per-head solves and the oracle; the autotuner's choice and cache."""
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


SPECS = [
    W.three_shell(0.006, 16, 40, seed=31, electrode_radius=0.009),
    W.three_shell(0.008, 32, 40, seed=32, r_out=0.1, electrode_radius=0.012),
    W.unit_sphere_point(h=0.2, n_electrodes=12, n_dipoles=30),
    W.three_shell(0.005, 64, 40, seed=33, r_out=0.085, electrode_radius=0.007),
]


def _build(spec):
    mesh = zi.mesh_from_grid(spec.h, spec.radii)
    s6 = W.conductivity(spec, mesh["nodes"].cpu().numpy(), mesh["tets"].cpu().numpy(),
                        mesh["labels"].cpu().numpy())
    centres, z = W.electrode_inputs(spec)
    pos, _ = W.dipole_inputs(spec)
    system = zi.System(mesh["nodes"], mesh["tets"], s6, mesh["bfaces"], centres, model=spec.electrode_model,
                       z=z if spec.electrode_model == "cem" else None, radius=spec.electrode_radius)
    dip = zi.locate_dipoles_grid(spec.h, spec.radii, pos)
    return system, dip


@pytest.mark.parametrize("schedule", ["tuned", "persistent"])
@pytest.mark.parametrize("precision", [zi.FP64, zi.MIXED], ids=["fp64", "mixed"])
def test_batched_matches_per_head_solves(precision, schedule):
    opts = zi.SolverOpts(tol=1e-10, precision=precision)
    built = [_build(sp) for sp in SPECS]
    systems = [b[0] for b in built]
    Tb, itb = zi.transfer_batched(systems, opts, want_T=True,
                                  persistent=None if schedule == "tuned" else [1] * len(systems))
    for (system, dip), spec, T, it in zip(built, SPECS, Tb, itb):
        assert np.all(it > 0)
        single = _build(spec)[0]
        Ts, its, rr = single.transfer(opts)
        assert rel(T.cpu().numpy(), Ts.cpu().numpy()) < 1e-8
        single.close()
        # the batched T feeds the lead field directly
        L = system.leadfield(dip).cpu().numpy()
        Lref, *_ = O.leadfield_from_spec(spec, W)
        assert rel(L, Lref) < (1e-8 if precision == zi.FP64 else 1e-6)
        system.close()


def test_batched_is_deterministic():
    opts = zi.SolverOpts(tol=1e-10, precision=zi.MIXED)
    outs = []
    for _ in range(2):
        systems = [_build(sp)[0] for sp in SPECS[:3]]
        Tb, itb = zi.transfer_batched(systems, opts, want_T=True)
        outs.append([t.cpu().numpy() for t in Tb])
        for s in systems:
            s.close()
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


def test_batched_rejects_duplicates():
    system, _ = _build(SPECS[2])
    with pytest.raises(zi.ZiError):
        zi.transfer_batched([system, system])
    system.close()


def test_barrier_timeout_is_reported_and_context_survives(monkeypatch):
    """Failure detection of the persistent launch: one block leaves before its
    first barrier (test-only injection), the other blocks of its head give up
    after their bounded wait and the call returns ZI_ERR_TIMEOUT; the GPU
    context stays usable and the next solve is correct."""
    built = [_build(sp) for sp in SPECS[:2]]
    systems = [b[0] for b in built]
    opts = zi.SolverOpts(tol=1e-10, precision=zi.FP64)
    monkeypatch.setenv("ZI_TEST_BARRIER_SKIP", "1")
    with pytest.raises(zi.ZiError) as e:
        zi.transfer_batched(systems, opts, persistent=[1, 1])
    assert e.value.status == zi.ZI_ERR_TIMEOUT
    monkeypatch.delenv("ZI_TEST_BARRIER_SKIP")
    Tb, itb = zi.transfer_batched(systems, opts, want_T=True, persistent=[1, 1])
    single = _build(SPECS[0])[0]
    Ts, _, _ = single.transfer(opts)
    assert rel(Tb[0].cpu().numpy(), Ts.cpu().numpy()) < 1e-8
    for s in systems + [single]:
        s.close()


def test_autotuner_picks_the_fastest_estimate_and_caches_it():
    """The tuned schedule's estimated time per iteration is no worse than
    every head alone or every head in the persistent launch (both are
    candidates); a second call of the same signature comes from the cache."""
    opts = zi.SolverOpts(tol=1e-10, precision=zi.MIXED)
    systems = [_build(sp)[0] for sp in SPECS[::-1]]
    mask, info = zi.batch_tune(systems, opts)
    assert info["source"] == zi.BATCH_TUNED and len(mask) == len(systems)
    assert info["est_window_ms"] <= info["est_window_ms_per_head"]
    assert info["est_window_ms"] <= info["est_window_ms_persistent"]
    assert sum(mask) != 1                       # a persistent set of one head is never chosen
    mask2, info2 = zi.batch_tune(systems, opts)
    assert info2["source"] == zi.BATCH_CACHED and mask2 == mask
    Tb, _ = zi.transfer_batched(systems, opts, want_T=True)
    Tp, _ = zi.transfer_batched(systems, opts, want_T=True, persistent=mask, chunk=16)
    for a, b in zip(Tb, Tp):
        assert torch.equal(a, b)               # zi_transfer_batched runs the cached schedule
    for s in systems:
        s.close()
