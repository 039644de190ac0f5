"""GPU parity of the IAS MAP inversion (App. B, zi_ias_map) against the CPU
oracle: random problems with ragged sizes, both hypermodels, a lead field of
the CUDA path itself, and the degenerate case of no rounds."""
import numpy as np
import pytest

from oracle import ias as I
from paper_1811_07717_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1811_07717_gb300 import zi  # noqa: E402


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def run_both(L, Y, nu, theta0, beta, hyper, iters):
    X, Th = zi.ias_map(torch.from_numpy(L).cuda(), torch.from_numpy(Y.T.copy()).cuda(), nu, theta0, beta, hyper,
                       iters)
    Xr, Thr = I.ias_map(L, Y, nu, theta0, beta, hyper, iters)
    return X.cpu().numpy().T, Th.cpu().numpy().T, Xr, Thr


@pytest.mark.parametrize("hyper", [zi.HYPER_G, zi.HYPER_IG], ids=["G", "IG"])
@pytest.mark.parametrize("Le,n,T", [(12, 40, 3), (37, 1000, 2), (64, 2049, 5)])
def test_ias_matches_oracle(hyper, Le, n, T):
    rng = np.random.default_rng(Le * 7 + n)
    L = rng.standard_normal((Le, n))
    x_true = np.zeros((n, T))
    x_true[rng.choice(n, 4, replace=False), :] = rng.standard_normal((4, T))
    Y = L @ x_true + 0.02 * rng.standard_normal((Le, T))
    X, Th, Xr, Thr = run_both(L, Y, 0.05, 0.1, 1.9, hyper, 12)
    assert rel(X, Xr) < 1e-9
    assert rel(Th, Thr) < 1e-9


def test_ias_on_a_lead_field():
    spec = W.three_shell(0.006, 32, 200, seed=21, electrode_radius=0.009)
    mesh = zi.mesh_from_grid(spec.h, spec.radii)
    s6 = W.conductivity(spec, mesh["nodes"].cpu().numpy(), mesh["tets"].cpu().numpy(),
                        mesh["labels"].cpu().numpy())
    centres, z = W.electrode_inputs(spec)
    pos, _ = W.dipole_inputs(spec)
    system = zi.System(mesh["nodes"], mesh["tets"], s6, mesh["bfaces"], centres, model="cem", z=z,
                       radius=spec.electrode_radius)
    dip = zi.locate_dipoles_grid(spec.h, spec.radii, pos)
    Lg = system.leadfield(dip, zi.SolverOpts(tol=1e-10))
    system.close()
    L = Lg.cpu().numpy()
    rng = np.random.default_rng(4)
    n = L.shape[1]
    x_true = np.zeros((n, 4))
    x_true[rng.choice(n, 3, replace=False), :] = rng.standard_normal((3, 4)) * 1e-8
    Y = L @ x_true
    nu = 0.02 * np.abs(Y).max()
    Y = Y + nu * rng.standard_normal(Y.shape)
    X, Th, Xr, Thr = run_both(L, Y, nu, 1e-16, 1.6, zi.HYPER_G, 10)
    assert rel(X, Xr) < 1e-9
    assert rel(Th, Thr) < 1e-9


def test_zero_rounds_and_argument_checks():
    L = torch.randn(8, 50, dtype=torch.float64, device="cuda")
    Y = torch.randn(2, 8, dtype=torch.float64, device="cuda")
    X, Th = zi.ias_map(L, Y, 0.1, 0.5, 2.0, zi.HYPER_IG, 0)
    assert torch.count_nonzero(X) == 0 and torch.all(Th == 0.5)
    with pytest.raises(zi.ZiError):
        zi.ias_map(L, Y, -0.1, 0.5, 2.0, zi.HYPER_G, 3)
    with pytest.raises(zi.ZiError):
        zi.ias_map(torch.randn(300, 10, dtype=torch.float64, device="cuda"), torch.randn(1, 300, dtype=torch.float64,
                                                                                          device="cuda"), 0.1, 0.5, 2.0)
