"""Linearised EIT on the GPU (App. A.3): the adjoint kernels behind the
torch.autograd.Function against the oracle's dense Jacobian and central
finite differences, and full-size properties on the 2 mm three-shell head."""
import math

import numpy as np
import pytest

from oracle import zi_oracle as O
from paper_1811_07717_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1811_07717_gb300 import eit, zi  # noqa: E402


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


def _setup(spec):
    mesh = zi.mesh_from_grid(spec.h, spec.radii)
    s6 = W.conductivity(spec, mesh["nodes"].cpu().numpy(), mesh["tets"].cpu().numpy(),
                        mesh["labels"].cpu().numpy())
    centres, z = W.electrode_inputs(spec)
    system = zi.System(mesh["nodes"], mesh["tets"], s6, mesh["bfaces"], centres, model="cem", z=z,
                       radius=spec.electrode_radius)
    return mesh, s6, centres, z, system


def test_autograd_vjp_matches_oracle_jacobian_unit_sphere():
    spec = W.unit_sphere_cem(h=0.1, n_electrodes=32)
    mesh, s6, centres, z, system = _setup(spec)
    I = W.injection_patterns(spec.n_electrodes)
    m = mesh["tets"].shape[0]
    log_s = torch.zeros(m, dtype=torch.float64, device="cuda", requires_grad=True)
    base = torch.from_numpy(s6).cuda()
    It = torch.from_numpy(I).cuda()
    y = eit.eit_voltages(log_s, system, base, It)
    G = torch.randn(y.shape, dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(3))
    (g,) = torch.autograd.grad((y * G).sum(), log_s)
    om = O.mesh_from_grid(spec.h, spec.radii)
    osys = O.System(om, s6, centres, "cem", radius=spec.electrode_radius, z=z)
    Jref, yref = O.eit_jacobian(osys, I)
    assert rel(y.detach().cpu().numpy(), yref) < 1e-9
    gref = np.einsum("pk,pkm->m", G.cpu().numpy(), Jref)
    assert rel(g.cpu().numpy(), gref) < 1e-8
    # full Jacobian on 50 random elements
    J, _ = eit.eit_jacobian(system, It)
    rng = np.random.default_rng(0)
    els = rng.choice(m, 50, replace=False)
    Jg = J.cpu().numpy()[els]                       # 50 x np x L
    Jr = np.transpose(Jref[:, :, els], (2, 0, 1))
    assert rel(Jg, Jr) < 1e-8
    system.close()


def test_jacobian_matches_central_differences():
    """GPU Jacobian against central differences (step 1e-6 in log s) of the
    oracle's direct-solve voltages on random elements of the h = 0.1 sphere."""
    spec = W.unit_sphere_cem(h=0.1, n_electrodes=32)
    mesh, s6, centres, z, system = _setup(spec)
    I = W.injection_patterns(spec.n_electrodes)
    J, y = eit.eit_jacobian(system, torch.from_numpy(I).cuda())
    J = J.cpu().numpy()
    om = O.mesh_from_grid(spec.h, spec.radii)
    rng = np.random.default_rng(7)
    eps = 1e-6
    for mi in rng.choice(mesh["tets"].shape[0], 8, replace=False):
        ys = []
        for sgn in (1, -1):
            sp = s6.copy()
            sp[mi] *= math.exp(sgn * eps)
            osys = O.System(om, sp, centres, "cem", radius=spec.electrode_radius, z=z)
            ys.append(O.eit_forward(osys, I)[0])
        fd = (ys[0] - ys[1]) / (2 * eps)
        assert np.linalg.norm(fd - J[mi]) <= 1e-6 * np.linalg.norm(J[mi]) + 1e-9 * np.linalg.norm(ys[0])
    system.close()


def test_backward_refuses_stale_system():
    spec = W.unit_sphere_cem(h=0.2, n_electrodes=16)
    mesh, s6, centres, z, system = _setup(spec)
    I = torch.from_numpy(W.injection_patterns(16)).cuda()
    log_s = torch.zeros(mesh["tets"].shape[0], dtype=torch.float64, device="cuda", requires_grad=True)
    base = torch.from_numpy(s6).cuda()
    y = eit.eit_voltages(log_s, system, base, I)
    system.set_conductivity(base)
    with pytest.raises(RuntimeError):
        y.sum().backward()
    system.close()


def test_full_size_eit_sum_rule_and_vjp_consistency():
    """2 mm three-shell head, 32 electrodes, 31 adjacent-pair 1 mA patterns.
    y is homogeneous of degree -1 in (sigma, 1/z): the Jacobian summed over
    all elements plus the derivative in a common log-scale of 1/z equals -y;
    and the VJP equals the contraction of the full Jacobian."""
    spec = W.config_eit_2mm()
    mesh, s6, centres, z, system = _setup(spec)
    I = torch.from_numpy(W.injection_patterns(spec.n_electrodes)).cuda()
    opts = zi.SolverOpts(tol=1e-12)
    J, y = eit.eit_jacobian(system, I, opts)
    Jsum = J.sum(dim=0).cpu().numpy()
    G = torch.randn(y.shape, dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(5))
    _, g = system.eit(I, mode=zi.EIT_VJP, grad_y=G, want_y=False, opts=opts)
    gJ = torch.einsum("mpk,pk->m", J, G)
    assert (torch.linalg.norm(g - gJ) / torch.linalg.norm(gJ)).item() < 1e-12
    del J
    eps = 1e-4
    yz = []
    for sgn in (1, -1):
        sz = zi.System(mesh["nodes"], mesh["tets"], s6, mesh["bfaces"], centres, model="cem",
                       z=z * math.exp(-sgn * eps), radius=spec.electrode_radius)
        yz.append(sz.eit(I, mode=None, opts=opts)[0].cpu().numpy())
        sz.close()
    dz = (yz[0] - yz[1]) / (2 * eps)
    yh = y.cpu().numpy()
    assert np.linalg.norm(Jsum + dz + yh) <= 1e-6 * np.linalg.norm(yh)
    system.close()


def test_log_conductivity_is_formed_in_the_library():
    """zi_system_set_log_conductivity assembles the same matrix as
    zi_system_set_conductivity of exp(log_s) * base (the EIT parametrisation
    is applied in libzi, not in torch)."""
    spec = W.unit_sphere_cem(h=0.2, n_electrodes=16)
    mesh, s6, centres, z, system = _setup(spec)
    m = mesh["tets"].shape[0]
    base = torch.from_numpy(s6).cuda()
    log_s = torch.from_numpy(np.random.default_rng(4).normal(0.0, 0.3, m)).cuda()
    system.set_log_conductivity(base, log_s)
    a = system.matrix()[2].cpu().numpy()
    system.set_conductivity((base * torch.exp(log_s)[:, None]).contiguous())
    b = system.matrix()[2].cpu().numpy()
    assert np.max(np.abs(a - b)) <= 1e-14 * np.max(np.abs(b))
    system.close()
