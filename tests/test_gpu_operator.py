"""Unit parity of the solver's own sparse operator and its fused column
reduction (the product of A, App. A.1, with the search directions of every
right-hand side, Sec. 2.3.1), through zi_apply_operator, row by row against
the oracle's assembled A:

* FP64: Y = S A~ S X, the FP64 CG's operator, S = diag(A)^-1/2 (Jacobi);
  per row within 1e-14 of sum_j |s_i a_ij s_j x_j| plus the couplings the
  FP64 copy omits as assembly noise (|a_ij| <= 2^-40 sqrt(a_ii a_jj));
* FP32: Y = A x16 by the difference form c_i x_i + sum_j a_ij (x_j - x_i),
  where x16 is X rounded to FP16 (round to nearest even), the storage of the
  FP32 path's search directions; per row within 20 unit roundoffs of FP32 of
  |c_i x_i| + sum_j |a_ij| |x_j - x_i| plus the couplings the FP32 copy
  leaves to c_i (|a_ij| <= 2^-24 sqrt(a_ii a_jj)) and the FP64 rounding of
  the reference A x16;
* the fused dots against FP64 host sums of the same x and y;
at 32, 128 and 256 right-hand sides on an anisotropic-skull head whose rows
overflow the eight ELL slots (the layout is asserted).  More than 256
right-hand sides are refused before any solver launch."""
import numpy as np
import pytest

from oracle import zi_oracle as O
from paper_1811_07717_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1811_07717_gb300 import zi  # noqa: E402

U32 = 2.0 ** -24
# right-hand sides and electrode radii (6 mm head), with the FP64 layout each
# gets: one, two or four 16-byte vectors of a row per thread
SIZES = [(32, 0.009), (128, 0.006), (256, 0.005)]
SIZE_IDS = ["ld32", "ld128", "ld256"]
VECTORS64 = {32: 1, 128: 2, 256: 4}


def head(L, radius):
    spec = W.three_shell(0.006, L, 10, seed=21, skull_aniso=(0.00132, 0.0132), electrode_radius=radius)
    mesh = zi.mesh_from_grid(spec.h, spec.radii)
    s6 = W.conductivity(spec, *(mesh[k].cpu().numpy() for k in ("nodes", "tets", "labels")))
    centres, z = W.electrode_inputs(spec)
    gs = zi.System(mesh["nodes"], mesh["tets"], s6, mesh["bfaces"], centres, model="cem", z=z,
                   radius=spec.electrode_radius)
    om = O.mesh_from_grid(spec.h, spec.radii)
    osys = O.System(om, W.conductivity(spec, om["nodes"], om["tets"], om["labels"]), centres, "cem",
                    radius=spec.electrode_radius, z=z)
    return gs, osys.A.tocsr()


def inputs(n, L, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, L))
    X[:, 0] = 1.0 + 1e-3 * rng.standard_normal(n)   # a nearly constant column: the difference form's case
    return X


def fp16_direction(X):
    """X as the FP32 path stores a search direction: FP16, round to nearest
    even (subnormals kept)."""
    return X.astype(np.float16).astype(np.float64)


def noise_mask(A, cut):
    """Off-diagonal couplings with |a_ij| <= cut * sqrt(|a_ii a_jj|)."""
    d = np.abs(A.diagonal())
    rows = np.repeat(np.arange(A.shape[0]), np.diff(A.indptr))
    return (rows != A.indices) & (np.abs(A.data) <= cut * np.sqrt(d[rows] * d[A.indices])), rows


@pytest.mark.parametrize("L,radius", SIZES, ids=SIZE_IDS)
def test_fp64_operator_and_dots(L, radius):
    gs, A = head(L, radius)
    n = A.shape[0]
    X = inputs(n, L, 1)
    Y, dots = gs.apply_operator(X, zi.SolverOpts(precision=zi.FP64))
    Y, dots = Y.cpu().numpy(), dots.cpu().numpy()
    s = 1.0 / np.sqrt(A.diagonal())
    As = A.multiply(s[:, None]).multiply(s[None, :]).tocsr()
    ref = As @ X
    absA = As.copy()
    absA.data = np.abs(absA.data)
    mask, rows = noise_mask(A, 2.0 ** -40)
    dropped = absA.copy()
    dropped.data = np.where(mask, dropped.data, 0.0)
    tol = 1e-14 * (absA @ np.abs(X)) + dropped @ np.abs(X)
    assert np.all(np.abs(Y - ref) <= tol)
    inf = gs.solver_info()
    assert inf["ld"] == L and inf["nnz64"] == A.nnz - int(mask.sum())
    assert inf["vectors_per_thread64"] == VECTORS64[L]
    assert inf["threads_per_row64"] * inf["vectors_per_thread64"] * 2 == L
    host = np.einsum("ic,ic->c", X, Y)
    assert np.all(np.abs(dots - host) <= 1e-12 * np.einsum("ic,ic->c", np.abs(X), np.abs(Y)))
    gs.close()


@pytest.mark.parametrize("order", ["rows", "tiles"])
@pytest.mark.parametrize("L,radius", SIZES, ids=SIZE_IDS)
def test_fp32_difference_form_operator_and_dots(L, radius, order, monkeypatch):
    """Both storage orders of the FP32 ELL copy (row order, and the tile
    columns used on large grids) give the same operator."""
    monkeypatch.setenv("ZI_ELL_ORDER", order)
    gs, A = head(L, radius)
    n = A.shape[0]
    X = inputs(n, L, 2)
    Y, dots = gs.apply_operator(X, zi.SolverOpts(precision=zi.MIXED))
    Y, dots = Y.cpu().numpy(), dots.cpu().numpy()
    x16 = fp16_direction(X)                            # the FP16 direction the kernel reads
    ref = A @ x16
    mask, rows = noise_mask(A, U32)
    c = np.asarray(A.sum(axis=1)).ravel()
    off = rows != A.indices
    diff = np.abs(x16[A.indices] - x16[rows])                       # |x_j - x_i| per stored entry
    w = (np.abs(A.data) * off)[:, None] * diff
    bound = np.zeros_like(X)
    dropped = np.zeros_like(X)
    np.add.at(bound, rows, w)
    np.add.at(dropped, rows, w * mask[:, None])
    # plus the reference's own FP64 rounding (rows hold at most 27 entries): it
    # matters where FP16 makes a row's neighbour values equal (bound = 0)
    absA = abs(A)
    tol = 20 * U32 * (np.abs(c)[:, None] * np.abs(x16) + bound) + dropped + 32 * 2.0 ** -53 * (absA @ np.abs(x16))
    assert np.all(np.abs(Y - ref) <= tol)
    inf = gs.solver_info()
    assert inf["spmm32"] == zi.SPMM32_ELL_OVERFLOW          # anisotropic rows overflow the 8 slots
    assert inf["ell_tiled"] == (order == "tiles")
    assert inf["vectors_per_thread32"] == 1
    assert inf["threads_per_row32"] * 4 == L
    kept_len = np.bincount(rows[~mask], minlength=n)
    assert inf["nnz32"] == int(kept_len.sum())
    assert inf["tail_rows"] == int((kept_len > 8).sum()) and inf["tail_rows"] * 20 > n
    host = np.einsum("ic,ic->c", x16, Y)
    assert np.all(np.abs(dots - host) <= 1e-5 * np.einsum("ic,ic->c", np.abs(x16), np.abs(Y)))
    gs.close()


def test_more_than_256_right_hand_sides_refused():
    """The solver keeps one shared-memory total per column, 256 at most: a
    320-electrode system is refused by the operator and the transfer solve
    before any solver kernel runs (and the SpMM timer finds no solver state)."""
    spec = W.three_shell(0.006, 320, 10, seed=21, electrode_radius=0.0045)
    mesh = zi.mesh_from_grid(spec.h, spec.radii)
    s6 = W.conductivity(spec, *(mesh[k].cpu().numpy() for k in ("nodes", "tets", "labels")))
    centres, z = W.electrode_inputs(spec)
    gs = zi.System(mesh["nodes"], mesh["tets"], s6, mesh["bfaces"], centres, model="cem", z=z,
                   radius=spec.electrode_radius)
    n = mesh["nodes"].shape[0]
    for prec in (zi.FP64, zi.MIXED):
        with pytest.raises(zi.ZiError, match="right-hand sides"):
            gs.apply_operator(np.zeros((n, 320)), zi.SolverOpts(precision=prec))
        with pytest.raises(zi.ZiError):                     # no solver state was ever built
            gs.time_spmm(prec, reps=1)
        with pytest.raises(zi.ZiError, match="right-hand sides"):
            gs.transfer(zi.SolverOpts(tol=1e-8, precision=prec), want_T=False)
    gs.close()


def test_operator_of_zero_block_is_zero():
    gs, A = head(32, 0.009)
    for prec in (zi.FP64, zi.MIXED):
        Y, dots = gs.apply_operator(np.zeros((A.shape[0], 32)), zi.SolverOpts(precision=prec))
        assert not torch.any(Y) and not torch.any(dots)
    gs.close()


@pytest.mark.parametrize("order", ["rows", "tiles"])
def test_mixed_lead_field_on_the_overflow_layout(order, monkeypatch):
    """The mixed-precision lead field of the anisotropic head runs the
    overflow-slot FP32 layout, in either storage order of the ELL copy, and
    stays within 1e-6 of the oracle."""
    monkeypatch.setenv("ZI_ELL_ORDER", order)
    spec = W.three_shell(0.006, 64, 100, seed=23, skull_aniso=(0.00132, 0.0132), electrode_radius=0.008)
    mesh = zi.mesh_from_grid(spec.h, spec.radii)
    s6 = W.conductivity(spec, *(mesh[k].cpu().numpy() for k in ("nodes", "tets", "labels")))
    centres, z = W.electrode_inputs(spec)
    pos, _ = W.dipole_inputs(spec)
    gs = zi.System(mesh["nodes"], mesh["tets"], s6, mesh["bfaces"], centres, model="cem", z=z,
                   radius=spec.electrode_radius)
    dip = zi.locate_dipoles_grid(spec.h, spec.radii, pos)
    Lg = gs.leadfield(dip, zi.SolverOpts(tol=1e-10, precision=zi.MIXED)).cpu().numpy()
    assert gs.solver_info()["spmm32"] == zi.SPMM32_ELL_OVERFLOW
    assert gs.solver_info()["ell_tiled"] == (order == "tiles")
    Lref, *_ = O.leadfield_from_spec(spec, W)
    assert np.linalg.norm(Lg - Lref) <= 1e-6 * np.linalg.norm(Lref)
    gs.close()
