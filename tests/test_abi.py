"""CPU-side checks of the C ABI: the library loads, exports every symbol that
include/zi.h declares, and answers its argument checks; no GPU work runs."""
import ctypes
import os
import re

import pytest

from paper_1811_07717_gb300 import zi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "zi.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1811_07717_gb300 import _build
    _build.build()
    return zi.load_library()


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(zi_[a-z0-9_]+)\s*\(", src)))


def test_header_and_binding_agree():
    assert sorted(zi.EXPORTS) == _declared()


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_version_and_status_strings(lib):
    assert lib.zi_version() >= 10000
    assert lib.zi_status_string(0) == b"ZI_OK"
    assert lib.zi_status_string(4) == b"ZI_ERR_NOT_CONVERGED"


def test_argument_errors_need_no_gpu(lib):
    n = ctypes.c_int64()
    radii = (ctypes.c_double * 1)(1.0)
    # negative step, descending radii, null size outputs: rejected before any CUDA call
    assert lib.zi_mesh_from_grid(-1.0, 1, radii, ctypes.byref(n), ctypes.byref(n), ctypes.byref(n),
                                 None, None, None, None, None) == zi.ZI_ERR_ARG
    r2 = (ctypes.c_double * 2)(1.0, 0.5)
    assert lib.zi_mesh_from_grid(0.1, 2, r2, ctypes.byref(n), ctypes.byref(n), ctypes.byref(n),
                                 None, None, None, None, None) == zi.ZI_ERR_ARG
    assert lib.zi_mesh_from_grid(0.1, 1, radii, None, None, None, None, None, None, None, None) == zi.ZI_ERR_ARG
    buf = ctypes.create_string_buffer(256)
    assert lib.zi_last_error(buf, 256) == zi.ZI_ERR_ARG
    assert b"non-null" in buf.value
    assert lib.zi_assemble(None, 0, None, 0, None, None, 0, None, None, None) == zi.ZI_ERR_ARG
    assert lib.zi_transfer(None, None, None, None, None, None) == zi.ZI_ERR_ARG
    assert lib.zi_leadfield(None, None, 0, None, None, None) == zi.ZI_ERR_ARG
    assert lib.zi_eit_jacobian(None, None, 0, 0, None, None, None, None, None) == zi.ZI_ERR_ARG
    assert lib.zi_transfer_batched(None, 0, None, None, None, None) == zi.ZI_ERR_ARG
    assert lib.zi_ias_map(None, 4, 10, None, 1, 0.1, 1.0, 2.0, 0, 5, None, None, None) == zi.ZI_ERR_ARG
    assert lib.zi_source_stencil(None, None, None, 1, zi.SOURCE_PBO10, 0.0, None, None, None) == zi.ZI_ERR_ARG
    assert lib.zi_leadfield_sparse(None, None, None, 1, 8, None, None, None) == zi.ZI_ERR_ARG
    assert lib.zi_source_pi(None, None, 1, None, None, None) == zi.ZI_ERR_ARG
    ms = ctypes.c_double()
    assert lib.zi_time_source_apply(None, None, None, 3, 8, 2, ctypes.byref(ms), None, None) == zi.ZI_ERR_ARG
    assert lib.zi_nearest_source(None, 4, None, 0, None, None) == zi.ZI_ERR_ARG
    assert lib.zi_nearest_source(None, 4, None, 3, None, None) == zi.ZI_ERR_ARG
    toff = (ctypes.c_int64 * 2)(0, 4)
    pr = (ctypes.c_int32 * 1)(1)
    assert lib.zi_mesh_from_surfaces(0.1, 1, toff, pr, None, 4, None, ctypes.byref(n), ctypes.byref(n),
                                     ctypes.byref(n), None, None, None, None, None) == zi.ZI_ERR_ARG
    assert lib.zi_mesh_from_surfaces(-1.0, 1, toff, pr, None, 4, None, ctypes.byref(n), ctypes.byref(n),
                                     ctypes.byref(n), None, None, None, None, None) == zi.ZI_ERR_ARG
    assert lib.zi_meg_rhs(None, None, None, None, 4, None, None) == zi.ZI_ERR_ARG
    assert lib.zi_meg_transfer(None, None, None, None, 4, None, None, None, None, None) == zi.ZI_ERR_ARG
    assert lib.zi_meg_leadfield(None, None, None, None, 4, None, 1, None, None, 4, None, None) == zi.ZI_ERR_ARG
    o = zi._Opts()
    lib.zi_solver_opts_default(ctypes.byref(o))
    assert lib.zi_apply_operator(None, ctypes.byref(o), None, None, None, None) == zi.ZI_ERR_ARG
    assert lib.zi_solver_get_info(None, None) == zi.ZI_ERR_ARG
    assert lib.zi_locate_points(None, 0, None, 0, None, 1, None, None) == zi.ZI_ERR_ARG
    assert lib.zi_system_set_log_conductivity(None, None, None, None) == zi.ZI_ERR_ARG
    assert lib.zi_leadfield_at(None, None, 1, ctypes.byref(o), None, None) == zi.ZI_ERR_ARG
    assert lib.zi_batch_tune(None, 0, ctypes.byref(o), None, None, None) == zi.ZI_ERR_ARG
    assert lib.zi_transfer_batched_schedule(None, 0, ctypes.byref(o), None, None, None, 0, None) == zi.ZI_ERR_ARG


def test_default_solver_options(lib):
    o = zi._Opts()
    lib.zi_solver_opts_default(ctypes.byref(o))
    assert o.tol == 1e-10 and o.precond == zi.PRECOND_JACOBI and o.precision == zi.FP64
    assert o.maxit > 0


def test_product_path_has_no_cpu_fallback():
    """The binding raises instead of computing anything on the CPU."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    with pytest.raises(RuntimeError):
        zi.mesh_from_grid(0.1, [1.0])
