"""Python binding of libzi (include/zi.h): argument marshalling only.

Every step of the lead-field build runs in the CUDA library; this module
turns torch CUDA tensors into raw device pointers, the current torch stream
into a cudaStream_t, and zi_status codes into exceptions.  There is no CPU
path: if libzi.so is missing or no GPU is present, calls raise.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libzi.so")

ZI_OK, ZI_ERR_ARG, ZI_ERR_BAD_MESH, ZI_ERR_NONFINITE = 0, 1, 2, 3
ZI_ERR_NOT_CONVERGED, ZI_ERR_TIMEOUT, ZI_ERR_CUDA, ZI_ERR_NOMEM = 4, 5, 6, 7
ELECTRODE_POINT, ELECTRODE_CEM = 0, 1
PRECOND_JACOBI, PRECOND_LDP = 0, 1
FP64, MIXED = 0, 1
EIT_FULL, EIT_VJP = 0, 1
HYPER_G, HYPER_IG = 0, 1
SOURCE_WHITNEY4, SOURCE_PBO10 = 0, 1
STENCIL_WIDTH = 8

# Every symbol include/zi.h declares.
EXPORTS = ("zi_version", "zi_last_error", "zi_status_string", "zi_mesh_from_grid", "zi_locate_dipoles_grid",
           "zi_mesh_from_surfaces", "zi_nearest_source", "zi_locate_points", "zi_leadfield_at",
           "zi_system_set_log_conductivity", "zi_assemble", "zi_system_set_conductivity",
           "zi_system_get_info", "zi_system_get_matrix", "zi_system_destroy", "zi_solver_opts_default",
           "zi_transfer", "zi_transfer_batched", "zi_leadfield", "zi_source_stencil", "zi_leadfield_sparse",
           "zi_source_pi", "zi_meg_rhs", "zi_meg_transfer", "zi_meg_leadfield", "zi_eit_jacobian",
           "zi_leadfield_noalloc", "zi_ias_map", "zi_time_spmm", "zi_time_source_apply", "zi_apply_operator",
           "zi_solver_get_info", "zi_batch_tune", "zi_transfer_batched_schedule", "zi_memory_stats",
           "zi_kernel_launches")

SPMM32_NONE, SPMM32_ELL, SPMM32_ELL_OVERFLOW = 0, 1, 2


class ZiError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (_status_name(status), msg))
        self.status = status


class NotConverged(ZiError):
    pass


class _Electrodes(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int32), ("n", ctypes.c_int32), ("centres", ctypes.c_void_p),
                ("z", ctypes.c_void_p), ("radius", ctypes.c_double)]


class _Info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("m", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("n_el", ctypes.c_int32), ("n_rhs", ctypes.c_int32), ("n_rows_L", ctypes.c_int32),
                ("model", ctypes.c_int32), ("ground", ctypes.c_int64), ("n_patch_faces", ctypes.c_int64),
                ("has_T", ctypes.c_int32)]


class _SolverInfo(ctypes.Structure):
    _fields_ = [("ld", ctypes.c_int32), ("threads_per_row64", ctypes.c_int32),
                ("vectors_per_thread64", ctypes.c_int32), ("threads_per_row32", ctypes.c_int32),
                ("vectors_per_thread32", ctypes.c_int32), ("spmm32", ctypes.c_int32),
                ("nnz64", ctypes.c_int64), ("nnz32", ctypes.c_int64), ("tail_rows", ctypes.c_int64),
                ("tail_entries", ctypes.c_int64), ("ell_tiled", ctypes.c_int32)]


class _BatchSchedule(ctypes.Structure):
    _fields_ = [("source", ctypes.c_int32), ("est_window_ms", ctypes.c_double),
                ("est_window_ms_per_head", ctypes.c_double),
                ("est_window_ms_persistent", ctypes.c_double)]


BATCH_TUNED, BATCH_CACHED = 1, 2


class _Opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("maxit", ctypes.c_int32), ("precond", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("inner_tol", ctypes.c_double),
                ("max_outer", ctypes.c_int32), ("check_every", ctypes.c_int32)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Loads libzi.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libzi.so not found at %s; build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`" % path)
    lib = ctypes.CDLL(path)
    P, I32, I64, D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    sig = {
        "zi_version": ([], ctypes.c_int),
        "zi_last_error": ([ctypes.c_char_p, ctypes.c_size_t], ctypes.c_int),
        "zi_status_string": ([ctypes.c_int], ctypes.c_char_p),
        "zi_mesh_from_grid": ([D, ctypes.c_int, P, P, P, P, P, P, P, P, P], ctypes.c_int),
        "zi_locate_dipoles_grid": ([D, ctypes.c_int, P, P, I64, P, P], ctypes.c_int),
        "zi_nearest_source": ([P, I64, P, I64, P, P], ctypes.c_int),
        "zi_locate_points": ([P, I64, P, I64, P, I64, P, P], ctypes.c_int),
        "zi_leadfield_at": ([P, P, I64, ctypes.POINTER(_Opts), P, P], ctypes.c_int),
        "zi_mesh_from_surfaces": ([D, ctypes.c_int, P, P, P, I64, P, P, P, P, P, P, P, P, P], ctypes.c_int),
        "zi_assemble": ([P, I64, P, I64, P, P, I64, ctypes.POINTER(_Electrodes), P, P], ctypes.c_int),
        "zi_system_set_conductivity": ([P, P, P], ctypes.c_int),
        "zi_system_set_log_conductivity": ([P, P, P, P], ctypes.c_int),
        "zi_system_get_info": ([P, ctypes.POINTER(_Info)], ctypes.c_int),
        "zi_system_get_matrix": ([P, P, P, P, P, P, P, P], ctypes.c_int),
        "zi_system_destroy": ([P], None),
        "zi_solver_opts_default": ([ctypes.POINTER(_Opts)], None),
        "zi_transfer": ([P, ctypes.POINTER(_Opts), P, P, P, P], ctypes.c_int),
        "zi_transfer_batched": ([P, ctypes.c_int, ctypes.POINTER(_Opts), P, P, P], ctypes.c_int),
        "zi_leadfield": ([P, P, I64, ctypes.POINTER(_Opts), P, P], ctypes.c_int),
        "zi_source_stencil": ([P, P, P, I64, ctypes.c_int, D, P, P, P], ctypes.c_int),
        "zi_leadfield_sparse": ([P, P, P, I64, ctypes.c_int, ctypes.POINTER(_Opts), P, P], ctypes.c_int),
        "zi_source_pi": ([P, P, I64, P, P, P], ctypes.c_int),
        "zi_meg_rhs": ([P, P, P, P, ctypes.c_int, P, P], ctypes.c_int),
        "zi_meg_transfer": ([P, P, P, P, ctypes.c_int, ctypes.POINTER(_Opts), P, P, P, P], ctypes.c_int),
        "zi_meg_leadfield": ([P, P, P, P, ctypes.c_int, P, I64, P, P, ctypes.c_int, P, P], ctypes.c_int),
        "zi_eit_jacobian": ([P, P, ctypes.c_int, ctypes.c_int, P, P, P, ctypes.POINTER(_Opts), P], ctypes.c_int),
        "zi_leadfield_noalloc": ([P, P, I64, P, P], ctypes.c_int),
        "zi_ias_map": ([P, I32, I64, P, I32, D, D, D, I32, I32, P, P, P], ctypes.c_int),
        "zi_time_spmm": ([P, ctypes.c_int, ctypes.c_int, ctypes.POINTER(D), ctypes.POINTER(D), P], ctypes.c_int),
        "zi_time_source_apply": ([P, P, P, I64, ctypes.c_int, ctypes.c_int, ctypes.POINTER(D),
                                  ctypes.POINTER(D), P], ctypes.c_int),
        "zi_apply_operator": ([P, ctypes.POINTER(_Opts), P, P, P, P], ctypes.c_int),
        "zi_solver_get_info": ([P, ctypes.POINTER(_SolverInfo)], ctypes.c_int),
        "zi_batch_tune": ([P, ctypes.c_int, ctypes.POINTER(_Opts), P, ctypes.POINTER(_BatchSchedule), P],
                          ctypes.c_int),
        "zi_transfer_batched_schedule": ([P, ctypes.c_int, ctypes.POINTER(_Opts), P, P, P, ctypes.c_int, P],
                                         ctypes.c_int),
        "zi_memory_stats": ([P, P, ctypes.c_int], ctypes.c_int),
        "zi_kernel_launches": ([], ctypes.c_int64),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _status_name(st: int) -> str:
    names = {0: "ZI_OK", 1: "ZI_ERR_ARG", 2: "ZI_ERR_BAD_MESH", 3: "ZI_ERR_NONFINITE",
             4: "ZI_ERR_NOT_CONVERGED", 5: "ZI_ERR_TIMEOUT", 6: "ZI_ERR_CUDA", 7: "ZI_ERR_NOMEM"}
    return names.get(st, "ZI_ERR_%d" % st)


def _check(st: int, allow_not_converged: bool = False):
    if st == ZI_OK:
        return
    buf = ctypes.create_string_buffer(1024)
    load_library().zi_last_error(buf, 1024)
    msg = buf.value.decode(errors="replace")
    if st == ZI_ERR_NOT_CONVERGED:
        if allow_not_converged:
            return
        raise NotConverged(st, msg)
    raise ZiError(st, msg)


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("libzi needs a CUDA device; none is available")
    return torch


def _stream():
    torch = _torch()
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t) -> ctypes.c_void_p:
    if t is None:
        return ctypes.c_void_p(0)
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _dev(x, dtype, device="cuda"):
    torch = _torch()
    if isinstance(x, np.ndarray):
        x = torch.from_numpy(np.ascontiguousarray(x))
    return x.to(device=device, dtype=dtype).contiguous()


def _radii_buf(radii):
    arr = (ctypes.c_double * len(radii))(*[float(r) for r in radii])
    return arr


@dataclass
class SolverOpts:
    """Options of the multi-RHS PCG (see zi_solver_opts in include/zi.h)."""
    tol: float = 1e-10
    maxit: int = 100000
    precond: int = PRECOND_JACOBI
    precision: int = FP64
    inner_tol: float = 5e-2
    max_outer: int = 30
    check_every: int = 25

    def c(self) -> _Opts:
        return _Opts(self.tol, self.maxit, self.precond, self.precision, self.inner_tol,
                     self.max_outer, self.check_every)


def version() -> int:
    return load_library().zi_version()


def memory_stats(reset_high: bool = False):
    """(bytes in use, high-water mark) of the library's device-memory pool on
    the current device (zi_memory_stats); reset_high zeroes the mark after
    reading it."""
    now, high = ctypes.c_int64(), ctypes.c_int64()
    _check(load_library().zi_memory_stats(ctypes.byref(now), ctypes.byref(high), int(bool(reset_high))))
    return now.value, high.value


def kernel_launches() -> int:
    """libzi kernels launched by this process so far (zi_kernel_launches)."""
    return int(load_library().zi_kernel_launches())


def mesh_from_grid(h: float, radii, device="cuda"):
    """Regular-grid Kuhn mesh of the ball (zi_mesh_from_grid); returns a dict
    of CUDA tensors nodes (n,3) f64, tets (m,4) i32, labels (m,) i32,
    bfaces (nb,3) i32."""
    torch = _torch()
    lib = load_library()
    rb = _radii_buf(radii)
    n, m, nb = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    st = _stream()
    _check(lib.zi_mesh_from_grid(h, len(radii), rb, ctypes.byref(n), ctypes.byref(m), ctypes.byref(nb),
                                 None, None, None, None, st))
    nodes = torch.empty((n.value, 3), dtype=torch.float64, device=device)
    tets = torch.empty((m.value, 4), dtype=torch.int32, device=device)
    labels = torch.empty((m.value,), dtype=torch.int32, device=device)
    bfaces = torch.empty((nb.value, 3), dtype=torch.int32, device=device)
    _check(lib.zi_mesh_from_grid(h, len(radii), rb, ctypes.byref(n), ctypes.byref(m), ctypes.byref(nb),
                                 _ptr(nodes), _ptr(tets), _ptr(labels), _ptr(bfaces), st))
    return dict(nodes=nodes, tets=tets, labels=labels, bfaces=bfaces, h=float(h), radii=tuple(radii))


def mesh_from_surfaces(h: float, surfaces, priority, device="cuda"):
    """Mesh of a surface segmentation (zi_mesh_from_surfaces): surfaces is a
    list of (verts (v,3), tris (t,3)) closed outward-oriented surfaces,
    innermost first; priority one int per surface (lower wins).  Returns a
    dict of CUDA tensors like mesh_from_grid."""
    torch = _torch()
    lib = load_library()
    if len(priority) != len(surfaces):
        raise ValueError("one priority per surface")
    vs, ts, off, base = [], [], [0], 0
    for v, t in surfaces:
        v = np.asarray(v, dtype=np.float64).reshape(-1, 3)
        t = np.asarray(t, dtype=np.int64).reshape(-1, 3)
        vs.append(v)
        ts.append(t + base)
        base += v.shape[0]
        off.append(off[-1] + t.shape[0])
    verts = _dev(np.concatenate(vs), torch.float64, device)
    tris = _dev(np.concatenate(ts).astype(np.int32), torch.int32, device)
    toff = (ctypes.c_int64 * len(off))(*off)
    pr = (ctypes.c_int32 * len(priority))(*[int(x) for x in priority])
    n, m, nb = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    st = _stream()
    args = (float(h), len(surfaces), toff, pr, _ptr(verts), verts.shape[0], _ptr(tris))
    _check(lib.zi_mesh_from_surfaces(*args, ctypes.byref(n), ctypes.byref(m), ctypes.byref(nb),
                                     None, None, None, None, st))
    nodes = torch.empty((n.value, 3), dtype=torch.float64, device=device)
    tets = torch.empty((m.value, 4), dtype=torch.int32, device=device)
    labels = torch.empty((m.value,), dtype=torch.int32, device=device)
    bfaces = torch.empty((nb.value, 3), dtype=torch.int32, device=device)
    _check(lib.zi_mesh_from_surfaces(*args, ctypes.byref(n), ctypes.byref(m), ctypes.byref(nb),
                                     _ptr(nodes), _ptr(tets), _ptr(labels), _ptr(bfaces), st))
    return dict(nodes=nodes, tets=tets, labels=labels, bfaces=bfaces, h=float(h))


def locate_points(nodes, tets, pos, device="cuda"):
    """Element of the mesh (nodes, tets) holding each position
    (zi_locate_points), as an int32 CUDA tensor."""
    torch = _torch()
    lib = load_library()
    V = _dev(nodes, torch.float64, device).reshape(-1, 3).contiguous()
    T = _dev(tets, torch.int32, device).reshape(-1, 4).contiguous()
    X = _dev(pos, torch.float64, device).reshape(-1, 3).contiguous()
    out = torch.empty(X.shape[0], dtype=torch.int32, device=device)
    _check(lib.zi_locate_points(_ptr(V), V.shape[0], _ptr(T), T.shape[0], _ptr(X), X.shape[0], _ptr(out),
                                _stream()))
    return out


def nearest_source(points, sources, device="cuda"):
    """Index of the nearest source for every point (zi_nearest_source), as
    an int32 CUDA tensor."""
    torch = _torch()
    lib = load_library()
    X = _dev(points, torch.float64, device).reshape(-1, 3).contiguous()
    S = _dev(sources, torch.float64, device).reshape(-1, 3).contiguous()
    out = torch.empty(X.shape[0], dtype=torch.int32, device=device)
    _check(lib.zi_nearest_source(_ptr(X), X.shape[0], _ptr(S), S.shape[0], _ptr(out), _stream()))
    return out


def locate_dipoles_grid(h: float, radii, pos):
    """Tet of a zi_mesh_from_grid mesh holding each point (zi_locate_dipoles_grid)."""
    torch = _torch()
    pos = _dev(pos, torch.float64)
    out = torch.empty((pos.shape[0],), dtype=torch.int32, device=pos.device)
    rb = _radii_buf(radii)
    _check(load_library().zi_locate_dipoles_grid(h, len(radii), rb, _ptr(pos), pos.shape[0], _ptr(out),
                                                 _stream()))
    return out


class System:
    """Grounded FEM system of one head (zi_assemble); owns a zi_system handle."""

    def __init__(self, nodes, tets, sigma6, bfaces, centres, model="cem", z=None, radius=0.0):
        torch = _torch()
        lib = load_library()
        self._lib = lib
        self.nodes = _dev(nodes, torch.float64)
        self.tets = _dev(tets, torch.int32)
        s6 = _dev(sigma6, torch.float64)
        self.sigma6 = s6  # kept for the MEG volume currents
        self.bfaces = _dev(bfaces, torch.int32)
        self.centres = _dev(centres, torch.float64)
        mdl = ELECTRODE_CEM if model in ("cem", ELECTRODE_CEM) else ELECTRODE_POINT
        self.model = mdl
        self.z = _dev(z, torch.float64) if z is not None else None
        el = _Electrodes(mdl, self.centres.shape[0], _ptr(self.centres).value,
                         _ptr(self.z).value if self.z is not None else None, float(radius))
        h = ctypes.c_void_p()
        _check(lib.zi_assemble(_ptr(self.nodes), self.nodes.shape[0], _ptr(self.tets), self.tets.shape[0],
                               _ptr(s6), _ptr(self.bfaces), self.bfaces.shape[0], ctypes.byref(el),
                               ctypes.byref(h), _stream()))
        self._h = h
        self.version = 0  # bumped whenever the matrix values change

    @property
    def handle(self):
        return self._h

    def info(self) -> dict:
        inf = _Info()
        _check(self._lib.zi_system_get_info(self._h, ctypes.byref(inf)))
        return {k: getattr(inf, k) for k, _ in _Info._fields_}

    def matrix(self):
        """(rowptr, colind, values, B, C or None, electrode nodes or None) as CUDA tensors."""
        torch = _torch()
        inf = self.info()
        n, nnz, nr, L = inf["n"], inf["nnz"], inf["n_rhs"], inf["n_el"]
        dev = self.nodes.device
        rowptr = torch.empty(n + 1, dtype=torch.int32, device=dev)
        colind = torch.empty(nnz, dtype=torch.int32, device=dev)
        vals = torch.empty(nnz, dtype=torch.float64, device=dev)
        B = torch.empty((n, nr), dtype=torch.float64, device=dev)
        cem = inf["model"] == ELECTRODE_CEM
        C = torch.empty(L, dtype=torch.float64, device=dev) if cem else None
        en = None if cem else torch.empty(L, dtype=torch.int32, device=dev)
        _check(self._lib.zi_system_get_matrix(self._h, _ptr(rowptr), _ptr(colind), _ptr(vals), _ptr(B),
                                              _ptr(C), _ptr(en), _stream()))
        return rowptr, colind, vals, B, C, en

    def set_conductivity(self, sigma6):
        torch = _torch()
        s6 = _dev(sigma6, torch.float64)
        _check(self._lib.zi_system_set_conductivity(self._h, _ptr(s6), _stream()))
        self.sigma6 = s6
        self.version += 1

    def set_log_conductivity(self, sigma_base6, log_s):
        """Element tensors exp(log_s[e]) * sigma_base6[e], formed and assembled in
        libzi (zi_system_set_log_conductivity)."""
        torch = _torch()
        base = _dev(sigma_base6, torch.float64, self.nodes.device).contiguous()
        ls = _dev(log_s, torch.float64, self.nodes.device).contiguous()
        _check(self._lib.zi_system_set_log_conductivity(self._h, _ptr(base), _ptr(ls), _stream()))
        self.sigma6 = None
        self.version += 1

    def transfer(self, opts: SolverOpts | None = None, want_T: bool = True, allow_not_converged=False):
        """T = A^-1 B (zi_transfer); returns (T or None, iters, relres)."""
        torch = _torch()
        opts = opts or SolverOpts()
        inf = self.info()
        nr = inf["n_rhs"]
        T = torch.empty((inf["n"], nr), dtype=torch.float64, device=self.nodes.device) if want_T else None
        it = (ctypes.c_int32 * nr)()
        rr = (ctypes.c_double * nr)()
        o = opts.c()
        st = self._lib.zi_transfer(self._h, ctypes.byref(o), _ptr(T), it, rr, _stream())
        _check(st, allow_not_converged)
        return T, np.array(it[:], dtype=np.int32), np.array(rr[:], dtype=np.float64)

    def leadfield(self, dip_tet, opts: SolverOpts | None = None, out=None):
        """L (zi_leadfield) for dipoles in tets dip_tet; columns 3p + d."""
        torch = _torch()
        opts = opts or SolverOpts()
        dt = _dev(dip_tet, torch.int32)
        inf = self.info()
        P = dt.shape[0]
        L = out if out is not None else torch.empty((inf["n_rows_L"], 3 * P), dtype=torch.float64,
                                                    device=self.nodes.device)
        o = opts.c()
        _check(self._lib.zi_leadfield(self._h, _ptr(dt), P, ctypes.byref(o), _ptr(L), _stream()))
        return L

    def leadfield_at(self, pos, opts: SolverOpts | None = None, out=None):
        """L (zi_leadfield_at) for dipoles at positions pos (P x 3, metres),
        located on the system's own mesh; columns 3p + d."""
        torch = _torch()
        opts = opts or SolverOpts()
        ps = _dev(pos, torch.float64, self.nodes.device).reshape(-1, 3).contiguous()
        inf = self.info()
        P = ps.shape[0]
        L = out if out is not None else torch.empty((inf["n_rows_L"], 3 * P), dtype=torch.float64,
                                                    device=self.nodes.device)
        o = opts.c()
        _check(self._lib.zi_leadfield_at(self._h, _ptr(ps), P, ctypes.byref(o), _ptr(L), _stream()))
        return L

    def source_stencil(self, pos, dip_tet, model=SOURCE_PBO10, lam: float = 0.0):
        """Source-matrix columns of Cartesian H(div) sources (zi_source_stencil):
        returns (F_nodes, F_w), each 3P x STENCIL_WIDTH; positions in metres."""
        torch = _torch()
        ps = _dev(pos, torch.float64).reshape(-1, 3).contiguous()
        dt = _dev(dip_tet, torch.int32)
        P = dt.shape[0]
        if ps.shape[0] != P:
            raise ValueError("pos and dip_tet disagree on the source count")
        Fn = torch.empty((3 * P, STENCIL_WIDTH), dtype=torch.int32, device=self.nodes.device)
        Fw = torch.empty((3 * P, STENCIL_WIDTH), dtype=torch.float64, device=self.nodes.device)
        _check(self._lib.zi_source_stencil(self._h, _ptr(ps), _ptr(dt), P, int(model), float(lam), _ptr(Fn),
                                           _ptr(Fw), _stream()))
        return Fn, Fw

    def leadfield_sparse(self, F_nodes, F_w, opts: SolverOpts | None = None, out=None):
        """L (zi_leadfield_sparse) for a source matrix given column by column
        (ncols x K node indices and loads)."""
        torch = _torch()
        opts = opts or SolverOpts()
        Fn = _dev(F_nodes, torch.int32).contiguous()
        Fw = _dev(F_w, torch.float64).contiguous()
        if Fn.dim() != 2 or Fn.shape != Fw.shape:
            raise ValueError("F_nodes and F_w must both be ncols x K")
        ncols, K = Fn.shape
        inf = self.info()
        L = out if out is not None else torch.empty((inf["n_rows_L"], ncols), dtype=torch.float64,
                                                    device=self.nodes.device)
        o = opts.c()
        _check(self._lib.zi_leadfield_sparse(self._h, _ptr(Fn), _ptr(Fw), ncols, K, ctypes.byref(o), _ptr(L),
                                             _stream()))
        return L

    def leadfield_hdiv(self, pos, dip_tet, model=SOURCE_PBO10, lam: float = 0.0,
                       opts: SolverOpts | None = None):
        """L for Cartesian H(div) sources (Sec. 2.1): the stencil columns, then
        the sparse lead field; columns 3p + d as in leadfield()."""
        Fn, Fw = self.source_stencil(pos, dip_tet, model, lam)
        return self.leadfield_sparse(Fn, Fw, opts)

    def source_pi(self, dip_tet):
        """Partial-integration source columns (zi_source_pi): (F_nodes, F_w), 3P x 4."""
        torch = _torch()
        dt = _dev(dip_tet, torch.int32)
        P = dt.shape[0]
        Fn = torch.empty((3 * P, 4), dtype=torch.int32, device=self.nodes.device)
        Fw = torch.empty((3 * P, 4), dtype=torch.float64, device=self.nodes.device)
        _check(self._lib.zi_source_pi(self._h, _ptr(dt), P, _ptr(Fn), _ptr(Fw), _stream()))
        return Fn, Fw

    def _sensors(self, sens_pos, sens_dir):
        torch = _torch()
        sp_ = _dev(sens_pos, torch.float64).reshape(-1, 3).contiguous()
        sd = _dev(sens_dir, torch.float64).reshape(-1, 3).contiguous()
        if sp_.shape != sd.shape:
            raise ValueError("sensor positions and orientations disagree")
        return sp_, sd

    def meg_rhs(self, sens_pos, sens_dir):
        """Bm (n x Ns) of the MEG volume currents (zi_meg_rhs)."""
        torch = _torch()
        sp_, sd = self._sensors(sens_pos, sens_dir)
        Ns = sp_.shape[0]
        Bm = torch.empty((self.info()["n"], Ns), dtype=torch.float64, device=self.nodes.device)
        _check(self._lib.zi_meg_rhs(self._h, _ptr(self.sigma6), _ptr(sp_), _ptr(sd), Ns, _ptr(Bm), _stream()))
        return Bm

    def meg_transfer(self, sens_pos, sens_dir, opts: SolverOpts | None = None, allow_not_converged=False):
        """T_meg = A^-1 Bm (zi_meg_transfer); returns (T_meg, iters, relres)."""
        torch = _torch()
        opts = opts or SolverOpts()
        sp_, sd = self._sensors(sens_pos, sens_dir)
        Ns = sp_.shape[0]
        Tm = torch.empty((self.info()["n"], Ns), dtype=torch.float64, device=self.nodes.device)
        it = (ctypes.c_int32 * Ns)()
        rr = (ctypes.c_double * Ns)()
        o = opts.c()
        st = self._lib.zi_meg_transfer(self._h, _ptr(self.sigma6), _ptr(sp_), _ptr(sd), Ns, ctypes.byref(o),
                                       _ptr(Tm), it, rr, _stream())
        _check(st, allow_not_converged)
        return Tm, np.array(it[:], dtype=np.int32), np.array(rr[:], dtype=np.float64)

    def meg_leadfield(self, T_meg, sens_pos, sens_dir, pos, F_nodes, F_w):
        """MEG lead field (zi_meg_leadfield), Ns x 3P, for Cartesian sources at pos
        with source columns (F_nodes, F_w) from source_pi or source_stencil."""
        torch = _torch()
        sp_, sd = self._sensors(sens_pos, sens_dir)
        ps = _dev(pos, torch.float64).reshape(-1, 3).contiguous()
        Fn = _dev(F_nodes, torch.int32).contiguous()
        Fw = _dev(F_w, torch.float64).contiguous()
        P = ps.shape[0]
        if Fn.shape != Fw.shape or Fn.dim() != 2 or Fn.shape[0] != 3 * P:
            raise ValueError("source columns must be 3P x K")
        Tm = _dev(T_meg, torch.float64).contiguous()
        Ns = sp_.shape[0]
        L = torch.empty((Ns, 3 * P), dtype=torch.float64, device=self.nodes.device)
        _check(self._lib.zi_meg_leadfield(self._h, _ptr(Tm), _ptr(sp_), _ptr(sd), Ns, _ptr(ps), P, _ptr(Fn),
                                          _ptr(Fw), Fn.shape[1], _ptr(L), _stream()))
        return L

    def eit(self, I, mode=EIT_FULL, grad_y=None, opts: SolverOpts | None = None, want_y=True):
        """Linearised EIT (zi_eit_jacobian): returns (y, out)."""
        torch = _torch()
        opts = opts or SolverOpts()
        I = _dev(I, torch.float64)
        np_, L = I.shape
        inf = self.info()
        dev = self.nodes.device
        y = torch.empty((np_, L), dtype=torch.float64, device=dev) if want_y else None
        if mode is None:
            out = None
            mode = EIT_FULL
        elif mode == EIT_FULL:
            out = torch.empty((inf["m"], np_, L), dtype=torch.float64, device=dev)
        else:
            out = torch.empty((inf["m"],), dtype=torch.float64, device=dev)
        gy = _dev(grad_y, torch.float64) if grad_y is not None else None
        o = opts.c()
        _check(self._lib.zi_eit_jacobian(self._h, _ptr(I), np_, mode, _ptr(gy), _ptr(out), _ptr(y),
                                         ctypes.byref(o), _stream()))
        return y, out

    def time_source_apply(self, F_nodes, F_w, reps=5):
        """(ms per launch, algorithmic bytes per launch) of the source
        application of leadfield_sparse (zi_time_source_apply); needs T."""
        torch = _torch()
        Fn = _dev(F_nodes, torch.int32).contiguous()
        Fw = _dev(F_w, torch.float64).contiguous()
        ms, b = ctypes.c_double(), ctypes.c_double()
        _check(self._lib.zi_time_source_apply(self._h, _ptr(Fn), _ptr(Fw), Fn.shape[0], Fn.shape[1], int(reps),
                                              ctypes.byref(ms), ctypes.byref(b), _stream()))
        return ms.value, b.value

    def time_spmm(self, precision=FP64, reps=5):
        """(ms per launch, algorithmic bytes per launch) of the solver's SpMM
        (zi_time_spmm); needs a prior transfer with the same precision."""
        ms, by = ctypes.c_double(), ctypes.c_double()
        _check(self._lib.zi_time_spmm(self._h, precision, reps, ctypes.byref(ms), ctypes.byref(by), _stream()))
        return ms.value, by.value

    def apply_operator(self, X, opts: "SolverOpts", want_dots=True):
        """(Y, dots): the solver's own operator applied to X (n x n_rhs) with its
        fused column dots (zi_apply_operator): S A S X for FP64, the FP32
        difference-form A X for MIXED."""
        torch = _torch()
        X = _dev(X, torch.float64, self.nodes.device)
        inf = self.info()
        Y = torch.empty((inf["n"], inf["n_rhs"]), dtype=torch.float64, device=X.device)
        dots = torch.empty(inf["n_rhs"], dtype=torch.float64, device=X.device) if want_dots else None
        o = opts.c()
        _check(self._lib.zi_apply_operator(self._h, ctypes.byref(o), _ptr(X), _ptr(Y), _ptr(dots), _stream()))
        return Y, dots

    def solver_info(self) -> dict:
        """The solver's layout and matrix-copy sizes (zi_solver_get_info)."""
        inf = _SolverInfo()
        _check(self._lib.zi_solver_get_info(self._h, ctypes.byref(inf)))
        return {k: getattr(inf, k) for k, _ in _SolverInfo._fields_}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.zi_system_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batch_tune(systems, opts: SolverOpts | None = None):
    """The autotuner's schedule for this batch (zi_batch_tune): (list of 0/1,
    1 = head in the persistent launch; dict with the source and the
    estimated ms per iteration of the schedule, of every head alone, and of
    every head in the persistent launch)."""
    lib = load_library()
    opts = opts or SolverOpts()
    nb = len(systems)
    hs = (ctypes.c_void_p * nb)(*[s.handle.value for s in systems])
    mask = (ctypes.c_int32 * nb)()
    info = _BatchSchedule()
    o = opts.c()
    _check(lib.zi_batch_tune(hs, nb, ctypes.byref(o), mask, ctypes.byref(info), _stream()))
    return list(mask), {k: getattr(info, k) for k, _ in _BatchSchedule._fields_}


def transfer_batched(systems, opts: SolverOpts | None = None, want_T: bool = False, persistent=None,
                     chunk: int = 0):
    """Transfer matrices of several systems in one batched solve
    (zi_transfer_batched, the tuned schedule; or zi_transfer_batched_schedule
    when `persistent` gives the schedule: one 0/1 per system); returns (list
    of T or None, list of iters)."""
    torch = _torch()
    lib = load_library()
    opts = opts or SolverOpts()
    nb = len(systems)
    hs = (ctypes.c_void_p * nb)(*[s.handle.value for s in systems])
    Ts, Tp, its, itp = [], (ctypes.c_void_p * nb)(), [], (ctypes.c_void_p * nb)()
    for b, s in enumerate(systems):
        inf = s.info()
        T = torch.empty((inf["n"], inf["n_rhs"]), dtype=torch.float64, device=s.nodes.device) if want_T else None
        Ts.append(T)
        Tp[b] = _ptr(T).value
        it = (ctypes.c_int32 * inf["n_rhs"])()
        its.append(it)
        itp[b] = ctypes.cast(it, ctypes.c_void_p).value
    o = opts.c()
    if persistent is None:
        _check(lib.zi_transfer_batched(hs, nb, ctypes.byref(o), Tp, itp, _stream()))
    else:
        if len(persistent) != nb:
            raise ValueError("one schedule flag per system")
        mask = (ctypes.c_int32 * nb)(*[1 if p else 0 for p in persistent])
        _check(lib.zi_transfer_batched_schedule(hs, nb, ctypes.byref(o), Tp, itp, mask, int(chunk), _stream()))
    return Ts, [np.array(it[:], dtype=np.int32) for it in its]


def ias_map(L, Y, nu: float, theta0: float, beta: float, hypermodel: int = HYPER_G, iters: int = 20):
    """IAS MAP inversion (App. B, zi_ias_map) of the data vectors Y (T x Le
    CUDA tensor, or Le for one) with the lead field L (Le x n CUDA tensor);
    returns X and Theta (T x n, or n for one data vector)."""
    torch = _torch()
    lib = load_library()
    L = L.contiguous().to(torch.float64)
    one = Y.dim() == 1
    Y = (Y[None, :] if one else Y).contiguous().to(torch.float64)
    Le, n = L.shape
    T = Y.shape[0]
    if Y.shape[1] != Le:
        raise ValueError("Y must have Le = %d columns" % Le)
    X = torch.empty((T, n), dtype=torch.float64, device=L.device)
    Th = torch.empty((T, n), dtype=torch.float64, device=L.device)
    _check(lib.zi_ias_map(_ptr(L), Le, n, _ptr(Y), T, float(nu), float(theta0), float(beta), int(hypermodel),
                          int(iters), _ptr(X), _ptr(Th), _stream()))
    return (X[0], Th[0]) if one else (X, Th)
