"""Lead-field build benchmark on GB300.

One step = one whole LF build of the three-shell head at h = 1 mm with a
transversely anisotropic skull (3,342,701 nodes, 19,573,872 tets, 256
complete-model electrodes, 100,000 dipoles x 3 orientations): dipole
location, assembly (element stiffness, pattern, CEM terms, grounding),
T = A^-1 B by multi-RHS PCG to a relative residual of 1e-10 per column,
source application and the electrode Schur step, from inputs resident in HBM
to L (256 x 300,000) in HBM.  (--workload shell2mm: the 2 mm isotropic head
with 128 electrodes and 20,000 dipoles.)

The headline is the mixed-precision build (FP32 inner PCG inside FP64
iterative refinement); the plain FP64 PCG build on the same GPU is reported
beside it, with the relative difference of the two lead fields.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Multi-GPU runs are independent replicas:
each rank builds the same lead field (no data-path collective).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "LF build s, mixed vs FP64 PCG at rel.err<=1e-6 on 1 GB300; SpMM HBM GB/s vs peak"
UNIT = "s"
WORKLOADS = {
    "aniso1mm": ("config_three_shell_1mm_aniso",
                 "three-shell sphere 80/86/92 mm, h=1 mm Kuhn grid (3342701 nodes, 19573872 tets), transversely "
                 "anisotropic skull (radial 0.00132, tangential 0.0132 S/m), 256 CEM electrodes r=5 mm "
                 "z=2e-3 Ohm m^2, 100000 dipoles x 3, PCG tol 1e-10"),
    "shell2mm": ("config_three_shell_2mm",
                 "three-shell sphere 80/86/92 mm, h=2 mm Kuhn grid (428185 nodes, 2447424 tets), "
                 "128 CEM electrodes r=5 mm z=2e-3 Ohm m^2, 20000 dipoles x 3, PCG tol 1e-10"),
}
DEFAULT_WORKLOAD = "aniso1mm"
# ncu DRAM traffic per launch of the FP32 SpMM on this workload, from the capture
# summarised in profiles/ (None until taken, or once the kernel source changed).
SPMM_TRAFFIC = {
    "shell2mm": {"source_sha": "9b1e26a920e49e63", "bytes": 137.207296e6 + 169.128960e6,
                 "note": "one ncu capture (--set full) of the standalone launch on this workload, taken on the "
                         "same kernel code (since then only its FP16 storage helpers were renamed and a "
                         "comment in the hashed region changed)"},
    "aniso1mm": {"source_sha": "9b1e26a920e49e63", "bytes": 2.93e9 + 3.38e9,
                 "note": "one ncu capture (dram__bytes_read.sum + dram__bytes_write.sum, one pass) of the "
                         "standalone launch on this workload at full size, on the same kernel code (a comment "
                         "in the hashed region changed since)"},
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparison build")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD,
                    choices=["aniso1mm", "shell2mm", "batch", "ias", "eit", "hdiv", "meg", "segmesh", "spmm"],
                    help="aniso1mm (default, the precision workload): 1 mm anisotropic-skull head, 256 "
                         "electrodes, 100k dipoles; shell2mm: 2 mm head, 128 electrodes, 20k dipoles; batch: 24 "
                         "heads, batched vs per-head solves; spmm: the solver's SpMM launched on its own (for a "
                         "profiler), see --h/--electrodes/--precision")
    ap.add_argument("--h", type=float, default=0.002, help="spmm: grid step of the three-shell head (m)")
    ap.add_argument("--electrodes", type=int, default=128, help="spmm: CEM electrodes (right-hand sides)")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"], help="spmm: which SpMM")
    ap.add_argument("--aniso", action="store_true", help="spmm: transversely anisotropic skull")
    ap.add_argument("--reps", type=int, default=3, help="spmm: standalone launches")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """The job's time is the slowest rank's: max of `value` over the process
    group (identity without one)."""
    if dist is None or not dist.is_initialized():
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# CPU oracle sample (the baseline leg and the reference arm)
# ---------------------------------------------------------------------------

ORACLE_SAMPLE = dict(h=0.004, electrodes=128, dipoles=20000)
ORACLE_SAMPLE_TEXT = ("oracle LF build (numpy + SuperLU direct solve, 1 thread) of the same three-shell head, "
                      "128 CEM electrodes and 20000 dipoles at h=4 mm (56235 nodes): the h=2 mm direct "
                      "factorisation does not fit a bounded CPU sample")
# the direct-solve sample of each LF workload: the same head at h = 4 mm
DIRECT_SAMPLES = {
    "shell2mm": ("W.three_shell(0.004, 128, 20000, seed=2)", ORACLE_SAMPLE_TEXT),
    "aniso1mm": ("W.three_shell(0.004, 256, 20000, seed=3, skull_aniso=(0.00132, 0.0132))",
                 "oracle LF build (numpy + SuperLU direct solve, 1 thread) of the same anisotropic-skull "
                 "three-shell head, 256 CEM electrodes and 20000 dipoles at h=4 mm (56235 nodes): a direct "
                 "factorisation at h=1 mm does not fit a bounded CPU sample"),
}


def oracle_once(workload: str = "shell2mm") -> float:
    """One oracle LF build of the workload's h = 4 mm sample, in a fresh
    single-threaded process (spawned with exec, so it never inherits a CUDA
    context)."""
    code = ("import sys,time; sys.path.insert(0, %r)\n"
            "from oracle import zi_oracle as O\n"
            "from paper_1811_07717_gb300 import workloads as W\n"
            "spec = %s\n"
            "t = time.perf_counter(); O.leadfield_from_spec(spec, W); print(time.perf_counter() - t)\n"
            % (ROOT, DIRECT_SAMPLES[workload][0]))
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env)
    if r.returncode != 0:
        raise RuntimeError("oracle sample failed: " + r.stderr[-500:])
    return float(r.stdout.strip().splitlines()[-1])


# CPU block PCG of the full workload (oracle/cpu_pcg.c, FP64, Jacobi, OpenMP over
# every host core) on the oracle's own assembly of the workload's system.
# A full solve of the 1 mm head takes minutes, so a step is bounded: the time
# of one iteration is the difference of two capped runs (K2 and K1
# iterations; allocation, first touch and set-up cancel), and the iteration
# count is the CPU's own, from a full solve of an evenly spaced sample of the
# columns.  LF seconds = s per iteration x that count (the transfer solve is
# all but a few percent of the LF build).
CPU_PCG_K1, CPU_PCG_K2, CPU_PCG_COLS = 1, 6, 8


def cpu_pcg_text(workload: str) -> str:
    return ("CPU block PCG (oracle/cpu_pcg.c: FP64 Jacobi PCG, OpenMP, all host cores) on the oracle's own "
            "assembly of the full workload: seconds per iteration with all %s columns (difference of %d- and "
            "%d-iteration runs) x the CPU's own iteration count to tol 1e-10 (the largest of a full solve of %d "
            "evenly spaced columns); the transfer solve only"
            % ({"aniso1mm": 256, "shell2mm": 128}[workload], CPU_PCG_K2, CPU_PCG_K1, CPU_PCG_COLS))


def cpu_pcg_workload(workload: str, steps: int) -> dict:
    """Runs the CPU block PCG measurement of the workload in a fresh process:
    `steps` per-iteration times, the sampled iteration count, threads."""
    code = ("import sys,time,os,json; import numpy as np; sys.path.insert(0, %r)\n"
            "from oracle import zi_oracle as O, cpu_pcg\n"
            "from paper_1811_07717_gb300 import workloads as W\n"
            "spec = W.%s()\n"
            "t0 = time.perf_counter()\n"
            "mesh = O.mesh_from_grid(spec.h, spec.radii)\n"
            "s6 = W.conductivity(spec, mesh['nodes'], mesh['tets'], mesh['labels'])\n"
            "c, z = W.electrode_inputs(spec)\n"
            "S = O.System(mesh, s6, c, spec.electrode_model, radius=spec.electrode_radius, z=z)\n"
            "A, B = S.A.tocsr(), np.ascontiguousarray(S.B)\n"
            "del mesh, s6\n"
            "setup = time.perf_counter() - t0\n"
            "th = len(os.sched_getaffinity(0))\n"
            "cols = np.unique(np.linspace(0, B.shape[1] - 1, %d).round().astype(int))\n"
            "t = time.perf_counter(); _, its, kmax = cpu_pcg.block_pcg(A, np.ascontiguousarray(B[:, cols]), "
            "tol=1e-10, threads=th); t_sample = time.perf_counter() - t\n"
            "def run(k):\n"
            "    t = time.perf_counter(); cpu_pcg.block_pcg(A, B, tol=1e-10, maxit=k, threads=th)\n"
            "    return time.perf_counter() - t\n"
            "per = []\n"
            "for _ in range(%d):\n"
            "    a = run(%d); b = run(%d); per.append((b - a) / %d)\n"
            "print(json.dumps({'s_per_iteration': per, 'iterations': int(kmax), 'threads': th, 'setup_s': setup, "
            "'sample_columns': int(cols.size), 'sample_solve_s': t_sample}))\n"
            % (ROOT, WORKLOADS[workload][0], CPU_PCG_COLS, max(1, steps), CPU_PCG_K1, CPU_PCG_K2,
               CPU_PCG_K2 - CPU_PCG_K1))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("cpu PCG measurement failed: " + r.stderr[-500:])
    return json.loads(r.stdout.strip().splitlines()[-1])


HDIV_SAMPLE_TEXT = ("oracle LF build with PBO 10-source H(div) sources (numpy stencils and KKT solves + SuperLU "
                    "direct solve, 1 thread) of the three-shell head, 128 CEM electrodes and 20000 sources at h=4 mm")
MEG_SAMPLE_TEXT = ("oracle MEG LF build (numpy right-hand sides + SuperLU direct solve, 1 thread) of the three-shell "
                   "head at h=4 mm, 32 of the 256 magnetometers, 20000 partial-integration dipoles")


def oracle_sample_once(kind: str) -> float:
    """One oracle build of the H(div) ("hdiv") or MEG ("meg") sample at h = 4 mm,
    in a fresh single-threaded process."""
    body = {
        "hdiv": ("mesh, s6, c, z, pos, q = O.build_head(spec, W)\n"
                 "S = O.System(mesh, s6, c, spec.electrode_model, radius=spec.electrode_radius, z=z)\n"
                 "dip = O.locate_dipoles(mesh, pos)\n"
                 "F = HD.source_matrix_hdiv(mesh['nodes'], mesh['tets'], dip, pos, HD.PBO10)\n"
                 "L = O.leadfield(S, F)\n"),
        "meg": ("mesh, s6, c, z, pos, q = O.build_head(spec, W)\n"
                "S = O.System(mesh, s6, c, spec.electrode_model, radius=spec.electrode_radius, z=z)\n"
                "sp_, sd = W.meg_sensors(256, spec.radii[-1] + 0.02)\n"
                "dip = O.locate_dipoles(mesh, pos)\n"
                "F = O.source_matrix(S.n, mesh['nodes'], mesh['tets'], dip)\n"
                "L = M.meg_leadfield(S, s6, sp_[:32], sd[:32], pos, F)\n"),
    }[kind]
    code = ("import sys,time; sys.path.insert(0, %r)\n"
            "from oracle import zi_oracle as O, hdiv as HD, meg as M\n"
            "from paper_1811_07717_gb300 import workloads as W\n"
            "spec = W.three_shell(%r, %d, %d, seed=2)\n"
            "t = time.perf_counter()\n%sprint(time.perf_counter() - t)\n"
            % (ROOT, ORACLE_SAMPLE["h"], ORACLE_SAMPLE["electrodes"], ORACLE_SAMPLE["dipoles"], body))
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env)
    if r.returncode != 0:
        raise RuntimeError("oracle sample failed: " + r.stderr[-500:])
    return float(r.stdout.strip().splitlines()[-1])


def reference_arm(args):
    """The oracle as it stands, on this machine's host cores, on the bench's own
    workload: the CPU block PCG of oracle/cpu_pcg.c on the oracle's assembly
    (rank 0 alone; the other ranks exit without work)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    wl = args.workload if args.workload in WORKLOADS else DEFAULT_WORKLOAD
    m = cpu_pcg_workload(wl, args.warmup + max(1, args.steps))
    per = m["s_per_iteration"][args.warmup:] or m["s_per_iteration"]
    v = statistics.mean(per) * m["iterations"]
    text = cpu_pcg_text(wl)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": v * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOADS[wl][1], "sample": text},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": m["threads"], "kind": "oracle", "sample": text},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "cpu_pcg": {"s_per_iteration": per, "iterations": m["iterations"], "threads": m["threads"],
                        "setup_s": m["setup_s"], "sample_columns": m["sample_columns"],
                        "sample_solve_s": m["sample_solve_s"]}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------

class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()

    def summary(self):
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.f.name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peak_gbs():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "of measured"
    except Exception:
        return 6800.0, "of fallback"


def spmm_source_sha():
    """Hash of the source that decides the FP32 ELL SpMM's code and its memory
    traffic: the shared header, zi_pcg.cu from its first include to the end
    of k_spmm_ell, and the code that chooses the copy's storage order (the
    tile kernels and ell_order).  The file's leading comment, the vector
    kernels, the batched kernel and the rest of the host code change
    neither."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_1811_07717_gb300", "csrc")
    with open(os.path.join(csrc, "zi_internal.cuh"), "rb") as f:
        head = f.read()
    with open(os.path.join(csrc, "zi_pcg.cu"), "rb") as f:
        body = f.read()

    def part(a, b):
        i = body.find(a)
        j = body.find(b, i + 1) if i >= 0 else -1
        return body[i:j] if i >= 0 and j > i else b""
    kernel = part(b"#include", b"// r -= alpha q, with the column partials")
    order = part(b"// Storage order of the FP32 ELL copy.", b"// Builds the padded, scaled right-hand side")
    order_host = part(b"// Storage position of every row of the FP32 ELL copy", b"// Scaled FP64 matrix, and the FP32")
    return hashlib.sha256(head + kernel + order + order_host).hexdigest()[:16]


# ---------------------------------------------------------------------------
# batched workload: 24 heads, one persistent launch vs per-head solves
# ---------------------------------------------------------------------------

def batch_workload(args):
    """24 heads: the autotuned batched solve against per-head solves, and the
    schedule with every head in the persistent launch.  The first batched
    call of each precision tunes (untimed warm-up); the timed calls use the
    cached schedule."""
    import torch
    from paper_1811_07717_gb300 import workloads as W
    from paper_1811_07717_gb300 import _build, zi
    _build.build()
    heads = W.config_batch()
    systems = []
    for spec in heads:
        mesh = zi.mesh_from_grid(spec.h, spec.radii)
        s6 = W.conductivity(spec, mesh["nodes"].cpu().numpy(), mesh["tets"].cpu().numpy(),
                            mesh["labels"].cpu().numpy())
        centres, z = W.electrode_inputs(spec)
        systems.append(zi.System(mesh["nodes"], mesh["tets"], s6, mesh["bfaces"], centres, model="cem", z=z,
                                 radius=spec.electrode_radius))
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, reps):
        torch.cuda.synchronize()
        t0.record()
        for _ in range(reps):
            fn()
        t1.record()
        torch.cuda.synchronize()
        return t0.elapsed_time(t1) / 1e3 / reps

    out = {}
    reps = max(1, args.steps)
    with Clocks(torch.cuda.current_device()) as clk:
        for name, prec in (("mixed", zi.MIXED), ("fp64", zi.FP64)):
            opts = zi.SolverOpts(tol=1e-10, precision=prec)
            t_tune = time.perf_counter()
            mask, info = zi.batch_tune(systems, opts)
            t_tune = time.perf_counter() - t_tune
            zi.transfer_batched(systems, opts)  # warm-up (allocations, graphs)
            seq = timed(lambda: [s.transfer(opts, want_T=False) for s in systems], reps)
            tuned = timed(lambda: zi.transfer_batched(systems, opts), reps)
            allp = timed(lambda: zi.transfer_batched(systems, opts, persistent=[1] * len(systems)), reps)
            out[name] = {"per_head_s": seq, "batched_tuned_s": tuned, "batched_all_persistent_s": allp,
                         "schedule": {"persistent_heads": [int(b) for b, m in enumerate(mask) if m],
                                      "n_persistent": int(sum(mask)), "tuning_s": t_tune,
                                      "est_window_ms": info["est_window_ms"],
                                      "est_window_ms_per_head": info["est_window_ms_per_head"],
                                      "est_window_ms_persistent": info["est_window_ms_persistent"]}}
    n = [s.info()["n"] for s in systems]
    L = [s.info()["n_rhs"] for s in systems]
    line = {"metric": "transfer solve s for 24 heads (autotuned batch schedule vs per-head launches)",
            "value": out["mixed"]["batched_tuned_s"], "unit": "s", "n_gpus": 1, "steps": reps, "warmup": 1,
            "higher_is_better": False, "dtype": "f32 inner PCG / f64 refinement", "data": "synthetic",
            "config": {"workload": "24 seeded three-shell heads, R 80-100 mm, h in {1.5, 2, 3} mm, "
                                   "32-256 CEM electrodes", "n_nodes_total": int(sum(n)), "tol": 1e-10,
                       "heads": [{"n": a, "n_rhs": b} for a, b in zip(n, L)]},
            "results": out, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# IAS MAP inversion (App. B) on the 2 mm lead field
# ---------------------------------------------------------------------------

def ias_oracle_once(L, Y, nu, theta0, beta, rounds) -> float:
    """The oracle's IAS on a bounded sample of the data vectors, in a fresh
    single-threaded process (seconds)."""
    import tempfile as _tf
    with _tf.TemporaryDirectory() as td:
        np.save(os.path.join(td, "L.npy"), L)
        np.save(os.path.join(td, "Y.npy"), Y)
        code = ("import sys,time,numpy as np; sys.path.insert(0, %r)\n"
                "from oracle import ias as I\n"
                "L = np.load(%r); Y = np.load(%r)\n"
                "t = time.perf_counter(); I.ias_map(L, Y, %r, %r, %r, I.HYPER_G, %d); print(time.perf_counter() - t)\n"
                % (ROOT, os.path.join(td, "L.npy"), os.path.join(td, "Y.npy"), nu, theta0, beta, rounds))
        env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env)
        if r.returncode != 0:
            raise RuntimeError("IAS oracle sample failed: " + r.stderr[-500:])
        return float(r.stdout.strip().splitlines()[-1])


def ias_workload(args):
    """IAS rounds for 16 data vectors with the 2 mm lead field (128 x 60000):
    time per round and the FP64 rate of the Gram product that bounds it."""
    import torch
    from paper_1811_07717_gb300 import workloads as W
    from paper_1811_07717_gb300 import _build, zi
    _build.build()
    spec = W.config_three_shell_2mm()
    mesh = zi.mesh_from_grid(spec.h, spec.radii)
    s6 = W.conductivity(spec, mesh["nodes"].cpu().numpy(), mesh["tets"].cpu().numpy(),
                        mesh["labels"].cpu().numpy())
    centres, z = W.electrode_inputs(spec)
    pos, _ = W.dipole_inputs(spec)
    system = zi.System(mesh["nodes"], mesh["tets"], s6, mesh["bfaces"], centres, model="cem", z=z,
                       radius=spec.electrode_radius)
    L = system.leadfield(zi.locate_dipoles_grid(spec.h, spec.radii, pos), zi.SolverOpts(tol=1e-10,
                                                                                        precision=zi.MIXED))
    system.close()
    Le, n = L.shape
    T, rounds = 16, 20
    rng = np.random.default_rng(7)
    Xt = np.zeros((n, T))
    Xt[rng.choice(n, 5, replace=False), :] = rng.standard_normal((5, T)) * 1e-8
    Yh = L.cpu().numpy() @ Xt
    nu = 0.05 * float(np.abs(Yh).max())
    Yh = Yh + nu * rng.standard_normal(Yh.shape)
    Y = torch.from_numpy(Yh.T.copy()).cuda()
    theta0, beta = 1e-16, 1.6
    for _ in range(max(1, args.warmup)):
        zi.ias_map(L, Y, nu, theta0, beta, zi.HYPER_G, rounds)
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    with Clocks(torch.cuda.current_device()) as clk:
        t0.record()
        for _ in range(args.steps):
            zi.ias_map(L, Y, nu, theta0, beta, zi.HYPER_G, rounds)
        t1.record()
        torch.cuda.synchronize()
    sec = t0.elapsed_time(t1) / 1e3 / args.steps
    tiles = ((Le + 31) // 32) * ((Le + 31) // 32 + 1) // 2
    flops = rounds * T * (2.0 * tiles * 32 * 32 * n + 2.0 * Le * n)   # Gram tiles computed + L^T z
    peak_tf = 1.25  # nominal FP64 rate of the part (no measured FP64 figure is available)
    line = {"metric": "IAS MAP inversion s (20 rounds, 16 data vectors, 2 mm lead field 128 x 60000)",
            "value": sec, "unit": "s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": False, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "IAS (App. B), gamma hypermodel, theta0 1e-16, beta 1.6, nu 5% of max |y|",
                       "Le": Le, "n": n, "data_vectors": T, "rounds": rounds},
            "roofline": {"bound": "alu", "kernel": "k_ias_gram (FP64 split-K Gram product)",
                         "achieved": flops / sec / 1e12, "peak": peak_tf, "unit": "TFLOP/s",
                         "frac": flops / sec / 1e12 / peak_tf, "peak_note": "nominal FP64", "traffic": None},
            "clocks": clk.summary()}
    if not args.no_cpu:
        try:
            c = ias_oracle_once(L.cpu().numpy(), Yh[:, :2], nu, theta0, beta, rounds)
            line["cpu_baseline"] = {"value": c * T / 2, "unit": "s", "cores": 1, "kind": "oracle",
                                    "sample": "2 of the 16 data vectors (numpy, 1 thread), scaled to 16"}
        except Exception as ex:
            line["cpu_baseline"] = {"value": None, "sample": "failed: %s" % ex}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# linearised EIT (App. A.3) on the 2 mm head with 32 electrodes
# ---------------------------------------------------------------------------

def eit_workload(args):
    """The EIT Jacobian of 31 adjacent-pair patterns on all 32 electrodes for
    every tet of the 2 mm head (m x 31 x 32, 19.4 GB written) and its VJP,
    from the head's transfer matrix (solved once, not timed)."""
    import torch
    from paper_1811_07717_gb300 import workloads as W
    from paper_1811_07717_gb300 import _build, zi
    _build.build()
    spec = W.config_eit_2mm()
    mesh = zi.mesh_from_grid(spec.h, spec.radii)
    s6 = W.conductivity(spec, mesh["nodes"].cpu().numpy(), mesh["tets"].cpu().numpy(),
                        mesh["labels"].cpu().numpy())
    centres, z = W.electrode_inputs(spec)
    system = zi.System(mesh["nodes"], mesh["tets"], s6, mesh["bfaces"], centres, model="cem", z=z,
                       radius=spec.electrode_radius)
    opts = zi.SolverOpts(tol=1e-10)
    system.transfer(opts)
    I = torch.from_numpy(W.injection_patterns(spec.n_electrodes)).cuda()
    gy = torch.ones((I.shape[0], spec.n_electrodes), dtype=torch.float64, device="cuda")
    m = system.info()["m"]

    def timed(mode, reps):
        system.eit(I, mode=mode, grad_y=gy if mode == zi.EIT_VJP else None, opts=opts, want_y=False)
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        t0.record()
        for _ in range(reps):
            _, out = system.eit(I, mode=mode, grad_y=gy if mode == zi.EIT_VJP else None, opts=opts, want_y=False)
            del out
        t1.record()
        torch.cuda.synchronize()
        return t0.elapsed_time(t1) / 1e3 / reps

    with Clocks(torch.cuda.current_device()) as clk:
        vjp = timed(zi.EIT_VJP, max(1, args.steps))
        full = timed(zi.EIT_FULL, max(1, args.steps))
    system.close()
    out_bytes = float(m) * I.shape[0] * spec.n_electrodes * 8
    L_el, n_pat = spec.n_electrodes, I.shape[0]
    flops = float(m) * 2.0 * L_el * (16 + 4 * n_pat)  # K w_k per electrode, then u_p . (K w_k)
    peak_tf = 1.25  # nominal FP64 rate of the part (no measured FP64 figure is available)
    line = {"metric": "linearised-EIT Jacobian s (31 patterns x 32 electrodes x every tet, 2 mm head)",
            "value": full, "unit": "s", "n_gpus": 1, "steps": args.steps, "warmup": 1,
            "higher_is_better": False, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "three-shell 2 mm head, 32 CEM electrodes, 31 adjacent-pair 1 mA patterns",
                       "tets": int(m), "jacobian_bytes": out_bytes},
            "vjp_s": vjp,
            "roofline": {"bound": "alu", "kernel": "k_eit_full (FP64: -u_p^T K_m w_k for every tet)",
                         "achieved": flops / full / 1e12, "peak": peak_tf, "unit": "TFLOP/s",
                         "frac": flops / full / 1e12 / peak_tf, "peak_note": "nominal FP64", "traffic": None,
                         "jacobian_write_GBps": out_bytes / full / 1e9},
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def cpu_leg(kind, text, args):
    """cpu_baseline of the H(div) and MEG lines (rank 0 at N=1 only; skipped
    by --no-cpu); a failure is reported, never replaced."""
    if args.no_cpu or dist_env()[1] != 1:
        return None
    try:
        return {"value": oracle_sample_once(kind), "unit": "s", "cores": 1, "kind": "oracle", "sample": text}
    except Exception as ex:
        return {"value": None, "unit": "s", "cores": 1, "kind": "oracle", "sample": "failed: %s" % ex}


def hdiv_workload(args):
    """The 2 mm lead-field build with Cartesian H(div) sources (PBO 10-source
    stencil, Sec. 2.1) in place of partial integration: the whole build, and
    the two source steps alone (stencil construction; T^T F and the electrode
    step) next to the partial-integration source step."""
    import torch
    from paper_1811_07717_gb300 import workloads as W
    from paper_1811_07717_gb300 import _build, zi
    _build.build()
    spec = W.config_three_shell_2mm()
    mesh = zi.mesh_from_grid(spec.h, spec.radii)
    s6 = torch.from_numpy(W.conductivity(spec, mesh["nodes"].cpu().numpy(), mesh["tets"].cpu().numpy(),
                                         mesh["labels"].cpu().numpy())).cuda()
    centres, z = W.electrode_inputs(spec)
    centres, z = torch.from_numpy(centres).cuda(), torch.from_numpy(z).cuda()
    pos = torch.from_numpy(W.dipole_inputs(spec)[0]).cuda()
    mixed = zi.SolverOpts(tol=1e-10, precision=zi.MIXED)

    def build_system():
        return zi.System(mesh["nodes"], mesh["tets"], s6, mesh["bfaces"], centres, model="cem", z=z,
                         radius=spec.electrode_radius)

    def lf_build():
        dip = zi.locate_dipoles_grid(spec.h, spec.radii, pos)
        system = build_system()
        L = system.leadfield_hdiv(pos, dip, zi.SOURCE_PBO10, opts=mixed)
        system.close()
        return L

    def ev_time(fn, reps):
        fn()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        t0.record()
        for _ in range(reps):
            fn()
        t1.record()
        torch.cuda.synchronize()
        return t0.elapsed_time(t1) / 1e3 / reps

    for _ in range(args.warmup):
        lf_build()
    torch.cuda.synchronize()
    l0 = zi.kernel_launches()
    with Clocks(torch.cuda.current_device()) as clk:
        sec = ev_time(lf_build, max(1, args.steps))
    launches = (zi.kernel_launches() - l0) // (max(1, args.steps) + 1)
    system = build_system()
    system.transfer(mixed, want_T=False)
    dip = zi.locate_dipoles_grid(spec.h, spec.radii, pos)
    Fn, Fw = system.source_stencil(pos, dip, zi.SOURCE_PBO10)
    t_stencil = ev_time(lambda: system.source_stencil(pos, dip, zi.SOURCE_PBO10), 5)
    t_sparse = ev_time(lambda: system.leadfield_sparse(Fn, Fw, mixed), 5)
    t_pi = ev_time(lambda: system.leadfield(dip, mixed), 5)
    ms_apply, bytes_apply = system.time_source_apply(Fn, Fw, reps=5)
    system.close()
    peak, peak_note = measured_peak_gbs()
    achieved = bytes_apply / (ms_apply * 1e-3) / 1e9
    line = {"metric": "EEG lead-field build s, Cartesian H(div) sources (PBO 10-source stencil)",
            "value": sec, "unit": "s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": False, "dtype": "f32 inner PCG / f64 refinement, assembly, LF",
            "data": "synthetic",
            "config": {"workload": "three-shell 2 mm head (428185 nodes, 2447424 tets), 128 CEM electrodes, "
                                   "20000 H(div) sources x 3 orientations, PCG tol 1e-10, mixed precision"},
            "cpu_baseline": cpu_leg("hdiv", HDIV_SAMPLE_TEXT, args),
            "source_stencil_s": t_stencil, "leadfield_sparse_s": t_sparse,
            "leadfield_partial_integration_s": t_pi,
            "roofline": {"bound": "hbm", "kernel": "k_source_apply_ell (H^T = F^T T over the stencil nodes)",
                         "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "peak_note": peak_note, "traffic": None, "algorithmic_bytes": bytes_apply,
                         "ms_per_launch": ms_apply},
            "gpu_launches": int(launches), "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def meg_workload(args):
    """The MEG lead field of the 2 mm head (App. A.2 by Biot-Savart): 256
    magnetometers 20 mm outside the scalp, 20,000 partial-integration dipoles
    x 3; the build = assembly, the sensors' right-hand sides, one mixed
    precision PCG solve per sensor, the source columns and L."""
    import torch
    from paper_1811_07717_gb300 import workloads as W
    from paper_1811_07717_gb300 import _build, zi
    _build.build()
    spec = W.config_three_shell_2mm()
    mesh = zi.mesh_from_grid(spec.h, spec.radii)
    s6 = torch.from_numpy(W.conductivity(spec, mesh["nodes"].cpu().numpy(), mesh["tets"].cpu().numpy(),
                                         mesh["labels"].cpu().numpy())).cuda()
    centres, z = W.electrode_inputs(spec)
    centres, z = torch.from_numpy(centres).cuda(), torch.from_numpy(z).cuda()
    pos = torch.from_numpy(W.dipole_inputs(spec)[0]).cuda()
    sp_np, sd_np = W.meg_sensors(256, spec.radii[-1] + 0.02)
    sp_, sd = torch.from_numpy(sp_np).cuda(), torch.from_numpy(sd_np).cuda()
    mixed = zi.SolverOpts(tol=1e-10, precision=zi.MIXED)

    def build_system():
        return zi.System(mesh["nodes"], mesh["tets"], s6, mesh["bfaces"], centres, model="cem", z=z,
                         radius=spec.electrode_radius)

    def lf_build():
        dip = zi.locate_dipoles_grid(spec.h, spec.radii, pos)
        system = build_system()
        Tm, _, _ = system.meg_transfer(sp_, sd, mixed)
        Fn, Fw = system.source_pi(dip)
        L = system.meg_leadfield(Tm, sp_, sd, pos, Fn, Fw)
        system.close()
        return L

    def ev_time(fn, reps):
        fn()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        t0.record()
        for _ in range(reps):
            fn()
        t1.record()
        torch.cuda.synchronize()
        return t0.elapsed_time(t1) / 1e3 / reps

    for _ in range(args.warmup):
        lf_build()
    torch.cuda.synchronize()
    l0 = zi.kernel_launches()
    with Clocks(torch.cuda.current_device()) as clk:
        sec = ev_time(lf_build, max(1, args.steps))
    launches = (zi.kernel_launches() - l0) // (max(1, args.steps) + 1)
    system = build_system()
    t_rhs = ev_time(lambda: system.meg_rhs(sp_, sd), 3)
    _, it, rr = system.meg_transfer(sp_, sd, mixed)
    system.close()
    m = int(mesh["tets"].shape[0])
    flops = 180.0 * m * 256  # per (tet, sensor): gradients, 4-point kernel integral, cross and sigma products
    peak_tf = 1.25
    line = {"metric": "MEG lead-field build s (Biot-Savart, 256 magnetometers)", "value": sec, "unit": "s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": False,
            "dtype": "f64 right-hand sides and L; f32 inner PCG / f64 refinement", "data": "synthetic",
            "config": {"workload": "three-shell 2 mm head (428185 nodes, 2447424 tets), 128 CEM electrodes "
                                   "attached, 256 magnetometers on a 112 mm sphere (radial + 0.6 tangential), "
                                   "20000 dipoles x 3, PCG tol 1e-10, mixed precision"},
            "cpu_baseline": cpu_leg("meg", MEG_SAMPLE_TEXT, args),
            "meg_rhs_s": t_rhs, "iterations_max": int(it.max()), "relres_max": float(rr.max()),
            "roofline": {"bound": "alu", "kernel": "k_meg_tet (FP64 kernel integrals per tet and sensor)",
                         "achieved": flops / t_rhs / 1e12, "peak": peak_tf, "unit": "TFLOP/s",
                         "frac": flops / t_rhs / 1e12 / peak_tf, "peak_note": "nominal FP64; the right-hand "
                         "side build (both of its kernels) timed", "traffic": None},
            "gpu_launches": int(launches), "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def segmesh_workload(args):
    """The mesher from a surface segmentation (Sec. 2.5) on three nested
    icosphere surfaces (80 / 86 / 92 mm, 5120 triangles each) at h = 2 mm,
    skull first by priority, then the nearest-DOF interpolation of the mesh
    nodes to 20,000 source positions."""
    import torch
    from paper_1811_07717_gb300 import workloads as W
    from paper_1811_07717_gb300 import _build, zi
    _build.build()
    centre = (0.00013, -0.00007, 0.00011)  # keeps the surfaces off the grid nodes
    surf = [W.icosphere(4, r, centre) for r in (0.080, 0.086, 0.092)]
    prio = (2, 1, 3)
    pos = torch.from_numpy(W.random_dipoles(20000, 0.078, 2)[0]).cuda()

    def ev_time(fn, reps):
        fn()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        t0.record()
        for _ in range(reps):
            out = fn()
        t1.record()
        torch.cuda.synchronize()
        return t0.elapsed_time(t1) / 1e3 / reps, out

    with Clocks(torch.cuda.current_device()) as clk:
        t_mesh, mesh = ev_time(lambda: zi.mesh_from_surfaces(0.002, surf, prio), max(1, args.steps))
        t_interp, _ = ev_time(lambda: zi.nearest_source(mesh["nodes"], pos), max(1, args.steps))
    G = 2 * (int(np.ceil(0.0921 / 0.002)) + 1) + 1
    n_tri = sum(t.shape[0] for _, t in surf)
    line = {"metric": "segmentation mesh s (3 surfaces, h = 2 mm)", "value": t_mesh, "unit": "s", "n_gpus": 1,
            "steps": args.steps, "warmup": 1, "higher_is_better": False, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "three nested icospheres 80/86/92 mm (5120 triangles each), h = 2 mm grid, "
                                   "priorities skull > brain > scalp; nearest of 20000 source positions per node",
                       "grid_nodes": G ** 3, "triangles": n_tri, "mesh_nodes": int(mesh["nodes"].shape[0]),
                       "mesh_tets": int(mesh["tets"].shape[0])},
            "interpolation_s": t_interp,
            "note": "winding numbers by brute force: grid nodes x triangles solid angles (two passes, counts "
                    "then outputs)",
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def spmm_workload(args):
    """The solver's SpMM on its own, for a profiler: builds one three-shell
    head's system, runs one CG iteration so the work vectors and the solver's
    matrix copies exist, then launches the SpMM `--reps` times after an L2
    flush (zi_time_spmm).  The first SpMM launch belongs to the one-iteration
    solve; select the standalone ones with ncu -s 1.  Prints the CUDA-event
    time per launch and the algorithmic bytes."""
    import torch
    from paper_1811_07717_gb300 import workloads as W
    from paper_1811_07717_gb300 import _build, zi
    _build.build()
    spec = W.three_shell(args.h, args.electrodes, 10, seed=2,
                         skull_aniso=(0.00132, 0.0132) if args.aniso else None)
    mesh = zi.mesh_from_grid(spec.h, spec.radii)
    s6 = W.conductivity(spec, mesh["nodes"].cpu().numpy(), mesh["tets"].cpu().numpy(),
                        mesh["labels"].cpu().numpy())
    centres, z = W.electrode_inputs(spec)
    system = zi.System(mesh["nodes"], mesh["tets"], s6, mesh["bfaces"], centres, model="cem", z=z,
                       radius=spec.electrode_radius)
    prec = zi.MIXED if args.precision == "mixed" else zi.FP64
    opts = zi.SolverOpts(tol=1e-10, precision=prec, maxit=1, check_every=1, max_outer=1)
    system.transfer(opts, want_T=False, allow_not_converged=True)
    ms, by = system.time_spmm(prec, reps=args.reps)
    torch.cuda.synchronize()
    info = system.info()
    print(json.dumps({"workload": "spmm", "h": args.h, "aniso": bool(args.aniso), "n": info["n"],
                      "nnz": info["nnz"], "ncol": info["n_rhs"], "precision": args.precision,
                      "spmm_kernel": info.get("spmm_kernel"), "ms_per_launch": ms, "algorithmic_bytes": by,
                      "GBps": by / ms / 1e6}), flush=True)
    system.close()


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
        return
    rank, world, local = dist_env()
    import torch
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    from paper_1811_07717_gb300 import workloads as W
    from paper_1811_07717_gb300 import _build, zi
    _build.build()

    if args.workload not in ("shell2mm", "aniso1mm") and world > 1:
        # the single-GPU workloads (batch, IAS, EIT, H(div), MEG, mesher, SpMM) run on rank 0 alone
        if rank != 0:
            dist.destroy_process_group()
            return
    if args.workload == "batch":
        return batch_workload(args)
    if args.workload == "ias":
        return ias_workload(args)
    if args.workload == "eit":
        return eit_workload(args)
    if args.workload == "hdiv":
        return hdiv_workload(args)
    if args.workload == "meg":
        return meg_workload(args)
    if args.workload == "segmesh":
        return segmesh_workload(args)
    if args.workload == "spmm":
        return spmm_workload(args)
    spec = getattr(W, WORKLOADS[args.workload][0])()
    workload = WORKLOADS[args.workload][1]
    dev = torch.device("cuda", local)
    mesh = zi.mesh_from_grid(spec.h, spec.radii)
    s6 = W.conductivity(spec, mesh["nodes"].cpu().numpy(), mesh["tets"].cpu().numpy(), mesh["labels"].cpu().numpy())
    centres, z = W.electrode_inputs(spec)
    pos, q = W.dipole_inputs(spec)
    d = dict(nodes=mesh["nodes"], tets=mesh["tets"], bfaces=mesh["bfaces"],
             s6=torch.from_numpy(s6).to(dev), centres=torch.from_numpy(centres).to(dev),
             z=torch.from_numpy(z).to(dev), pos=torch.from_numpy(pos).to(dev))
    torch.cuda.synchronize()

    def lf_build(opts):
        dip = zi.locate_dipoles_grid(spec.h, spec.radii, d["pos"])
        system = zi.System(d["nodes"], d["tets"], d["s6"], d["bfaces"], d["centres"], model="cem", z=d["z"],
                           radius=spec.electrode_radius)
        L = system.leadfield(dip, opts)
        system.close()
        return L

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def timed(opts, warmup, steps, tag):
        for _ in range(warmup):
            L = lf_build(opts)
        barrier()
        l0 = zi.kernel_launches()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with Clocks(torch.cuda.current_device()) as clk:
            torch.cuda.nvtx.range_push(tag)  # lets a profiler select the timed builds (ncu --nvtx-include)
            t0.record()
            for _ in range(steps):
                L = lf_build(opts)
            t1.record()
            torch.cuda.nvtx.range_pop()
            barrier()
        launches = zi.kernel_launches() - l0
        sec = max_over_ranks(t0.elapsed_time(t1) / 1e3 / steps, dist, dev)
        return sec, L, launches, clk.summary()

    mixed = zi.SolverOpts(tol=1e-10, precision=zi.MIXED)
    fp64 = zi.SolverOpts(tol=1e-10, precision=zi.FP64)
    sec_mixed, L_mixed, launches, clocks = timed(mixed, args.warmup, args.steps, "timed_mixed")

    extra = {}
    if not args.no_fp64:
        sec64, L64, _, clocks64 = timed(fp64, 1, 1, "timed_fp64")
        diff = float(torch.linalg.norm(L_mixed - L64) / torch.linalg.norm(L64))
        extra = {"fp64_lf_build_s": sec64, "speedup_mixed_vs_fp64": sec64 / sec_mixed,
                 "mixed_vs_fp64_rel_frobenius": diff, "fp64_clocks": clocks64}
        del L64

    # iteration counts and the SpMM roofline on one more build
    system = zi.System(d["nodes"], d["tets"], d["s6"], d["bfaces"], d["centres"], model="cem", z=d["z"],
                       radius=spec.electrode_radius)
    _, it_mixed, rr_mixed = system.transfer(mixed, want_T=False)
    sinfo = system.solver_info()
    n_p = float(system.info()["n"]) * system.info()["n_rhs"]  # P elements (unpadded)
    ms32, bytes32 = system.time_spmm(zi.MIXED, reps=5)
    it64 = None
    if not args.no_fp64:
        _, it64, _ = system.transfer(fp64, want_T=False)
        ms64, bytes64 = system.time_spmm(zi.FP64, reps=3)
        extra["spmm_fp64"] = {"ms_per_launch": ms64, "algorithmic_GBps": bytes64 / ms64 / 1e6,
                              "bound": "fp64 FMA pipe (ncu: sm__pipe_fp64_cycles_active ~94%)"}
    system.close()
    peak, peak_note = measured_peak_gbs()
    achieved = bytes32 / (ms32 * 1e-3) / 1e9
    cap = SPMM_TRAFFIC.get(args.workload)
    traffic = cap["bytes"] if cap and cap["source_sha"] == spmm_source_sha() else None
    kname = {zi.SPMM32_ELL: "k_spmm_ell<%d, false>", zi.SPMM32_ELL_OVERFLOW: "k_spmm_ell<%d, true>"}.get(
        sinfo["spmm32"], "k_spmm_ell<%d, ?>") % sinfo["vectors_per_thread32"]
    # the bytes the kernel moves: P is read in FP16 (2 B), Q written in FP32 (4 B).  The same launch counted
    # with P at 4 B (the accounting of an FP32 direction) is reported beside it.
    bytes_p32 = bytes32 + 2.0 * n_p
    roofline = {"bound": "hbm", "kernel": kname + " (FP32 SpMM in difference form on the FP16 direction, "
                                                  "fused with the p.q column dots)",
                "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "peak_note": peak_note, "traffic": traffic,
                "traffic_note": cap["note"] if cap and traffic is not None else None,
                "algorithmic_bytes": bytes32, "ms_per_launch": ms32, "solver_layout": sinfo,
                "p_fp32_accounting": {"algorithmic_bytes": bytes_p32,
                                      "achieved": bytes_p32 / (ms32 * 1e-3) / 1e9,
                                      "frac": bytes_p32 / (ms32 * 1e-3) / 1e9 / peak}}

    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        host = {k: v.cpu().pin_memory() for k, v in d.items()}
        h2d = sum(v.numel() * v.element_size() for v in host.values())

        def e2e_build():
            dd = {k: v.to(dev, non_blocking=True) for k, v in host.items()}
            dip = zi.locate_dipoles_grid(spec.h, spec.radii, dd["pos"])
            system = zi.System(dd["nodes"], dd["tets"], dd["s6"], dd["bfaces"], dd["centres"], model="cem",
                               z=dd["z"], radius=spec.electrode_radius)
            L = system.leadfield(dip, mixed).cpu()
            system.close()
            return L
        e2e_build()
        barrier()
        t = time.perf_counter()
        for _ in range(max(1, args.steps)):
            Lh = e2e_build()
        barrier()
        e2e_sec = (time.perf_counter() - t) / max(1, args.steps)
        e2e = {"value": e2e_sec, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(Lh.numel() * Lh.element_size())}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        text = cpu_pcg_text(args.workload)
        try:
            m = cpu_pcg_workload(args.workload, 1)
            cpu = {"value": m["s_per_iteration"][0] * m["iterations"], "unit": UNIT, "cores": m["threads"],
                   "kind": "oracle", "sample": text}
            extra["cpu_pcg"] = dict(m, gpu_fp64_s_per_iteration=(
                None if it64 is None else extra["fp64_lf_build_s"] / max(1, int(it64.max()))),
                gpu_fp64_iterations=None if it64 is None else int(it64.max()))
        except Exception as ex:  # reported, never silently replaced
            cpu = {"value": None, "unit": UNIT, "cores": None, "kind": "oracle", "sample": "failed: %s" % ex}
        try:
            extra["cpu_oracle_direct"] = {"value": oracle_once(args.workload), "unit": UNIT, "cores": 1,
                                          "kind": "oracle", "sample": DIRECT_SAMPLES[args.workload][1]}
        except Exception as ex:
            extra["cpu_oracle_direct"] = {"value": None, "sample": "failed: %s" % ex}

    if rank == 0:
        line = {"metric": METRIC, "value": sec_mixed, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": sec_mixed * 1e3, "higher_is_better": False,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32 inner PCG / f64 refinement, assembly, LF",
                "data": "synthetic",
                "config": {"workload": workload, "n_nodes": int(d["nodes"].shape[0]),
                           "n_tets": int(d["tets"].shape[0]), "electrodes": spec.n_electrodes,
                           "dipoles": spec.n_dipoles,
                           "precision": "mixed",
                           "l2": "inputs larger than L2 (T alone is %.0f MB)" % (
                               d["nodes"].shape[0] * spec.n_electrodes * 8 / 1e6),
                           "parallelism": "replicas" if world > 1 else "single GPU"},
                "iterations_mixed_max": int(it_mixed.max()), "relres_mixed_max": float(rr_mixed.max()),
                "iterations_fp64_max": None if it64 is None else int(it64.max()),
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
                "clocks": clocks}
        line.update(extra)
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
