"""Profiling driver: builds one head's system, runs a short transfer so the
solver's work vectors and scaled matrices exist, then launches the solver's
SpMM on its own (zi_time_spmm) so an ncu capture can select it:

    ncu --set full --clock-control none -k regex:k_spmm_dot -s 1 -c 1 \\
        -o prof python -m paper_1811_07717_gb300.prof --h 0.002 --precision mixed

The first k_spmm_dot launch belongs to the one-iteration transfer; the
second is the standalone one.  Prints the CUDA-event time of the standalone
launches and the algorithmic GB/s.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--h", type=float, default=0.002)
    ap.add_argument("--electrodes", type=int, default=128)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--iters", type=int, default=1, help="CG iterations before the standalone launches")
    ap.add_argument("--aniso", action="store_true", help="transversely anisotropic skull (radial 0.00132, "
                    "tangential 0.0132 S/m)")
    a = ap.parse_args()
    import torch

    from paper_1811_07717_gb300 import workloads as W
    from paper_1811_07717_gb300 import zi

    spec = W.three_shell(a.h, a.electrodes, 10, seed=2, skull_aniso=(0.00132, 0.0132) if a.aniso else None)
    mesh = zi.mesh_from_grid(spec.h, spec.radii)
    s6 = W.conductivity(spec, mesh["nodes"].cpu().numpy(), mesh["tets"].cpu().numpy(),
                        mesh["labels"].cpu().numpy())
    centres, z = W.electrode_inputs(spec)
    system = zi.System(mesh["nodes"], mesh["tets"], s6, mesh["bfaces"], centres, model="cem", z=z,
                       radius=spec.electrode_radius)
    prec = zi.MIXED if a.precision == "mixed" else zi.FP64
    opts = zi.SolverOpts(tol=1e-10, precision=prec, maxit=a.iters, check_every=a.iters, max_outer=1)
    system.transfer(opts, want_T=False, allow_not_converged=True)
    ms, by = system.time_spmm(prec, reps=a.reps)
    torch.cuda.synchronize()
    info = system.info()
    print(json.dumps({"n": info["n"], "nnz": info["nnz"], "ncol": info["n_rhs"], "precision": a.precision,
                      "ms_per_launch": ms, "algorithmic_bytes": by, "GBps": by / ms / 1e6}))
    system.close()


if __name__ == "__main__":
    main()
