"""Run the oracle to convergence on the full-size workloads and store the
results in oracle/reference_runs.json -- TEST INFRASTRUCTURE ONLY.

The stored eigenvalues are the FP64 oracle's answer for the full-size
operators (used as full-size parity references), and the stored cycle counts
and per-phase timings let the CPU-baseline measurement extrapolate a bounded
sample of the oracle to a whole solve.  Calls only ``oracle/`` and the seeded
input generators.  Usage:
  python -m oracle.reference_runs [name ...]                  run and store
  python -m oracle.reference_runs --time-on-this-host NAME OUT.json
  python -m oracle.reference_runs --add-host-timing OUT.json  add that run's timing
"""
from __future__ import annotations

import json
import os
import platform
import sys
import time

import numpy as np

from oracle import trplk as O

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "reference_runs.json")


def workloads():
    from paper_1711_10128_gb300 import workloads as W
    return {
        # 3D 7-point lognormal(0,1) diffusion on 128^3, 10 smallest, Jacobi, q=40, p_hat=15, +K=1, tol 1e-8
        "diffusion128": dict(build=lambda: (W.diffusion_3d(128, W.lognormal_field(128, 1.0, 1)), None),
                             p=10, q=40, k=15, l=1, tol=1e-8, seed=0),
        # the 128^3 diffusion operator above at tol 1e-12: there the Kato-Temple bound of every pair falls
        # below 1e-10 relative, so the eigenvalues of any two converged runs compare at 1e-10
        "diffusion128_tight": dict(build=lambda: (W.diffusion_3d(128, W.lognormal_field(128, 1.0, 1)), None),
                                   p=10, q=40, k=15, l=1, tol=1e-12, seed=0),
        # 2D 5-point Laplacian on 100x100, 5 smallest, Jacobi, q=20, p_hat=8, +K=5, tol 1e-8
        "laplace100": dict(build=lambda: (W.laplacian_2d(100), None), p=5, q=20, k=8, l=5, tol=1e-8, seed=0),
        # Q1 stiffness/mass pencil on 96^3 elements, E ~ U[1,10] (seed 2), 20 smallest, q=50, p_hat=25, +K=1
        "q1pencil96": dict(build=lambda: W.fem_q1_pencil(96, np.random.default_rng(2).uniform(1.0, 10.0,
                                                                                            (96, 96, 96))),
                           p=20, q=50, k=25, l=1, tol=1e-8, seed=0),
        # L + 1e-3 I of a Chung-Lu graph (2^22 vertices, mean degree 16, gamma 2.1, seed 3, largest component),
        # 16 smallest, q=40, p_hat=20, +K=1
        "chunglu22": dict(build=lambda: (W.chung_lu_laplacian(1 << 22, 16.0, 2.1, 3), None),
                          p=16, q=40, k=20, l=1, tol=1e-8, seed=0),
        # the Chung-Lu operator above at tol 1e-12: there the Kato-Temple bound of its clustered pairs
        # (gap ~2e-5, ||A||_1 ~1.6e4) falls below 1e-10 relative, so eigenvalues compare at 1e-10
        "chunglu22_tight": dict(build=lambda: (W.chung_lu_laplacian(1 << 22, 16.0, 2.1, 3), None),
                                p=16, q=40, k=20, l=1, tol=1e-12, seed=0),
        # anisotropic 7-point diffusion on 128^3 (seed 2000), 20 smallest, q=50, p_hat=25, +K=1
        "aniso128": dict(build=lambda: (W.anisotropic_diffusion(128, 2000), None),
                         p=20, q=50, k=25, l=1, tol=1e-8, seed=0),
    }


def run(name):
    from paper_1711_10128_gb300 import workloads as W
    cfg = workloads()[name]
    A, B = cfg["build"]()
    As = A.to_scipy()
    X0 = W.start_block(A.n, cfg["k"], cfg["seed"])
    t0 = time.perf_counter()
    r = O.solve(As, None if B is None else B.to_scipy(), cfg["p"], cfg["q"], cfg["k"], cfg["l"], cfg["tol"], X0,
                "jacobi")
    secs = time.perf_counter() - t0
    return dict(n=A.n, nnz=A.nnz, p=cfg["p"], q=cfg["q"], k=cfg["k"], l=cfg["l"], tol=cfg["tol"],
                status=r["status"], cycles=r["cycles"], mv_A=r["mv_A"], evals=[float(x) for x in r["evals"]],
                resid=[float(x) for x in r["resid"]], seconds=secs, cores=os.cpu_count(),
                host=f"{platform.machine()}, {os.cpu_count()} cores")


def main(names):
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    for name in names:
        data[name] = run(name)
        json.dump(data, open(OUT, "w"), indent=1)
        print(name, data[name]["status"], data[name]["cycles"], data[name]["seconds"], flush=True)


def time_on_this_host(name, path):
    """Run one workload to convergence and write the run alone to `path` (for
    timing the oracle on another machine without touching the stored runs)."""
    r = run(name)
    r["workload"] = name
    json.dump(r, open(path, "w"), indent=1)
    print(name, r["status"], r["cycles"], r["seconds"], r["host"], flush=True)


def add_host_timing(path):
    """Record a run written by `time_on_this_host` as an extra timing of its
    stored workload: host, seconds, cycles, and the largest relative
    difference of its eigenvalues from the stored ones."""
    r = json.load(open(path))
    data = json.load(open(OUT))
    ent = data[r["workload"]]
    ev, ref = np.array(r["evals"]), np.array(ent["evals"])
    timing = dict(host=r["host"], seconds=r["seconds"], cores=r["cores"], cycles=r["cycles"], mv_A=r["mv_A"],
                  status=r["status"], max_rel_eval_diff=float(np.max(np.abs(ev - ref) / np.abs(ref))))
    ent["other_host_timings"] = [t for t in ent.get("other_host_timings", []) if t["host"] != timing["host"]]
    ent["other_host_timings"].append(timing)
    json.dump(data, open(OUT, "w"), indent=1)
    print(r["workload"], timing, flush=True)


if __name__ == "__main__":
    if len(sys.argv) == 4 and sys.argv[1] == "--time-on-this-host":
        time_on_this_host(sys.argv[2], sys.argv[3])
    elif len(sys.argv) == 3 and sys.argv[1] == "--add-host-timing":
        add_host_timing(sys.argv[2])
    else:
        main(sys.argv[1:] or ["laplace100", "diffusion128"])
