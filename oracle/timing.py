"""Time the FP64 oracle on a bounded sample of a workload (oracle; test infrastructure).

Used only by bench.py (its cpu_baseline leg and its reference arm).  Runs the
oracle as it stands -- no tuning -- on the first `n_gates` gates of instance 0's
mesh, starting from the initial state, and reports beam-splitter updates per
second of wall time plus the observables at the end of the sample.

Run as a module so that the caller can pin the BLAS thread count in the child's
environment:  python -m oracle.timing <workload> <n_gates> [repeats]
"""
from __future__ import annotations

import json
import os
import sys
import time


def _cores(threads: dict) -> int:
    """Threads the BLAS/OpenMP environment allows (all host cores when unset)."""
    vals = [int(v) for v in threads.values() if v and v.isdigit()]
    return min(vals) if vals else (os.cpu_count() or 1)


def run(name: str, n_gates: int, repeats: int = 1) -> dict:
    import gbs_workloads as w
    from . import u1mpo
    wl = w.workload(name)
    mesh = wl.mesh(0)
    n = min(n_gates, mesh.n_gates)
    times = []
    P = None
    for _ in range(max(1, repeats)):
        t0 = time.perf_counter()
        P = u1mpo.U1MPO(wl.M, wl.d, wl.r[0], wl.eta[0], chi_max=wl.chis[0])
        t1 = time.perf_counter()
        P.run_mesh(mesh.k[:n], mesh.theta[:n], mesh.phi[:n])
        t2 = time.perf_counter()
        times.append(t2 - t1)
    tr, n1, n2 = P.observables()
    threads = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    return {
        "workload": name, "gates": n, "seconds": times, "init_seconds": t1 - t0,
        "updates_per_s": [n / t for t in times], "trace": tr, "n_mean": list(n1), "n2_mean": list(n2),
        "entropy": list(P.entropy), "discarded_sum": float(sum(P.discarded)),
        "cores": _cores(threads), "threads_env": threads,
    }


def run_asymptotic(n_points: int, repeats: int = 1) -> dict:
    """The App. C estimator of the oracle on the first n_points of the Fig. 1 grid."""
    import gbs_workloads as w
    from . import asymptotic
    g = w.asymptotic_grid()
    n = min(n_points, g.size)
    times, S = [], []
    for _ in range(max(1, repeats)):
        t0 = time.perf_counter()
        S = [asymptotic.system_entropy(int(g.N[i]), float(g.beta[i]), float(g.gamma[i]), g.r, g.n_max)
             for i in range(n)]
        times.append(time.perf_counter() - t0)
    threads = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    return {"workload": g.name, "points": n, "seconds": times, "points_per_s": [n / t for t in times],
            "S": S, "cores": _cores(threads), "threads_env": threads}


if __name__ == "__main__":
    if sys.argv[1] == "asymptotic":
        n = int(sys.argv[2])
        rep = int(sys.argv[3]) if len(sys.argv) > 3 else 1
        print(json.dumps(run_asymptotic(n, rep)))
        sys.exit(0)
    name = sys.argv[1]
    n = int(sys.argv[2])
    rep = int(sys.argv[3]) if len(sys.argv) > 3 else 1
    print(json.dumps(run(name, n, rep)))
