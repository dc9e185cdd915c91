"""Write the oracle's results for the large-mesh parity tests (test infrastructure).

The FP64 oracle (oracle/u1mpo.py: App. D, Eq. `theta`, block SVD, keep-chi rule and
Vidal re-split) runs a standard workload's Clements mesh gate by gate from the
initial state and records, after each requested prefix of gates, what the GPU
parity tests compare: Tr rho, <n_j>, <n_j^2>, the entropy and purity at every cut,
the bond dimensions, the largest bond weights of every bond, and the per-gate
discarded weights.  A prefix equal to the whole mesh also applies the final phase
screen, as the benchmark's step does.

Only `oracle/` and the seeded input generators (`gbs_workloads`) are called; no
value comes from the CUDA path.  The oracle takes about 1 s per gate at chi = 512 on
one x86 core, so the 48-mode mesh takes about 20 minutes:

    OPENBLAS_NUM_THREADS=1 python tests/golden/make_mesh_goldens.py M32_d8_chi256 120,496
    OPENBLAS_NUM_THREADS=1 python tests/golden/make_mesh_goldens.py M48_d8_chi512 60,1128
"""
from __future__ import annotations

import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

LAM_TOP = 8  # largest bond weights recorded per bond


def largest_block(P, j: int):
    """(Gram side, long side) of the largest Theta(m) of the gate on modes (j, j+1):
    for every centre charge m, rows = indices of bond j whose charge dominates m and
    columns = indices of bond j+2 dominated by m (App. D); Gram side = min(rows, cols)."""
    import numpy as np
    A, B = P.charges[j], P.charges[j + 2]
    best = (0, 0)
    for cm in range(P.n_cap + 1):
        for cbm in range(P.n_cap + 1):
            r = int(np.count_nonzero((A[:, 0] >= cm) & (A[:, 1] >= cbm)))
            c = int(np.count_nonzero((B[:, 0] <= cm) & (B[:, 1] <= cbm)))
            if min(r, c) > best[0]:
                best = (min(r, c), max(r, c))
    return best


def snapshot(P, n_done: int) -> dict:
    tr, n1, n2 = P.observables()
    lam_top = []
    for l in P.lam:
        s = sorted((float(x) for x in l), reverse=True)
        lam_top.append(s[:LAM_TOP])
    return {"gates": n_done, "trace": float(tr), "n_mean": [float(x) for x in n1],
            "n2_mean": [float(x) for x in n2], "entropy": [float(x) for x in P.entropy],
            "purity": [float(x) for x in P.purities()], "chi": [int(len(l)) for l in P.lam],
            "lam_top": lam_top}


def make(name: str, prefixes) -> str:
    import gbs_workloads as w
    from oracle import u1mpo
    wl = w.workload(name)
    mesh = wl.mesh(0)
    prefixes = sorted(set(min(int(p), mesh.n_gates) for p in prefixes))
    P = u1mpo.U1MPO(wl.M, wl.d, wl.r[0], wl.eta[0], chi_max=wl.chis[0])
    snaps = []
    t0 = time.time()
    done = 0
    big = (0, 0)
    for p in prefixes:
        for i in range(done, p):
            big = max(big, largest_block(P, int(mesh.k[i])))
            P.apply_gate(int(mesh.k[i]), float(mesh.theta[i]), float(mesh.phi[i]))
        done = p
        if p == mesh.n_gates:
            P.apply_phases(mesh.final_phase)
        s = snapshot(P, p)
        s["final_phases"] = p == mesh.n_gates
        s["largest_block"] = {"gram_side": big[0], "long_side": big[1]}
        snaps.append(s)
        print(f"{name}: {p} gates, max chi {max(s['chi'])}, {time.time() - t0:.0f} s", flush=True)
    out = {"workload": name, "M": wl.M, "d": wl.d, "chi": wl.chi, "seed": int(wl.seeds[0]),
           "r": float(wl.r[0, 0]), "eta": float(wl.eta[0, 0]), "n_gates_mesh": mesh.n_gates,
           "source": "oracle/u1mpo.py (FP64; App. D Eq. theta, LAPACK SVD per block, keep chi)",
           "discarded": [float(x) for x in P.discarded], "snapshots": snaps}
    path = os.path.join(HERE, f"mesh_{name}.json")
    with open(path, "w") as f:
        json.dump(out, f, separators=(",", ":"))
    return path


if __name__ == "__main__":
    print(make(sys.argv[1], [int(x) for x in sys.argv[2].split(",")]))
