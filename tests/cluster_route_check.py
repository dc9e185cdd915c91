"""Run as a script by test_gpu_cluster.py, in a process whose environment sends every
block of every gate (Gram side >= 1) through the thread-block-cluster SVD.  Prints one
JSON line of results; the oracle runs on the same seeded inputs."""
import json
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import gbs_workloads as w  # noqa: E402
from oracle import u1mpo  # noqa: E402
from paper_2301_12814_gb300 import build, mpo  # noqa: E402


def rel(a, b, atol=1e-12):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return float(np.max(np.abs(a - b) / (atol + np.abs(b))))


def run(name, ngates, precision):
    wl = w.workload(name)
    mesh = wl.mesh()
    n = mesh.n_gates if ngates is None else ngates
    P = u1mpo.U1MPO(wl.M, wl.d, wl.r[0], wl.eta[0], chi_max=wl.chis[0])
    P.run_mesh(mesh.k[:n], mesh.theta[:n], mesh.phi[:n], mesh.final_phase if n == mesh.n_gates else None)
    G = mpo.MPO(wl.M, wl.d, wl.r[0], wl.eta[0], chi_max=wl.chis[0], precision=precision)
    disc = G.sweep_mesh([n], mesh.k[:n], mesh.theta[:n], mesh.phi[:n],
                        mesh.final_phase if n == mesh.n_gates else None)
    tr, n1, n2 = P.observables()
    gtr, gn1, gn2 = G.observables()
    S, _, _ = G.operator_entropy()
    chi, _, _ = G.bonds()
    out = {"tr": abs(float(gtr[0]) - tr), "n1": rel(gn1[0], n1), "n2": rel(gn2[0], n2),
           "S": float(np.max(np.abs(S[0] - np.array(P.entropy)))),
           "disc_abs": float(np.max(np.abs(disc - P.discarded))), "disc_max": float(np.max(P.discarded)),
           "chi_equal": list(map(int, chi)) == [len(l) for l in P.lam]}
    # bitwise reproducible under the cluster path too
    G.reset()
    disc2 = G.sweep_mesh([n], mesh.k[:n], mesh.theta[:n], mesh.phi[:n],
                         mesh.final_phase if n == mesh.n_gates else None)
    out["bitwise_replay"] = bool(np.array_equal(disc, disc2))
    G.close()
    return out


def main():
    mpo.load_library(build.build())
    res = {"exact_fp64": run("exact_M4_d4", None, "fp64"),
           "chi64_fp64": run("M16_d6_chi64", None, "fp64"),
           "chi64_mixed": run("M16_d6_chi64", None, "mixed_tf32"),
           "chi256_fp64_prefix": run("M32_d8_chi256", 24, "fp64")}
    print(json.dumps(res))


if __name__ == "__main__":
    main()
