"""Launch choices (mpo_set_tuning) and the autotuner change the split of the work over
the GPU, never the method: every choice must meet the oracle at the path's bar.

* FP64 path, 16-mode chi = 64 mesh: each cluster choice (no clusters, 2 / 8 CTAs, all
  blocks of Gram side >= 16 on clusters) and both Gram kernels, within 1e-10.
* TF32 path, same mesh: both contraction forms and the no-cluster route, within the
  stated mixed prefix bounds.
* The autotuner on four instances of the batched workload: it returns the fastest of
  its table, leaves that choice installed, and the run under it meets the oracle.
* Out-of-range values are refused with MPO_ERR_ARG and leave the handle unchanged.
"""
import numpy as np
import pytest

import gbs_workloads as w
from oracle import u1mpo

pytestmark = pytest.mark.gpu

MIXED = dict(n=1e-4, n2=1e-4, S=1e-3, tr=1e-4)


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2301_12814_gb300 import build, mpo
    mpo.load_library(build.build())
    return mpo


@pytest.fixture(scope="module")
def chi64():
    wl = w.workload("M16_d6_chi64")
    mesh = wl.mesh()
    P = u1mpo.U1MPO(wl.M, wl.d, wl.r[0], wl.eta[0], chi_max=wl.chi)
    P.run_mesh(mesh.k, mesh.theta, mesh.phi, mesh.final_phase)
    return wl, mesh, P


def _errors(G, P, disc):
    tr, n1, n2 = G.observables()
    S = G.operator_entropy()[0][0]
    otr, on1, on2 = P.observables()
    rel = lambda a, b: float(np.max(np.abs(np.asarray(a) - np.asarray(b)) / np.abs(np.asarray(b))))
    return dict(tr=abs(tr[0] - otr), n=rel(n1[0], on1), n2=rel(n2[0], on2),
                S=float(np.max(np.abs(S - np.asarray(P.entropy)))),
                eps=float(np.max(np.abs(disc - np.asarray(P.discarded)))))


@pytest.mark.parametrize("choice", [
    dict(svd_cluster_size=1), dict(svd_cluster_size=2), dict(svd_cluster_size=8),
    dict(svd_cluster_min_n=16), dict(svd_cluster_min_n=-1), dict(gram_tc_min=1 << 20), dict(gram_tc_min=16),
])
def test_fp64_choices_meet_oracle(lib, chi64, choice):
    wl, mesh, P = chi64
    G = lib.MPO(wl.M, wl.d, wl.r[0], wl.eta[0], chi_max=wl.chi)
    got = G.set_tuning(**choice)
    for k_, v in choice.items():
        assert got[k_] == v
    plan = G.plan_mesh([mesh.n_gates], mesh.k, mesh.theta, mesh.phi, mesh.final_phase)
    plan.run()
    err = _errors(G, P, plan.discarded())
    G.close()
    tr = P.observables()[0]
    assert err["tr"] <= 1e-12 + 1e-10 * tr and err["n"] <= 1e-10 and err["n2"] <= 1e-10, err
    assert err["S"] <= 1e-10 * 4 and err["eps"] <= 1e-12 + 1e-10 * max(P.discarded), err


@pytest.mark.parametrize("choice", [dict(theta_form=1), dict(theta_form=2), dict(svd_cluster_min_n=-1)])
def test_tf32_choices_meet_oracle(lib, chi64, choice):
    wl, mesh, P = chi64
    G = lib.MPO(wl.M, wl.d, wl.r[0], wl.eta[0], chi_max=wl.chi, precision="mixed_tf32")
    G.set_tuning(**choice)
    disc = G.sweep_mesh([mesh.n_gates], mesh.k, mesh.theta, mesh.phi, mesh.final_phase)
    err = _errors(G, P, disc)
    G.close()
    for k_, b in MIXED.items():
        assert err[k_] <= b, (k_, err)


def test_tuning_rejects_bad_values(lib):
    G = lib.MPO(4, 4, [0.5] * 4, [0.5] * 4)
    before = G.get_tuning()
    for bad in [dict(theta_form=3), dict(svd_cluster_size=3), dict(gram_tc_min=-1), dict(svd_cluster_seed_max=-2)]:
        with pytest.raises(lib.MPOError) as ei:
            G.set_tuning(**bad)
        assert ei.value.status == 1
        assert G.get_tuning() == before
    G.close()


def test_autotune_installs_fastest_and_meets_oracle(lib):
    from paper_2301_12814_gb300 import autotune as at
    wl = w.workload("batched_64x_M16_d6")
    insts = [3, 20, 41, 60]
    meshes = [wl.mesh(i) for i in insts]
    n_gates = [m.n_gates for m in meshes]
    cat = lambda f: np.concatenate([getattr(m, f) for m in meshes])
    k, th, ph, fp = cat("k"), cat("theta"), cat("phi"), cat("final_phase")
    G = lib.MPO(wl.M, wl.d, np.stack([wl.r[i] for i in insts]), np.stack([wl.eta[i] for i in insts]),
                chi_max=[wl.chis[i] for i in insts], batch=len(insts), precision="mixed_tf32")
    res = at.autotune(G, n_gates, k, th, ph, fp, precision="mixed_tf32",
                      space={"theta_form": [1, 2], "svd_cluster_min_n": [0, -1]})
    assert len(res["table"]) == 4
    assert res["best_ms"] <= res["default_ms"]
    assert res["best_ms"] <= min(ms for ms, _ in res["table"])
    assert G.get_tuning() == res["best"]
    disc = G.sweep_mesh(n_gates, k, th, ph, fp)
    tr, n1, n2 = G.observables()
    off = np.concatenate([[0], np.cumsum(n_gates)])
    for b, i in enumerate(insts):
        P = u1mpo.U1MPO(wl.M, wl.d, wl.r[i], wl.eta[i], chi_max=wl.chis[i])
        P.run_mesh(meshes[b].k, meshes[b].theta, meshes[b].phi, meshes[b].final_phase)
        otr, on1, _ = P.observables()
        assert abs(tr[b] - otr) <= MIXED["tr"]
        assert np.max(np.abs(n1[b] - on1) / on1) <= MIXED["n"]
        assert np.max(np.abs(disc[off[b]:off[b + 1]] - np.asarray(P.discarded))) <= 1e-2 * max(P.discarded) + 1e-9
    G.close()
