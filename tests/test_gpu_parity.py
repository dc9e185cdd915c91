"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

FP64 bar (stated for the FP64 mode): every observable within 1e-10 relative of the
oracle, absolute floor 1e-12 -- Tr rho, <n_j>, <n_j^2>, the entropy at every cut and
the per-gate discarded weights; bond dimensions identical.  The oracle runs on the
same seeded inputs (gbs_workloads); no expected value comes from the CUDA path.
"""
import numpy as np
import pytest

import gbs_workloads as w
from oracle import u1mpo

pytestmark = pytest.mark.gpu

RTOL, ATOL = 1e-10, 1e-12


def close(a, b, rtol=RTOL, atol=ATOL):
    a, b = np.asarray(a, dtype=float), np.asarray(b, dtype=float)
    return np.all(np.abs(a - b) <= atol + rtol * np.abs(b))


@pytest.fixture(scope="module")
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2301_12814_gb300 import build, mpo
    mpo.load_library(build.build())
    return mpo


def oracle_run(wl, inst=0, ngates=None, phases=True):
    mesh = wl.mesh(inst)
    n = mesh.n_gates if ngates is None else ngates
    P = u1mpo.U1MPO(wl.M, wl.d, wl.r[inst], wl.eta[inst], chi_max=wl.chis[inst])
    P.run_mesh(mesh.k[:n], mesh.theta[:n], mesh.phi[:n],
               mesh.final_phase if (phases and n == mesh.n_gates) else None)
    return P


def gpu_handle(lib, wl, insts=(0,), precision="fp64"):
    r = np.stack([wl.r[i] for i in insts]); eta = np.stack([wl.eta[i] for i in insts])
    chis = [wl.chis[i] for i in insts]
    return lib.MPO(wl.M, wl.d, r, eta, chi_max=chis, batch=len(insts), precision=precision)


def compare(P, G, inst=0, rtol=RTOL, atol=ATOL, lam_rel=1e-6):
    tr, n1, n2 = P.observables()
    gtr, gn1, gn2 = G.observables()
    assert close(gtr[inst], tr, rtol, atol), (gtr[inst], tr)
    assert close(gn1[inst], n1, rtol, atol), np.max(np.abs(gn1[inst] - n1) / n1)
    assert close(gn2[inst], n2, rtol, atol), np.max(np.abs(gn2[inst] - n2) / n2)
    S, pur, smax = G.operator_entropy()
    assert close(S[inst], P.entropy, rtol, atol), np.max(np.abs(S[inst] - np.array(P.entropy)))
    assert close(pur[inst], P.purities(), rtol, atol)
    chi, lams, chs = G.bonds(inst)
    for b in range(P.M + 1):
        lo = np.sort(P.lam[b])[::-1]
        lg = np.sort(lams[b])[::-1]
        lo = lo[lo > lam_rel * lo[0]]
        lg = lg[lg > lam_rel * lg[0]]
        assert len(lo) == len(lg), (b, len(lo), len(lg))
        assert np.all(np.abs(lo - lg) <= 1e-10 * lo[0]), b


def test_exact_small_mesh_vs_oracle(lib):
    """No truncation, 4 modes, cutoff 4, Haar seed 0, final phases: the exact workload."""
    wl = w.workload("exact_M4_d4")
    mesh = wl.mesh()
    P = oracle_run(wl)
    G = gpu_handle(lib, wl)
    disc = G.sweep_mesh([mesh.n_gates], mesh.k, mesh.theta, mesh.phi, mesh.final_phase)
    assert np.all(np.abs(disc) < 1e-12)
    compare(P, G)
    tr, _, _ = G.observables()
    assert abs(tr[0] - 1.0) < 1e-12


def test_initial_state_vs_oracle(lib):
    for name in ["M16_d6_chi64", "M32_d8_chi256"]:
        wl = w.workload(name)
        P = u1mpo.U1MPO(wl.M, wl.d, wl.r[0], wl.eta[0], chi_max=wl.chi)
        G = gpu_handle(lib, wl)
        compare(P, G, rtol=1e-12, atol=1e-14)
        chi, _, chs = G.bonds()
        assert list(chi) == [len(l) for l in P.lam]
        for b in range(wl.M + 1):
            assert np.array_equal(chs[b], P.charges[b])


@pytest.fixture(scope="module")
def chi64_oracle():
    wl = w.workload("M16_d6_chi64")
    return wl, oracle_run(wl)


def test_chi64_mesh_plan_vs_oracle(lib, chi64_oracle):
    """16 modes, cutoff 6, chi 64, 120 gates + phases, through the CUDA-graph plan
    (the launch configuration the benchmark times)."""
    wl, P = chi64_oracle
    mesh = wl.mesh()
    G = gpu_handle(lib, wl)
    plan = G.plan_mesh([mesh.n_gates], mesh.k, mesh.theta, mesh.phi, mesh.final_phase)
    plan.run()
    disc = plan.discarded()
    assert close(disc, P.discarded)
    assert close(np.sum(disc), np.sum(P.discarded))
    compare(P, G)
    chi, _, _ = G.bonds()
    assert list(chi) == [len(l) for l in P.lam]
    # replay after reset is bitwise reproducible
    S1 = G.operator_entropy()[0].copy()
    o1 = G.observables()
    G.reset(); plan.run()
    assert np.array_equal(plan.discarded(), disc)
    assert np.array_equal(G.operator_entropy()[0], S1)
    o2 = G.observables()
    assert all(np.array_equal(x, y) for x, y in zip(o1, o2))
    plan.close()


def test_plan_stage_times_and_profile(lib, chi64_oracle):
    """The event nodes inside the plan's graph time every stage of the last replay;
    the instrumented replay (eager, flop counters) gives the same results."""
    import torch
    wl, _ = chi64_oracle
    mesh = wl.mesh()
    stream = torch.cuda.Stream()
    G = lib.MPO(wl.M, wl.d, wl.r[0], wl.eta[0], chi_max=wl.chi, stream=stream)
    plan = G.plan_mesh([mesh.n_gates], mesh.k, mesh.theta, mesh.phi, mesh.final_phase)
    with pytest.raises(lib.MPOError):
        plan.stage_times()          # never run yet
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    G.sync()
    e0.record(stream); plan.run(); e1.record(stream)
    st = plan.stage_times()
    total = e0.elapsed_time(e1)
    assert all(v >= 0.0 for v in st.values())
    assert st["svd"] > 0.0 and st["theta"] > 0.0
    assert sum(st.values()) <= total * 1.05 + 0.05
    d_plan = plan.discarded()
    G.reset()
    prof, jac = plan.profile(with_jacobi=True)
    assert np.array_equal(plan.discarded(), d_plan)
    assert prof["svd"][1] == prof["theta"][1] > 0 and prof["svd"][2] > 0
    assert jac["blocks"] > 0 and jac["refine_flops"] > 0
    plan.close()


def test_chi64_sweep_equals_plan(lib, chi64_oracle):
    wl, _ = chi64_oracle
    mesh = wl.mesh()
    G1 = gpu_handle(lib, wl)
    d1 = G1.sweep_mesh([mesh.n_gates], mesh.k, mesh.theta, mesh.phi, mesh.final_phase)
    G2 = gpu_handle(lib, wl)
    plan = G2.plan_mesh([mesh.n_gates], mesh.k, mesh.theta, mesh.phi, mesh.final_phase)
    plan.run()
    assert np.array_equal(d1, plan.discarded())
    assert all(np.array_equal(x, y) for x, y in zip(G1.observables(), G2.observables()))


def test_single_gate_api_vs_oracle(lib):
    wl = w.workload("M16_d6_chi64")
    mesh = wl.mesh()
    P = u1mpo.U1MPO(wl.M, wl.d, wl.r[0], wl.eta[0], chi_max=wl.chi)
    G = gpu_handle(lib, wl)
    for i in range(12):
        e_o = P.apply_gate(int(mesh.k[i]), mesh.theta[i], mesh.phi[i])
        e_g = G.apply_bs(int(mesh.k[i]), mesh.theta[i], mesh.phi[i])
        assert close(e_g, e_o), (i, e_g, e_o)
    compare(P, G)


def test_batched_instances_equal_single(lib):
    """Independent instances in one handle run in the same layer launches; each must
    equal the instance run alone to the FP64 parity bar.  (A block may take the
    cluster path in one run and the single-CTA path in the other, because that choice
    depends on the whole layer's load, so equality is not bitwise.)"""
    wl = w.batched_instances(n=3)
    meshes = [wl.mesh(i) for i in range(3)]
    n = [m.n_gates for m in meshes]
    k = np.concatenate([m.k for m in meshes]); th = np.concatenate([m.theta for m in meshes])
    ph = np.concatenate([m.phi for m in meshes]); fp = np.concatenate([m.final_phase for m in meshes])
    Gb = gpu_handle(lib, wl, insts=(0, 1, 2))
    db = Gb.sweep_mesh(n, k, th, ph, fp)
    trb, n1b, n2b = Gb.observables()
    Sb = Gb.operator_entropy()[0]
    off = 0
    for i in range(3):
        Gi = gpu_handle(lib, wl, insts=(i,))
        di = Gi.sweep_mesh([n[i]], meshes[i].k, meshes[i].theta, meshes[i].phi, meshes[i].final_phase)
        assert close(db[off:off + n[i]], di)
        tr, n1, n2 = Gi.observables()
        assert close(trb[i], tr[0]) and close(n1b[i], n1[0]) and close(n2b[i], n2[0])
        assert close(Sb[i], Gi.operator_entropy()[0][0])
        off += n[i]
    # the batched run itself is bitwise reproducible
    Gb.reset()
    assert np.array_equal(Gb.sweep_mesh(n, k, th, ph, fp), db)


def test_batched_instance_vs_oracle(lib):
    wl = w.batched_instances(n=2)
    meshes = [wl.mesh(i) for i in range(2)]
    G = gpu_handle(lib, wl, insts=(0, 1))
    G.sweep_mesh([m.n_gates for m in meshes], np.concatenate([m.k for m in meshes]),
                 np.concatenate([m.theta for m in meshes]), np.concatenate([m.phi for m in meshes]),
                 np.concatenate([m.final_phase for m in meshes]))
    P = oracle_run(wl, inst=1)
    compare(P, G, inst=1)


@pytest.mark.parametrize("name,ngates", [("M32_d8_chi256", 24), ("M48_d8_chi512", 6)])
def test_large_workload_prefix_vs_oracle(lib, name, ngates):
    """Full-size workloads, sampled: the first gates of the mesh against the oracle."""
    wl = w.workload(name)
    P = oracle_run(wl, ngates=ngates, phases=False)
    mesh = wl.mesh()
    G = gpu_handle(lib, wl)
    disc = G.sweep_mesh([ngates], mesh.k[:ngates], mesh.theta[:ngates], mesh.phi[:ngates])
    assert close(disc, P.discarded)
    compare(P, G)


@pytest.mark.parametrize("name", ["M32_d8_chi256", "M48_d8_chi512"])
def test_large_workload_full_mesh_properties(lib, name):
    """Whole meshes at full size: properties that hold at any size (Tr in (0, 1],
    chi within the cap, non-negative entropies and discarded weights, the ket/bra
    mirror symmetry of every bond spectrum)."""
    wl = w.workload(name)
    mesh = wl.mesh()
    G = gpu_handle(lib, wl)
    plan = G.plan_mesh([mesh.n_gates], mesh.k, mesh.theta, mesh.phi, mesh.final_phase)
    plan.run()
    disc = plan.discarded()
    assert np.all(disc >= 0) and np.all(disc < 1), (disc.min(), disc.max())
    tr, n1, n2 = G.observables()
    assert 0.0 < tr[0] <= 1.0 + 1e-12
    assert np.all(n1 > 0) and np.all(n2 >= n1 - 1e-12)
    S, pur, smax = G.operator_entropy()
    assert np.all(S >= -1e-12) and smax[0] == S[0].max()
    chi, lams, chs = G.bonds()
    assert chi.max() <= wl.chi
    for b in range(wl.M + 1):
        for c in range(wl.d):
            for cb in range(c + 1, wl.d):
                x = np.sort(lams[b][(chs[b][:, 0] == c) & (chs[b][:, 1] == cb)])
                y = np.sort(lams[b][(chs[b][:, 0] == cb) & (chs[b][:, 1] == c)])
                assert np.array_equal(x, y)
    plan.close()


def test_edge_cases(lib):
    # two modes, one gate; vacuum inputs; eta = 0 and eta = 1; theta = 0 and pi/2
    G = lib.MPO(2, 3, [0.7, 0.0], [1.0, 0.5], chi_max=None)
    P = u1mpo.U1MPO(2, 3, [0.7, 0.0], [1.0, 0.5])
    for th, ph in [(0.0, 0.3), (np.pi / 2, 0.0), (0.4, 1.1)]:
        assert close(G.apply_bs(0, th, ph), P.apply_gate(0, th, ph))
    compare(P, G)
    # all loss: the vacuum stays the vacuum
    G0 = lib.MPO(4, 4, [0.8] * 4, [0.0] * 4, chi_max=8)
    mesh = w.clements(w.haar_unitary(4, 3))
    G0.sweep_mesh([mesh.n_gates], mesh.k, mesh.theta, mesh.phi, mesh.final_phase)
    tr, n1, _ = G0.observables()
    assert abs(tr[0] - 1) < 1e-14 and np.all(np.abs(n1) < 1e-14)
    # smallest cutoff, chi = 1, empty mesh
    G1 = lib.MPO(5, 2, [0.5] * 5, [0.5] * 5, chi_max=1)
    P1 = u1mpo.U1MPO(5, 2, [0.5] * 5, [0.5] * 5, chi_max=1)
    m5 = w.clements(w.haar_unitary(5, 9))
    d = G1.sweep_mesh([m5.n_gates], m5.k, m5.theta, m5.phi)
    assert close(d, P1.run_mesh(m5.k, m5.theta, m5.phi))
    compare(P1, G1)
    assert G1.sweep_mesh([0], np.zeros(0), np.zeros(0), np.zeros(0)).size == 0


def test_invalid_arguments_rejected_on_host(lib):
    G = lib.MPO(4, 4, [0.5] * 4, [0.5] * 4, chi_max=16)
    with pytest.raises(lib.MPOError) as ei:
        G.apply_bs(3, 0.1, 0.1)          # k = M - 1 has no partner mode
    assert ei.value.status == 1
    with pytest.raises(lib.MPOError):
        G.sweep_mesh([1], [7], [0.1], [0.2])
    with pytest.raises(lib.MPOError):
        G.apply_bs(0, float("nan"), 0.0)
    G.sync()   # the handle is still usable


# Mixed path (FP32 contraction, Gram, eigensolver and back-multiplication; FP64
# selection, lambda, entropy, state): errors against the FP64 oracle at the same chi.
MIXED_BOUNDS = {"n_rel": 1e-4, "n2_rel": 1e-4, "S_abs": 1e-3, "tr_abs": 1e-4, "eps_rel": 1e-2}


def mixed_errors(P, G):
    tr, n1, n2 = P.observables()
    gtr, gn1, gn2 = G.observables()
    S = G.operator_entropy()[0][0]
    return {"n_rel": float(np.max(np.abs(gn1[0] - n1) / n1)),
            "n2_rel": float(np.max(np.abs(gn2[0] - n2) / n2)),
            "S_abs": float(np.max(np.abs(S - np.array(P.entropy)))),
            "tr_abs": float(abs(gtr[0] - tr))}


@pytest.mark.parametrize("name,ngates", [("M16_d6_chi64", None), ("M32_d8_chi256", 24), ("M48_d8_chi512", 6)])
def test_mixed_precision_vs_oracle(lib, name, ngates):
    wl = w.workload(name)
    mesh = wl.mesh()
    n = mesh.n_gates if ngates is None else ngates
    P = oracle_run(wl, ngates=n, phases=(ngates is None))
    G = gpu_handle(lib, wl, precision="mixed_tf32")
    fp = mesh.final_phase if ngates is None else None
    disc = G.sweep_mesh([n], mesh.k[:n], mesh.theta[:n], mesh.phi[:n], fp)
    err = mixed_errors(P, G)
    err["eps_rel"] = float(abs(np.sum(disc) - np.sum(P.discarded)) / max(np.sum(P.discarded), 1e-300))
    print(name, "mixed errors", err)
    for k, v in MIXED_BOUNDS.items():
        assert err[k] <= v, (k, err[k], v)
