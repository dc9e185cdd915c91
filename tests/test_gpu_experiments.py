"""The App. A run protocols (paper_2301_12814_gb300.experiments) on the GPU against the
oracle replaying the same gates: the per-layer maximum operator entanglement and the
stop of the depth protocol, and the truncation error at every bond dimension the
search visits (the search is a deterministic function of those errors, so equal
errors mean the same search path and the same answer)."""
import numpy as np
import pytest

import gbs_workloads as w
from oracle import u1mpo

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ex():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2301_12814_gb300 import build, experiments, mpo
    mpo.load_library(build.build())
    return experiments


def test_ee_over_depth_vs_oracle(ex):
    wl = w.workload("M16_d6_chi64")
    mesh = wl.mesh()
    layer_of = w.layer_schedule(mesh.k, wl.M)
    res = ex.ee_over_depth(wl.M, wl.d, wl.r[0], wl.eta[0], wl.chi, mesh.k, mesh.theta, mesh.phi, layer_of,
                           patience=3)
    P = u1mpo.U1MPO(wl.M, wl.d, wl.r[0], wl.eta[0], chi_max=wl.chi)
    want = []
    for l in range(res["layers"]):
        for g in np.nonzero(layer_of == l)[0]:
            P.apply_gate(int(mesh.k[g]), mesh.theta[g], mesh.phi[g])
        want.append(max(P.entropy[1:wl.M]))
    got = np.array(res["max_ee"])
    assert np.all(np.abs(got - np.array(want)) <= 1e-10 * np.abs(np.array(want)) + 1e-12)
    # the same stop decision on the oracle's values
    stop = ex.plateau_stop(want, 3)
    assert res["stopped"] == (stop is not None)
    if stop is not None:
        assert res["layers"] == stop + 1
    else:
        assert res["layers"] == int(layer_of.max()) + 1
    tr, _, _ = P.observables()
    assert abs(res["trace"] - tr) <= 1e-10 * tr


def test_bond_dimension_search_vs_oracle(ex):
    wl = w.workload("M16_d6_chi64")
    mesh = wl.mesh()
    res = ex.bond_dimension_search(wl.M, wl.d, wl.r[0], wl.eta[0], mesh.k, mesh.theta, mesh.phi,
                                   mesh.final_phase, chi0=8, target=0.4, refine=2)
    assert res["chi"] is not None and res["error"] <= 0.4
    for chi, e in res["visited"]:
        P = u1mpo.U1MPO(wl.M, wl.d, wl.r[0], wl.eta[0], chi_max=chi)
        P.run_mesh(mesh.k, mesh.theta, mesh.phi, mesh.final_phase)
        tr, _, _ = P.observables()
        assert abs(e - (1.0 - tr)) <= 1e-10 * max(tr, 1e-300) + 1e-12, (chi, e, 1.0 - tr)
    # doubling then bisection: the answer passes, every smaller visited value failed
    assert all(e > 0.4 for c, e in res["visited"] if c < res["chi"])


def test_truncated_probability_vs_oracle(ex):
    """Per-instance truncated probability of a batched handle (kernel-computed kept
    probability) against the oracle's, with different r and eta per instance and an
    explicit photon-number cap below d - 1."""
    from paper_2301_12814_gb300 import mpo
    rng = np.random.default_rng(7)
    M, d, B = 6, 8, 3
    r = rng.uniform(0.4, 1.2, (B, M))
    eta = rng.uniform(0.2, 0.9, (B, M))
    for n_cap in (None, 5):
        G = mpo.MPO(M, d, r, eta, chi_max=16, batch=B, n_cap=n_cap)
        try:
            got = G.truncated_probability()
        finally:
            G.close()
        for i in range(B):
            want = u1mpo.U1MPO(M, d, r[i], eta[i], n_cap=n_cap).truncated_probability
            assert abs(got[i] - want) <= 1e-13, (n_cap, i, got[i], want)


def test_choose_d_vs_oracle(ex):
    """App. A's choice of d: every visited d carries the oracle's tail, the answer is
    the first below 1%, and each smaller d was at or above it."""
    M = 8
    r = [0.9] * 2 + [0.0] * (M - 2)  # N = M / 4 squeezed inputs, as in App. A
    eta = [0.5] * M
    res = ex.choose_d(M, r, eta, threshold=0.01, d_min=4)
    tail_of = lambda d: u1mpo.U1MPO(M, ex.D_IN, r, eta, n_cap=d - 1, chi_max=1).truncated_probability
    want_d = next(d for d in range(4, 17) if tail_of(d) < 0.01)
    assert res["d"] == want_d and res["tail"] < 0.01
    assert res["n_cap"] == want_d - 1 and res["d_in"] == ex.D_IN
    for d, tail in res["visited"]:
        want = tail_of(d)
        assert abs(tail - want) <= 1e-13, (d, tail, want)
    assert all(t >= 0.01 for d, t in res["visited"] if d < res["d"])
    assert res["visited"][-1][0] == res["d"]


def test_truncation_curve_vs_oracle(ex):
    """1 - Tr rho against chi as one batched run (one instance per chi) equals separate
    oracle runs, with the input cut above the cap (the choose_d setting)."""
    M, cap = 8, 5
    r = [0.88] * M
    eta = [0.3] * M
    mesh = w.dialled_mesh(M, 4)
    curve = ex.truncation_curve(M, ex.D_IN, r, eta, mesh.k, mesh.theta, mesh.phi, mesh.final_phase,
                                chis=(4, 8, 16, 32), n_cap=cap)
    errs = [e for _, e in curve]
    assert all(a >= b - 1e-12 for a, b in zip(errs, errs[1:]))  # more chi, less error
    for chi, e in curve:
        P = u1mpo.U1MPO(M, ex.D_IN, r, eta, chi_max=chi, n_cap=cap)
        P.run_mesh(mesh.k, mesh.theta, mesh.phi, mesh.final_phase)
        tr, _, _ = P.observables()
        assert abs(e - (1.0 - tr)) <= 1e-10 * max(tr, 1e-300) + 1e-12, (chi, e, 1.0 - tr)


def test_dialled_mesh_vs_oracle(ex):
    """A direct-dialled Haar mesh (the paper's M-layer array, App. A) through the whole
    GPU path against the oracle on the same gates."""
    from paper_2301_12814_gb300 import mpo
    wl = w.workload("M16_d6_chi64")
    mesh = wl.mesh(dialled=True)
    G = mpo.MPO(wl.M, wl.d, wl.r[0], wl.eta[0], chi_max=wl.chi)
    try:
        disc = G.sweep_mesh([mesh.n_gates], mesh.k, mesh.theta, mesh.phi, mesh.final_phase)
        tr, n1, _ = G.observables()
        S, _, _ = G.operator_entropy()
    finally:
        G.close()
    P = u1mpo.U1MPO(wl.M, wl.d, wl.r[0], wl.eta[0], chi_max=wl.chi)
    P.run_mesh(mesh.k, mesh.theta, mesh.phi, mesh.final_phase)
    ptr, pn1, _ = P.observables()
    assert abs(tr[0] - ptr) <= 1e-10 * ptr
    assert np.allclose(n1[0], pn1, rtol=1e-10, atol=1e-12)
    assert np.allclose(S[0], np.asarray(P.entropy), rtol=1e-10, atol=1e-12)
    assert np.allclose(disc, P.discarded, rtol=1e-10, atol=1e-12)
