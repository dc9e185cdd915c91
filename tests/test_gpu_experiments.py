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
