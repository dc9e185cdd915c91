"""The per-layer workspace pools (Theta, W, Gram-sized arrays shared by a layer's
gates, laid out by k_setup from the actual block sizes): a budget too small for a
layer fails that call with MPO_ERR_CAPACITY and poisons the handle, with no device
fault; a handle built afterwards with the normal budget runs the same mesh to the
oracle's numbers."""

import numpy as np
import pytest

import gbs_workloads as w
from oracle import u1mpo

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2301_12814_gb300 import build, mpo
    mpo.load_library(build.build())
    return mpo


def test_pool_overflow_is_reported(lib, monkeypatch):
    wl = w.workload("M16_d6_chi64")
    mesh = wl.mesh()
    monkeypatch.setenv("GBS_MPO_WORKSPACE_GB", "1e-7")  # ~107 bytes: far below one layer
    G = lib.MPO(wl.M, wl.d, wl.r[0], wl.eta[0], chi_max=wl.chi)
    with pytest.raises(lib.MPOError) as ei:
        G.sweep_mesh([mesh.n_gates], mesh.k, mesh.theta, mesh.phi)
    assert ei.value.status == 6
    with pytest.raises(lib.MPOError) as ei:
        G.observables()
    assert ei.value.status == 8  # poisoned
    G.close()
    monkeypatch.delenv("GBS_MPO_WORKSPACE_GB")
    H = lib.MPO(wl.M, wl.d, wl.r[0], wl.eta[0], chi_max=wl.chi)
    disc = H.sweep_mesh([mesh.n_gates], mesh.k, mesh.theta, mesh.phi, mesh.final_phase)
    tr, _, _ = H.observables()
    H.close()
    P = u1mpo.U1MPO(wl.M, wl.d, wl.r[0], wl.eta[0], chi_max=wl.chi)
    P.run_mesh(mesh.k, mesh.theta, mesh.phi, mesh.final_phase)
    ptr, _, _ = P.observables()
    assert abs(tr[0] - ptr) <= 1e-10 * ptr
    assert np.allclose(disc, P.discarded, rtol=1e-10, atol=1e-12)
