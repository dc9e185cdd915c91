"""Allocation failures injected on the host through the allocator hook
(mpo_set_allocator): for every device allocation of a full scenario -- handle
creation, an eager mesh, a planned mesh and its replay, observables -- the k-th
allocation is made to fail.  Each call that hits it must return MPO_ERR_OOM, the
handle must close cleanly, every byte taken from the allocator must be given back
(torch's accounting returns to its base), and a fresh handle must still match the
oracle afterwards.  No GPU fault is involved: the failure is a NULL from the host-side
allocator."""
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
    yield mpo
    mpo.set_allocator(None, None)


def _scenario(lib, wl, mesh):
    G = lib.MPO(wl.M, wl.d, wl.r[0], wl.eta[0], chi_max=wl.chi)
    try:
        G.sweep_mesh([mesh.n_gates], mesh.k, mesh.theta, mesh.phi, mesh.final_phase)
        P = G.plan_mesh([mesh.n_gates], mesh.k, mesh.theta, mesh.phi, mesh.final_phase)
        G.reset()
        P.run()
        P.discarded()
        G.observables()
    finally:
        G.close()


def test_every_allocation_failure_is_clean(lib):
    import torch
    dev = torch.cuda.current_device()
    wl = w.workload("M16_d6_chi64")
    mesh = wl.mesh()
    state = {"n": 0, "fail_at": -1}

    def alloc(n, st):
        state["n"] += 1
        if state["n"] == state["fail_at"]:
            return 0
        return torch.cuda.caching_allocator_alloc(n, device=dev, stream=st)

    def free(p, st):
        torch.cuda.caching_allocator_delete(p)

    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    lib.set_allocator(alloc, free)
    try:
        _scenario(lib, wl, mesh)          # count the allocations of a clean run
        total = state["n"]
        assert total >= 10
        assert torch.cuda.memory_allocated() == base
        for k in range(1, total + 1):
            state["n"], state["fail_at"] = 0, k
            with pytest.raises(lib.MPOError) as ei:
                _scenario(lib, wl, mesh)
            assert ei.value.status == 2, (k, ei.value.status)
            torch.cuda.synchronize()
            assert torch.cuda.memory_allocated() == base, k
    finally:
        lib.set_allocator(None, None)
    # the library is unharmed: a fresh handle still matches the oracle
    G = lib.MPO(wl.M, wl.d, wl.r[0], wl.eta[0], chi_max=wl.chi)
    disc = G.sweep_mesh([mesh.n_gates], mesh.k, mesh.theta, mesh.phi, mesh.final_phase)
    tr, _, _ = G.observables()
    G.close()
    P = u1mpo.U1MPO(wl.M, wl.d, wl.r[0], wl.eta[0], chi_max=wl.chi)
    P.run_mesh(mesh.k, mesh.theta, mesh.phi, mesh.final_phase)
    assert abs(tr[0] - P.observables()[0]) <= 1e-10 * tr[0]
    assert np.allclose(disc, P.discarded, rtol=1e-10, atol=1e-12)
