"""Caller-provided device allocator (mpo_set_allocator): a handle whose memory comes
from PyTorch's caching allocator computes bitwise the same mesh as one on cudaMalloc;
its memory appears in and returns to torch's accounting; plans and checkpoints work on
it; handles created before the switch keep freeing through the CUDA runtime."""
import numpy as np
import pytest

import gbs_workloads as w

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


def _run(lib, wl, mesh, plan=False):
    G = lib.MPO(wl.M, wl.d, wl.r[0], wl.eta[0], chi_max=wl.chi)
    if plan:
        P = G.plan_mesh([mesh.n_gates], mesh.k, mesh.theta, mesh.phi, mesh.final_phase)
        P.run()
        disc = P.discarded()
    else:
        disc = G.sweep_mesh([mesh.n_gates], mesh.k, mesh.theta, mesh.phi, mesh.final_phase)
    tr, n1, _ = G.observables()
    S, _, _ = G.operator_entropy()
    return G, (disc, tr, n1, S)


def test_torch_allocator_same_results(lib):
    import torch
    wl = w.workload("M16_d6_chi64")
    mesh = wl.mesh()
    A, ref = _run(lib, wl, mesh)            # cudaMalloc
    base = torch.cuda.memory_allocated()
    lib.use_torch_allocator()
    try:
        B, got = _run(lib, wl, mesh)
        held = torch.cuda.memory_allocated() - base
        assert held > 0                      # the handle's buffers came from torch
        for x, y in zip(ref, got):
            assert np.array_equal(x, y)
        C, got_plan = _run(lib, wl, mesh, plan=True)
        for x, y in zip(ref, got_plan):
            assert np.array_equal(x, y)
        ck = B.save(cursor=3)
        assert C.load(ck) == 3
        B.close(); C.close()
        assert torch.cuda.memory_allocated() == base  # everything went back to torch
    finally:
        lib.set_allocator(None, None)
    A.close()                                # created before the switch: frees with cudaFree
    D, again = _run(lib, wl, mesh)
    for x, y in zip(ref, again):
        assert np.array_equal(x, y)
    D.close()
