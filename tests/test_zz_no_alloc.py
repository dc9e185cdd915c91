"""mpo_observables_static: the allocation-free observables entry point.

It exists for callers that cannot call cudaMalloc when they need the observables
(an application or framework that owns all device memory and forbids direct
allocation, which would also synchronise the device).  It runs the trace-environment
kernel on an MPO held in the caller's device buffers with its scratch in a
file-scope device array.

Here the caller's buffers are torch tensors holding the oracle's state after ten
gates of the 16-mode, chi = 64 mesh.  Two calls in a row must give the oracle's own
Tr rho, <n_j> Tr rho, <n_j^2> Tr rho and bond purities within the FP64 tolerance of
the parity tests, agree with mpo_observables on a handle that ran the same ten gates,
and allocate nothing: the device's free memory and torch's allocation count are
unchanged across the calls, and a counting allocator installed through
mpo_set_allocator is never called.

The file is named to be collected last, so that a run stopping at the first failure
has already run every other test if this one fails.
"""
import ctypes

import numpy as np
import pytest

import gbs_workloads as w
from oracle import u1mpo

pytestmark = pytest.mark.gpu

RTOL, ATOL = 1e-10, 1e-12


def _close(a, b):
    a, b = np.asarray(a, dtype=float), np.asarray(b, dtype=float)
    return np.all(np.abs(a - b) <= ATOL + RTOL * np.abs(b))


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2301_12814_gb300 import build, mpo
    mpo.load_library(build.build())
    yield torch, mpo
    mpo.set_allocator(None, None)


def _device_state(torch, P, D):
    """The oracle MPO in the handle's device layout (one instance, capacity D)."""
    M, q = P.M, P.n_cap + 1
    Pn = q * q
    chi = np.array([len(l) for l in P.lam], dtype=np.int32)
    charge = np.zeros((M + 1, D), dtype=np.int32)
    segoff = np.zeros((M + 1, Pn + 1), dtype=np.int32)
    lam = np.zeros((M + 1, D), dtype=np.float64)
    gam = np.zeros((M, D, D), dtype=np.complex128)
    for b in range(M + 1):
        p = P.charges[b][:, 0] * q + P.charges[b][:, 1]
        charge[b, :chi[b]] = p
        lam[b, :chi[b]] = P.lam[b]
        segoff[b] = np.searchsorted(p, np.arange(Pn + 1), side="left")
    for j in range(M):
        gam[j, :chi[j], :chi[j + 1]] = P.gam[j]
    dev = torch.device("cuda", 0)
    return {k: torch.from_numpy(v).to(dev) for k, v in
            dict(chi=chi, charge=charge, segoff=segoff, lam=lam, gam=gam).items()}


def test_static_observables_match_oracle_two_calls_no_allocation(env):
    torch, mpo = env
    lib = mpo.load_library()
    wl = w.workload("M16_d6_chi64")
    mesh = wl.mesh()
    n = 10
    P = u1mpo.U1MPO(wl.M, wl.d, wl.r[0], wl.eta[0], chi_max=wl.chi)
    P.run_mesh(mesh.k[:n], mesh.theta[:n], mesh.phi[:n])
    otr, on1, on2 = P.observables()
    oracle = np.concatenate([[otr], on1 * otr, on2 * otr, P.purities()])

    G = mpo.MPO(wl.M, wl.d, wl.r[0], wl.eta[0], chi_max=wl.chi)
    G.sweep_mesh([n], mesh.k[:n], mesh.theta[:n], mesh.phi[:n])
    tr, n1, n2 = G.observables(normalize=False)
    pur = G.operator_entropy()[1][0]
    handle = np.concatenate([[tr[0]], n1[0], n2[0], pur])
    G.close()

    D = 64
    st = _device_state(torch, P, D)
    out = torch.zeros(3 * wl.M + 2, dtype=torch.float64, device="cuda:0")
    stream = torch.cuda.current_stream().cuda_stream
    calls = {"alloc": 0, "free": 0}

    def count_alloc(nbytes, s):
        calls["alloc"] += 1
        return 0

    def count_free(ptr, s):
        calls["free"] += 1

    mpo.set_allocator(count_alloc, count_free)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    n_alloc0 = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
    got = []
    try:
        for call in range(2):
            out.fill_(float("nan"))
            status = lib.mpo_observables_static(
                wl.M, wl.d - 1, D, ctypes.c_void_p(st["chi"].data_ptr()), ctypes.c_void_p(st["charge"].data_ptr()),
                ctypes.c_void_p(st["segoff"].data_ptr()), ctypes.c_void_p(st["lam"].data_ptr()),
                ctypes.c_void_p(st["gam"].data_ptr()), ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))
            assert status == 0, lib.mpo_status_string(status)
            torch.cuda.synchronize()
            got.append(out.cpu().numpy())
        free1, _ = torch.cuda.mem_get_info()
        n_alloc1 = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
    finally:
        mpo.set_allocator(None, None)
    assert calls == {"alloc": 0, "free": 0}
    assert free1 == free0
    assert n_alloc1 == n_alloc0
    for call, g in enumerate(got):
        assert np.all(np.isfinite(g)), call
        assert _close(g, oracle), (call, np.max(np.abs(g - oracle) / np.abs(oracle)))
        assert _close(g, handle), (call, np.max(np.abs(g - handle) / np.abs(handle)))


def test_static_observables_rejects_oversize(env):
    torch, mpo = env
    lib = mpo.load_library()
    dummy = ctypes.c_void_p(16)   # never dereferenced: the size check comes first
    # 2 (M + 1) D complex values exceed the 65536-element scratch array
    assert lib.mpo_observables_static(48, 7, 1024, dummy, dummy, dummy, dummy, dummy, dummy, None) == 6
    assert lib.mpo_observables_static(1, 7, 64, dummy, dummy, dummy, dummy, dummy, dummy, None) == 1
