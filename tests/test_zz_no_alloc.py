"""mpo_observables_static: the allocation-free observables entry point.

It exists for callers that cannot call cudaMalloc when they need the observables
(an application or framework that owns all device memory and forbids direct
allocation, which would also synchronise the device).  It runs the trace-environment
kernel on an MPO held in the caller's device buffers with its scratch in a
file-scope device array.  Here the caller's buffers are torch tensors holding the
oracle's state after ten gates of the 16-mode, chi = 64 mesh; two calls in a row
must agree with mpo_observables on a handle that ran the same ten gates, within the
FP64 tolerance of the parity tests.  This file is collected last on purpose.
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
    return torch, mpo


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


def test_static_observables_match_handle_two_calls(env):
    torch, mpo = env
    lib = mpo.load_library()
    wl = w.workload("M16_d6_chi64")
    mesh = wl.mesh()
    n = 10
    P = u1mpo.U1MPO(wl.M, wl.d, wl.r[0], wl.eta[0], chi_max=wl.chi)
    P.run_mesh(mesh.k[:n], mesh.theta[:n], mesh.phi[:n])
    G = mpo.MPO(wl.M, wl.d, wl.r[0], wl.eta[0], chi_max=wl.chi)
    G.sweep_mesh([n], mesh.k[:n], mesh.theta[:n], mesh.phi[:n])
    tr, n1, n2 = G.observables(normalize=False)
    pur = G.operator_entropy()[1][0]
    want = np.concatenate([[tr[0]], n1[0], n2[0], pur])

    D = 64
    st = _device_state(torch, P, D)
    out = torch.zeros(3 * wl.M + 2, dtype=torch.float64, device="cuda:0")
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        out.fill_(float("nan"))
        status = lib.mpo_observables_static(
            wl.M, wl.d - 1, D, ctypes.c_void_p(st["chi"].data_ptr()), ctypes.c_void_p(st["charge"].data_ptr()),
            ctypes.c_void_p(st["segoff"].data_ptr()), ctypes.c_void_p(st["lam"].data_ptr()),
            ctypes.c_void_p(st["gam"].data_ptr()), ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))
        assert status == 0, lib.mpo_status_string(status)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got)), call
        assert _close(got, want), (call, np.max(np.abs(got - want) / np.abs(want)))


def test_static_observables_rejects_oversize(env):
    torch, mpo = env
    lib = mpo.load_library()
    dummy = ctypes.c_void_p(16)   # never dereferenced: the size check comes first
    # 2 (M + 1) D complex values exceed the 65536-element scratch array
    assert lib.mpo_observables_static(48, 7, 1024, dummy, dummy, dummy, dummy, dummy, dummy, None) == 6
    assert lib.mpo_observables_static(1, 7, 64, dummy, dummy, dummy, dummy, dummy, dummy, None) == 1
