"""Checkpoints (mpo_checkpoint_bytes / mpo_save / mpo_load) on the GPU: a run that is
saved halfway, loaded into a fresh handle and finished gives bitwise the same state,
observables and per-gate discarded weights as the uninterrupted run; the oracle agrees
with the resumed run; corrupted, truncated or mismatched checkpoints are refused and
leave the state unchanged."""
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


def _state(G):
    tr, n1, n2 = G.observables(normalize=False)
    S, _, _ = G.operator_entropy()
    bonds = [G.bonds(i) for i in range(G.batch)]
    return tr, n1, n2, S, bonds


def _same(a, b):
    for x, y in zip(a[:4], b[:4]):
        assert np.array_equal(x, y)
    for (c1, l1, q1), (c2, l2, q2) in zip(a[4], b[4]):
        assert np.array_equal(c1, c2)
        for u, v in zip(l1, l2):
            assert np.array_equal(u, v)
        for u, v in zip(q1, q2):
            assert np.array_equal(u, v)


@pytest.mark.parametrize("precision", ["fp64", "mixed_tf32"])
def test_resume_is_bitwise_identical(lib, precision):
    wl = w.workload("M16_d6_chi64")
    mesh = wl.mesh()
    half = mesh.n_gates // 2
    k, th, ph = mesh.k, mesh.theta, mesh.phi
    A = lib.MPO(wl.M, wl.d, wl.r[0], wl.eta[0], chi_max=wl.chi, precision=precision)
    dA1 = A.sweep_mesh([half], k[:half], th[:half], ph[:half])
    ck = A.save(cursor=half)
    dA2 = A.sweep_mesh([mesh.n_gates - half], k[half:], th[half:], ph[half:], mesh.final_phase)
    full = _state(A)
    B = lib.MPO(wl.M, wl.d, wl.r[0], wl.eta[0], chi_max=wl.chi, precision=precision)
    assert B.load(ck) == half
    dB2 = B.sweep_mesh([mesh.n_gates - half], k[half:], th[half:], ph[half:], mesh.final_phase)
    assert np.array_equal(dA2, dB2)
    _same(full, _state(B))
    if precision == "fp64":
        P = u1mpo.U1MPO(wl.M, wl.d, wl.r[0], wl.eta[0], chi_max=wl.chi)
        P.run_mesh(k, th, ph, mesh.final_phase)
        tr, _, _ = P.observables()
        assert abs(full[0][0] - tr) <= 1e-10 * tr
        assert np.allclose(np.concatenate([dA1, dB2]), P.discarded, rtol=1e-10, atol=1e-12)
    # reset still returns to the initial state, not to the loaded one
    B.reset()
    C = lib.MPO(wl.M, wl.d, wl.r[0], wl.eta[0], chi_max=wl.chi, precision=precision)
    _same(_state(B), _state(C))
    for G in (A, B, C):
        G.close()


def test_batched_checkpoint(lib):
    wl = w.batched_instances(n=4)
    meshes = [wl.mesh(i) for i in range(wl.batch)]
    n_g = [m.n_gates for m in meshes]
    cat = lambda f: np.concatenate([f(m) for m in meshes])
    A = lib.MPO(wl.M, wl.d, wl.r, wl.eta, chi_max=wl.chis, batch=wl.batch)
    A.sweep_mesh(n_g, cat(lambda m: m.k), cat(lambda m: m.theta), cat(lambda m: m.phi))
    ck = A.save(cursor=7)
    B = lib.MPO(wl.M, wl.d, wl.r, wl.eta, chi_max=wl.chis, batch=wl.batch)
    assert B.load(ck) == 7
    _same(_state(A), _state(B))
    assert np.array_equal(A.truncated_probability(), B.truncated_probability())
    A.close(); B.close()


def test_bad_checkpoints_are_refused(lib):
    wl = w.workload("M16_d6_chi64")
    mesh = wl.mesh()
    A = lib.MPO(wl.M, wl.d, wl.r[0], wl.eta[0], chi_max=wl.chi)
    A.sweep_mesh([10], mesh.k[:10], mesh.theta[:10], mesh.phi[:10])
    ck = A.save()
    before = _state(A)
    bad = ck.copy(); bad[200] ^= 0xFF          # payload byte: checksum mismatch
    bad2 = ck.copy(); bad2[0] ^= 0x01           # magic
    for b in (bad, bad2, ck[:100], ck[:-1]):
        with pytest.raises(lib.MPOError) as ei:
            A.load(b)
        assert ei.value.status == 1
    _same(before, _state(A))
    # another shape (other chi cap -> other bond capacity D) is refused
    B = lib.MPO(wl.M, wl.d, wl.r[0], wl.eta[0], chi_max=2 * wl.chi)
    with pytest.raises(lib.MPOError):
        B.load(ck)
    # other precision is refused
    C = lib.MPO(wl.M, wl.d, wl.r[0], wl.eta[0], chi_max=wl.chi, precision="mixed_tf32")
    with pytest.raises(lib.MPOError):
        C.load(ck)
    for G in (A, B, C):
        G.close()
