"""The ABI's size limits on the GPU against the oracle: the most modes (M = 256), the
largest charge cap (n_cap = 15, 256 charge pairs per bond), the largest bond capacity
(D = 4096) and one past it (refused on the host).  FP64 bar as in the parity tests."""
import numpy as np
import pytest

from oracle import u1mpo

pytestmark = pytest.mark.gpu

RTOL, ATOL = 1e-10, 1e-12


def close(a, b):
    a, b = np.asarray(a, dtype=float), np.asarray(b, dtype=float)
    return np.all(np.abs(a - b) <= ATOL + RTOL * np.abs(b))


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2301_12814_gb300 import build, mpo
    mpo.load_library(build.build())
    return mpo


def brickwork(M, layers, seed):
    """Gates on (0,1), (2,3), ... then (1,2), (3,4), ...; seeded angles and phases."""
    rng = np.random.default_rng(seed)
    k = np.concatenate([np.arange(l % 2, M - 1, 2) for l in range(layers)]).astype(np.int32)
    return k, rng.uniform(0, np.pi / 2, k.size), rng.uniform(0, 2 * np.pi, k.size)


def run_both(lib, M, d, r, eta, chi, k, th, ph, n_cap=None):
    G = lib.MPO(M, d, r, eta, chi_max=chi, n_cap=n_cap)
    disc = G.sweep_mesh([k.size], k, th, ph)
    tr, n1, n2 = G.observables()
    S, _, _ = G.operator_entropy()
    G.close()
    P = u1mpo.U1MPO(M, d, r, eta, chi_max=chi, n_cap=n_cap)
    P.run_mesh(k, th, ph)
    ptr, pn1, pn2 = P.observables()
    assert close(tr[0], ptr)
    assert close(n1[0], pn1) and close(n2[0], pn2)
    assert close(S[0], np.asarray(P.entropy))
    assert close(disc, P.discarded)
    return disc


def test_most_modes(lib):
    M = 256
    rng = np.random.default_rng(5)
    r = rng.uniform(0.2, 0.8, M)
    eta = rng.uniform(0.3, 0.9, M)
    k, th, ph = brickwork(M, 2, 11)
    run_both(lib, M, 3, r, eta, 8, k, th, ph)


def test_largest_charge_cap(lib):
    M, d = 4, 16                      # n_cap = d - 1 = 15: 256 charge pairs per bond
    k, th, ph = brickwork(M, 4, 12)
    disc = run_both(lib, M, d, [1.2, 0.9, 1.1, 0.7], [0.9, 0.8, 0.95, 0.85], 48, k, th, ph)
    assert np.max(disc) > 0            # the cap of chi = 48 truncates


def test_largest_bond_capacity(lib):
    M = 4
    k, th, ph = brickwork(M, 4, 13)
    G = lib.MPO(M, 4, [0.6] * M, [0.5] * M, chi_max=4096)
    assert G.D == 4096
    G.close()
    run_both(lib, M, 4, [0.6] * M, [0.5] * M, 4096, k, th, ph)
    with pytest.raises(lib.MPOError) as ei:
        lib.MPO(M, 4, [0.6] * M, [0.5] * M, chi_max=4097)
    assert ei.value.status == 1
