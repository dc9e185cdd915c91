"""Seeded random small configurations through the whole GPU path against the oracle
(FP64 bar): modes 3..12, local cutoff 3..8 with a random cap n_cap <= d - 1, bond caps
from 1 to 64 (or none), per-mode squeezing and transmission (vacuum and lossless modes
included), and a direct-dialled mesh.  Catches corner cases of the charge structure
(ragged and empty blocks, single-index bonds, caps below d - 1) that the fixed
workloads do not reach."""
import numpy as np
import pytest

import gbs_workloads as w
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


def _config(seed):
    rng = np.random.default_rng(1000 + seed)
    M = int(rng.integers(3, 13))
    d = int(rng.integers(3, 9))
    n_cap = int(rng.integers(1, d)) if rng.uniform() < 0.4 else None
    chi = int(rng.choice([1, 2, 3, 5, 8, 13, 24, 40, 64]))
    if M * d <= 30 and rng.uniform() < 0.3:
        chi = None  # exact runs only where the exact bond dimension stays small
    r = rng.uniform(0.0, 1.3, M)
    r[rng.uniform(size=M) < 0.2] = 0.0           # some vacuum inputs
    eta = rng.uniform(0.05, 1.0, M)
    eta[rng.uniform(size=M) < 0.15] = 1.0        # some lossless modes
    mesh = w.dialled_mesh(M, 2000 + seed)
    return M, d, n_cap, chi, r, eta, mesh


@pytest.mark.parametrize("seed", range(32))
def test_random_configuration_vs_oracle(lib, seed):
    M, d, n_cap, chi, r, eta, mesh = _config(seed)
    G = lib.MPO(M, d, r, eta, chi_max=chi, n_cap=n_cap)
    disc = G.sweep_mesh([mesh.n_gates], mesh.k, mesh.theta, mesh.phi, mesh.final_phase)
    tr, n1, n2 = G.observables()
    S, pur, _ = G.operator_entropy()
    G.close()
    P = u1mpo.U1MPO(M, d, r, eta, chi_max=chi, n_cap=n_cap)
    P.run_mesh(mesh.k, mesh.theta, mesh.phi, mesh.final_phase)
    ptr, pn1, pn2 = P.observables()
    cfg = dict(M=M, d=d, n_cap=n_cap, chi=chi)
    assert close(tr[0], ptr), (cfg, tr[0], ptr)
    assert close(n1[0], pn1), cfg
    assert close(n2[0], pn2), cfg
    assert close(S[0], np.asarray(P.entropy)), cfg
    assert close(pur[0], P.purities()), cfg
    assert close(disc, P.discarded), cfg
