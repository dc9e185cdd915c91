"""Pins for the dense oracle O1 and the U(1) MPO oracle O2.

O1 is pinned by closed forms (Gaussian first and second moments of lossy squeezed
light through a passive interferometer; exact first moments of the cap-projected
state by brute-force enumeration) and by unitarity.  O2 is pinned against O1 by
brute force (dense density matrix, Schmidt spectra of the charge-split vec(rho))
and by invariants that the paper's method fixes: trace, Hermiticity, positivity,
U(1) conservation, the bond-0 register weights, and the ket/bra mirror symmetry.
"""
import itertools
import math

import numpy as np
import pytest

import gbs_workloads as w
from oracle import dense, fock, u1mpo


def _mesh(M, seed):
    U = w.haar_unitary(M, seed)
    return U, w.clements(U)


def _run_dense(D, mesh):
    for kk, th, ph in zip(mesh.k, mesh.theta, mesh.phi):
        D.apply_gate(int(kk), w.gate_block(float(th), float(ph)))
    D.apply_phases(mesh.final_phase)


def _cap_mean_brute(M, d, n_cap, r, eta):
    """<n_j> of P_cap (x) rho_j P_cap / Tr by enumerating every configuration."""
    diags = [np.diag(fock.lossy_mode_state(r[j], eta[j], d)[0]).real for j in range(M)]
    tot = 0.0; acc = np.zeros(M)
    for conf in itertools.product(range(d), repeat=M):
        if sum(conf) > n_cap:
            continue
        p = np.prod([diags[j][conf[j]] for j in range(M)])
        tot += p
        acc += p * np.array(conf)
    return acc / tot


# ---------------------------------------------------------------- O1 pins
def test_dense_gate_unitary_on_cap_space():
    D = dense.DenseState(4, 4, [0.5] * 4, [0.5] * 4)
    S = w.gate_block(0.7, 1.1)
    G = D.gate_matrix(1, S)
    keep = np.nonzero(D.occ.sum(axis=1) <= D.n_cap)[0]
    Gs = G[np.ix_(keep, keep)]
    assert np.abs(Gs.conj().T @ Gs - np.eye(len(keep))).max() < 1e-12
    # the cap space is invariant: no amplitude leaves it
    out = np.setdiff1d(np.arange(G.shape[0]), keep)
    assert np.abs(G[np.ix_(out, keep)]).max() == 0.0


def test_dense_gaussian_moments():
    """<n_i> = sum_j |U_ij|^2 eta sinh^2 r and <n_i^2> = n_i + 2 n_i^2 + |m_i|^2,
    m_i = sum_j U_ij^2 eta (-sinh r cosh r), for Gaussian light; the cutoff tail here
    is ~1e-9, so both hold to ~1e-6 relative."""
    M, d, r, eta = 3, 12, 0.15, 0.6
    U, mesh = _mesh(M, 5)
    D = dense.DenseState(M, d, [r] * M, [eta] * M)
    _run_dense(D, mesh)
    tr, n1, n2 = D.moments()
    nG = (np.abs(U) ** 2) @ np.full(M, eta * math.sinh(r) ** 2)
    mG = (U ** 2) @ np.full(M, -eta * math.sinh(r) * math.cosh(r))
    n2G = nG + 2 * nG ** 2 + np.abs(mG) ** 2
    assert abs(tr - 1) < 1e-12
    assert np.max(np.abs(n1 - nG) / nG) < 1e-6
    assert np.max(np.abs(n2 - n2G) / n2G) < 1e-5


def test_dense_first_moments_exact_with_cap():
    """With the cap active, <a_j^dag a_k> = 0 (j != k) in the projected product state,
    so <n_out> = |U|^2 <n_in>_cap exactly; <n_in>_cap by brute-force enumeration."""
    M, d, r, eta = 4, 4, 0.9, 0.7
    U, mesh = _mesh(M, 11)
    D = dense.DenseState(M, d, [r] * M, [eta] * M)
    _run_dense(D, mesh)
    _, n1, _ = D.moments()
    want = (np.abs(U) ** 2) @ _cap_mean_brute(M, d, d - 1, [r] * M, [eta] * M)
    assert np.abs(n1 - want).max() < 1e-13


# ---------------------------------------------------------------- O2 vs O1
@pytest.mark.parametrize("M,d,n_cap,r,eta", [(4, 4, None, 0.5, 0.5), (3, 5, 3, 0.8, 0.6),
                                            (5, 3, None, 1.0, 0.4)])
def test_init_mpo_rebuilds_dense(M, d, n_cap, r, eta):
    D = dense.DenseState(M, d, [r] * M, [eta] * M, n_cap=n_cap)
    P = u1mpo.U1MPO(M, d, [r] * M, [eta] * M, n_cap=n_cap)
    assert np.abs(P.to_dense() - D.rho).max() < 1e-14
    pur = float(np.sum(np.abs(D.rho) ** 2))
    assert np.abs(P.purities() - pur).max() < 1e-14
    for b in range(M + 1):
        s = D.u1_schmidt(b)
        s = s[s > 1e-14 * s[0]]
        assert np.abs(np.sort(s) - np.sort(P.lam[b])).max() < 1e-14


def test_init_mpo_canonical():
    """Left and right orthonormality of the initial Vidal form (sums over the implied
    physical indices: entries with different (i, ibar) never mix)."""
    M, d = 5, 4
    P = u1mpo.U1MPO(M, d, [0.7, 0.9, 0.4, 1.1, 0.6], [0.5, 0.3, 0.8, 0.45, 0.6])
    for j in range(M):
        G = P.gam[j]
        A, B = P.charges[j], P.charges[j + 1]
        iA = A[:, 0][:, None] - B[:, 0][None, :]
        ibA = A[:, 1][:, None] - B[:, 1][None, :]
        for i in range(d):
            for ib in range(d):
                sel = (iA == i) & (ibA == ib)
                Gi = G * sel
                left = (Gi * P.lam[j][:, None]).conj().T @ (Gi * P.lam[j][:, None])
                right = (Gi * P.lam[j + 1][None, :]) @ (Gi * P.lam[j + 1][None, :]).conj().T
                if i == 0 and ib == 0:
                    accl, accr = left, right
                else:
                    accl = accl + left; accr = accr + right
        assert np.abs(accl - np.eye(B.shape[0])).max() < 1e-13
        assert np.abs(accr - np.eye(A.shape[0])).max() < 1e-13


@pytest.mark.parametrize("M,d,seed", [(4, 4, 0), (5, 3, 7), (3, 6, 2)])
def test_mesh_exact_matches_dense(M, d, seed):
    """No truncation: O2 after the whole mesh equals the brute-force rho (entries,
    moments, U(1)-form entanglement at every cut)."""
    r = [0.5 + 0.1 * j for j in range(M)]
    eta = [0.5 + 0.05 * j for j in range(M)]
    _, mesh = _mesh(M, seed)
    D = dense.DenseState(M, d, r, eta)
    P = u1mpo.U1MPO(M, d, r, eta)
    lam0 = P.lam[0].copy()
    _run_dense(D, mesh)
    P.run_mesh(mesh.k, mesh.theta, mesh.phi, mesh.final_phase)
    rho = P.to_dense()
    assert np.abs(rho - D.rho).max() < 1e-13
    assert abs(np.trace(rho).real - 1.0) < 1e-13
    assert np.abs(rho - rho.conj().T).max() < 1e-13
    assert np.linalg.eigvalsh(0.5 * (rho + rho.conj().T)).min() > -1e-13
    trD, n1D, n2D = D.moments()
    trP, n1P, n2P = P.observables()
    assert abs(trP - trD) < 1e-13
    assert np.abs(n1P - n1D).max() < 1e-13 and np.abs(n2P - n2D).max() < 1e-13
    for b in range(M + 1):
        assert abs(P.entropy[b] - D.u1_entropy(b)) < 1e-11
    # the bond-0 register weights never change (no gate touches bond 0)
    assert np.array_equal(P.lam[0], lam0)
    # U(1): the total-photon distribution is invariant
    tot = D.occ.sum(axis=1)
    D0 = dense.DenseState(M, d, r, eta)
    for n in range(d):
        sel = tot == n
        assert abs(np.diag(D.rho).real[sel].sum() - np.diag(D0.rho).real[sel].sum()) < 1e-13


@pytest.mark.parametrize("seed", range(10))
def test_random_exact_configurations_match_dense(seed):
    """Seeded random exact cases: 2-4 modes, cutoffs up to 5 (d^M <= 256), a random cap
    n_cap <= d - 1, per-mode r and eta (vacuum and lossless modes included), random
    nearest-neighbour gates.  O2 must equal O1 entry by entry, and in its moments and
    U(1)-form entanglement at every cut."""
    rng = np.random.default_rng(300 + seed)
    M = int(rng.integers(2, 5))
    d = int(rng.integers(2, 6))
    while d ** M > 256:
        d -= 1
    n_cap = int(rng.integers(1, d)) if rng.uniform() < 0.5 else None
    r = rng.uniform(0.0, 1.3, M)
    r[rng.uniform(size=M) < 0.2] = 0.0
    eta = rng.uniform(0.0, 1.0, M)
    eta[rng.uniform(size=M) < 0.2] = 1.0
    ng = int(rng.integers(1, 3 * M))
    k = rng.integers(0, M - 1, ng)
    th = rng.uniform(0, np.pi / 2, ng)
    ph = rng.uniform(0, 2 * np.pi, ng)
    D = dense.DenseState(M, d, r, eta, n_cap=n_cap)
    P = u1mpo.U1MPO(M, d, r, eta, n_cap=n_cap)
    for kk, t, p in zip(k, th, ph):
        D.apply_gate(int(kk), w.gate_block(float(t), float(p)))
    P.run_mesh(k, th, ph)
    assert np.abs(P.to_dense() - D.rho).max() < 1e-13
    trD, n1D, n2D = D.moments()
    trP, n1P, n2P = P.observables()
    assert abs(trP - trD) < 1e-13
    assert np.abs(n1P - n1D).max() < 1e-13 and np.abs(n2P - n2D).max() < 1e-13
    for b in range(M + 1):
        assert abs(P.entropy[b] - D.u1_entropy(b)) < 1e-11


def test_first_moments_exact_larger_mesh():
    """M = 8 with the cap active and no truncation: O2's <n> equals |U|^2 <n_in>_cap;
    this also fixes the U versus U^T convention of the gate list."""
    M, d = 8, 3
    r = [0.9, 0.3, 0.0, 1.2, 0.6, 0.8, 0.5, 1.0]
    eta = [0.6, 0.9, 0.5, 0.3, 0.7, 0.5, 0.4, 0.8]
    U, mesh = _mesh(M, 21)
    P = u1mpo.U1MPO(M, d, r, eta)
    P.run_mesh(mesh.k, mesh.theta, mesh.phi, mesh.final_phase)
    tr, n1, _ = P.observables()
    want = (np.abs(U) ** 2) @ _cap_mean_brute(M, d, d - 1, r, eta)
    assert abs(tr - 1.0) < 1e-12
    assert np.abs(n1 - want).max() < 1e-12


# ---------------------------------------------------------------- truncation
def test_select_rule_drops_split_degenerate_pair():
    c = [(5.0, 0, 0, None), (3.0, 1, 0, None), (3.0, 2, 0, None), (2.0, 3, 0, None),
         (1e-20, 4, 0, None)]
    kept, eps = u1mpo.select_kept(c, 2)
    assert [t[1] for t in kept] == [0]           # the 3.0 pair straddles the cut: both go
    assert abs(eps - (9 + 9 + 4 + 1e-40) / (25 + 9 + 9 + 4 + 1e-40)) < 1e-15
    kept, _ = u1mpo.select_kept(c, 3)
    assert [t[1] for t in kept] == [0, 1, 2]
    kept, _ = u1mpo.select_kept(c, 10)
    assert [t[1] for t in kept] == [0, 1, 2, 3]  # 1e-20 < 1e-14 * s_max is dropped
    kept, _ = u1mpo.select_kept([(1.0, 0, 0, None), (1.0, 1, 0, None)], 1)
    assert len(kept) == 1                        # everything degenerate: plain cut


def test_truncated_prefix_invariants():
    """chi-truncated updates keep Tr <= 1, the mirror symmetry of the spectra
    (Hermiticity: the lambda multiset of charge (c, cb) equals that of (cb, c)),
    chi <= chi_max and non-negative discarded weights."""
    wl = w.workload("M16_d6_chi64")
    mesh = wl.mesh()
    P = u1mpo.U1MPO(wl.M, wl.d, wl.r[0], wl.eta[0], chi_max=24)
    P.run_mesh(mesh.k[:40], mesh.theta[:40], mesh.phi[:40])
    tr, n1, n2 = P.observables()
    assert tr <= 1.0 + 1e-12 and tr > 0.5
    assert min(P.discarded) >= 0.0 and sum(P.discarded) > 0.0
    for b in range(wl.M + 1):
        assert len(P.lam[b]) <= max(24, 18)
        ch = P.charges[b]
        for c in range(wl.d):
            for cb in range(c + 1, wl.d):
                x = np.sort(P.lam[b][(ch[:, 0] == c) & (ch[:, 1] == cb)])
                y = np.sort(P.lam[b][(ch[:, 0] == cb) & (ch[:, 1] == c)])
                assert len(x) == len(y) and (len(x) == 0 or np.abs(x - y).max() < 1e-12 * x.max())


# ------------------------------------------------- planted mistakes (CPU only)
@pytest.mark.parametrize("mistake", ["transposed_S", "unconjugated_bra"])
def test_pins_catch_planted_mistakes(monkeypatch, mistake):
    """A transposed mode matrix or a missing conjugate on the bra side must break
    the O1/O2 agreement that the pins above rely on."""
    M, d = 3, 4
    r, eta = [0.7, 0.5, 0.9], [0.6, 0.5, 0.7]
    _, mesh = _mesh(M, 4)
    D = dense.DenseState(M, d, r, eta)
    _run_dense(D, mesh)
    if mistake == "transposed_S":
        orig = u1mpo._gate_S
        monkeypatch.setattr(u1mpo, "_gate_S", lambda th, ph: orig(th, ph).T)
    else:
        monkeypatch.setattr(u1mpo.np, "conj", lambda x: x)
    P = u1mpo.U1MPO(M, d, r, eta)
    P.run_mesh(mesh.k, mesh.theta, mesh.phi, mesh.final_phase)
    monkeypatch.undo()
    assert np.abs(P.to_dense() - D.rho).max() > 1e-3


def _photon_count_kept(r, eta, d, n_cap):
    """Kept probability from photon-number statistics alone: a squeezed vacuum holds
    2m photons with the negative-binomial weight NB(m; 1/2, 1/cosh^2 r) (its
    generating function is (1 - tanh^2 r)^(1/2) (1 - x tanh^2 r)^(-1/2)); keep n < d,
    thin each photon with survival eta (binomial), keep a total <= n_cap."""
    from scipy import stats
    tot = np.zeros(1); tot[0] = 1.0
    for rj, ej in zip(r, eta):
        q = np.zeros(d)
        for n in range(0, d, 2):
            pn = stats.nbinom.pmf(n // 2, 0.5, 1.0 / math.cosh(rj) ** 2)
            q[:n + 1] += pn * stats.binom.pmf(np.arange(n + 1), n, ej)
        tot = np.convolve(tot, q)
    return float(tot[:n_cap + 1].sum())


@pytest.mark.parametrize("M,d,n_cap", [(4, 6, None), (5, 5, 3), (3, 9, None), (6, 4, 2)])
def test_truncated_probability_matches_photon_statistics(M, d, n_cap):
    """App. A's truncated probability from the oracle's Kraus-built state equals the
    same number from squeezed-vacuum photon statistics and binomial loss."""
    rng = np.random.default_rng(M * 100 + d)
    r = rng.uniform(0.3, 1.2, M)
    eta = rng.uniform(0.2, 0.9, M)
    P = u1mpo.U1MPO(M, d, r, eta, n_cap=n_cap)
    cap = d - 1 if n_cap is None else n_cap
    assert abs(P.truncated_probability - (1.0 - _photon_count_kept(r, eta, d, cap))) < 1e-13


def test_truncated_probability_limits():
    """No squeezing truncates nothing; the tail shrinks as d grows and vanishes in the
    limit (the squeezed vacuum's weights sum to one)."""
    M = 3
    P = u1mpo.U1MPO(M, 5, [0.0] * M, [0.5] * M)
    assert abs(P.truncated_probability) < 1e-15
    tails = [u1mpo.U1MPO(M, d, [0.8] * M, [0.6] * M).truncated_probability for d in range(3, 17)]
    assert all(a > b for a, b in zip(tails, tails[1:]))
    assert tails[-1] < 2e-3 and tails[0] > 0.1
