"""Pins for the oracle's single-mode states, loss channel and two-mode Fock elements.

Each check is against a fact fixed independently of the code under test: the
paper's Eq. `kun` (App. B), closed forms of squeezed vacuum, trace preservation of
the Kraus channel, the group homomorphism of U(S), and scipy's matrix exponential
of the number-conserving generator on the n-photon sector.
"""
import math

import numpy as np
import pytest
import scipy.linalg

from oracle import fock


def _rand_su2(rng):
    z = rng.standard_normal((2, 2)) + 1j * rng.standard_normal((2, 2))
    q, r = np.linalg.qr(z)
    return q * (np.diag(r) / np.abs(np.diag(r)))[None, :]


@pytest.mark.parametrize("n", range(0, 9))
def test_fock_block_unitary(n):
    rng = np.random.default_rng(10 + n)
    S = _rand_su2(rng)
    B = fock.two_mode_block(S, n)
    assert np.abs(B.conj().T @ B - np.eye(n + 1)).max() < 1e-12


@pytest.mark.parametrize("n", [1, 2, 5, 8])
def test_fock_eq_kun_single_input_column(n):
    """App. B, Eq. `kun`: <k_u, k_d| U |n> = sqrt(C(n, k_u)) cos^k_u sin^k_d (all photons in
    one input mode), for the real rotation a^dag -> cos a_u^dag + sin a_d^dag."""
    th = 0.37
    S = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
    B = fock.two_mode_block(S, n)
    for ku in range(n + 1):
        want = math.sqrt(math.comb(n, ku)) * math.cos(th) ** ku * math.sin(th) ** (n - ku)
        assert abs(B[ku, n] - want) < 1e-13


@pytest.mark.parametrize("n", [1, 3, 6])
def test_fock_homomorphism(n):
    rng = np.random.default_rng(99 + n)
    S1, S2 = _rand_su2(rng), _rand_su2(rng)
    lhs = fock.two_mode_block(S1 @ S2, n)
    rhs = fock.two_mode_block(S1, n) @ fock.two_mode_block(S2, n)
    assert np.abs(lhs - rhs).max() < 1e-12


@pytest.mark.parametrize("n", [1, 2, 4, 7])
def test_fock_matches_expm_of_generator(n):
    """U(S) = exp(i sum_{jk} H_jk a_j^dag a_k) with S = exp(iH), restricted to the
    n-photon sector (exact: the sector is invariant).  Basis |i, n-i>, i = photons in
    mode 1.  Textbook special case computed by scipy.linalg.expm."""
    rng = np.random.default_rng(3 + n)
    S = _rand_su2(rng)
    H = -1j * scipy.linalg.logm(S)
    H = 0.5 * (H + H.conj().T)
    gen = np.zeros((n + 1, n + 1), dtype=np.complex128)
    for i in range(n + 1):
        gen[i, i] = H[0, 0] * i + H[1, 1] * (n - i)
        if i + 1 <= n:
            # a_1^dag a_2 |i, n-i> = sqrt((i+1)(n-i)) |i+1, n-i-1>
            gen[i + 1, i] += H[0, 1] * math.sqrt((i + 1) * (n - i))
            gen[i, i + 1] += H[1, 0] * math.sqrt((i + 1) * (n - i))
    want = scipy.linalg.expm(1j * gen)
    got = fock.two_mode_block(S, n)
    assert np.abs(got - want).max() < 1e-11


def test_squeezed_closed_forms():
    """Untruncated squeezed vacuum: sum |c|^2 = 1 and <n> = sinh^2 r; odd amplitudes vanish."""
    for r in (0.3, 0.8, 1.2):
        c = fock.squeezed_amplitudes(r, 400)
        assert abs(np.sum(c ** 2) - 1.0) < 1e-12
        assert abs(np.sum(np.arange(400) * c ** 2) - math.sinh(r) ** 2) < 1e-10
        assert np.all(c[1::2] == 0.0)


def test_kraus_trace_preserving_and_mean_scaling():
    """sum_l K^(l)T K^(l) = I on the truncated space; <n> after loss = eta <n> exactly."""
    d, eta = 9, 0.37
    K = fock.kraus_loss(eta, d)
    assert np.abs(np.einsum("lij,lik->jk", K, K) - np.eye(d)).max() < 1e-13
    rng = np.random.default_rng(0)
    psi = rng.standard_normal(d) + 1j * rng.standard_normal(d)
    psi /= np.linalg.norm(psi)
    rho = np.outer(psi, psi.conj())
    out = sum(K[l] @ rho @ K[l].T for l in range(d))
    n = np.arange(d)
    assert abs(np.trace(out).real - 1.0) < 1e-13
    assert abs(np.sum(n * np.diag(out).real) - eta * np.sum(n * np.diag(rho).real)) < 1e-13


def test_lossy_mode_parity_and_mean():
    """rho[m, n] = 0 unless m = n mod 2 (App. B); <n> = eta sinh^2 r for a large cutoff."""
    r, eta = 0.7, 0.4
    rho, tail = fock.lossy_mode_state(r, eta, 80)
    m = np.arange(80)
    par = (m[:, None] - m[None, :]) % 2 == 1
    assert np.all(rho[par] == 0)
    assert tail < 1e-14
    assert abs(np.sum(m * np.diag(rho).real) - eta * math.sinh(r) ** 2) < 1e-12
    assert np.abs(rho - rho.conj().T).max() < 1e-15
    assert np.linalg.eigvalsh(rho).min() > -1e-14
