"""Pins of the App. C asymptotic estimator in the oracle (oracle/asymptotic.py) against
results it does not compute itself:

* lossless input (mu = 1): the split squeezed vacuum is a pure two-mode Gaussian state
  whose reduced state has symplectic eigenvalue nu = sqrt(1 + sin^2(2 theta) sinh^2 r);
  the vectorised pure state's operator spectrum is the product of two copies of that
  thermal spectrum, so S_alpha(operator) = 2 S_alpha(thermal, nbar = (nu - 1) / 2);
* the lossy mode against the dense oracle O1 on two modes (squeezed + vacuum) with one
  beam splitter, whose plain operator entanglement is computed from the full d^2 x d^2
  density matrix by an unrelated route;
* App. C's eigenvalue structure for small transmission: exactly one O(1) value, the
  next ones O(mu^2);
* special cases: mu = 0 (vacuum output) and theta = 0 (nothing reaches the other half)
  carry no entanglement; the Renyi entropy tends to S_1 as alpha -> 1.
"""
import math

import numpy as np
import pytest

from oracle import asymptotic as asy
from oracle import dense


def _thermal_renyi(nbar: float, alpha: float) -> float:
    """Renyi entropy (bits) of the thermal spectrum (1 - x) x^k, x = nbar / (nbar + 1)."""
    if alpha == 1.0:
        return (nbar + 1) * math.log2(nbar + 1) - (nbar * math.log2(nbar) if nbar > 0 else 0.0)
    return math.log2((nbar + 1) ** alpha - nbar ** alpha) / (alpha - 1.0)


@pytest.mark.parametrize("theta", [math.pi / 4, 0.3])
@pytest.mark.parametrize("alpha", [1.0, 2.0, 0.5])
def test_lossless_split_matches_gaussian_closed_form(theta, alpha):
    r, n_max = 0.4, 28
    nu = math.sqrt(1.0 + math.sin(2 * theta) ** 2 * math.sinh(r) ** 2)
    want = 2.0 * _thermal_renyi((nu - 1.0) / 2.0, alpha)
    got = asy.mode_entropy(r, 1.0, n_max, theta, None if alpha == 1.0 else alpha)
    # the photons above n_max carry ~1e-14 of the probability; orders alpha < 1 weigh
    # that missing tail by p^alpha, so their bound is its square root
    tol = 1e-9 if alpha >= 1.0 else 5e-6  # alpha = 1/2: 1.9e-6 at n_max = 28, 4e-8 at 36
    assert abs(got - want) < tol, (got, want)


@pytest.mark.parametrize("r,mu,theta", [(0.8, 0.6, math.pi / 4), (0.88, 0.3, 0.7), (1.1, 0.9, 0.2)])
def test_lossy_mode_matches_dense_two_mode_state(r, mu, theta):
    n_max = 5
    D = dense.DenseState(2, n_max + 1, [r, 0.0], [mu, mu])
    S = np.array([[math.cos(theta), -math.sin(theta)], [math.sin(theta), math.cos(theta)]])
    D.apply_gate(0, S)
    want = D.plain_operator_entropy(1)
    got = asy.mode_entropy(r, mu, n_max, theta)
    assert abs(got - want) < 1e-10, (got, want)


def test_small_transmission_eigenvalue_orders():
    """App. C: one O(1) eigenvalue, none of first order, the rest at least O(mu^2)."""
    r, n_max = 0.88, 8
    p1 = asy.mode_spectrum(r, 1e-3, n_max)
    p2 = asy.mode_spectrum(r, 5e-4, n_max)
    assert abs(p1[0] - 1.0) < 1e-5
    # the second value scales as mu^2: halving mu divides it by 4
    assert abs(p1[1] / p2[1] - 4.0) < 0.01
    assert p1[1] / 1e-6 < 10.0  # no first-order term
    # the entropy is O(mu^2 log mu): S / (mu^2 log2(1/mu)) settles
    s1 = asy.entropy(p1) / (1e-6 * math.log2(1e3))
    s2 = asy.entropy(p2) / (0.25e-6 * math.log2(2e3))
    assert abs(s1 / s2 - 1.0) < 0.15


def test_special_cases():
    assert asy.mode_entropy(0.88, 0.0, 8) == 0.0
    assert abs(asy.mode_entropy(0.88, 0.7, 8, theta=0.0)) < 1e-14
    assert abs(asy.mode_entropy(0.0, 0.7, 8)) < 1e-14  # vacuum input
    s1 = asy.mode_entropy(0.88, 0.5, 8)
    assert abs(asy.mode_entropy(0.88, 0.5, 8, alpha=1.0 + 1e-6) - s1) < 1e-5
    assert abs(asy.mode_entropy(0.88, 0.5, 8, alpha=1.0 - 1e-6) - s1) < 1e-5
    p = asy.mode_spectrum(0.88, 0.5, 8)
    assert abs(p.sum() - 1.0) < 1e-14 and np.all(np.diff(p) <= 0)


def test_system_entropy_scales_mode_value():
    N, beta, gamma = 64, 1.0, 0.5
    mu = beta * N ** gamma / N
    assert abs(asy.system_entropy(N, beta, gamma, 0.88, 6) - N * asy.mode_entropy(0.88, mu, 6)) < 1e-12


def test_transposed_vectorisation_is_caught():
    """A transposed reshape (rows (k_u, k_d) instead of (k_u, k_u')) makes the pure
    lossless state look unentangled; the closed-form pin rejects it."""
    r, theta, n_max = 0.4, math.pi / 4, 16
    rho = asy.mode_output(r, 1.0, n_max, theta)
    d = n_max + 1
    s = np.linalg.svd(rho.reshape(d * d, d * d), compute_uv=False)  # wrong grouping
    p = s * s / np.sum(s * s)
    nu = math.sqrt(1.0 + math.sinh(r) ** 2)
    assert abs(asy.entropy(p) - 2.0 * _thermal_renyi((nu - 1.0) / 2.0, 1.0)) > 0.1
