"""Property-based pins of the oracle's building blocks (oracle/fock.py) over random
inputs (hypothesis; skipped where it is not installed):
* the two-mode Fock block of any U(2) mode matrix is unitary, and the map S -> U(S) is
  a homomorphism, U(S1 S2) = U(S1) U(S2), in every photon-number sector;
* the lossy single-mode state is a density matrix (Hermitian, unit trace, positive)
  whose mean photon number is exactly eta times the truncated input's (binomial loss);
* the squeezed amplitudes' weights are the negative-binomial law NB(m; 1/2, 1/cosh^2 r)
  on 2m photons."""
import math

import numpy as np
import pytest

from oracle import fock

try:
    from hypothesis import given, settings
    from hypothesis import strategies as st
except ImportError:
    # Without hypothesis each test skips on its own.  A module-level skip would be
    # reported as a skipped test even in runs that deselect this CPU-only file.
    class _NoStrategies:
        def __getattr__(self, name):
            return lambda *a, **k: None

    st = _NoStrategies()

    def settings(**kwargs):
        return lambda f: f

    def given(**kwargs):
        def wrap(f):
            def skipped():
                pytest.skip("hypothesis is not installed")
            skipped.__name__, skipped.__doc__ = f.__name__, f.__doc__
            return skipped
        return wrap


def _u2(a, b, c, d):
    """A U(2) matrix from four angles (Euler form with a global phase)."""
    return np.exp(1j * a) * np.array([[np.exp(1j * b) * math.cos(c), -np.exp(1j * d) * math.sin(c)],
                                      [np.exp(-1j * d) * math.sin(c), np.exp(-1j * b) * math.cos(c)]])


angles = st.floats(min_value=-math.pi, max_value=math.pi, allow_nan=False)


@settings(max_examples=40, deadline=None)
@given(a=angles, b=angles, c=angles, d=angles, n=st.integers(min_value=0, max_value=8))
def test_fock_block_unitary(a, b, c, d, n):
    B = fock.two_mode_block(_u2(a, b, c, d), n)
    assert np.abs(B @ B.conj().T - np.eye(n + 1)).max() < 1e-12


@settings(max_examples=30, deadline=None)
@given(x=st.lists(angles, min_size=8, max_size=8), n=st.integers(min_value=0, max_value=7))
def test_fock_homomorphism(x, n):
    S1, S2 = _u2(*x[:4]), _u2(*x[4:])
    lhs = fock.two_mode_block(S1 @ S2, n)
    rhs = fock.two_mode_block(S1, n) @ fock.two_mode_block(S2, n)
    assert np.abs(lhs - rhs).max() < 1e-11


@settings(max_examples=40, deadline=None)
@given(r=st.floats(min_value=0.0, max_value=1.5), eta=st.floats(min_value=0.0, max_value=1.0),
       d=st.integers(min_value=2, max_value=14))
def test_lossy_state_is_a_density_matrix_with_scaled_mean(r, eta, d):
    rho, tail = fock.lossy_mode_state(r, eta, d)
    assert abs(np.trace(rho).real - 1.0) < 1e-12
    assert np.abs(rho - rho.conj().T).max() < 1e-14
    assert np.linalg.eigvalsh(rho).min() > -1e-12
    c = fock.squeezed_amplitudes(r, d)
    kept = float(np.sum(c * c))
    n_in = float(np.sum(np.arange(d) * c * c)) / kept if kept > 0 else 0.0
    n_out = float(np.sum(np.arange(d) * np.diag(rho).real))
    assert abs(n_out - eta * n_in) < 1e-12 * max(1.0, n_in)
    assert abs(tail - (1.0 - kept)) < 1e-15


@settings(max_examples=40, deadline=None)
@given(r=st.floats(min_value=0.01, max_value=1.5), d=st.integers(min_value=1, max_value=30))
def test_squeezed_weights_negative_binomial(r, d):
    from scipy import stats
    c = fock.squeezed_amplitudes(r, d)
    for n in range(d):
        want = stats.nbinom.pmf(n // 2, 0.5, 1.0 / math.cosh(r) ** 2) if n % 2 == 0 else 0.0
        assert abs(c[n] ** 2 - want) < 1e-13
