"""Single-mode input states, the pure-loss channel, and two-mode Fock beam-splitter
elements, in float64 (oracle; test infrastructure only).

Paper references (arXiv:2301.12814):
* squeezed vacuum amplitudes: App. C, the input wavefunction of one squeezed mode
  (tanh^n r / (2^n n! sqrt(cosh r)) a^{dag 2n}|0>);  the sign (-tanh r)^j used here
  differs from the paper's +tanh r by the phase e^{i pi N/2}, which commutes with
  the mesh and leaves every observable and every lambda unchanged;
* pure-loss Kraus operators: App. B, K^{(l)}_{out,in} = sqrt(C(in,out) mu^out (1-mu)^l)
  for in - out = l, with mu the transmission;
* the two-mode beam-splitter element: App. B, Eq. `kun` gives the column with all
  input photons in one mode;  the general element used here follows from the
  mode transformation a_1^dag -> S11 a_1^dag + S21 a_2^dag,
  a_2^dag -> S12 a_1^dag + S22 a_2^dag by the binomial expansion.
"""
from __future__ import annotations

import math
from typing import Tuple

import numpy as np


def squeezed_amplitudes(r: float, d: int) -> np.ndarray:
    """c_n, n = 0..d-1, of single-mode squeezed vacuum truncated at d levels (App. C).

    c_{2j} = (-tanh r)^j sqrt((2j)!) / (2^j j! sqrt(cosh r)); odd n are zero.
    Not renormalised: sum |c_n|^2 = 1 - (truncation tail)."""
    c = np.zeros(d, dtype=np.float64)
    t = math.tanh(r)
    for j in range(0, (d - 1) // 2 + 1):
        n = 2 * j
        # sqrt((2j)!) / (2^j j!) = sqrt(C(2j, j) / 4^j), evaluated in exact integers
        c[n] = ((-t) ** j) * math.sqrt(math.comb(n, j) / 4 ** j) / math.sqrt(math.cosh(r))
    return c


def kraus_loss(eta: float, d: int) -> np.ndarray:
    """Pure-loss Kraus operators K[l] (d x d), l = 0..d-1 photons lost (App. B).

    K[l][out, in] = sqrt(C(in, out) eta^out (1-eta)^l) when in - out = l."""
    K = np.zeros((d, d, d), dtype=np.float64)
    for l in range(d):
        for out in range(d - l):
            n_in = out + l
            K[l, out, n_in] = math.sqrt(math.comb(n_in, out) * (eta ** out) * ((1.0 - eta) ** l))
    return K


def lossy_mode_state(r: float, eta: float, d: int) -> Tuple[np.ndarray, float]:
    """rho_j = sum_l K^(l) |psi><psi| K^(l)^dag for one mode, renormalised to trace 1.

    Returns (rho, tail) with tail = 1 - sum |c_n|^2 (the truncation tail of |psi>).
    The state and the Kraus operators are both truncated to d levels (App. C)."""
    c = squeezed_amplitudes(r, d)
    rho_in = np.outer(c, c).astype(np.complex128)
    K = kraus_loss(eta, d)
    rho = np.zeros((d, d), dtype=np.complex128)
    for l in range(d):
        rho += K[l] @ rho_in @ K[l].T
    tail = 1.0 - float(np.sum(c * c))
    return rho / np.trace(rho).real, tail


def two_mode_block(S: np.ndarray, n: int) -> np.ndarray:
    """U_n[i, j] = <i, n-i| U(S) |j, n-j> for the two-mode passive unitary with mode
    matrix S (a_1^dag -> S11 a_1^dag + S21 a_2^dag, a_2^dag -> S12 a_1^dag + S22 a_2^dag).

    Closed form, summing over p photons that go from input mode 1 to output mode 1:
    sqrt(i!(n-i)!/(j!(n-j)!)) sum_p C(j,p) C(n-j,i-p) S11^p S21^(j-p) S12^(i-p) S22^(n-j-i+p).
    For S = [[cos, .], [sin, .]] and j = n this is Eq. `kun` of App. B."""
    S11, S12, S21, S22 = complex(S[0, 0]), complex(S[0, 1]), complex(S[1, 0]), complex(S[1, 1])
    B = np.zeros((n + 1, n + 1), dtype=np.complex128)
    for i in range(n + 1):
        for j in range(n + 1):
            acc = 0j
            for p in range(0, min(i, j) + 1):
                if i - p > n - j:
                    continue
                acc += (math.comb(j, p) * math.comb(n - j, i - p)
                        * S11 ** p * S21 ** (j - p) * S12 ** (i - p) * S22 ** (n - j - i + p))
            B[i, j] = acc * math.sqrt(math.factorial(i) * math.factorial(n - i)
                                      / (math.factorial(j) * math.factorial(n - j)))
    return B


def fock_tables(S: np.ndarray, n_max: int):
    """[U_0, U_1, ..., U_{n_max}] for one gate."""
    return [two_mode_block(S, n) for n in range(n_max + 1)]
