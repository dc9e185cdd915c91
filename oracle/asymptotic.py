"""App. C of arXiv:2301.12814: the asymptotic estimate of the MPO operator entanglement
from a single input mode (oracle; test infrastructure only).

For large systems the paper estimates the operator EE by treating one squeezed input
mode at a time.  Loss is uniform, so it acts on the input state first (Method); the
interferometer then spreads the lossy mode over the two halves of the bipartition, and
the whole-system operator EE is the single-mode contribution times the number N of
squeezed inputs, because the output is a product over input modes (App. C).

Steps, in the paper's order:
1. |psi_in>: squeezed vacuum amplitudes up to n_max photons (App. C; truncated, not
   renormalised; the sign convention of ``fock.squeezed_amplitudes`` is a local phase
   that leaves every entropy unchanged);
2. rho_lossy = sum_l K^(l) rho_in K^(l)^T with the pure-loss Kraus operators, both the
   state and the operators truncated to n_max photons (App. C, Eq. `lossy`);
3. the basis transform of Eq. `transform` / Eq. `kun`:
   <k_u, k_d| U |n> = sqrt(C(n, k_u)) cos^k_u(theta) sin^k_d(theta), k_u + k_d = n,
   so rho_out[k_u, k_d; k_u', k_d'] = sum_{m,n} <k_u,k_d|U|m> rho_lossy[m,n] <n|U^T|k_u',k_d'>
   (Eq. `out`); theta = pi/4 in the asymptotic limit (App. C, Eq. `normalization`);
4. vectorisation: K_u = (k_u, k_u'), K_d = (k_d, k_d'), X[K_u, K_d] = rho_out[k_u, k_d; k_u', k_d'];
5. the eigenvalues of rho' = tr_u |rho_out>><<rho_out| (rho'[K_d, K_d'] = sum_K_u X[K_u, K_d] X*[K_u, K_d'])
   are the squared singular values of X (App. C names the singular values lambda and the
   eigenvalues lambda^2); they are normalised to sum 1 because the vectorised state is
   not L2-normalised (App. C);
6. S_1 = -sum p log2 p, and the Renyi entropy S_alpha = log2(sum p^alpha) / (1 - alpha)
   (App. C);
7. the system estimate is N S with the transmission mu = beta N^gamma / N (Results:
   N_out = beta N^gamma surviving photons).

The singular values come from LAPACK (numpy.linalg.svd); nothing is blocked or reordered.
"""
from __future__ import annotations

import math
from typing import Optional

import numpy as np

from . import fock


def lossy_input(r: float, mu: float, n_max: int) -> np.ndarray:
    """Steps 1-2: rho_lossy on Fock levels 0..n_max (real, not renormalised)."""
    d = n_max + 1
    c = fock.squeezed_amplitudes(r, d)
    K = fock.kraus_loss(mu, d)
    rho_in = np.outer(c, c)
    rho = np.zeros((d, d))
    for l in range(d):
        rho += K[l] @ rho_in @ K[l].T
    return rho


def split_matrix(theta: float, n_max: int) -> np.ndarray:
    """Step 3: W[k_u, k_d, n] = <k_u, k_d| U |n> (Eq. `kun`)."""
    d = n_max + 1
    c, s = math.cos(theta), math.sin(theta)
    W = np.zeros((d, d, d))
    for n in range(d):
        for ku in range(n + 1):
            W[ku, n - ku, n] = math.sqrt(math.comb(n, ku)) * c ** ku * s ** (n - ku)
    return W


def mode_output(r: float, mu: float, n_max: int, theta: float = math.pi / 4) -> np.ndarray:
    """Step 3: rho_out[k_u, k_d, k_u', k_d'] (Eq. `out`)."""
    W = split_matrix(theta, n_max)
    rho = lossy_input(r, mu, n_max)
    return np.einsum("abm,mn,cdn->abcd", W, rho, W)


def vectorised(rho_out: np.ndarray) -> np.ndarray:
    """Step 4: X[(k_u, k_u'), (k_d, k_d')]."""
    d = rho_out.shape[0]
    return rho_out.transpose(0, 2, 1, 3).reshape(d * d, d * d)


def mode_spectrum(r: float, mu: float, n_max: int, theta: float = math.pi / 4) -> np.ndarray:
    """Step 5: normalised eigenvalues of the reduced operator, descending."""
    s = np.linalg.svd(vectorised(mode_output(r, mu, n_max, theta)), compute_uv=False)
    p = s * s
    tot = p.sum()
    return np.sort(p / tot)[::-1] if tot > 0.0 else p


def entropy(p: np.ndarray, alpha: Optional[float] = None) -> float:
    """Step 6: S_1 (alpha None or 1) or the Renyi entropy S_alpha, in bits."""
    p = p[p > 0.0]
    if alpha is None or alpha == 1.0:
        return float(-np.sum(p * np.log2(p)))
    return float(math.log2(np.sum(p ** alpha)) / (1.0 - alpha))


def mode_entropy(r: float, mu: float, n_max: int, theta: float = math.pi / 4,
                 alpha: Optional[float] = None) -> float:
    """Steps 1-6: the operator EE contributed by one squeezed input mode."""
    return entropy(mode_spectrum(r, mu, n_max, theta), alpha)


def system_entropy(N: int, beta: float, gamma: float, r: float, n_max: int,
                   alpha: Optional[float] = None) -> float:
    """Step 7: N S at mu = beta N^gamma / N, theta = pi/4."""
    mu = beta * N ** gamma / N
    return N * mode_entropy(r, mu, n_max, math.pi / 4, alpha)
