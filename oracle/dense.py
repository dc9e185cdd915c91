"""O1: brute-force dense density matrix of a few modes (oracle; test infrastructure only).

rho lives on (C^d)^{(x)M} as a d^M x d^M complex128 matrix, mode 0 the most
significant digit.  Steps (arXiv:2301.12814):
1. rho_0 = P_cap (x)_j rho_j P_cap / Tr, with rho_j the lossy squeezed mode (App. B/C:
   uniform loss is moved to the input state, Method section) and P_cap the projector
   on total photon number <= n_cap (the left-most charge is the total photon number,
   App. A);
2. every mesh gate rho <- G rho G^dag, G = U(S) on modes (k, k+1) (Method: the
   vectorised update U_{jk} U^*_{j'k'});
3. final phase screen;
4. observables: Tr rho, <n_k>, <n_k^2>, and the U(1)-form operator entanglement.

The U(1)-form entanglement at bond b (modes [0,b) | [b,M)): reshape vec(rho) into
rows (ket, bra digits of modes < b) and columns (ket, bra digits of modes >= b),
split the columns by the right charge pair (total ket photons right of b, total bra
photons right of b), take the singular values of every column group, pool them,
p = s^2 / sum s^2, S = -sum p log2 p (log base 2 as in App. B).  This is the
Schmidt spectrum of vec(rho) augmented by the left-boundary charge register, which
is what the U(1) MPO's lambda hold (App. D; the Results note that a product state
can carry non-zero U(1)-symmetric MPO entanglement).
"""
from __future__ import annotations

from typing import List, Sequence

import numpy as np

from . import fock


def _digits(M: int, d: int) -> np.ndarray:
    """occ[s, j] = photons in mode j of basis state s."""
    s = np.arange(d ** M)
    occ = np.zeros((d ** M, M), dtype=np.int64)
    for j in range(M - 1, -1, -1):
        occ[:, j] = s % d
        s = s // d
    return occ


class DenseState:
    def __init__(self, M: int, d: int, r: Sequence[float], eta: Sequence[float],
                 n_cap: int | None = None):
        self.M, self.d = M, d
        self.n_cap = d - 1 if n_cap is None else n_cap
        self.occ = _digits(M, d)
        rho = np.ones((1, 1), dtype=np.complex128)
        for j in range(M):
            rj, _ = fock.lossy_mode_state(float(r[j]), float(eta[j]), d)
            rho = np.kron(rho, rj)
        keep = (self.occ.sum(axis=1) <= self.n_cap).astype(np.float64)
        rho = keep[:, None] * rho * keep[None, :]
        self.cap_trace = float(np.trace(rho).real)
        self.rho = rho / self.cap_trace

    def gate_matrix(self, k: int, S: np.ndarray) -> np.ndarray:
        """Full d^M x d^M matrix of U(S) on modes (k, k+1); identity elsewhere."""
        occ, d = self.occ, self.d
        blocks = fock.fock_tables(S, 2 * (d - 1))
        N = d ** self.M
        G = np.zeros((N, N), dtype=np.complex128)
        place = d ** (self.M - 1 - np.arange(self.M))
        for s in range(N):
            j1, j2 = occ[s, k], occ[s, k + 1]
            n = j1 + j2
            base = s - j1 * place[k] - j2 * place[k + 1]
            for i1 in range(max(0, n - (d - 1)), min(n, d - 1) + 1):
                t = base + i1 * place[k] + (n - i1) * place[k + 1]
                G[t, s] = blocks[n][i1, j1]
        return G

    def apply_gate(self, k: int, S: np.ndarray) -> None:
        G = self.gate_matrix(k, S)
        self.rho = G @ self.rho @ G.conj().T

    def apply_phases(self, phases: Sequence[float]) -> None:
        ph = np.exp(1j * (self.occ * np.asarray(phases)[None, :]).sum(axis=1))
        self.rho = ph[:, None] * self.rho * ph.conj()[None, :]

    # --- observables ---------------------------------------------------------
    def trace(self) -> float:
        return float(np.trace(self.rho).real)

    def moments(self):
        """(Tr rho, <n_j>, <n_j^2>) with the moments divided by Tr rho."""
        diag = np.diag(self.rho).real
        tr = diag.sum()
        n1 = (diag[:, None] * self.occ).sum(axis=0) / tr
        n2 = (diag[:, None] * self.occ ** 2).sum(axis=0) / tr
        return tr, n1, n2

    def u1_schmidt(self, b: int) -> np.ndarray:
        """Pooled singular values of the charge-split vec(rho) at bond b (descending)."""
        M, d, occ = self.M, self.d, self.occ
        # tensor indices: ket digits (M), bra digits (M)
        t = self.rho.reshape([d] * (2 * M))
        left = list(range(b)) + list(range(M, M + b))
        right = list(range(b, M)) + list(range(M + b, 2 * M))
        t = np.transpose(t, left + right).reshape(d ** (2 * b), d ** (2 * (M - b)))
        nr = M - b
        if nr > 0:
            rocc = _digits(nr, d).sum(axis=1)
        else:
            rocc = np.zeros(1, dtype=np.int64)
        # column (ket right config, bra right config) -> charge pair
        ck = np.repeat(rocc, d ** nr)
        cb = np.tile(rocc, d ** nr)
        svals: List[np.ndarray] = []
        for c in np.unique(ck):
            for cbar in np.unique(cb):
                cols = np.nonzero((ck == c) & (cb == cbar))[0]
                if cols.size == 0:
                    continue
                sub = t[:, cols]
                svals.append(np.linalg.svd(sub, compute_uv=False))
        s = np.sort(np.concatenate(svals))[::-1]
        return s

    def u1_entropy(self, b: int, rel_cut: float = 1e-14) -> float:
        s = self.u1_schmidt(b)
        s = s[s > rel_cut * s[0]]
        p = s ** 2 / np.sum(s ** 2)
        return float(-np.sum(p * np.log2(p)))

    def plain_operator_entropy(self, b: int) -> float:
        """Operator entanglement of vec(rho) without the charge register (context only)."""
        M, d = self.M, self.d
        t = self.rho.reshape([d] * (2 * M))
        left = list(range(b)) + list(range(M, M + b))
        right = list(range(b, M)) + list(range(M + b, 2 * M))
        t = np.transpose(t, left + right).reshape(d ** (2 * b), d ** (2 * (M - b)))
        s = np.linalg.svd(t, compute_uv=False)
        s = s[s > 1e-14 * s[0]]
        p = s ** 2 / np.sum(s ** 2)
        return float(-np.sum(p * np.log2(p)))
