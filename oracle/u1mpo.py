"""O2: the U(1)-symmetric vectorised MPO of arXiv:2301.12814, App. D, in plain FP64
loops over charges (oracle; test infrastructure only).

State (Vidal form, App. D).  Modes j = 0..M-1; bond b = 0..M sits left of mode b
(bond 0 is the left boundary, bond M the right one).  Every index of bond b carries
a charge pair (c, cbar) = (ket photons, bra photons) in modes b..M-1, i.e. to the
RIGHT of the bond (App. D; the left-most charge is then the total photon number,
App. A).  Gamma_j is a chi_j x chi_{j+1} matrix whose physical ket/bra indices are
implied by the charges, i = c_row - c_col and ibar = cbar_row - cbar_col (the delta
constraint of App. D), lambda_b are the bond weights.  The amplitude of a
(ket, bra) configuration is  sum over bond indices of
lambda_0 Gamma_0 lambda_1 Gamma_1 ... Gamma_{M-1} lambda_M.
Bond 0 ranges over the total-charge pairs (a charge register) with weights
lambda_0; bond M has the single charge (0, 0).

Charges are capped: 0 <= c, cbar <= n_cap (default n_cap = d - 1: d - 1 caps the
total photon number on each side, App. A and App. D.5).

Gate (App. D, Eq. `theta`, the block SVD and keep-chi rule, and the Vidal re-split):
for the beam splitter S on modes (j, j+1), bonds A = j, C = j+1, B = j+2:

  Theta(m)[alpha, beta] = lambda_A[alpha] lambda_B[beta]
        * sum_gamma u(a, b, c, m) Gamma_j[alpha, gamma] lambda_C[gamma] Gamma_{j+1}[gamma, beta]

with a, b, c the charges of alpha, beta, gamma and m the new centre charge,
u = U_Delta[c_a - m, c_a - c] * conj(U_Deltabar[cbar_a - mbar, cbar_a - cbar]),
Delta = c_a - c_b.  Each Theta(m) is factorised by LAPACK's SVD, the singular values
of all blocks are pooled and the chi largest kept; lambda_C = kept values (never
renormalised), Gamma_j = X / lambda_A, Gamma_{j+1} = Y / lambda_B.

Readings of points the paper leaves open (each is listed in the design notes):
* ordering of the pooled values: (s descending, m ascending, index ascending);
* values s <= 1e-14 * s_max are dropped before the cut;
* when the cut at chi would split a run of values whose consecutive relative gap is
  <= 1e-9 (Hermiticity makes blocks m and its ket/bra mirror carry identical
  spectra), the whole run is dropped; if that would drop everything, the plain cut
  at chi is used;
* discarded weight = (sum of dropped s^2) / (sum of all s^2) per gate.
"""
from __future__ import annotations

import math
from typing import List, Optional, Sequence

import numpy as np

from . import fock

REL_DROP = 1e-14
TIE_REL = 1e-9


def _gate_S(theta: float, phi: float) -> np.ndarray:
    """Mode matrix of one mesh gate: [[e^{i phi} cos, -sin], [e^{i phi} sin, cos]]."""
    e = complex(math.cos(phi), math.sin(phi))
    c, s = math.cos(theta), math.sin(theta)
    return np.array([[e * c, -s], [e * s, c]], dtype=np.complex128)


def _entropy(lam: np.ndarray) -> float:
    """-sum p log2 p with p = lambda^2 / sum lambda^2 (Method, Eq. `schmidt`; App. B)."""
    p = lam.astype(np.float64) ** 2
    tot = p.sum()
    if tot <= 0:
        return 0.0
    p = p / tot
    p = p[p > 0]
    return float(-np.sum(p * np.log2(p)))


def _conv2(a: np.ndarray, w: np.ndarray, cap: int) -> np.ndarray:
    """(a (*) w)[c, cb] = sum_{n <= c, nb <= cb} w[n, nb] a[c - n, cb - nb], c, cb <= cap."""
    out = np.zeros((cap + 1, cap + 1), dtype=np.float64)
    for c in range(cap + 1):
        for cb in range(cap + 1):
            acc = 0.0
            for n in range(min(c, w.shape[0] - 1) + 1):
                for nb in range(min(cb, w.shape[1] - 1) + 1):
                    acc += w[n, nb] * a[c - n, cb - nb]
            out[c, cb] = acc
    return out


def select_kept(cands, chi_max: Optional[int]):
    """Pool the block singular values and keep the chi largest (App. D: "keep the chi
    largest singular values" over all Theta(c) blocks), with the readings stated in
    the module docstring.  cands = [(s, m_index, i, payload)]; returns the kept
    entries ordered by (m_index, i) and the discarded weight."""
    cands = sorted(cands, key=lambda t: (-t[0], t[1], t[2]))
    total = sum(t[0] ** 2 for t in cands)
    smax = cands[0][0] if cands else 0.0
    alive = [t for t in cands if t[0] > REL_DROP * smax]
    keep = len(alive)
    if chi_max is not None and keep > chi_max:
        jcut = chi_max
        while jcut > 0 and alive[jcut][0] >= alive[jcut - 1][0] * (1.0 - TIE_REL):
            jcut -= 1
        keep = jcut if jcut > 0 else chi_max
    kept = alive[:keep]
    dropped_w = total - sum(t[0] ** 2 for t in kept)
    eps = dropped_w / total if total > 0 else 0.0
    kept.sort(key=lambda t: (t[1], t[2]))
    return kept, eps


class U1MPO:
    """The U(1) MPO with dense per-site matrices and explicit charge vectors."""

    def __init__(self, M: int, d: int, r: Sequence[float], eta: Sequence[float],
                 chi_max: Optional[int] = None, n_cap: Optional[int] = None):
        self.M, self.d = M, d
        self.n_cap = d - 1 if n_cap is None else int(n_cap)
        if self.n_cap > d - 1:
            raise ValueError("n_cap must be <= d - 1")
        self.chi_max = chi_max
        self.discarded: List[float] = []
        self._init_state([float(x) for x in r], [float(x) for x in eta])

    # ------------------------------------------------------------------ init
    def _init_state(self, r: List[float], eta: List[float]) -> None:
        """Exactly canonical U(1) Vidal form of rho_0 = P_cap (x)_j rho_j P_cap / T.

        Per-mode weights w_j(n, nb) = |rho_j[n, nb]|^2.  R_b(c, cb)^2 = weight of the
        configurations of modes b..M-1 with totals (c, cb); W_b(x, xb) = weight of the
        configurations of modes 0..b-1 with totals (x, xb); L_b(c, cb)^2 = sum of W_b
        over x <= n_cap - c, xb <= n_cap - cb.  Then lambda_b = L_b R_b / T and
        Gamma_j[a, b'] = T rho_j[c_a - c_b', cbar_a - cbar_b'] / (R_j(a) L_{j+1}(b')),
        which is left and right orthonormal by the convolution identities.
        The paper credits the loss-in-the-initial-state construction to the Method
        section and gives no formulas for the MPO initialisation; this is the
        construction written out."""
        M, cap = self.M, self.n_cap
        self.rho_modes = []
        kept_modes = 1.0
        for j in range(M):
            rho_j, tail_j = fock.lossy_mode_state(r[j], eta[j], self.d)
            self.rho_modes.append(rho_j[:cap + 1, :cap + 1])
            kept_modes *= 1.0 - tail_j
        w = [np.abs(rj) ** 2 for rj in self.rho_modes]
        R2 = [None] * (M + 1)
        R2[M] = np.zeros((cap + 1, cap + 1)); R2[M][0, 0] = 1.0
        for b in range(M - 1, -1, -1):
            R2[b] = _conv2(R2[b + 1], w[b], cap)
        W = [None] * (M + 1)
        W[0] = np.zeros((cap + 1, cap + 1)); W[0][0, 0] = 1.0
        for b in range(M):
            W[b + 1] = _conv2(W[b], w[b], cap)
        L2 = []
        for b in range(M + 1):
            Lb = np.zeros((cap + 1, cap + 1))
            for c in range(cap + 1):
                for cb in range(cap + 1):
                    Lb[c, cb] = W[b][:cap - c + 1, :cap - cb + 1].sum()
            L2.append(Lb)
        # trace normalisation T = Tr(P_cap (x) rho_j P_cap)
        t = np.zeros(cap + 1); t[0] = 1.0
        for j in range(M):
            dj = np.real(np.diag(self.rho_modes[j]))
            nt = np.zeros(cap + 1)
            for x in range(cap + 1):
                for n in range(x + 1):
                    nt[x] += dj[n] * t[x - n]
            t = nt
        T = float(t.sum())
        self.cap_trace = T
        # App. A: the probability cut by the local dimension (each mode's squeezed
        # vacuum keeps its first d Fock levels) and then by the photon-number cap
        self.truncated_probability = 1.0 - kept_modes * T
        self.charges: List[np.ndarray] = []
        self.lam: List[np.ndarray] = []
        for b in range(M + 1):
            ch = [(c, cb) for c in range(cap + 1) for cb in range(cap + 1)
                  if R2[b][c, cb] > 0.0 and L2[b][c, cb] > 0.0]
            self.charges.append(np.array(ch, dtype=np.int64).reshape(-1, 2))
            self.lam.append(np.array([math.sqrt(L2[b][c, cb] * R2[b][c, cb]) / T
                                      for (c, cb) in ch]))
        self.gam: List[np.ndarray] = []
        for j in range(M):
            A, B = self.charges[j], self.charges[j + 1]
            G = np.zeros((len(A), len(B)), dtype=np.complex128)
            for ia, (ca, cba) in enumerate(A):
                for ib, (cbb, cbbb) in enumerate(B):
                    i, ib_ = ca - cbb, cba - cbbb
                    if i < 0 or ib_ < 0:
                        continue
                    G[ia, ib] = T * self.rho_modes[j][i, ib_] / (
                        math.sqrt(R2[j][ca, cba]) * math.sqrt(L2[j + 1][cbb, cbbb]))
            self.gam.append(G)
        self.entropy = [_entropy(l) for l in self.lam]

    # ------------------------------------------------------------------ gate
    def theta_blocks(self, j: int, theta: float, phi: float):
        """Eq. `theta` for every new centre charge m: {m: (rows, cols, Theta(m))}.

        Plain loops over (m, a, b) as in the CPU algorithm of App. D.1: fix the centre
        charge, select the bonds of each left charge a and right charge b, look up the
        unitary elements for every centre bond gamma, and contract."""
        cap = self.n_cap
        tabs = fock.fock_tables(_gate_S(theta, phi), cap)
        # U[n, i, q] = <i, n-i| U(S) |q, n-q>, zero-padded to (cap+1)^3 for lookups
        U = np.zeros((cap + 1, cap + 1, cap + 1), dtype=np.complex128)
        for n, t in enumerate(tabs):
            U[n, :n + 1, :n + 1] = t
        A, C, B = self.charges[j], self.charges[j + 1], self.charges[j + 2]
        lA, lC, lB = self.lam[j], self.lam[j + 1], self.lam[j + 2]
        G1, G2 = self.gam[j], self.gam[j + 1]
        out = {}
        for cm in range(cap + 1):
            for cbm in range(cap + 1):
                rows = np.nonzero((A[:, 0] >= cm) & (A[:, 1] >= cbm))[0]
                cols = np.nonzero((B[:, 0] <= cm) & (B[:, 1] <= cbm))[0]
                if rows.size == 0 or cols.size == 0:
                    continue
                Th = np.zeros((rows.size, cols.size), dtype=np.complex128)
                a_pairs = sorted(set(map(tuple, A[rows])))
                b_pairs = sorted(set(map(tuple, B[cols])))
                for (ca, cba) in a_pairs:
                    ra = np.nonzero((A[rows, 0] == ca) & (A[rows, 1] == cba))[0]
                    for (cb, cbb) in b_pairs:
                        rb = np.nonzero((B[cols, 0] == cb) & (B[cols, 1] == cbb))[0]
                        dk, db = ca - cb, cba - cbb
                        # u(a, b, c, m) for every centre bond gamma (zero unless a >= c >= b)
                        ok = ((C[:, 0] <= ca) & (C[:, 0] >= cb)
                              & (C[:, 1] <= cba) & (C[:, 1] >= cbb))
                        qk = np.where(ok, ca - C[:, 0], 0)
                        qb = np.where(ok, cba - C[:, 1], 0)
                        u = np.where(ok, U[dk, ca - cm, qk] * np.conj(U[db, cba - cbm, qb]), 0)
                        left = G1[rows[ra], :] * (u * lC)[None, :]
                        blk = left @ G2[:, cols[rb]]
                        Th[np.ix_(ra, rb)] = (lA[rows[ra]][:, None] * blk
                                              * lB[cols[rb]][None, :])
                out[(cm, cbm)] = (rows, cols, Th)
        return out

    def apply_gate(self, j: int, theta: float, phi: float) -> float:
        """One two-site update on modes (j, j+1); returns the discarded weight."""
        cap = self.n_cap
        blocks = self.theta_blocks(j, theta, phi)
        cands = []   # (s, m_index, i)
        svd = {}
        for m, (rows, cols, Th) in blocks.items():
            X, s, Yh = np.linalg.svd(Th, full_matrices=False)
            svd[m] = (X, s, Yh)
            mi = m[0] * (cap + 1) + m[1]
            for i, sv in enumerate(s):
                cands.append((float(sv), mi, i, m))
        kept, eps = select_kept(cands, self.chi_max)
        A, B = self.charges[j], self.charges[j + 2]
        lA, lB = self.lam[j], self.lam[j + 2]
        newC = np.array([t[3] for t in kept], dtype=np.int64).reshape(-1, 2)
        newl = np.array([t[0] for t in kept])
        G1 = np.zeros((A.shape[0], len(kept)), dtype=np.complex128)
        G2 = np.zeros((len(kept), B.shape[0]), dtype=np.complex128)
        for col, (sv, mi, i, m) in enumerate(kept):
            rows, cols, _ = blocks[m]
            X, s, Yh = svd[m]
            G1[rows, col] = X[:, i] / lA[rows]
            G2[col, cols] = Yh[i, :] / lB[cols]
        self.charges[j + 1] = newC
        self.lam[j + 1] = newl
        self.gam[j] = G1
        self.gam[j + 1] = G2
        self.entropy[j + 1] = _entropy(newl)
        self.discarded.append(eps)
        return eps

    def apply_phases(self, phases: Sequence[float]) -> None:
        """Final phase screen: Gamma_j *= exp(i phi_j (i - ibar)), i = c_row - c_col."""
        for j in range(self.M):
            A, B = self.charges[j], self.charges[j + 1]
            i = A[:, 0][:, None] - B[:, 0][None, :]
            ib = A[:, 1][:, None] - B[:, 1][None, :]
            self.gam[j] = self.gam[j] * np.exp(1j * phases[j] * (i - ib))

    def run_mesh(self, k: Sequence[int], theta: Sequence[float], phi: Sequence[float],
                 final_phase: Optional[Sequence[float]] = None) -> List[float]:
        eps = [self.apply_gate(int(kk), float(t), float(p)) for kk, t, p in zip(k, theta, phi)]
        if final_phase is not None:
            self.apply_phases(final_phase)
        return eps

    # ----------------------------------------------------------- observables
    def _diag_mask(self, j: int) -> np.ndarray:
        A, B = self.charges[j], self.charges[j + 1]
        i = A[:, 0][:, None] - B[:, 0][None, :]
        ib = A[:, 1][:, None] - B[:, 1][None, :]
        return (i == ib) & (i >= 0), i

    def observables(self):
        """(Tr rho, <n_j>, <n_j^2>) with moments divided by Tr rho.

        Left trace environment E_0 = lambda_0, E_{j+1}(b) = sum_a E_j(a) Gamma_j[a, b]
        lambda_{j+1}(b) over entries whose ket and bra local photon numbers agree;
        right environment F_M = 1, F_j(a) = sum_b Gamma_j[a, b] lambda_{j+1}(b) F_{j+1}(b);
        <n_j^p> = sum_{a,b} E_j(a) Gamma_j[a, b] i^p lambda_{j+1}(b) F_{j+1}(b) / Tr."""
        M = self.M
        E = [None] * (M + 1)
        E[0] = self.lam[0].astype(np.complex128)
        masks = [self._diag_mask(j) for j in range(M)]
        for j in range(M):
            mk, _ = masks[j]
            E[j + 1] = (E[j] @ (self.gam[j] * mk)) * self.lam[j + 1]
        F = [None] * (M + 1)
        F[M] = np.ones(self.lam[M].shape[0], dtype=np.complex128)
        for j in range(M - 1, -1, -1):
            mk, _ = masks[j]
            F[j] = (self.gam[j] * mk) @ (self.lam[j + 1] * F[j + 1])
        tr = complex(E[M].sum())
        n1 = np.zeros(M); n2 = np.zeros(M)
        for j in range(M):
            mk, i = masks[j]
            core = self.gam[j] * mk
            rgt = self.lam[j + 1] * F[j + 1]
            n1[j] = (E[j] @ (core * i) @ rgt).real / tr.real
            n2[j] = (E[j] @ (core * i * i) @ rgt).real / tr.real
        return tr.real, n1, n2

    def purities(self) -> np.ndarray:
        return np.array([float(np.sum(l ** 2)) for l in self.lam])

    # ----------------------------------------------------- dense rebuild (tiny)
    def to_dense(self) -> np.ndarray:
        """vec(rho) rebuilt as a d^M x d^M matrix (only for a few modes)."""
        M, d = self.M, self.d
        # T[ket_prefix, bra_prefix, bond]
        T = self.lam[0][None, None, :].astype(np.complex128)
        for j in range(M):
            A, B = self.charges[j], self.charges[j + 1]
            nk, nb = T.shape[0], T.shape[1]
            NT = np.zeros((nk * d, nb * d, B.shape[0]), dtype=np.complex128)
            for i in range(d):
                for ib in range(d):
                    sel = ((A[:, 0][:, None] - B[:, 0][None, :]) == i) & \
                          ((A[:, 1][:, None] - B[:, 1][None, :]) == ib)
                    core = self.gam[j] * sel * self.lam[j + 1][None, :]
                    part = np.tensordot(T, core, axes=([2], [0]))
                    NT[i::d, ib::d, :] += part
            T = NT
        return T[:, :, 0]
