"""Seeded synthetic inputs for the lossy-GBS MPO mesh (shared by the CUDA path and the oracle).

This module holds no arithmetic of the MPO method itself. It only produces the
inputs both sides consume:

* a Haar-random M x M unitary drawn from a seed (complex Ginibre matrix, QR,
  phases of diag(R) divided out, Mezzadri 2007);
* its Clements decomposition (Clements et al., Optica 3, 1460 (2016)) into an
  ordered list of nearest-neighbour beam splitters (mode k, theta, phi) and a
  final diagonal phase screen;
* the workload recipes (M, d, chi, r, eta, seeds) of the five standard workloads
  and the per-instance draws of the batched one;
* a greedy layering of the gate list into layers of gates on disjoint mode pairs;
* a direct-dialled rectangular mesh (Russell et al., New J. Phys. 19, 033007 (2017)):
  the same M-layer layout with every beam-splitter angle and phase drawn
  independently from position-dependent laws that make the product Haar-random,
  with no matrix drawn or decomposed;
* the parameter grid of the asymptotic-entanglement sweep (Results, Fig. 1): numbers
  N of squeezed inputs, surviving-photon prefactors beta and exponents gamma.

The paper builds its interferometers as Haar-random global unitaries realised by
an M-layer nearest-neighbour array (Appendix A); the decomposition used here is
the Clements rectangular mesh, whose depth is also M layers.

Conventions. A gate T(k; theta, phi) acts on modes (k, k+1) (0-based) through the
2 x 2 block  [[e^{i phi} cos theta, -sin theta], [e^{i phi} sin theta, cos theta]],
i.e. a_k^dag -> t_00 a_k^dag + t_10 a_{k+1}^dag and a_{k+1}^dag -> t_01 a_k^dag +
t_11 a_{k+1}^dag.  The list is in application order: U = D T_L ... T_2 T_1.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

__all__ = [
    "haar_unitary", "clements", "mesh_unitary", "gate_block", "Mesh",
    "Workload", "workload", "WORKLOADS", "layer_schedule", "batched_instances", "AsymptoticGrid",
    "asymptotic_grid", "elimination_steps", "dialled_mesh",
]


def haar_unitary(M: int, seed: int) -> np.ndarray:
    """Haar-random unitary from numpy's default_rng(seed) (Ginibre -> QR -> phase fix)."""
    rng = np.random.default_rng(seed)
    z = (rng.standard_normal((M, M)) + 1j * rng.standard_normal((M, M))) / math.sqrt(2.0)
    q, r = np.linalg.qr(z)
    ph = np.diag(r) / np.abs(np.diag(r))
    return q * ph[None, :]


def gate_block(theta: float, phi: float) -> np.ndarray:
    """The 2 x 2 mode matrix of one mesh gate (the Clements T block)."""
    c, s, e = math.cos(theta), math.sin(theta), complex(math.cos(phi), math.sin(phi))
    return np.array([[e * c, -s], [e * s, c]], dtype=np.complex128)


def _embed(M: int, k: int, t: np.ndarray) -> np.ndarray:
    T = np.eye(M, dtype=np.complex128)
    T[k:k + 2, k:k + 2] = t
    return T


@dataclasses.dataclass
class Mesh:
    """An ordered nearest-neighbour mesh: gates[i] = (k, theta, phi); final phases D."""
    M: int
    k: np.ndarray          # int32 [L]
    theta: np.ndarray      # float64 [L]
    phi: np.ndarray        # float64 [L]
    final_phase: np.ndarray  # float64 [M]

    @property
    def n_gates(self) -> int:
        return int(self.k.shape[0])


def _null_by_column(U: np.ndarray, row: int, n: int) -> Tuple[float, float]:
    """(theta, phi) such that (U T_n^{-1})[row, n] = 0."""
    x, y = U[row, n], U[row, n + 1]
    if abs(y) == 0.0:
        return (math.pi / 2, 0.0) if abs(x) > 0 else (0.0, 0.0)
    theta = math.atan2(abs(x), abs(y))
    phi = math.atan2((x / y).imag, (x / y).real) if abs(x) > 0 else 0.0
    return theta, phi


def _null_by_row(U: np.ndarray, n: int, col: int) -> Tuple[float, float]:
    """(theta, phi) such that (T_n U)[n + 1, col] = 0."""
    x, y = U[n, col], U[n + 1, col]
    if abs(x) == 0.0:
        return (math.pi / 2, 0.0) if abs(y) > 0 else (0.0, 0.0)
    theta = math.atan2(abs(y), abs(x))
    z = -y / x
    phi = math.atan2(z.imag, z.real) if abs(y) > 0 else 0.0
    return theta, phi


def clements(U: np.ndarray) -> Mesh:
    """Decompose U = D T_L ... T_1 into M(M-1)/2 nearest-neighbour gates.

    Elements below the anti-diagonal are nulled alternately by column
    operations (right multiplication by T^{-1}) and row operations (left
    multiplication by T), which leaves a diagonal D'.  Each left factor T^{-1}
    is then moved through the diagonal with  T^{-1}(theta, phi) diag(d1, d2) =
    diag(-e^{-i phi} d2, d2) T(theta, phi')  with  e^{i phi'} = -d1/d2.
    """
    U = np.array(U, dtype=np.complex128)
    N = U.shape[0]
    right: List[Tuple[int, float, float]] = []
    left: List[Tuple[int, float, float]] = []
    W = U.copy()
    for i in range(N - 1):
        if i % 2 == 0:
            for j in range(i + 1):
                n, row = i - j, N - 1 - j
                th, ph = _null_by_column(W, row, n)
                W = W @ _embed(N, n, gate_block(th, ph)).conj().T
                right.append((n, th, ph))
        else:
            for j in range(1, i + 2):
                n, col = N + j - i - 3, j - 1
                th, ph = _null_by_row(W, n, col)
                W = _embed(N, n, gate_block(th, ph)) @ W
                left.append((n, th, ph))
    d = np.diag(W).copy()
    moved: List[Tuple[int, float, float]] = []
    for (n, th, ph) in reversed(left):
        d1, d2 = d[n], d[n + 1]
        z = -d1 / d2
        moved.append((n, th, math.atan2(z.imag, z.real)))
        d[n] = -complex(math.cos(ph), -math.sin(ph)) * d2
    # U = D * moved[0] ... moved[-1] * right[-1] ... right[0]; right[0] acts first
    order = list(right) + list(moved)
    k = np.array([g[0] for g in order], dtype=np.int32)
    theta = np.array([g[1] for g in order], dtype=np.float64)
    phi = np.array([g[2] for g in order], dtype=np.float64)
    return Mesh(N, k, theta, phi, np.angle(d).astype(np.float64))


def elimination_steps(N: int) -> List[Tuple[int, str, int, int]]:
    """(mode n, side, diagonal i, position p) of every nulling step of ``clements`` in
    its order: side 'R' = column operation (right factor), 'L' = row operation."""
    steps = []
    for i in range(N - 1):
        if i % 2 == 0:
            for j in range(i + 1):
                steps.append((i - j, "R", i, j))
        else:
            for j in range(1, i + 2):
                steps.append((N + j - i - 3, "L", i, j - 1))
    return steps


def dialled_mesh(M: int, seed: int) -> Mesh:
    """A Haar-random M-layer rectangular mesh dialled gate by gate.

    For a Haar-random U the nulling step at position p of diagonal i of ``clements``
    has sin^2(theta) ~ Beta(a, 1) with a = min(2p + 1, 2(i + 1 - p)), independently of
    every other step, and every phase (gate phases, final screen) is uniform on
    [0, 2 pi).  So theta = asin(xi^(1 / 2a)) with xi uniform on [0, 1] (the inverse of
    the Beta(a, 1) CDF x^a).  The gates come out in ``clements``' layout and order, so
    the mesh is interchangeable with ``clements(haar_unitary(M, seed))``.  Draws
    (numpy default_rng(seed)): per step in elimination order xi then phi, then the M
    final phases."""
    rng = np.random.default_rng(seed)
    right: List[Tuple[int, float, float]] = []
    left: List[Tuple[int, float, float]] = []
    for n, side, i, p in elimination_steps(M):
        a = min(2 * p + 1, 2 * (i + 1 - p))
        xi = rng.uniform()
        th = math.asin(min(1.0, xi ** (1.0 / (2 * a))))
        ph = rng.uniform(0.0, 2 * math.pi)
        (right if side == "R" else left).append((n, th, ph))
    order = right + list(reversed(left))
    final = rng.uniform(0.0, 2 * math.pi, M)
    return Mesh(M, np.array([g[0] for g in order], dtype=np.int32), np.array([g[1] for g in order]),
                np.array([g[2] for g in order]), final)


def mesh_unitary(mesh: Mesh) -> np.ndarray:
    """Rebuild D T_L ... T_1 from a mesh (used to check a decomposition)."""
    V = np.eye(mesh.M, dtype=np.complex128)
    for k, th, ph in zip(mesh.k, mesh.theta, mesh.phi):
        V = _embed(mesh.M, int(k), gate_block(float(th), float(ph))) @ V
    return np.diag(np.exp(1j * mesh.final_phase)) @ V


def layer_schedule(k: Sequence[int], M: int) -> np.ndarray:
    """Greedy layering: each gate goes to the first layer after the last one using
    either of its modes.  Gates of one layer act on disjoint pairs and commute."""
    last = np.full(M, -1, dtype=np.int64)
    layer = np.zeros(len(k), dtype=np.int32)
    for i, kk in enumerate(k):
        l = max(last[kk], last[kk + 1]) + 1
        layer[i] = l
        last[kk] = last[kk + 1] = l
    return layer


@dataclasses.dataclass
class Workload:
    """One synthetic instance family: M modes, cutoff d, bond cap chi (None = no cap)."""
    name: str
    M: int
    d: int
    chi: Optional[int]
    r: np.ndarray        # [batch, M]
    eta: np.ndarray      # [batch, M]
    seeds: List[int]
    chis: List[Optional[int]]
    precision: str = "fp64"

    @property
    def batch(self) -> int:
        return len(self.seeds)

    @property
    def n_cap(self) -> int:
        return self.d - 1

    def mesh(self, i: int = 0, dialled: bool = False) -> Mesh:
        """Instance i's mesh: the Clements decomposition of haar_unitary(M, seed), or
        with ``dialled`` the direct-dialled mesh of the same seed (another unitary)."""
        if dialled:
            return dialled_mesh(self.M, self.seeds[i])
        return clements(haar_unitary(self.M, self.seeds[i]))

    def unitary(self, i: int = 0) -> np.ndarray:
        return haar_unitary(self.M, self.seeds[i])


def _uniform(name, M, d, chi, r, eta, seed, precision="fp64") -> Workload:
    return Workload(name, M, d, chi, np.full((1, M), r), np.full((1, M), eta), [seed], [chi],
                    precision)


def batched_instances(n: int = 64, M: int = 16, d: int = 6, first_seed: int = 100) -> Workload:
    """The batched workload: per instance seed s, default_rng(s) first draws the
    Haar unitary (inside haar_unitary), then a separate default_rng(s + 10**6)
    draws r ~ U[0.5, 1.2], eta ~ U[0.1, 0.5] and chi from {32, 64, 96, 128}."""
    seeds = list(range(first_seed, first_seed + n))
    r = np.zeros((n, M)); eta = np.zeros((n, M)); chis = []
    for i, s in enumerate(seeds):
        rng = np.random.default_rng(s + 10 ** 6)
        r[i, :] = rng.uniform(0.5, 1.2)
        eta[i, :] = rng.uniform(0.1, 0.5)
        chis.append(int(rng.choice([32, 64, 96, 128])))
    return Workload("batched_64x_M16_d6", M, d, max(chis), r, eta, seeds, chis, "mixed_tf32")


def _sqrt_n_eta(M: int, r: float) -> float:
    n_in = M * math.sinh(r) ** 2
    return 1.0 / math.sqrt(n_in)


def workload(name: str) -> Workload:
    return WORKLOADS[name]()


WORKLOADS = {
    # exact, no truncation, checked against the dense density matrix
    "exact_M4_d4": lambda: _uniform("exact_M4_d4", 4, 4, None, 0.5, 0.5, 0),
    # dense FP64 on the GPU against the oracle
    "M16_d6_chi64": lambda: _uniform("M16_d6_chi64", 16, 6, 64, 0.8, 0.3, 1),
    # U(1) block-sparse, precision form
    "M32_d8_chi256": lambda: _uniform("M32_d8_chi256", 32, 8, 256, 1.0, 0.2, 2, "mixed_tf32"),
    # batched form
    "batched_64x_M16_d6": lambda: batched_instances(),
    # sqrt(N) loss sweep point
    "M48_d8_chi512": lambda: _uniform("M48_d8_chi512", 48, 8, 512, 0.9, _sqrt_n_eta(48, 0.9), 3,
                                      "mixed_bf16"),
}


@dataclasses.dataclass
class AsymptoticGrid:
    """Flattened (N, beta, gamma) points of the asymptotic sweep at squeezing r and
    photon cutoff n_max."""
    name: str
    N: np.ndarray
    beta: np.ndarray
    gamma: np.ndarray
    r: float
    n_max: int

    @property
    def size(self) -> int:
        return int(self.N.size)


def asymptotic_grid(n_N: int = 64, N_min: float = 10.0, N_max: float = 1e5, n_max: int = 8) -> AsymptoticGrid:
    """Fig. 1's sweep: N_out = beta N^gamma surviving photons for gamma = 1/4, 1/2, 1
    and beta = 0.25, 0.5, 0.75, 1 (a linear trend in beta is what the figure shows),
    N at n_N log-spaced values in [N_min, N_max] (rounded to integers), r = 0.88 (about
    one photon per squeezed mode), n_max = 8."""
    Ns = np.unique(np.round(np.logspace(math.log10(N_min), math.log10(N_max), n_N)))
    g, b, n = np.meshgrid([0.25, 0.5, 1.0], [0.25, 0.5, 0.75, 1.0], Ns, indexing="ij")
    return AsymptoticGrid(f"asymptotic_fig1_{Ns.size}N", n.ravel(), b.ravel(), g.ravel(), 0.88, n_max)
