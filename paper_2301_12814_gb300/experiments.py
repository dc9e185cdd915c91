"""Two run protocols of the paper's experiments (App. A), driven over the C ABI.

Every gate still runs in the library's kernels; this module only decides how far to
run and with which bond dimension.

* ``ee_over_depth``: apply the mesh layer by layer and record, after each layer, the
  largest operator entanglement over the cuts between modes; stop once the running
  maximum has not increased for ``patience`` layers (App. A: simulate until there is no
  MPO EE increase for at least 10 layers; only the maximum over depth matters).
* ``bond_dimension_search``: run the full mesh with a small bond dimension and double
  it while the truncation error 1 - Tr rho exceeds the target (App. A: start small,
  double while the error exceeds 0.02), then narrow the bracket by bisection a few
  more times (App. A: the bond dimension is refined a few more times).
* ``choose_d``: the smallest local dimension d whose initial state loses less than a
  threshold of the probability to the truncation (App. A: d is chosen so that under
  1 % is truncated; the left-most charge is the total photon number, so the cap
  n_cap = d - 1 on that total is what binds, and d grows with r and with the number
  of squeezed inputs).  The input state is cut generously (32 photons per mode)
  before loss, so the cap is the binding cut.
* ``truncation_curve`` / ``fig4b``: 1 - Tr rho after the full mesh against the bond
  dimension, every chi of the curve as one instance of a single batched handle (Fig.
  4(b): (M, mu) = (10, 0.2), (15, 0.15), (20, 0.1), every mode squeezed at r = 0.88
  so that mu M ~ 2 photons survive; d by the 1 % rule; a dialled M-layer mesh).
* ``asymptotic_ee`` / ``n_max_convergence``: the App. C estimate N S(mu = beta N^gamma / N)
  behind Fig. 1 (EE against the number N of squeezed inputs for surviving photons
  N_out = beta N^gamma, r = 0.88, n_max = 8) and its convergence in the photon cutoff
  (Fig. 1(d): N = 50, beta = 1, gamma = 1/2).
"""
from __future__ import annotations

import math
from typing import Dict, List, Optional, Sequence

import numpy as np

from . import mpo as _mpo


def plateau_stop(values: Sequence[float], patience: int) -> Optional[int]:
    """Index of the layer after which a run stops: the first layer whose running
    maximum has not strictly increased for ``patience`` consecutive layers (None if
    that never happens)."""
    best = -np.inf
    since = 0
    for i, v in enumerate(values):
        if v > best:
            best = v
            since = 0
        else:
            since += 1
            if since >= patience:
                return i
    return None


def _layers(layer_of: Sequence[int]) -> List[np.ndarray]:
    layer_of = np.asarray(layer_of)
    return [np.nonzero(layer_of == l)[0] for l in range(int(layer_of.max()) + 1)] if layer_of.size else []


def ee_over_depth(M: int, d: int, r, eta, chi: Optional[int], k: Sequence[int], theta: Sequence[float],
                  phi: Sequence[float], layer_of: Sequence[int], patience: int = 10,
                  precision: str = "fp64", n_cap: Optional[int] = None) -> Dict[str, object]:
    """Apply the gates layer by layer (``layer_of[g]`` = layer of gate g; gates of one
    layer act on disjoint mode pairs) and stop by the App. A rule.

    Returns ``{"max_ee": [largest S over the cuts 1..M-1 after each simulated layer],
    "layers": simulated layers, "stopped": whether the rule fired, "max_over_depth":
    the largest of them, "trace": Tr rho at the end}``."""
    k = np.asarray(k, dtype=np.int32)
    theta = np.asarray(theta, dtype=np.float64)
    phi = np.asarray(phi, dtype=np.float64)
    G = _mpo.MPO(M, d, r, eta, chi_max=chi, precision=precision, n_cap=n_cap)
    try:
        max_ee: List[float] = []
        stopped = False
        for idx in _layers(layer_of):
            if idx.size:
                G.sweep_mesh([idx.size], k[idx], theta[idx], phi[idx])
            S = G.operator_entropy()[0][0]
            max_ee.append(float(np.max(S[1:M])))
            if plateau_stop(max_ee, patience) is not None:
                stopped = True
                break
        tr = G.observables(normalize=False)[0][0]
    finally:
        G.close()
    return {"max_ee": max_ee, "layers": len(max_ee), "stopped": stopped,
            "max_over_depth": max(max_ee) if max_ee else 0.0, "trace": float(tr)}


def _truncation_error(M, d, r, eta, chi, k, theta, phi, final_phase, precision, n_cap=None) -> float:
    G = _mpo.MPO(M, d, r, eta, chi_max=chi, precision=precision, n_cap=n_cap)
    try:
        G.sweep_mesh([len(k)], k, theta, phi, final_phase)
        return float(1.0 - G.observables(normalize=False)[0][0])
    finally:
        G.close()


def bond_dimension_search(M: int, d: int, r, eta, k: Sequence[int], theta: Sequence[float],
                          phi: Sequence[float], final_phase=None, chi0: int = 8, target: float = 0.02,
                          refine: int = 3, chi_limit: int = 4096, precision: str = "fp64",
                          n_cap: Optional[int] = None) -> Dict[str, object]:
    """The smallest bond dimension found whose full-mesh truncation error 1 - Tr rho is
    at most ``target``: double from ``chi0`` until the error is within the target, then
    bisect the last bracket ``refine`` times.  Returns ``{"chi": ..., "error": ...,
    "visited": [(chi, error), ...]}`` (``chi`` is None if ``chi_limit`` is reached)."""
    k = np.asarray(k, dtype=np.int32)
    theta = np.asarray(theta, dtype=np.float64)
    phi = np.asarray(phi, dtype=np.float64)
    visited = []

    def err(chi):
        e = _truncation_error(M, d, r, eta, chi, k, theta, phi, final_phase, precision, n_cap)
        visited.append((chi, e))
        return e

    chi = chi0
    e = err(chi)
    while e > target:
        if chi >= chi_limit:
            return {"chi": None, "error": e, "visited": visited}
        chi = min(2 * chi, chi_limit)
        e = err(chi)
    lo, hi, e_hi = chi // 2, chi, e  # error(lo) > target (or lo below chi0), error(hi) <= target
    if chi == chi0:
        lo = 0
    for _ in range(refine):
        if hi - lo <= 1:
            break
        mid = (lo + hi) // 2
        e_mid = err(mid)
        if e_mid <= target:
            hi, e_hi = mid, e_mid
        else:
            lo = mid
    return {"chi": hi, "error": e_hi, "visited": visited}


def truncation_curve(M: int, d: int, r, eta, k: Sequence[int], theta: Sequence[float], phi: Sequence[float],
                     final_phase=None, chis: Sequence[int] = (8, 16, 32, 64, 128), precision: str = "fp64",
                     n_cap: Optional[int] = None) -> List[tuple]:
    """[(chi, 1 - Tr rho)] after the whole mesh for every chi in ``chis``; the curve is
    one batched run (instance i capped at chis[i], all on the same mesh)."""
    chis = [int(c) for c in chis]
    B = len(chis)
    k = np.tile(np.asarray(k, dtype=np.int32), B)
    th = np.tile(np.asarray(theta, dtype=np.float64), B)
    ph = np.tile(np.asarray(phi, dtype=np.float64), B)
    fp = None if final_phase is None else np.tile(np.asarray(final_phase, dtype=np.float64), B)
    n = len(k) // B
    G = _mpo.MPO(M, d, r, eta, chi_max=chis, batch=B, precision=precision, n_cap=n_cap)
    try:
        G.sweep_mesh([n] * B, k, th, ph, fp)
        tr = G.observables(normalize=False)[0]
    finally:
        G.close()
    return [(c, float(1.0 - t)) for c, t in zip(chis, tr)]


FIG4B = ((10, 0.2), (15, 0.15), (20, 0.1))


def fig4b(seed: int = 0, r: float = 0.88, chi_max: int = 256, target: float = 0.02, refine: int = 3,
          precision: str = "fp64", report=None) -> List[Dict[str, object]]:
    """Fig. 4(b)'s three configurations on the dialled M-layer mesh of ``seed``: d by the
    1 % rule, then App. A's chi search done as two batched runs -- the doubling phase
    (chi = 8, 16, ..., chi_max in one handle) and the refinement (``refine`` evenly
    spaced chi inside the first bracket that meets ``target``, in a second handle).
    ``report`` (callable or None) receives each configuration's result when done."""
    import gbs_workloads as w
    out = []
    for M, mu in FIG4B:
        rr, ee = [r] * M, [mu] * M
        dsel = choose_d(M, rr, ee)
        if dsel["d"] is None:
            raise ValueError(f"no d <= 16 truncates under 1% at M = {M}")
        d, d_in, cap = dsel["d"], dsel["d_in"], dsel["n_cap"]
        mesh = w.dialled_mesh(M, seed)
        run = lambda chis: truncation_curve(M, d_in, rr, ee, mesh.k, mesh.theta, mesh.phi, mesh.final_phase,
                                            chis, precision, n_cap=cap)
        doubling = [8]
        while doubling[-1] * 2 <= chi_max:
            doubling.append(doubling[-1] * 2)
        curve = run(doubling)
        hit = next((i for i, (_, e) in enumerate(curve) if e <= target), None)
        chi_t, err_t, refined = None, None, []
        if hit is not None:
            chi_t, err_t = curve[hit]
            lo = curve[hit - 1][0] if hit > 0 else 0
            step = (chi_t - lo) / (refine + 1)
            mids = sorted({int(round(lo + step * (i + 1))) for i in range(refine)} - {lo, chi_t} - {0})
            if mids:
                refined = run(mids)
                for c, e in refined:
                    if e <= target and c < chi_t:
                        chi_t, err_t = c, e
                        break
        res = {"M": M, "mu": mu, "d": d, "n_cap": cap, "d_in": d_in, "truncated": dsel["tail"], "curve": curve,
               "refined": refined, "chi_for_target": chi_t, "error_at_chi": err_t}
        if report is not None:
            report(res)
        out.append(res)
    return out


D_IN = 32  # input cutoff per mode (photons before loss) for the App. A choice of d; MPO_D_LOCAL_MAX


def choose_d(M: int, r, eta, threshold: float = 0.01, d_min: int = 2, d_max: int = 16,
             d_in: int = D_IN) -> Dict[str, object]:
    """App. A's choice of d: the smallest local dimension d whose cap on the total
    photon number, n_cap = d - 1 (the left-most charge), leaves less than ``threshold``
    of the probability truncated.  Each mode's squeezed vacuum is cut at ``d_in``
    photons before loss, so the cap is the binding truncation; the reported tail
    (``MPO.truncated_probability``, computed by the kernels) includes both cuts.  The
    kept set only grows with d, so the first hit is the smallest.  A run then uses
    ``MPO(M, d_in, r, eta, n_cap=d - 1)``.  Returns ``{"d", "n_cap", "d_in", "tail",
    "visited": [(d, tail), ...]}`` (``d`` is None if d_max is not enough)."""
    visited = []
    for d in range(int(d_min), int(d_max) + 1):
        G = _mpo.MPO(M, d_in, r, eta, chi_max=1, n_cap=d - 1)
        try:
            tail = float(G.truncated_probability()[0])
        finally:
            G.close()
        visited.append((d, tail))
        if tail < threshold:
            return {"d": d, "n_cap": d - 1, "d_in": d_in, "tail": tail, "visited": visited}
    return {"d": None, "n_cap": None, "d_in": d_in, "tail": visited[-1][1] if visited else None,
            "visited": visited}


def transmission(N, beta, gamma) -> np.ndarray:
    """mu = beta N^gamma / N: the transmission that leaves N_out = beta N^gamma of the
    N input photons (Results)."""
    N, beta, gamma = np.broadcast_arrays(np.asarray(N, dtype=np.float64), np.asarray(beta, dtype=np.float64),
                                         np.asarray(gamma, dtype=np.float64))
    mu = beta * N ** gamma / N
    if np.any(mu > 1.0) or np.any(mu < 0.0):
        raise ValueError("beta N^gamma / N must lie in [0, 1]")
    return mu


def asymptotic_ee(N, beta, gamma, r: float = 0.88, n_max: int = 8, alpha: Optional[float] = None) -> Dict[str, np.ndarray]:
    """App. C estimate of the system's operator EE for every (N, beta, gamma) of the
    broadcast inputs: mu = beta N^gamma / N, theta = pi / 4, S_system = N S_mode.
    Returns ``{"mu": ..., "S1": ..., "S_alpha": ... or None}`` with the inputs' shape.
    Every mode entropy is computed by the library's kernels in one batch."""
    mu = transmission(N, beta, gamma)
    N = np.broadcast_to(np.asarray(N, dtype=np.float64), mu.shape)
    res = _mpo.asymptotic_ee(np.full(mu.size, float(r)), mu.ravel(), np.full(mu.size, math.pi / 4), n_max, alpha)
    out = {"mu": mu, "S1": (N.ravel() * res["S1"]).reshape(mu.shape), "S_alpha": None}
    if alpha is not None:
        out["S_alpha"] = (N.ravel() * res["S_alpha"]).reshape(mu.shape)
    return out


def n_max_convergence(N: int = 50, beta: float = 1.0, gamma: float = 0.5, r: float = 0.88,
                      n_maxes: Sequence[int] = tuple(range(2, 17))) -> List[tuple]:
    """[(n_max, N S)] for increasing photon cutoffs (Fig. 1(d))."""
    return [(int(n), float(asymptotic_ee(N, beta, gamma, r, int(n))["S1"])) for n in n_maxes]


if __name__ == "__main__":
    import json
    import sys
    import time
    from . import build as _build
    _mpo.load_library(_build.build())
    if len(sys.argv) > 1 and sys.argv[1] == "fig4b":
        t0 = time.perf_counter()
        seed = int(sys.argv[2]) if len(sys.argv) > 2 else 0
        chi_max = int(sys.argv[3]) if len(sys.argv) > 3 else 256
        fig4b(seed=seed, chi_max=chi_max,
              report=lambda res: print(json.dumps(dict(res, seconds=time.perf_counter() - t0)), flush=True))
    else:
        print("usage: python -m paper_2301_12814_gb300.experiments fig4b [seed]")
