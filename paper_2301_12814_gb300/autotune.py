"""Autotuner of a handle's launch choices (mpo_tuning) for one workload.

The choices -- contraction form, the Gram side from which Gram matrices run on the
tensor cores, the SVD kernel's cluster size, and which blocks go to a cluster -- change
how a layer's work is spread over the GPU, not what is computed.  The best set depends
on the workload: many small instances (the batched form) keep every block on single
CTAs, a few large ones want clusters for their critical blocks.

`autotune` captures the workload's mesh as a plan under each candidate set, replays it
and keeps the fastest.  Time = the summed device time of the replay's stages, from the
event nodes inside the plan's graph (mpo_plan_stage_times), best of `reps` replays
after one warm-up replay; the state is reset before each replay.  The search is a plain
grid over a small space (at most a few dozen candidates); every candidate runs the same
mesh from the same initial state.  The chosen set stays installed on the handle and is
returned with the whole table, so a benchmark can record it; the handle is reset to
its initial state before `autotune` returns.
"""
from __future__ import annotations

import itertools
from typing import Dict, Iterable, List, Optional

NEVER = 1 << 20  # a Gram side no block reaches


def default_space(precision: str) -> Dict[str, List[int]]:
    """Candidate values per choice.  The FP64 path has one contraction form."""
    space = {
        "svd_cluster_size": [2, 4, 8],
        "svd_cluster_min_n": [0, -1],
        "gram_tc_min": [48, NEVER],
    }
    if precision != "fp64":
        space["theta_form"] = [1, 2]
    return space


def _candidates(space: Dict[str, Iterable[int]]):
    keys = sorted(space)
    for vals in itertools.product(*(list(space[k]) for k in keys)):
        cand = dict(zip(keys, vals))
        # without clusters the cluster size is moot: keep one representative
        if cand.get("svd_cluster_min_n", 0) < 0 and cand.get("svd_cluster_size", 4) != 4:
            continue
        yield cand


def autotune(G, n_gates, k, theta, phi, final_phase=None, precision: str = "fp64",
             space: Optional[Dict[str, Iterable[int]]] = None, reps: int = 2) -> dict:
    """Time the mesh under each candidate set of launch choices on handle G and
    install the fastest.  Returns {"best": choices, "best_ms": ms per mesh,
    "default_ms": ms under the defaults, "table": [(ms, choices), ...]}."""
    space = default_space(precision) if space is None else space
    table = []

    def time_plan() -> float:
        plan = G.plan_mesh(n_gates, k, theta, phi, final_phase)
        try:
            G.reset()
            plan.run()
            best = float("inf")
            for _ in range(max(1, reps)):
                G.reset()
                plan.run()
                best = min(best, sum(plan.stage_times().values()))
            return best
        finally:
            plan.close()

    base = G.get_tuning()
    default_ms = time_plan()
    for cand in _candidates(space):
        G.set_tuning(**{**base, **cand})
        table.append((time_plan(), dict(cand)))
    table.sort(key=lambda t: t[0])
    G.reset()  # every candidate ran the mesh: back to the initial state
    best_ms, best = table[0]
    if best_ms < default_ms:
        G.set_tuning(**{**base, **best})
        chosen = G.get_tuning()
    else:  # the defaults were at least as fast
        G.set_tuning(**base)
        chosen, best_ms = G.get_tuning(), default_ms
    return {"best": chosen, "best_ms": best_ms, "default_ms": default_ms,
            "table": table}
