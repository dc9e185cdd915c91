"""FP64 CPU oracle for the lossy-GBS U(1) MPO mesh.  TEST INFRASTRUCTURE ONLY.

Only `tests/`, `__graft_entry__.smoke()` and the `cpu_baseline` / reference leg of
`bench.py` may import anything from this package.  The CUDA library never calls
it, and it never calls the CUDA library: the two share no code.  The only module
both sides import is `gbs_workloads` (seeded inputs, no method arithmetic).

Contents (paper: Liu et al., "Simulating lossy Gaussian boson sampling with
matrix product operators", arXiv:2301.12814):

* `fock`   -- single-mode squeezed amplitudes (App. C), pure-loss Kraus channel
              (App. B, Kraus equations), two-mode Fock elements of a beam splitter
              (App. B, Eq. `kun` is its single-input special case).
* `dense`  -- O1: brute-force dense density matrix for a few modes, and the
              U(1)-form operator entanglement defined from it.
* `u1mpo`  -- O2: the U(1)-symmetric vectorised MPO of App. D written out in
              plain loops over charges (Eq. `theta`, the block SVD and the keep-chi
              rule, the Vidal re-split), plus the canonical initial state and the
              trace-environment observables.

Every number here is float64 / complex128.  Every function is pinned by a
`-m "not gpu"` test against an independent fact (closed forms, a library routine
on a special case, brute force); none is "parity unpinned".
"""
