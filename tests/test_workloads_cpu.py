"""The seeded input generators (gbs_workloads): the Clements decomposition and the
direct-dialled Haar mesh.

The dialled mesh draws each angle from a position-dependent Beta law; these tests
check its product against what Haar measure fixes independently of any
decomposition: E|U_ij|^2 = 1/M, E|U_ij|^4 = 2/(M(M+1)), |U_ij|^2 ~ Beta(1, M-1),
E|Tr U|^2 = 1 and E|Tr U|^4 = 2 (M >= 2), and the law of |Tr U|^2 against
QR-sampled Haar unitaries.  A mesh with uniform angles fails the same checks."""
import math

import numpy as np
import pytest

import gbs_workloads as w

stats = pytest.importorskip("scipy.stats")


@pytest.mark.parametrize("M", [2, 3, 4, 7, 10])
def test_clements_round_trip(M):
    U = w.haar_unitary(M, 11 * M)
    m = w.clements(U)
    assert m.n_gates == M * (M - 1) // 2
    assert np.allclose(w.mesh_unitary(m), U, atol=1e-12)
    assert w.layer_schedule(m.k, M).max() + 1 <= M  # an M-layer array


@pytest.mark.parametrize("M", [2, 3, 4, 5, 8, 9])
def test_dialled_layout_and_round_trip(M):
    d = w.dialled_mesh(M, 3)
    assert np.array_equal(d.k, w.clements(w.haar_unitary(M, 0)).k)
    assert np.all((d.theta >= 0) & (d.theta <= math.pi / 2))
    # decomposing the dialled unitary returns the dialled angles in place
    back = w.clements(w.mesh_unitary(d))
    assert np.allclose(back.theta, d.theta, atol=1e-9)
    assert np.allclose(w.mesh_unitary(back), w.mesh_unitary(d), atol=1e-12)


def _haar_checks(Us, M):
    n = len(Us)
    a2 = np.array([np.abs(U) ** 2 for U in Us])           # [n, M, M]
    tr2 = np.array([abs(np.trace(U)) ** 2 for U in Us])
    fails = []
    se = lambda x: x.std() / math.sqrt(n)
    m1 = a2.mean(axis=0)
    if np.max(np.abs(m1 - 1.0 / M)) > 5 * se(a2[:, 0, 0]):
        fails.append("E|U|^2")
    m2 = (a2 ** 2).mean(axis=0)
    if np.max(np.abs(m2 - 2.0 / (M * (M + 1)))) > 5 * se(a2[:, 0, 0] ** 2):
        fails.append("E|U|^4")
    if abs(tr2.mean() - 1.0) > 5 * se(tr2):
        fails.append("E|Tr U|^2")
    if abs((tr2 ** 2).mean() - 2.0) > 5 * se(tr2 ** 2):
        fails.append("E|Tr U|^4")
    for (i, j) in [(0, 0), (M - 1, 0), (M // 2, M - 1)]:
        if stats.kstest(a2[:, i, j], stats.beta(1, M - 1).cdf).pvalue < 1e-4:
            fails.append(f"KS |U_{i}{j}|^2")
    return fails, tr2


def test_dialled_mesh_is_haar():
    M, n = 5, 4000
    Us = [w.mesh_unitary(w.dialled_mesh(M, 10_000 + s)) for s in range(n)]
    fails, tr2 = _haar_checks(Us, M)
    assert not fails, fails
    ref = np.array([abs(np.trace(w.haar_unitary(M, 50_000 + s))) ** 2 for s in range(n)])
    assert stats.ks_2samp(tr2, ref).pvalue > 1e-4


def test_uniform_angles_are_not_haar():
    """The checks have power: uniform theta instead of the Beta laws is rejected."""
    M, n = 5, 4000
    Us = []
    for s in range(n):
        d = w.dialled_mesh(M, 20_000 + s)
        rng = np.random.default_rng(s)
        d.theta = rng.uniform(0.0, math.pi / 2, d.n_gates)
        Us.append(w.mesh_unitary(d))
    fails, _ = _haar_checks(Us, M)
    assert fails
