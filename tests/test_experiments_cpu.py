"""The App. A stopping rule of the depth protocol, as host logic (no GPU)."""


def _plateau_stop():
    import paper_2301_12814_gb300.experiments as ex  # importing the package needs no GPU
    return ex.plateau_stop


def test_plateau_stop_rule():
    stop = _plateau_stop()
    # rising all the way: never stops
    assert stop([0.1, 0.2, 0.3, 0.4], patience=2) is None
    # rises to layer 2, then 3 layers without a strict rise: stops at the third of them
    assert stop([0.1, 0.5, 0.9, 0.9, 0.8, 0.7, 0.95], patience=3) == 5
    # an equal value is not a rise
    assert stop([1.0, 1.0, 1.0], patience=2) == 2
    # a rise resets the count
    assert stop([0.1, 0.2, 0.1, 0.3, 0.2, 0.2, 0.2], patience=3) == 6
    # patience 10 as in App. A
    seq = [0.1 * i for i in range(12)] + [1.0] * 10
    assert stop(seq, patience=10) == 21


def _fake_protocol(monkeypatch, err_of_chi):
    """Run experiments.fig4b / bond_dimension_search with the GPU calls replaced by a
    known error curve, recording every chi the protocol asks for."""
    import paper_2301_12814_gb300.experiments as ex
    asked = []

    def fake_curve(M, d, r, eta, k, theta, phi, final_phase=None, chis=(), precision="fp64", n_cap=None):
        asked.append(list(chis))
        return [(int(c), float(err_of_chi(M, int(c)))) for c in chis]

    monkeypatch.setattr(ex, "truncation_curve", fake_curve)
    monkeypatch.setattr(ex, "choose_d", lambda M, r, eta, **kw: {"d": 9, "n_cap": 8, "d_in": 32, "tail": 0.005,
                                                                   "visited": [(9, 0.005)]})
    monkeypatch.setattr(ex, "_truncation_error",
                        lambda M, d, r, eta, chi, *a, **kw: float(err_of_chi(M, int(chi))))
    return ex, asked


def test_fig4b_bracket_and_refinement(monkeypatch):
    """Doubling phase in one batch, then evenly spaced chi inside the first bracket
    that meets the target; the answer is the smallest refined chi within target."""
    err = lambda M, chi: 8.0 / chi  # 0.02 is first met at chi = 400: bracket (256, 512]
    ex, asked = _fake_protocol(monkeypatch, err)
    res = ex.fig4b(chi_max=1024, target=0.02, refine=3)
    assert len(res) == 3
    r0 = res[0]
    assert [c for c, _ in r0["curve"]] == [8, 16, 32, 64, 128, 256, 512, 1024]
    assert [c for c, _ in r0["refined"]] == [320, 384, 448]
    assert r0["chi_for_target"] == 448 and abs(r0["error_at_chi"] - 8.0 / 448) < 1e-15
    # two batched calls per configuration
    assert len(asked) == 6 and asked[1] == [320, 384, 448]


def test_fig4b_target_not_reached(monkeypatch):
    ex, asked = _fake_protocol(monkeypatch, lambda M, chi: 0.5)
    res = ex.fig4b(chi_max=64)
    assert all(r["chi_for_target"] is None and r["refined"] == [] for r in res)
    assert len(asked) == 3  # no refinement batch


def test_bond_dimension_search_doubling_then_bisection(monkeypatch):
    """App. A: double from chi0 while the error exceeds the target, then bisect the
    last bracket; every visited chi below the answer failed the target."""
    ex, _ = _fake_protocol(monkeypatch, lambda M, chi: 10.0 / chi)  # target 0.02 met from chi = 500
    res = ex.bond_dimension_search(8, 9, [0.88] * 8, [0.3] * 8, [0], [0.1], [0.2], chi0=8, target=0.02, refine=4)
    chis = [c for c, _ in res["visited"]]
    assert chis[:7] == [8, 16, 32, 64, 128, 256, 512]
    assert res["chi"] >= 500 and 10.0 / res["chi"] <= 0.02
    assert all(e > 0.02 for c, e in res["visited"] if c < res["chi"])
    assert len(chis) == 7 + 4


def test_transmission_rule():
    """mu = beta N^gamma / N (Results), refused outside [0, 1]."""
    import numpy as np
    import pytest
    import paper_2301_12814_gb300.experiments as ex
    mu = ex.transmission([10, 100, 1000], 1.0, 0.5)
    assert np.allclose(mu, [10 ** -0.5, 0.1, 1000 ** -0.5])
    assert np.allclose(ex.transmission(50, 0.4, 1.0), 0.4)
    with pytest.raises(ValueError):
        ex.transmission(10, 2.0, 1.0)


def test_asymptotic_bench_flop_count():
    """The App. C roofline's flop count, pinned by hand-counted cases.

    Block sizes: the columns (k, k') of X, k, k' = 0..n_max, split into symmetric
    and antisymmetric combinations under the swap and by the parity of k + k';
    enumerated here one by one.  Flops: a block of nb columns has nb (nb - 1) / 2
    pairs; per pair and sweep 3 FMAs per row for the dot products (6 nb flops), and
    6 nb for a rotation (two products and two FMAs per row) in every sweep but the
    last.  For n_max = 1 the blocks have 2, 1, 0, 1 columns; with sweeps (3, 2, 1, 4)
    only the first block has a pair: 3 sweeps x 12 + 2 x 12 = 60 flops.  For
    n_max = 2 the blocks have 4, 2, 1, 2 columns: 6 pairs x 24 x (3 + 2) = 720,
    12 x (2 + 1) = 36, 0 and 12 x (4 + 3) = 84, in total 840."""
    import os
    import sys
    import numpy as np
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench

    def block_sizes(n_max):
        sizes = [0, 0, 0, 0]  # sym/even, sym/odd, antisym/even, antisym/odd
        for k in range(n_max + 1):
            for kk in range(k, n_max + 1):
                odd = (k + kk) % 2
                sizes[0 + odd] += 1
                if kk > k:
                    sizes[2 + odd] += 1
        return sizes

    assert block_sizes(1) == [2, 1, 0, 1]
    assert block_sizes(2) == [4, 2, 1, 2]
    for n_max in range(1, 12):
        assert sum(block_sizes(n_max)) == (n_max + 1) ** 2
        # a single sweep of each block is its dot products alone
        want = sum(nb * (nb - 1) / 2 * 6 * nb for nb in block_sizes(n_max))
        assert abs(bench.asym_flops(n_max, np.ones(4, dtype=int)) - want) <= 1e-9 * max(want, 1.0)
    sweeps = np.array([3, 2, 1, 4])
    assert bench.asym_flops(1, sweeps) == 60.0
    assert bench.asym_flops(2, sweeps) == 840.0
