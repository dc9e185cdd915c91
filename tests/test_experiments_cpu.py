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
