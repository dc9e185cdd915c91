"""Pins from numbers the paper prints (fixtures under tests/golden/, each with its
citation)."""
import os

from oracle import u1mpo

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _fixture(name):
    vals = {}
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v = line.split()
            vals[k] = int(v)
    return vals


def test_charge_space_at_d15():
    """App. D: 225 charge values per bond at d = 15, 225^2 (row, column) charge
    combinations for the Theta fill.  The oracle's charge space is the cap square;
    a strongly squeezed 3-mode state at d = 15 puts weight on every pair the parity
    rule allows (c = cbar mod 2) and on no other."""
    g = _fixture("charge_space_d15.txt")
    P = u1mpo.U1MPO(3, g["d"], [1.2] * 3, [0.9] * 3)
    q = P.n_cap + 1
    assert q * q == g["pairs_per_bond"]
    assert (q * q) ** 2 == g["theta_pair_iterations"]
    seen = set()
    for b in range(P.M + 1):
        ch = P.charges[b]
        assert ch.min() >= 0 and ch.max() <= P.n_cap
        seen |= set(map(tuple, ch))
    allowed = {(c, cb) for c in range(q) for cb in range(q) if (c - cb) % 2 == 0}
    assert seen == allowed
