"""The round-robin schedule of the cluster block Jacobi (k_svd, cluster blocks), checked
on the CPU: the same index arithmetic as the kernel, for ragged sizes, every cluster
size K and every column split w.  In one sweep every pair of columns must be rotated
exactly once, and within a round no column may sit in two CTAs (the CTAs of a round
work on disjoint columns in parallel) nor in two pairs of one inner round."""
import itertools

import pytest


def circle_pair(rnd, k, np_):
    """Pair k of round rnd of the circle method over np_ (even) players, (p < q)."""
    if k == 0:
        p, q = rnd, np_ - 1
    else:
        p, q = (rnd + k) % (np_ - 1), (rnd - k + np_ - 1) % (np_ - 1)
    return (min(p, q), max(p, q))


def sweep(n, K, w):
    nb = 2 * K * w
    b = -(-n // nb)
    seen = {}
    for rho in range(nb - 1):
        round_cols = []
        for kr in range(K):
            for pi in range(kr, nb // 2, K):           # this CTA's w block pairs
                I, J = circle_pair(rho, pi, nb)
                i0, j0 = I * b, J * b
                nI = max(0, min(n, i0 + b) - i0)
                nJ = max(0, min(n, j0 + b) - j0)

                def gc(l):
                    return i0 + l if l < nI else j0 + (l - nI)
                round_cols += [gc(l) for l in range(nI + nJ)]
                inner = []
                if rho == 0:                            # pairs inside each block
                    pI, pJ = nI + (nI & 1), nJ + (nJ & 1)
                    for r in range(max(pI, pJ) - 1):
                        hI = pI // 2 if r < pI - 1 else 0
                        hJ = pJ // 2 if r < pJ - 1 else 0
                        pairs = []
                        for k in range(hI + hJ):
                            if k < hI:
                                p, q = circle_pair(r, k, pI)
                                if q >= nI:
                                    continue
                            else:
                                p, q = circle_pair(r, k - hI, pJ)
                                if q >= nJ:
                                    continue
                                p, q = p + nI, q + nI
                            pairs.append((p, q))
                        inner.append(pairs)
                for r in range(b):                      # pairs across the two blocks
                    inner.append([(i, nI + (i + r) % b) for i in range(nI) if (i + r) % b < nJ])
                for pairs in inner:
                    cols = [c for pq in pairs for c in pq]
                    assert len(cols) == len(set(cols)), "a column in two pairs of one inner round"
                    for p, q in pairs:
                        key = (min(gc(p), gc(q)), max(gc(p), gc(q)))
                        seen[key] = seen.get(key, 0) + 1
        assert len(round_cols) == len(set(round_cols)), "a column in two CTAs in one round"
    return seen


@pytest.mark.parametrize("K", [1, 2, 4, 8])
@pytest.mark.parametrize("w", [1, 2, 4, 8])
def test_every_pair_once_per_sweep(K, w):
    for n in list(range(1, 34)) + [48, 64, 100, 257, 300]:
        seen = sweep(n, K, w)
        assert set(seen) == set(itertools.combinations(range(n), 2)), (n, K, w)
        assert all(v == 1 for v in seen.values()), (n, K, w)
