"""Pins of the oracle's mutual-nomination matching.

With distinct edge keys, repeating rounds of "every free bead nominates its
best edge to a free partner, mutually nominated edges are matched" until
nothing changes is the locally-dominant matching, which equals the sequential
greedy matching over edges sorted by key (a textbook equivalence).  A single
round is exactly the set of mutually best edges (the paper's one nomination
per bead, Appendix steps 2-4).  Both are stated here independently.
"""

import numpy as np
import pytest

from oracle import oracle as O


def greedy(n, k1, a, b):
    order = sorted(range(len(k1)), key=lambda e: (k1[e], a[e], b[e]))
    used = [False] * n
    out = np.zeros(len(k1), bool)
    for e in order:
        if not used[a[e]] and not used[b[e]]:
            used[a[e]] = used[b[e]] = True
            out[e] = True
    return out


def mutual_best(n, k1, a, b):
    best = [None] * n
    for e in range(len(k1)):
        key = (k1[e], a[e], b[e])
        for x in (a[e], b[e]):
            if best[x] is None or key < best[x][0]:
                best[x] = (key, e)
    out = np.zeros(len(k1), bool)
    for e in range(len(k1)):
        if best[a[e]][1] == e and best[b[e]][1] == e:
            out[e] = True
    return out


def random_graph(rng, n, m, key_range):
    pairs = set()
    while len(pairs) < m:
        i, j = rng.integers(0, n, 2)
        if i != j:
            pairs.add((min(i, j), max(i, j)))
    pairs = sorted(pairs)
    a = np.array([p[0] for p in pairs], np.int32)
    b = np.array([p[1] for p in pairs], np.int32)
    k1 = rng.integers(-key_range, key_range + 1, len(pairs)).astype(np.int64)
    return k1, a, b


@pytest.mark.parametrize("seed", range(40))
def test_rounds_to_fixpoint_equal_greedy(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 40))
    m = int(rng.integers(1, min(120, n * (n - 1) // 2) + 1))
    # small key ranges force many equal first keys, exercising the id tie-break
    k1, a, b = random_graph(rng, n, m, key_range=int(rng.choice([0, 2, 1000])))
    got, rounds = O.match(n, k1, a, b, 0)
    assert np.array_equal(got, greedy(n, k1, a, b))
    # maximal: no edge has both endpoints free
    used = np.zeros(n, bool)
    used[a[got]] = True
    used[b[got]] = True
    assert not np.any(~used[a] & ~used[b])


@pytest.mark.parametrize("seed", range(20))
def test_single_round_is_mutual_best(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(2, 30))
    m = int(rng.integers(1, min(80, n * (n - 1) // 2) + 1))
    k1, a, b = random_graph(rng, n, m, key_range=5)
    got, rounds = O.match(n, k1, a, b, 1)
    assert np.array_equal(got, mutual_best(n, k1, a, b))
    assert rounds == (1 if got.any() else 0)


def test_chain_needs_one_round_per_link():
    # a path 0-1-2-...-9 with keys decreasing along it: only the last edge is
    # mutually best in round 1, then every second edge from the end
    n = 10
    a = np.arange(9, dtype=np.int32)
    b = a + 1
    k1 = (100 - np.arange(9)).astype(np.int64)
    got, rounds = O.match(n, k1, a, b, 0)
    assert list(np.nonzero(got)[0]) == [0, 2, 4, 6, 8]
    assert rounds == 5
    got1, r1 = O.match(n, k1, a, b, 1)
    assert list(np.nonzero(got1)[0]) == [8] and r1 == 1


def test_all_equal_keys_tie_to_lower_partner_id():
    # a star: bead 5 with partners 0..4 and 6..9 at equal distance; it takes bead 0
    a = np.array([0, 1, 2, 3, 4, 5, 5, 5, 5], np.int32)
    b = np.array([5, 5, 5, 5, 5, 6, 7, 8, 9], np.int32)
    k1 = np.zeros(9, np.int64)
    got, rounds = O.match(10, k1, a, b, 0)
    assert list(np.nonzero(got)[0]) == [0] and rounds == 1
