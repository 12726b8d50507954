"""Pins for oracle.stamp (eq. StampSet, Lemma StampSetCardinality, Lemma
StampSizeUpperBound)."""
import itertools

import numpy as np
import pytest

from oracle import stamp
from tests.golden.loader import stamp_cases


def brute_minkowski(F, A, N):
    """{f + a_1 + ... + a_N}: every N-tuple of supp(a_hat) (0 included, so the
    shorter sums are in), plus the first level reaching each point."""
    F = [tuple(f) for f in np.asarray(F).tolist()]
    A = [tuple(a) for a in np.asarray(A).tolist()]
    first = {}
    for n in range(N + 1):
        for f in F:
            for steps in itertools.product(A, repeat=n):
                k = tuple(sum(c) for c in zip(f, *steps))
                first.setdefault(k, n)
    return first


@pytest.mark.parametrize("case", stamp_cases(), ids=lambda c: c["name"])
def test_hand_worked_order(case):
    S, lvl = stamp.stamp_bfs(case["A"], case["F"], case["N"])
    np.testing.assert_array_equal(S, case["S"])
    np.testing.assert_array_equal(lvl, case["L"])


@pytest.mark.parametrize("seed", range(8))
def test_set_and_levels_match_brute_force(seed):
    rng = np.random.default_rng(seed)
    d = int(rng.integers(1, 4))
    n_a = int(rng.integers(1, 3))
    P = rng.integers(-3, 4, size=(n_a, d))
    P = P[P.any(axis=1)]
    A = np.unique(np.vstack([np.zeros((1, d), int), P, -P]), axis=0)
    F = np.unique(rng.integers(-4, 5, size=(3, d)), axis=0)
    N = int(rng.integers(0, 4))
    S, lvl = stamp.stamp_bfs(A, F, N)
    first = brute_minkowski(F, A, N)
    got = {tuple(k): int(l) for k, l in zip(S.tolist(), lvl)}
    assert len(got) == len(S)                      # no duplicates
    assert got == first
    # levels appear in non-decreasing order, level 0 is F sorted
    assert np.all(np.diff(lvl.astype(int)) >= 0)
    l0 = S[lvl == 0].tolist()
    assert l0 == sorted(l0)


def count_tuples(r, n):
    """|T_n| from the proof of Lemma StampSetCardinality by enumeration:
    multiplicity vectors m in {0..n}^r with |m|_1 = n, each nonzero entry
    signed +-1."""
    tot = 0
    for m in itertools.product(range(n + 1), repeat=r):
        if sum(m) == n:
            tot += 2 ** sum(1 for x in m if x)
    return tot


@pytest.mark.parametrize("r,N", [(1, 3), (2, 3), (3, 2), (4, 3), (5, 2)])
def test_cardinality_formula_matches_enumeration(r, N):
    s = 2 * r + 1
    assert stamp.cardinality_bound(1, s, N) == sum(count_tuples(r, n) for n in range(N + 1))


@pytest.mark.parametrize("seed,d,r,nf,N", [(0, 6, 3, 4, 3), (1, 8, 5, 6, 2), (2, 5, 2, 3, 4)])
def test_generic_position_count_is_exact(seed, d, r, nf, N):
    # large random frequencies: no two sums coincide, so the bound is attained
    rng = np.random.default_rng(seed)
    P = rng.integers(-10**4, 10**4, size=(r, d))
    A = np.vstack([np.zeros((1, d), int), P, -P])
    F = rng.integers(-10**4, 10**4, size=(nf, d))
    S, _ = stamp.stamp_bfs(A, F, N)
    assert len(S) == stamp.cardinality_bound(nf, 2 * r + 1, N)


@pytest.mark.parametrize("s,N", [(3, 1), (3, 3), (5, 2), (7, 1), (9, 2)])
def test_simple_bound_holds(s, N):
    rng = np.random.default_rng(s * 10 + N)
    d = 3
    P = rng.integers(-2, 3, size=((s - 1) // 2, d))
    A = np.unique(np.vstack([np.zeros((1, d), int), P, -P]), axis=0)
    F = np.unique(rng.integers(-2, 3, size=(min(s, 4), d)), axis=0)
    S, _ = stamp.stamp_bfs(A, F, N)
    assert len(S) <= stamp.cardinality_bound(len(F), len(A), N) <= stamp.simple_bound(len(A), N)


def test_symmetric_F_gives_symmetric_S():
    rng = np.random.default_rng(4)
    d = 3
    P = rng.integers(-3, 4, size=(3, d))
    A = np.vstack([np.zeros((1, d), int), P, -P])
    q = rng.integers(-3, 4, size=(2, d))
    F = np.unique(np.vstack([q, -q]), axis=0)
    S, _ = stamp.stamp_bfs(A, F, 3)
    keys = {tuple(k) for k in S.tolist()}
    assert keys == {tuple(-x for x in k) for k in keys}


def test_duplicate_F_rejected():
    with pytest.raises(ValueError):
        stamp.stamp_bfs([[0], [1], [-1]], [[2], [2]], 1)


def multiset_bound(n_f, s_a, n):
    """|F| C(s_a - 1 + n, n): F plus a multiset of at most n of the s_a - 1
    nonzero steps (the count the GPU build presizes its table and keys by)."""
    from math import comb
    return n_f * comb(s_a - 1 + n, n)


@pytest.mark.parametrize("seed,symmetric", [(0, True), (1, True), (2, False), (3, False), (4, True)])
def test_multiset_count_bounds_every_level(seed, symmetric):
    # |S^n| <= |F| C(s_a - 1 + n, n) for every level n, whatever the steps
    rng = np.random.default_rng(seed)
    d = 3
    P = rng.integers(-2, 3, size=(3, d))
    P = P[np.any(P != 0, axis=1)]
    A = np.vstack([np.zeros((1, d), int), P, -P]) if symmetric else np.vstack([np.zeros((1, d), int), P])
    A = np.unique(A, axis=0)
    F = np.unique(rng.integers(-3, 4, size=(5, d)), axis=0)
    S, lvl = stamp.stamp_bfs(A, F, 4)
    for n in range(5):
        assert int(np.sum(lvl <= n)) <= multiset_bound(len(F), len(A), n)


@pytest.mark.parametrize("seed,d,s_a,nf,N", [(0, 6, 5, 3, 3), (1, 4, 7, 2, 2), (2, 8, 4, 4, 4)])
def test_multiset_count_attained_without_cancellation(seed, d, s_a, nf, N):
    # generic steps without their negations: every multiset of at most N steps
    # gives a distinct sum, so |S^N| equals the count (it is exact, not slack)
    rng = np.random.default_rng(seed)
    P = rng.integers(-10**4, 10**4, size=(s_a - 1, d))
    A = np.vstack([np.zeros((1, d), int), P])
    F = rng.integers(-10**4, 10**4, size=(nf, d))
    S, lvl = stamp.stamp_bfs(A, F, N)
    for n in range(N + 1):
        assert int(np.sum(lvl <= n)) == multiset_bound(nf, s_a, n)
