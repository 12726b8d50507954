"""Stamping sets (oracle; test infrastructure only).

eq. StampSet (Proposition SolutionSupport): S^0 = F and
S^N = S^{N-1} + supp(a_hat) (Minkowski sum).  Because 0 is in supp(a_hat),
S^{N-1} is a subset of S^N and S^N is reached level by level: level n holds the
frequencies first reached after n stamps (the decomposition used in the proof
of Lemma StampSetCardinality).

Canonical order (the paper defines S only as a set; this is the reading used
throughout): level 0 is F in signed lexicographic order; level n lists, in
order of first discovery, the new frequencies parent + p over the parents of
level n-1 in index order and, for each parent, the nonzero p in supp(a_hat)
in signed lexicographic order.  The canonical index of a frequency is its
position in this order.

Lemma StampSetCardinality gives |S^N| <= |F| sum_{n<=N} sum_t 2^t C(r,t) C(n-1,t-1)
with r = (s-1)/2 (with C(n-1, -1) = [n = 0]), an equality when no sums
coincide; Lemma StampSizeUpperBound simplifies it to 7 max(s,2N+1)^min(s,2N+1)
when |F| <= s.

Pins: brute-force Minkowski sums on tiny inputs; equality with the count of
Lemma StampSetCardinality in generic position; symmetry S = -S when F = -F
(tests/test_oracle_stamp.py).
"""
from __future__ import annotations

from math import comb

import numpy as np


def lex_order(freq):
    """Indices sorting the rows of ``freq`` in signed lexicographic order."""
    f = np.asarray(freq, np.int64)
    if len(f) == 0:
        return np.zeros(0, np.int64)
    return np.lexsort(f.T[::-1])


def stamp_bfs(a_freq, f_freq, N):
    """S^N[a](F) in canonical order.  Returns (S [n, d] int64, level [n] int8)."""
    F = np.asarray(f_freq, np.int64)
    A = np.asarray(a_freq, np.int64)
    d = F.shape[1]
    F = F[lex_order(F)]
    A = A[lex_order(A)]
    if len({tuple(r) for r in F.tolist()}) != len(F):
        raise ValueError("duplicate frequencies in F")
    steps = [p for p in A.tolist() if any(p)]
    S = [tuple(r) for r in F.tolist()]
    index = {k: i for i, k in enumerate(S)}
    level = [0] * len(S)
    start, stop = 0, len(S)
    for n in range(1, N + 1):
        for i in range(start, stop):
            parent = S[i]
            for p in steps:
                c = tuple(x + y for x, y in zip(parent, p))
                if c not in index:
                    index[c] = len(S)
                    S.append(c)
                    level.append(n)
        start, stop = stop, len(S)
    return np.array(S, dtype=np.int64).reshape(len(S), d), np.array(level, dtype=np.int8)


def index_map(S):
    return {tuple(int(x) for x in row): i for i, row in enumerate(np.asarray(S))}


def cardinality_bound(n_f, s, N):
    """Right-hand side of Lemma StampSetCardinality."""
    r = (s - 1) // 2
    total = 0
    for n in range(N + 1):
        for t in range(0, min(n, r) + 1):
            if t == 0:
                binom_n = 1 if n == 0 else 0
            else:
                binom_n = comb(n - 1, t - 1)
            total += 2 ** t * comb(r, t) * binom_n
    return n_f * total


def simple_bound(s, N):
    """Lemma StampSizeUpperBound: 7 max(s, 2N+1)^min(s, 2N+1)."""
    return 7 * max(s, 2 * N + 1) ** min(s, 2 * N + 1)
