"""Rank-1 lattices (oracle; test infrastructure only).

Section "Previous results on SFTs", Definition (rank-1 lattice): the lattice
Lambda(z, M) = { (j/M) z mod 1 : j = 0..M-1 } is *reconstructing* for a
frequency set I when k.z != l.z (mod M) for all k != l in I.

Lemma RandomRank1Lattice: with K the expansion of I (the side of the smallest
cube holding I) and M the smallest prime greater than max(K, |I|^2/sigma),
z drawn uniformly from {1..M-1}^d is reconstructing with probability at
least 1 - sigma (the paper's statement of the probability is read as 1 - sigma).

Component-by-component (CBC) construction is only named by the paper; the
reading used here: z_1 = 1 and, for j = 2..d, the first candidate from a
seeded stream such that the projections of I onto coordinates 1..j that are
distinct points have distinct residues mod M.  The CBC check is exact and
needs no primality (only the random-lattice lemma does), so M is the smallest
7-smooth integer (prime factors 2, 3, 5, 7) not below max(M_min, K + 1): a
length that a mixed-radix FFT handles directly.

Pins: exact integer arithmetic throughout; checked against a closed-form
bijective box lattice, a brute-force pairwise collision check, forced
collisions and an independent primality routine (tests/test_oracle_lattice.py).
"""
from __future__ import annotations

import numpy as np


def residues(freq, z, M):
    """k.z mod M for every row k of ``freq`` (exact, Python integers)."""
    freq = np.asarray(freq, dtype=object)
    z = np.asarray(z, dtype=object)
    out = [int(sum(int(a) * int(b) for a, b in zip(row, z)) % int(M)) for row in freq]
    return np.array(out, dtype=np.int64)


def is_reconstructing(freq, z, M):
    """True when the residues of the distinct rows of ``freq`` are distinct."""
    uniq = {tuple(int(x) for x in row) for row in np.asarray(freq)}
    pts = np.array(sorted(uniq), dtype=np.int64).reshape(len(uniq), -1)
    r = residues(pts, z, M)
    return len(set(r.tolist())) == len(r)


def expansion(freq):
    """K = max_j (max_k k_j - min_l l_j) over the rows of ``freq``."""
    f = np.asarray(freq, dtype=np.int64)
    if f.size == 0:
        return 0
    return int((f.max(axis=0) - f.min(axis=0)).max())


def is_prime(n):
    """Trial division (n < 2^62 in practice: the largest sizes here are ~2^27)."""
    n = int(n)
    if n < 2:
        return False
    if n % 2 == 0:
        return n == 2
    i = 3
    while i * i <= n:
        if n % i == 0:
            return False
        i += 2
    return True


def next_prime(n):
    """Smallest prime >= n."""
    n = max(int(n), 2)
    while not is_prime(n):
        n += 1
    return n


def random_lattice_size(K, n_I, sigma, M_min=0):
    """Lemma RandomRank1Lattice: the smallest prime greater than
    max(K, |I|^2/sigma), and not below ``M_min`` when a size is prescribed."""
    bound = max(float(K), float(n_I) ** 2 / float(sigma))
    lo = int(np.floor(bound)) + 1            # strictly greater than the bound
    return next_prime(max(lo, int(M_min)))


def is_smooth(n, primes=(2, 3, 5, 7)):
    """True when every prime factor of n is in ``primes``."""
    n = int(n)
    if n < 1:
        return False
    for p in primes:
        while n % p == 0:
            n //= p
    return n == 1


def next_smooth(n):
    """Smallest 7-smooth integer >= n."""
    n = max(int(n), 1)
    while not is_smooth(n):
        n += 1
    return n


def z_from_raw(raw, M):
    """Map raw non-negative integers onto {1..M-1}."""
    return np.array([1 + int(r) % (int(M) - 1) for r in np.asarray(raw).ravel()], dtype=np.int64)


def random_lattice(freq, draws):
    """Choose (z, M, attempt) for the frequency set ``freq`` from the raw draws
    of ``workloads.random_lattice_draws``: M by Lemma RandomRank1Lattice, then
    the first attempt whose z is reconstructing."""
    uniq = np.unique(np.asarray(freq, np.int64), axis=0)
    M = random_lattice_size(expansion(uniq), len(uniq), draws["sigma"], draws["M_min"])
    for att, raw in enumerate(np.asarray(draws["raw"])):
        z = z_from_raw(raw, M)
        if is_reconstructing(uniq, z, M):
            return z, M, att
    raise ValueError("no reconstructing lattice among the attempts")


def cbc_lattice(freq, draws):
    """Component-by-component search (reading stated in the module header).
    M is the smallest 7-smooth integer >= max(M_min, K + 1)."""
    uniq = np.unique(np.asarray(freq, np.int64), axis=0)
    d = uniq.shape[1]
    M = next_smooth(max(int(draws["M_min"]), expansion(uniq) + 1))
    raw = np.asarray(draws["raw"])
    z = [1]
    for j in range(1, d):
        proj = np.unique(uniq[:, : j + 1], axis=0)
        for r in raw[j]:
            c = 1 + int(r) % (M - 1)
            if is_reconstructing(proj, z + [c], M):
                z.append(c)
                break
        else:
            raise ValueError(f"CBC: no candidate for coordinate {j}")
    return np.array(z, dtype=np.int64), M
