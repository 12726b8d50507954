"""Pins for oracle.lattice (rank-1 lattices; Definition of Lambda(z, M) and the
reconstructing property, Lemma RandomRank1Lattice)."""
import itertools

import numpy as np
import pytest

from oracle import lattice as lat


def pairwise_reconstructing(I, z, M):
    """Brute force over all pairs: (k - l).z != 0 mod M."""
    pts = [np.array(p) for p in {tuple(r) for r in np.asarray(I).tolist()}]
    for k, l in itertools.combinations(pts, 2):
        if int(np.dot(k - l, z)) % M == 0:
            return False
    return True


def test_box_lattice_is_a_bijection():
    # z = (1, 33), M = 33^2: k.z = k1 + 33 k2 runs over 33 consecutive blocks of
    # 33 consecutive integers for k in [-16,16]^2, so every residue appears once.
    g = np.arange(-16, 17)
    box = np.stack(np.meshgrid(g, g, indexing="ij"), -1).reshape(-1, 2)
    r = lat.residues(box, [1, 33], 1089)
    assert sorted(r.tolist()) == list(range(1089))
    assert lat.is_reconstructing(box, [1, 33], 1089)
    # one step wider collides: (17, 0) and (-16, 1) share 17 = -16 + 33
    wide = np.vstack([box, [[17, 0]]])
    assert not lat.is_reconstructing(wide, [1, 33], 1089)


@pytest.mark.parametrize("seed", range(6))
def test_reconstructing_matches_pairwise(seed):
    rng = np.random.default_rng(seed)
    d = int(rng.integers(1, 5))
    I = rng.integers(-5, 6, size=(30, d))
    M = int(rng.choice([31, 61, 101, 211]))
    z = rng.integers(1, M, size=d)
    assert lat.is_reconstructing(I, z, M) == pairwise_reconstructing(I, z, M)


def test_forced_collision_detected():
    z = np.array([7, 11, 13])
    M = 1009
    k = np.array([1, 2, 3])
    v = np.array([z[1], -z[0], 0])          # v.z = 0
    assert not lat.is_reconstructing(np.stack([k, k + v]), z, M)
    assert lat.is_reconstructing(np.stack([k, k + np.array([1, 0, 0])]), z, M)


def test_next_prime_against_sieve():
    n = 5000
    sieve = np.ones(n + 200, bool)
    sieve[:2] = False
    for i in range(2, int((n + 200) ** 0.5) + 1):
        if sieve[i]:
            sieve[i * i::i] = False
    primes = np.flatnonzero(sieve)
    for m in range(0, n, 37):
        assert lat.next_prime(m) == int(primes[primes >= m][0])
    assert lat.next_prime(10**6) == 1000003
    assert lat.is_prime(2**26 + 15) and all(not lat.is_prime(2**26 + i) for i in range(15))


def test_smooth_sizes():
    assert lat.next_smooth(10**6) == 10**6               # 2^6 5^6
    assert lat.next_smooth(1000003) == 1000188           # 2^2 3^2 7^3 ... checked by factoring
    assert lat.is_smooth(1000188) and not lat.is_smooth(1000003)
    assert [m for m in range(1, 21) if lat.is_smooth(m)] == [1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 12, 14, 15, 16, 18, 20]


def test_random_lattice_size_rule():
    # smallest prime strictly greater than max(K, |I|^2 / sigma)
    assert lat.random_lattice_size(2048, 35, 0.05) == lat.next_prime(24501)
    assert lat.random_lattice_size(100, 3, 0.05) == 181   # 9/0.05 = 180 > K; 181 is prime
    assert lat.random_lattice_size(400, 3, 0.05) == 401   # K dominates; 401 is prime
    M = lat.random_lattice_size(10, 3, 0.05)
    assert M > 180 and lat.is_prime(M) and not any(lat.is_prime(m) for m in range(181, M))
    assert lat.random_lattice_size(10, 3, 0.05, M_min=2**26) == 2**26 + 15


def test_random_lattice_failure_rate_below_sigma():
    rng = np.random.default_rng(1)
    I = np.unique(rng.integers(-3, 4, size=(12, 3)), axis=0)
    sigma = 0.5
    M = lat.random_lattice_size(lat.expansion(I), len(I), sigma)
    fails = sum(not pairwise_reconstructing(I, rng.integers(1, M, size=3), M) for _ in range(400))
    assert fails / 400 <= sigma


def test_cbc_lattice_reconstructs():
    rng = np.random.default_rng(3)
    I = np.unique(rng.integers(-8, 9, size=(80, 6)), axis=0)
    I = np.unique(np.vstack([I, -I]), axis=0)
    draws = {"raw": rng.integers(0, 2**62, size=(6, 16)), "M_min": 100000}
    z, M = lat.cbc_lattice(I, draws)
    assert z[0] == 1 and lat.is_smooth(M) and M >= 100000
    assert not any(lat.is_smooth(m) for m in range(100000, M))
    assert pairwise_reconstructing(I, z, M)
    for j in range(1, 6):
        assert pairwise_reconstructing(np.unique(I[:, : j + 1], axis=0), z[: j + 1], M)
