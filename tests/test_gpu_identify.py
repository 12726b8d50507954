"""Support identification without a candidate set (shifted lattices; the
paper's SFT in its identify role).  The GPU result equals the oracle's: the
same frequencies in the same order (bit-exact integers) and values within
1e-12 (FP64) / 1e-5 (FP32) of sum |c|; and the identified support is the true
one (closed form of the generating trigonometric sum)."""
import numpy as np
import pytest

import workloads as W
from oracle import lattice as olat
from oracle import sft as osft

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2302_00752_gb300 import binding
    return binding


def random_problem(seed, d, K, n_terms, M_min):
    rng = np.random.default_rng([seed, 0x1d])
    freqs, _ = W.draw_freqs(rng, n_terms, d, -K, K)
    g = W.random_cos_sin(rng, freqs)
    freq = np.vstack([np.zeros((1, d), np.int32), g.freq])
    coef = np.concatenate([[0.5 + 0j], g.coef])
    true = osft.true_coefficients(freq, coef)
    I = np.array(sorted(true), np.int64)
    M = olat.next_prime(max(M_min, 2 * K + 1))
    while True:
        z = rng.integers(1, M, size=d)
        if olat.is_reconstructing(I, z, M):
            break
    return freq, coef, true, z, M, olat.next_prime(2 * K + 1)


@pytest.mark.parametrize("seed,d,K,n,M_min", [(0, 2, 8, 5, 500), (1, 3, 20, 12, 3000), (2, 5, 6, 9, 2000),
                                              (3, 1, 50, 7, 400)])
def test_identify_matches_oracle_and_truth(B, seed, d, K, n, M_min):
    freq, coef, true, z, M, P = random_problem(seed, d, K, n, M_min)
    f_ref, v_ref = osft.identify(freq, coef, z, M, P, tau=1e-9)
    f, v = B.sft_identify(z, M, freq, coef, P, s_max=64, tau=1e-9)
    assert np.array_equal(f.cpu().numpy(), f_ref)
    scale = np.abs(coef).sum()
    assert np.max(np.abs(v.cpu().numpy() - v_ref)) <= 1e-12 * scale
    got = {tuple(k): val for k, val in zip(f.cpu().numpy().tolist(), v.cpu().numpy())}
    assert set(got) == set(true)


def test_identify_fp32(B):
    freq, coef, true, z, M, P = random_problem(7, 3, 15, 10, 5000)
    f, v = B.sft_identify(z, M, freq, coef, P, s_max=64, tau=1e-4, precision="fp32")
    got = {tuple(k): val for k, val in zip(f.cpu().numpy().tolist(), v.cpu().numpy())}
    assert set(got) == set(true)
    assert max(abs(got[k] - true[k]) for k in true) <= 1e-5 * np.abs(coef).sum()


def test_identify_limits(B):
    freq, coef, true, z, M, P = random_problem(8, 2, 8, 6, 800)
    with pytest.raises(B.SSError):
        B.sft_identify(z, M, freq, coef, P, s_max=len(true) - 1)
    # a lattice that folds two frequencies into one bin is reported
    M2 = 7
    with pytest.raises(B.SSError):
        B.sft_identify(np.array([1, 3]), M2, freq, coef, P, s_max=64)
