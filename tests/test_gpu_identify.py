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


def poisson(k0, r, z, M, P):
    from tests.test_oracle_sft import poisson_samples
    return poisson_samples(np.asarray(k0), r, z, M, P)


@pytest.mark.parametrize("r,keep,tau", [(0.5, 6, 1e-12), (0.7, 12, 0.0), (0.9, 60, 0.0)])
def test_compressible_identify_matches_oracle(B, r, keep, tau):
    # Poisson kernel along k0 (coefficients r^|m| at m k0): the keep largest
    # bins, aliased ones dropped; same frequencies and values as the oracle
    k0, z, M, P = [3, -2, 5], np.array([1, 77, 340]), 1021, 101
    X = poisson(k0, r, z, M, P)
    f_ref, v_ref = osft.identify_samples(X, z, M, P, tau=tau, keep=keep, robust=True)
    f, v = B.sft_identify_samples(z, M, X, P, s_max=4 * keep + 2, tau=tau, keep=keep, robust=True)
    assert np.array_equal(f.cpu().numpy(), f_ref)
    assert np.max(np.abs(v.cpu().numpy() - v_ref)) <= 1e-12 * np.abs(X[0]).max()


def test_samples_form_equals_trig_form(B):
    freq, coef, true, z, M, P = random_problem(9, 3, 10, 8, 1500)
    rows = [osft.sample(freq, coef, z, M)] + [osft.sample_shifted(freq, coef, z, M, P, i) for i in range(3)]
    f1, v1 = B.sft_identify(z, M, freq, coef, P, s_max=64)
    f2, v2 = B.sft_identify_samples(z, M, np.stack(rows), P, s_max=64)
    assert np.array_equal(f1.cpu().numpy(), f2.cpu().numpy())
    assert np.max(np.abs(v1.cpu().numpy() - v2.cpu().numpy())) <= 1e-12 * np.abs(coef).sum()


def test_radix_selection_keeps_exactly_the_largest(B):
    # random bins: keep = 17 out of many above threshold -> exactly the 17
    # largest half-spectrum magnitudes (robust drops none: consistent data)
    rng = np.random.default_rng(4)
    d, K = 2, 30
    freqs, _ = W.draw_freqs(rng, 40, d, -K, K)
    g = W.random_cos_sin(rng, freqs)
    true = osft.true_coefficients(g.freq, g.coef)
    I = np.array(sorted(true), np.int64)
    M = olat.next_prime(8000)
    while True:
        z = rng.integers(1, M, size=d)
        if olat.is_reconstructing(I, z, M):
            break
    P = olat.next_prime(2 * K + 1)
    rows = [osft.sample(g.freq, g.coef, z, M)] + [osft.sample_shifted(g.freq, g.coef, z, M, P, i) for i in range(d)]
    f, v = B.sft_identify_samples(z, M, np.stack(rows), P, s_max=64, tau=1e-9, keep=17, robust=False)
    got = {tuple(k) for k in f.cpu().numpy().tolist()}
    mags = sorted({abs(val) for val in true.values()}, reverse=True)
    cut = mags[17]
    want = {k for k, val in true.items() if abs(val) > cut}
    assert got == want
