"""Pins for oracle.sft (lattice sampling; recovery of Fourier coefficients by the
DFT of lattice samples, Section 2 coefficient definition and the
reconstructing-lattice premise of Theorem SFTRecovery)."""
import numpy as np
import pytest

from oracle import lattice as lat
from oracle import sft


def eval_at_float_points(freq, coef, z, M, js):
    """g at x_j = (j z / M) mod 1 computed in floating point (no residues)."""
    x = np.mod(np.outer(js, np.asarray(z, np.float64)) / M, 1.0)
    ph = 2 * np.pi * x @ np.asarray(freq, np.float64).T
    return (np.exp(1j * ph) * np.asarray(coef)[None, :]).real.sum(axis=1)


def test_sample_equals_pointwise_evaluation():
    rng = np.random.default_rng(0)
    d, M = 3, 1009
    z = rng.integers(1, M, size=d)
    freq = rng.integers(-7, 8, size=(6, d))
    coef = rng.standard_normal(6) + 1j * rng.standard_normal(6)
    js = np.arange(M)
    np.testing.assert_allclose(sft.sample(freq, coef, z, M), eval_at_float_points(freq, coef, z, M, js),
                               atol=1e-11)


def test_recover_closed_form_cos_sin_mean():
    # g = 0.7 + 0.3 cos(2pi p.x) - 0.2 sin(2pi q.x):
    # g_hat_0 = 0.7, g_hat_{+-p} = 0.15, g_hat_{+q} = -0.2/(2i) = 0.1i, g_hat_{-q} = -0.1i
    d = 3
    p = np.array([2, -1, 3])
    q = np.array([-4, 0, 1])
    freq = np.array([[0, 0, 0], p, q])
    coef = np.array([0.7, 0.3, -0.2 * -1j])       # sine term c sin = Re(-i c e)
    # box lattice z = (1, 9, 81), M = 9^3: a bijection of [-4,4]^3 onto Z_M
    g = np.arange(-4, 5)
    cand = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    z, M = np.array([1, 9, 81]), 729
    assert lat.is_reconstructing(cand, z, M)
    samples = sft.sample(freq, coef, z, M)
    kf, kv = sft.recover_known(samples, cand, z, M, tau=1e-9)
    got = {tuple(k): v for k, v in zip(kf.tolist(), kv)}
    want = {(0, 0, 0): 0.7, tuple(p): 0.15, tuple(-p): 0.15, tuple(q): 0.1j, tuple(-q): -0.1j}
    assert set(got) == set(want)
    for k, v in want.items():
        assert abs(got[k] - v) < 1e-12 * 1.2


def test_dft_equals_library_fft_on_box_lattice():
    rng = np.random.default_rng(2)
    M = 1089
    samples = rng.standard_normal(M)
    bins = np.arange(M)
    np.testing.assert_allclose(sft.dft_bins(samples, bins, M), np.fft.fft(samples) / M, atol=1e-13)


def test_true_coefficients_definition():
    c = sft.true_coefficients([[0, 0], [1, 2], [1, 2]], [2.0, 1.0 + 1j, 0.5])
    assert c[(0, 0)] == 2.0
    assert c[(1, 2)] == pytest.approx((1.5 + 1j) / 2)
    assert c[(-1, -2)] == pytest.approx((1.5 - 1j) / 2)


def test_recover_rejects_bad_inputs():
    cand = np.array([[1, 0], [-1, 0], [0, 1], [0, -1]])
    s = np.zeros(7)
    with pytest.raises(ValueError):
        sft.recover_known(s, cand[:3], [1, 2], 7)            # not symmetric
    with pytest.raises(ValueError):
        sft.recover_known(s, cand, [1, 1], 7)                # (1,0) ~ (0,1)


def test_threshold_and_cap():
    d, M = 1, 101
    freq = np.array([[3], [5]])
    coef = np.array([1.0, 1e-12])
    cand = np.arange(-10, 11).reshape(-1, 1)
    s = sft.sample(freq, coef, [1], M)
    kf, _ = sft.recover_known(s, cand, [1], M, tau=1e-9)
    assert sorted(kf.ravel().tolist()) == [-3, 3]
    kf, _ = sft.recover_known(s, cand, [1], M, tau=1e-14)
    assert sorted(kf.ravel().tolist()) == [-5, -3, 3, 5]
    with pytest.raises(ValueError):
        sft.recover_known(s, cand, [1], M, tau=1e-14, s_max=3)


def test_identify_single_term_phase_ratio():
    # g = cos(2 pi p.x): the shifted spectrum at p's bin is the plain one
    # times exp(2 pi i p_i / P)
    from oracle.sft import sample, sample_shifted
    p = np.array([[5, -3, 7]])
    z, M, P = np.array([1, 23, 529]), 12167, 17
    b = int((p[0] @ z) % M)
    X0 = np.fft.fft(sample(p, [1.0], z, M))
    for i in range(3):
        Xi = np.fft.fft(sample_shifted(p, [1.0], z, M, P, i))
        np.testing.assert_allclose(Xi[b] / X0[b], np.exp(2j * np.pi * p[0, i] / P), atol=1e-12)


@pytest.mark.parametrize("seed", range(4))
def test_identify_recovers_random_sparse_sums(seed):
    from oracle.lattice import is_reconstructing, next_prime
    from oracle.sft import identify, true_coefficients
    rng = np.random.default_rng(seed)
    d, K = 3, 12
    freqs = np.unique(rng.integers(-K, K + 1, size=(6, d)), axis=0)
    freqs = freqs[freqs.any(axis=1)]
    coef = rng.uniform(-1, 1, len(freqs)) + 1j * rng.uniform(-1, 1, len(freqs))
    freqs = np.vstack([np.zeros((1, d), int), freqs])
    coef = np.concatenate([[0.7], coef])
    true = true_coefficients(freqs, coef)
    I = np.array(sorted(true))
    M = next_prime(4000)
    while True:
        z = rng.integers(1, M, size=d)
        if is_reconstructing(I, z, M):
            break
    P = next_prime(2 * K + 1)
    f, v = identify(freqs, coef, z, M, P, tau=1e-9)
    got = {tuple(int(x) for x in k): val for k, val in zip(f.tolist(), v)}
    assert set(got) == set(true)
    for k in true:
        assert abs(got[k] - true[k]) < 1e-12


def poisson_samples(k0, r, z, M, P):
    """Samples of the Poisson kernel along k0, g(x) = (1 - r^2)/(1 - 2 r cos(2 pi k0.x) + r^2)
    (coefficients r^|m| at m k0), on the lattice and the d shifted lattices,
    phases k0.x taken as exact rationals."""
    M, P = int(M), int(P)
    j = np.arange(M, dtype=np.int64)
    q = int(np.dot(k0, z) % M)
    rows = []
    for i in [None] + list(range(len(k0))):
        num = ((j * q) % M) * P + (0 if i is None else int(k0[i]) * M)
        th = 2 * np.pi * ((num % (M * P)) / (M * P))
        rows.append((1 - r * r) / (1 - 2 * r * np.cos(th) + r * r))
    return np.stack(rows)


def test_identify_compressible_poisson_kernel():
    # compressible data: the s largest coefficients r^|m| (m = 0, +-1, ...) are
    # identified at the right frequencies; their values carry only the
    # aliasing of the tail, sum over |m| >= M / |.| of r^|m|, below 1e-12 here
    from oracle.sft import identify_samples
    k0 = np.array([3, -2, 5])
    z = np.array([1, 77, 340])
    M, P, r, keep = 1021, 101, 0.5, 6
    X = poisson_samples(k0, r, z, M, P)
    f, v = identify_samples(X, z, M, P, tau=1e-12, keep=keep, robust=True)
    got = {tuple(k): val for k, val in zip(f.tolist(), v)}
    want = {tuple(m * k0): r ** abs(m) for m in range(-5, 6)}
    assert set(got) == set(want)
    for k in want:
        assert abs(got[k] - want[k]) < 1e-12


def test_identify_robust_drops_aliased_bins():
    # with keep large enough to reach bins where the tail aliases, robust
    # mode keeps only bins whose k maps back, and never raises
    from oracle.sft import identify_samples
    k0 = np.array([3, -2, 5])
    z = np.array([1, 77, 340])
    M, P, r = 1021, 101, 0.9
    X = poisson_samples(k0, r, z, M, P)
    f, v = identify_samples(X, z, M, P, tau=0.0, keep=200, robust=True)
    assert len(f) > 0
    assert len({tuple(k) for k in f.tolist()}) == len(f)        # no frequency twice
    # every output frequency lies on the line m k0 with |m| < P/2
    for k in f.tolist():
        m = k[0] // 3
        assert k == [3 * m, -2 * m, 5 * m]
