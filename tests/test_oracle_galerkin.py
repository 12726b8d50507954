"""Pins for oracle.galerkin (eq. GF, Proposition GalerkinBilinearForm,
Proposition LExpansion, eq. FiniteGalerkinOperator)."""
import numpy as np
import pytest

from oracle import galerkin, stamp
from oracle.sft import true_coefficients


def coeff_arrays(d):
    return np.array(list(d.keys()), np.int64), np.array(list(d.values()), np.complex128)


def grid(n, dim):
    g = np.arange(n) / n
    return np.stack(np.meshgrid(*([g] * dim), indexing="ij"), -1).reshape(-1, dim)


def series(x, freq, val):
    """sum_k val_k exp(2 pi i k.x) and its gradient, at points x [P, dim]."""
    ph = np.exp(2j * np.pi * x @ np.asarray(freq, np.float64).T)       # [P, T]
    s = ph @ val
    grad = np.stack([ph @ (2j * np.pi * np.asarray(freq)[:, i] * val) for i in range(x.shape[1])], -1)
    return s, grad


def random_problem(seed, dim=2, deg_a=3, deg_u=4, n_a=3, n_u=4, hermitian_u=False):
    rng = np.random.default_rng(seed)
    pa = rng.integers(-deg_a, deg_a + 1, size=(n_a, dim))
    a_trig_f = np.vstack([np.zeros((1, dim), int), pa])
    a_trig_c = np.concatenate([[2.0], rng.uniform(-0.4, 0.4, n_a) + 1j * rng.uniform(-0.4, 0.4, n_a)])
    af, av = coeff_arrays(true_coefficients(a_trig_f, a_trig_c))
    uf = np.unique(rng.integers(-deg_u, deg_u + 1, size=(n_u, dim)), axis=0)
    uf = uf[uf.any(axis=1)]
    uv = rng.standard_normal(len(uf)) + 1j * rng.standard_normal(len(uf))
    if hermitian_u:      # u real: u_hat_{-k} = conj(u_hat_k)
        d = {}
        for k, v in zip(uf.tolist(), uv):
            d[tuple(k)] = d.get(tuple(k), 0) + v / 2
            d[tuple(-x for x in k)] = d.get(tuple(-x for x in k), 0) + np.conj(v) / 2
        uf, uv = coeff_arrays(d)
    return af, av, uf, uv


@pytest.mark.parametrize("seed", range(4))
def test_bilinear_form_identity_by_quadrature(seed):
    # <L[a] u_hat, v_hat> = integral a grad u . conj(grad v); the trapezoidal rule
    # on a 32^2 grid is exact for these trigonometric integrands (degree <= 11).
    af, av, uf, uv = random_problem(seed)
    # v lives on the support of L u (plus part of u's): the pairing is nontrivial
    Lf0, _ = galerkin.convolve(af, av, uf, uv)
    rng = np.random.default_rng(seed + 100)
    vf = np.unique(np.vstack([Lf0[rng.choice(len(Lf0), 8, replace=False)], uf[:2]]), axis=0)
    vf = vf[vf.any(axis=1)]
    vv = rng.standard_normal(len(vf)) + 1j * rng.standard_normal(len(vf))
    x = grid(32, 2)
    a_x, _ = series(x, af, av)
    _, gu = series(x, uf, uv)
    _, gv = series(x, vf, vv)
    lhs = np.mean(a_x * np.sum(gu * np.conj(gv), axis=1))
    Lf, Lv = galerkin.convolve(af, av, uf, uv)
    vd = {tuple(k): c for k, c in zip(vf.tolist(), vv)}
    rhs = sum(c * np.conj(vd.get(tuple(k), 0)) for k, c in zip(Lf.tolist(), Lv))
    assert abs(rhs) > 1.0
    assert abs(lhs - rhs) <= 1e-12 * np.linalg.norm(Lv) * np.linalg.norm(vv)


@pytest.mark.parametrize("seed", range(3))
def test_manufactured_forcing_matches_pointwise_operator(seed):
    # f = -div(a grad u) = -(grad a . grad u + a lap u), evaluated pointwise and
    # transformed with numpy's FFT, equals the convolution L[a] u_hat.
    af, av, uf, uv = random_problem(seed, hermitian_u=False)
    n = 32
    x = grid(n, 2)
    a_x, ga = series(x, af, av)
    _, gu = series(x, uf, uv)
    lap_u, _ = series(x, uf, -4 * np.pi ** 2 * (uf ** 2).sum(1) * uv)
    f_x = -(np.sum(ga * gu, axis=1) + a_x * lap_u)
    fhat = np.fft.fftn(f_x.reshape(n, n)) / n ** 2
    Lf, Lv = galerkin.convolve(af, av, uf, uv)
    for k, c in zip(Lf.tolist(), Lv):
        assert abs(fhat[k[0] % n, k[1] % n] - c) <= 1e-9 * (1 + abs(c))
    mask = np.zeros((n, n), bool)
    for k in Lf.tolist():
        mask[k[0] % n, k[1] % n] = True
    assert np.abs(fhat[~mask]).max() < 1e-9


def small_stamp(seed=0, N=2):
    rng = np.random.default_rng(seed)
    d = 3
    P = rng.integers(-3, 4, size=(3, d))
    af = np.vstack([np.zeros((1, d), int), P, -P])
    c = rng.uniform(-0.2, 0.2, 3) + 1j * rng.uniform(-0.2, 0.2, 3)
    av = np.concatenate([[1.0], c, np.conj(c)])
    q = rng.integers(-3, 4, size=(2, d))
    F = np.unique(np.vstack([q, -q]), axis=0)
    S, lvl = stamp.stamp_bfs(af, F, N)
    return af, av, S, lvl


def test_matrix_matches_convolution_when_support_inside():
    af, av, S, _ = small_stamp()
    rng = np.random.default_rng(1)
    inner = np.flatnonzero(stamp.stamp_bfs(af, S[:4], 0)[1] == 0)[:4]
    u = np.zeros(len(S), complex)
    u[inner] = rng.standard_normal(len(inner)) + 1j * rng.standard_normal(len(inner))
    L, nnz = galerkin.galerkin_matrix(S, af, av)
    Lf, Lv = galerkin.convolve(af, av, S[inner], u[inner])
    idx = stamp.index_map(S)
    y = L @ u
    for k, c in zip(Lf.tolist(), Lv):
        if tuple(k) in idx:
            assert abs(y[idx[tuple(k)]] - c) < 1e-12 * (1 + abs(c))
    assert nnz == galerkin.nnz_count(S, af)


def test_hermitian_and_zero_row():
    af, av, S, _ = small_stamp(2, N=3)
    L, _ = galerkin.galerkin_matrix(S, af, av)
    D = L.toarray()
    np.testing.assert_allclose(D, D.conj().T, atol=0, rtol=0)
    z = np.flatnonzero(~S.any(axis=1))
    if len(z):
        row = D[z[0]]
        assert row[z[0]] == 1 and np.count_nonzero(row) == 1
        assert np.count_nonzero(D[:, z[0]]) == 1


def test_constant_coefficient_is_diagonal():
    _, _, S, _ = small_stamp(3)
    d = S.shape[1]
    L, _ = galerkin.galerkin_matrix(S, np.zeros((1, d), int), np.array([2.5]))
    n2 = (S ** 2).sum(1)
    want = np.where(n2 == 0, 1.0, 4 * np.pi ** 2 * 2.5 * n2)
    np.testing.assert_allclose(L.toarray(), np.diag(want), rtol=1e-15)


def test_level_structure():
    # Proposition LExpansion: v on level n => L v on levels n-1 .. n+1
    af, av, S, lvl = small_stamp(4, N=3)
    L, _ = galerkin.galerkin_matrix(S, af, av)
    rng = np.random.default_rng(0)
    for n in range(3):
        v = np.where(lvl == n, rng.standard_normal(len(S)), 0)
        y = L @ v
        hit = set(lvl[np.abs(y) > 0].tolist())
        assert hit <= {n - 1, n, n + 1}


def test_apply_rows_matches_matrix():
    af, av, S, _ = small_stamp(5)
    L, _ = galerkin.galerkin_matrix(S, af, av)
    rng = np.random.default_rng(3)
    u = rng.standard_normal(len(S)) + 1j * rng.standard_normal(len(S))
    rows = rng.choice(len(S), 10, replace=False)
    np.testing.assert_allclose(galerkin.apply_rows(S, af, av, u, rows), (L @ u)[rows], rtol=1e-13, atol=1e-12)


def test_proxy_error_against_pointwise_residual():
    # Lemma ProxyError by Plancherel: ||f - L[a]u||_{L2} from the pointwise
    # residual -div(a grad u) - f on a grid (trapezoidal rule, exact here)
    af, av, uf, uv = random_problem(11)
    rng = np.random.default_rng(12)
    ff = np.unique(rng.integers(-5, 6, size=(6, 2)), axis=0)
    ff = ff[ff.any(axis=1)]
    fv = rng.standard_normal(len(ff)) + 1j * rng.standard_normal(len(ff))
    n = 32
    x = grid(n, 2)
    a_x, ga = series(x, af, av)
    _, gu = series(x, uf, uv)
    lap_u, _ = series(x, uf, -4 * np.pi ** 2 * (uf ** 2).sum(1) * uv)
    f_x, _ = series(x, ff, fv)
    res = -(np.sum(ga * gu, axis=1) + a_x * lap_u) - f_x
    want = np.sqrt(np.mean(np.abs(res) ** 2)) / np.linalg.norm(fv)
    got = galerkin.proxy_error(af, av, uf, uv, ff, fv)
    assert abs(got - want) <= 1e-12 * want


def test_proxy_error_vanishes_for_manufactured_data():
    af, av, uf, uv = random_problem(13)
    Lf, Lv = galerkin.convolve(af, av, uf, uv)
    assert galerkin.proxy_error(af, av, uf, uv, Lf, Lv) < 1e-15


def test_mc_point_values_against_closed_form():
    # sin(2 pi k.x) and cos(2 pi k.x) written as Re(-i e_k) and Re(e_k), at
    # points whose coordinates are exact binary fractions
    rng = np.random.default_rng(21)
    k = np.array([[3, -5, 7]])
    X = rng.integers(0, 1 << 32, size=(50, 3), dtype=np.int64)
    x = X / 2.0 ** 32
    np.testing.assert_allclose(galerkin.trig_at(k, [-1j], X), np.sin(2 * np.pi * x @ k[0]), atol=1e-9)
    np.testing.assert_allclose(galerkin.trig_at(k, [2.0], X), 2 * np.cos(2 * np.pi * x @ k[0]), atol=1e-9)
    # a point where k.x = 1/4 exactly: sin = 1, cos = 0
    Xq = np.array([[1 << 30, 0, 0]])
    assert abs(galerkin.trig_at([[1, 0, 0]], [-1j], Xq)[0] - 1.0) < 1e-15
    assert abs(galerkin.trig_at([[1, 0, 0]], [1.0], Xq)[0]) < 1e-15
    # coordinates far out: the phase is taken mod 1 in integers
    big = np.array([[2 ** 30 + 1, -(2 ** 30) + 3, 5]])
    np.testing.assert_allclose(galerkin.trig_at(big, [1.0], X[:5]),
                               np.cos(2 * np.pi * ((X[:5] @ big[0]) % (1 << 32)) / 2.0 ** 32), atol=1e-12)


def power_of_two_lattice(freq, m, seed):
    from oracle.lattice import is_reconstructing
    rng = np.random.default_rng(seed)
    M = 1 << m
    for _ in range(1000):
        z = rng.integers(1, M, size=freq.shape[1]) | 1
        if is_reconstructing(freq, z, M):
            return z, M
    raise AssertionError("no reconstructing lattice")


@pytest.mark.parametrize("seed", range(3))
def test_mc_on_a_reconstructing_lattice_equals_exact_proxy(seed):
    # averaging |r|^2 over a rank-1 lattice that separates supp(r_hat) is exact
    # (Parseval on the lattice), so the Monte Carlo form reproduces the exact
    # proxy to rounding
    af, av, uf, uv = random_problem(40 + seed, hermitian_u=True)
    rng = np.random.default_rng(seed)
    f_trig = np.unique(rng.integers(-6, 7, size=(5, 2)), axis=0)
    f_trig = f_trig[f_trig.any(axis=1)]
    f_coef = rng.standard_normal(len(f_trig)) + 1j * rng.standard_normal(len(f_trig))
    fF, fV = coeff_arrays(true_coefficients(f_trig, f_coef))
    gF, _ = galerkin.convolve(af, av, uf, uv)
    z, M = power_of_two_lattice(np.vstack([fF, gF]), 12, seed)
    j = np.arange(M, dtype=np.int64)
    X = ((j[:, None] * z[None, :]) % M) * ((1 << 32) // M)
    r, fx = galerkin.proxy_mc(af, av, uf, uv, f_trig, f_coef, X)
    want = galerkin.proxy_error(af, av, uf, uv, fF, fV)
    assert want > 1e-3
    assert abs(galerkin.mc_estimate(r, fx) - want) <= 1e-12 * want
    # and the pointwise r is real-valued data: r = f - f^{s,N} with f^{s,N} real
    assert np.isfinite(r).all()


def test_mc_estimate_is_statistically_consistent():
    af, av, uf, uv = random_problem(50, hermitian_u=True)
    rng = np.random.default_rng(51)
    f_trig = np.array([[1, 2], [3, -1], [0, 4]])
    f_coef = np.array([1.0, 0.5j, -0.7 + 0.2j])
    fF, fV = coeff_arrays(true_coefficients(f_trig, f_coef))
    X = rng.integers(0, 1 << 32, size=(20000, 2), dtype=np.int64)
    r, fx = galerkin.proxy_mc(af, av, uf, uv, f_trig, f_coef, X)
    want = galerkin.proxy_error(af, av, uf, uv, fF, fV)
    num, den = np.mean(r ** 2), np.mean(fx ** 2)
    se = np.std(r ** 2) / np.sqrt(len(r)) / np.sum(np.abs(fV) ** 2)
    assert abs(num / den - want ** 2) < 5 * se + 5 * np.std(fx ** 2) / np.sqrt(len(r)) * want ** 2
