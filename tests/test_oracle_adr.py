"""Pins for oracle.adr (Remark ADR): the Fourier-side operator against the PDE
evaluated pointwise, the pure-diffusion special case, the explicit matrix
against the convolution, manufactured solutions."""
import numpy as np
import pytest

import workloads as W
from oracle import adr, galerkin, stamp
from oracle.sft import true_coefficients


def coeffs(trig):
    dct = true_coefficients(trig.freq, trig.coef)
    keys = sorted(dct)
    return np.array(keys, np.int64).reshape(len(keys), -1), np.array([dct[k] for k in keys], np.complex128)


def small_adr(seed, kmax=3, manufactured_u=3, n_a=2, n_bc=5):
    inst = W.make_adr(seed, N=1, kmax=kmax, n_a=n_a, n_bc=n_bc, manufactured_u=manufactured_u)
    a = coeffs(inst.a)
    b = [coeffs(t) for t in inst.b]
    c = coeffs(inst.c)
    return inst, a, b, c


def grid(n, dim):
    g = np.arange(n) / n
    return np.stack(np.meshgrid(*([g] * dim), indexing="ij"), -1).reshape(-1, dim)


def series(x, freq, val):
    ph = np.exp(2j * np.pi * x @ np.asarray(freq, np.float64).T)
    s = ph @ val
    grad = np.stack([ph @ (2j * np.pi * np.asarray(freq)[:, i] * val) for i in range(x.shape[1])], -1)
    lap = ph @ (-4 * np.pi ** 2 * (np.asarray(freq, np.float64) ** 2).sum(1) * val)
    return s, grad, lap


@pytest.mark.parametrize("seed", range(3))
def test_convolution_against_pointwise_pde(seed):
    # -div(a grad u) + b.grad u + c u on a 16^3 grid, transformed by numpy's
    # FFT: exact for frequencies below 8 per coordinate (|k_c| <= 6 here)
    inst, a, b, c = small_adr(seed)
    n, d = 16, 3
    x = grid(n, d)
    a_x, ga, _ = series(x, *a)
    u_x, gu, lu = series(x, inst.u_freq, inst.u_val)
    f_x = -(np.sum(ga * gu, axis=1) + a_x * lu)
    for j in range(d):
        bj, _, _ = series(x, *b[j])
        f_x += bj * gu[:, j]
    c_x, _, _ = series(x, *c)
    f_x += c_x * u_x
    F = np.fft.fftn(f_x.reshape(n, n, n)) / n ** d
    kf, kv = adr.convolve(a, b, c, inst.u_freq, inst.u_val)
    assert np.abs(kf).max() < n // 2
    got = np.array([F[tuple(k % n)] for k in kf])
    np.testing.assert_allclose(kv, got, atol=1e-10 * np.abs(kv).max())
    # every other grid coefficient vanishes
    mask = np.ones((n, n, n), bool)
    for k in kf:
        mask[tuple(k % n)] = False
    assert np.abs(F[mask]).max() < 1e-10 * np.abs(kv).max()


def test_pure_diffusion_is_eq_gf():
    inst, a, b, c = small_adr(4)
    zero = (np.zeros((0, 3), np.int64), np.zeros(0, complex))
    kf, kv = adr.convolve(a, [zero] * 3, zero, inst.u_freq, inst.u_val)
    gf, gv = galerkin.convolve(*a, inst.u_freq, inst.u_val)
    assert np.array_equal(kf, gf)
    np.testing.assert_allclose(kv, gv, rtol=1e-14, atol=1e-12)


def test_union_step_set():
    inst, a, b, c = small_adr(5)
    U, A, Bv, C = adr.coefficient_maps(a, b, c)
    want = {tuple(k) for k in a[0].tolist()} | {tuple(k) for k in c[0].tolist()}
    for bf, _ in b:
        want |= {tuple(k) for k in bf.tolist()}
    assert {tuple(k) for k in U.tolist()} == want
    assert np.array_equal(U, U[stamp.lex_order(U)])
    assert {tuple(-x for x in k) for k in U.tolist()} == want     # real data: symmetric


@pytest.mark.parametrize("seed", range(2))
def test_matrix_equals_convolution_on_the_stamp(seed):
    inst, a, b, c = small_adr(seed)
    U, _, _, _ = adr.coefficient_maps(a, b, c)
    S, _ = stamp.stamp_bfs(U, inst.u_freq, 1)      # supp u and all its neighbours
    L, nnz = adr.adr_matrix(S, a, b, c)
    idx = stamp.index_map(S)
    u = np.zeros(len(S), complex)
    for k, v in zip(inst.u_freq.tolist(), inst.u_val):
        u[idx[tuple(k)]] = v
    kf, kv = adr.convolve(a, b, c, inst.u_freq, inst.u_val)
    want = np.zeros(len(S), complex)
    for k, v in zip(kf.tolist(), kv):
        want[idx[tuple(k)]] = v
    np.testing.assert_allclose(L @ u, want, rtol=1e-13, atol=1e-12 * np.abs(want).max())
    assert nnz == L.nnz or nnz >= L.nnz


@pytest.mark.parametrize("N,n_u,n_a,n_bc", [(1, 2, 2, 5), (2, 1, 1, 1)])
def test_manufactured_solution_reproduced(N, n_u, n_a, n_bc):
    inst, a, b, c = small_adr(6, kmax=4, manufactured_u=n_u, n_a=n_a, n_bc=n_bc)
    ff, fv = adr.convolve(a, b, c, inst.u_freq, inst.u_val)
    U, _, _, _ = adr.coefficient_maps(a, b, c)
    S, _ = stamp.stamp_bfs(U, ff, N)
    u, _ = adr.solve(S, a, b, c, ff, fv)
    idx = stamp.index_map(S)
    want = np.zeros(len(S), complex)
    for k, v in zip(inst.u_freq.tolist(), inst.u_val):
        want[idx[tuple(k)]] = v
    np.testing.assert_allclose(u, want, atol=1e-12 * np.abs(want).max())
    assert adr.proxy_error(a, b, c, S, u, ff, fv) < 1e-12
