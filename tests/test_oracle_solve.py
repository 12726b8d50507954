"""Pins for oracle.solve and oracle.pipeline (Algorithm 1; eq.
SparseSpectralSFTEquation; the low-sparsity test of Section "Low sparsity")."""
import numpy as np
import pytest

import workloads as W
from oracle import galerkin, pipeline, solve, stamp
from oracle.sft import true_coefficients


def coeff_arrays(d):
    return np.array(list(d.keys()), np.int64), np.array(list(d.values()), np.complex128)


def test_constant_coefficient_closed_form():
    # a = a0: u_hat_k = f_hat_k / (4 pi^2 a0 |k|^2)
    rng = np.random.default_rng(0)
    d, a0 = 4, 1.7
    q = rng.integers(-5, 6, size=(6, d))
    q = q[q.any(axis=1)]
    F = np.vstack([q, -q])
    fv = rng.standard_normal(len(q)) + 1j * rng.standard_normal(len(q))
    fval = np.concatenate([fv, np.conj(fv)])
    res = pipeline.solve_recovered(2, np.zeros((1, d), int), np.array([a0]), F, fval, tol=1e-15)
    want = res.f_on_S / np.where((res.S ** 2).sum(1) == 0, 1, 4 * np.pi ** 2 * a0 * (res.S ** 2).sum(1))
    assert solve.rel_l2(res.u, want) < 1e-14
    assert res.iters <= 2


@pytest.mark.parametrize("seed", range(3))
def test_manufactured_solution_is_reproduced(seed):
    inst = W.make_tiny(seed, d=3, n_cos=2, n_u=3, N=2)
    res = pipeline.run(inst)
    idx = stamp.index_map(res.S)
    want = np.zeros(len(res.S), complex)
    for k, v in zip(inst.u_freq.tolist(), inst.u_val):
        want[idx[tuple(k)]] = v
    assert solve.rel_l2(res.u, want) < 1e-12


@pytest.mark.parametrize("seed", range(3))
def test_pcg_equals_dense_lu(seed):
    inst = W.make_tiny(seed + 10, d=2, n_cos=2, n_u=2, N=3, manufactured_u=False)
    res = pipeline.run(inst)
    L, _ = galerkin.galerkin_matrix(res.S, res.a_freq, res.a_val)
    x = solve.dense_solve(L, res.f_on_S)
    assert len(res.S) <= 2000
    assert solve.rel_l2(res.u, x) < 1e-12


def chain_solution(N, a0, c, gff, gfa, gaa, fk):
    """Tridiagonal system on the chain k_m = k_f + m k_a, |m| <= N, from the Gram
    values k_f.k_f, k_f.k_a, k_a.k_a only: diagonal 4pi^2 a0 |k_m|^2, off-diagonal
    4pi^2 (k_m.k_{m+-1}) c/2; right-hand side fk at m = 0."""
    m = np.arange(-N, N + 1)
    dot = lambda i, j: gff + (i + j) * gfa + i * j * gaa
    diag = 4 * np.pi ** 2 * a0 * np.array([dot(i, i) for i in m], float)
    off = np.array([4 * np.pi ** 2 * dot(i, i + 1) * c / 2 for i in m[:-1]], float)
    lower = np.concatenate([[0], off])
    upper = np.concatenate([off, [0]])
    rhs = np.zeros(len(m), complex)
    rhs[N] = fk
    return m, solve.thomas(lower, diag, upper, rhs)


@pytest.mark.parametrize("d", [1, 2, 5, 16])
def test_one_term_chain_and_dimension_independence(d):
    inst = W.make_one_term(d, seed=7)
    ka = inst.a.freq[1].astype(np.int64)
    kf = inst.f.freq[0].astype(np.int64)
    c = float(inst.a.coef[1].real)
    for N in (1, 3):
        af, av = coeff_arrays(true_coefficients(inst.a.freq, inst.a.coef))
        ff, fv = coeff_arrays(true_coefficients(inst.f.freq, inst.f.coef))
        res = pipeline.solve_recovered(N, af, av, ff, fv, tol=1e-15)
        idx = stamp.index_map(res.S)
        m, x = chain_solution(N, 4.0, c, kf @ kf, kf @ ka, ka @ ka, fv[0] if tuple(ff[0]) == tuple(kf) else fv[1])
        got = np.array([res.u[idx[tuple(kf + i * ka)]] for i in m])
        assert solve.rel_l2(got, x) < 1e-12
        # the mirror chain carries the conjugate solution
        mirror = np.array([res.u[idx[tuple(-kf - i * ka)]] for i in m])
        assert solve.rel_l2(mirror, np.conj(x)) < 1e-12


def test_invariance_under_coordinate_maps():
    inst = W.make_tiny(4, d=3, n_cos=2, n_u=2, N=2, manufactured_u=False)
    base = pipeline.run(inst)
    sol = {tuple(k): v for k, v in zip(base.S.tolist(), base.u)}
    perm, sign = np.array([2, 0, 1]), np.array([1, -1, 1])
    for fmap in (lambda f: f[:, perm], lambda f: f * sign, lambda f: np.hstack([f, np.zeros((len(f), 1), f.dtype)])):
        a_freq = fmap(base.a_freq.astype(np.int64))
        f_freq = fmap(base.f_freq.astype(np.int64))
        res = pipeline.solve_recovered(2, a_freq, base.a_val, f_freq, base.f_val, tol=1e-15)
        # map every original frequency and compare values
        img = fmap(base.S.astype(np.int64))
        idx = stamp.index_map(res.S)
        assert len(res.S) == len(base.S)
        got = np.array([res.u[idx[tuple(k)]] for k in img.tolist()])
        assert solve.rel_l2(got, base.u) < 1e-12


def test_hermitian_solution_and_positivity_check():
    inst = W.make_tiny(6, d=2, n_cos=3, n_u=2, N=3, manufactured_u=False)
    res = pipeline.run(inst)
    idx = stamp.index_map(res.S)
    for k, v in zip(res.S.tolist(), res.u):
        mk = tuple(-x for x in k)
        if mk in idx:
            assert abs(res.u[idx[mk]] - np.conj(v)) < 1e-12 * np.abs(res.u).max()
    assert solve.is_elliptic(res.a_freq, res.a_val)
    assert not solve.is_elliptic(np.array([[0, 0], [1, 0], [-1, 0]]), np.array([1.0, 0.6, 0.6]))


def test_cfg1_end_to_end():
    inst = W.make_cfg1()
    res = pipeline.run(inst)
    assert res.M == 1089 and list(res.z) == [1, 33]
    assert len(res.a_freq) == 9
    idx = stamp.index_map(res.S)
    want = np.zeros(len(res.S), complex)
    for k, v in zip(inst.u_freq.tolist(), inst.u_val):
        want[idx[tuple(k)]] = v
    assert solve.rel_l2(res.u, want) < 1e-12
