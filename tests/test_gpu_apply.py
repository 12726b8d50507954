"""galerkin_apply parity with the oracle's explicit matrix (eq.
FiniteGalerkinOperator).  FP64: relative l2 error <= 1e-14 (a row sums at most
|supp a_hat| terms with exact integer coefficients; the only differences are the
summation order and one rounding of 4 pi^2 a_hat_p).  FP32: <= 2e-6 (FP32
storage of u and a_hat, FP32 accumulation over <= 41 terms)."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import galerkin as ogal
from oracle import stamp as ostamp
from tests.helpers import rel_l2, stamp_inputs

pytestmark = pytest.mark.gpu

TOL64, TOL32 = 1e-14, 2e-6


@pytest.fixture(scope="module")
def B():
    from paper_2302_00752_gb300 import binding
    return binding


def rand_u(n, seed=0):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(n) + 1j * rng.standard_normal(n)


def check_full(B, af, av, F, N):
    S, _ = ostamp.stamp_bfs(af, F, N)
    L, nnz = ogal.galerkin_matrix(S, af, av)
    u = rand_u(len(S))
    with B.stamp_build(af, av, F, N) as s:
        assert s.nnz == nnz
        y64 = B.galerkin_apply(s, torch.as_tensor(u).cuda()).cpu().numpy()
        y32 = B.galerkin_apply(s, torch.as_tensor(u.astype(np.complex64)).cuda()).cpu().numpy()
    ref = L @ u
    assert rel_l2(y64, ref) <= TOL64
    assert rel_l2(y32, ref) <= TOL32


@pytest.mark.parametrize("seed", range(4))
def test_tiny(B, seed):
    inst = W.make_tiny(seed, d=2 + seed % 2, n_cos=3, n_u=3, N=2 + seed % 2)
    _, af, av, ff, _ = stamp_inputs(inst)
    check_full(B, af, av, ff, inst.N)


@pytest.mark.parametrize("name", ["cfg1", "cfg3"])
def test_configs(B, name):
    inst, af, av, ff, _ = stamp_inputs(name)
    check_full(B, af, av, ff, inst.N)


def test_complex_coefficients(B):
    # a with sine terms: a_hat not real, L Hermitian but complex
    rng = np.random.default_rng(7)
    d = 3
    P = rng.integers(-3, 4, size=(3, d))
    c = 0.1 * (rng.standard_normal(3) + 1j * rng.standard_normal(3))
    af = np.vstack([np.zeros((1, d), int), P, -P])
    av = np.concatenate([[1.0], c, np.conj(c)])
    F = np.unique(rng.integers(-4, 5, size=(6, d)), axis=0)
    F = F[F.any(axis=1)]
    check_full(B, af, av, F, 3)


@pytest.mark.parametrize("name,rows", [("cfg2", 400), ("cfg5", 300)])
def test_full_size_sampled_rows(B, name, rows):
    inst, af, av, ff, _ = stamp_inputs(name)
    with B.stamp_build(af, av, ff, inst.N) as s:
        S = s.export()[0].cpu().numpy()
        u = rand_u(len(S), 1)
        y64 = B.galerkin_apply(s, torch.as_tensor(u).cuda()).cpu().numpy()
        y32 = B.galerkin_apply(s, torch.as_tensor(u.astype(np.complex64)).cuda()).cpu().numpy()
        # Hermitian: <L x, v> = <x, L v>
        v = rand_u(len(S), 2)
        Lv = B.galerkin_apply(s, torch.as_tensor(v).cuda()).cpu().numpy()
    rng = np.random.default_rng(3)
    pick = np.concatenate([rng.choice(len(S), rows, replace=False), [0, len(S) - 1]])
    ref = ogal.apply_rows(S, af, av, u, pick)
    assert rel_l2(y64[pick], ref) <= TOL64
    assert rel_l2(y32[pick], ref) <= TOL32
    lhs, rhs = np.vdot(v, y64), np.vdot(Lv, u)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
