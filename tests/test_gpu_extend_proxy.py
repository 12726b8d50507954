"""N-sweep reuse (stamp_extend) and the exact proxy error (Lemma ProxyError).

stamp_extend grows S^N to S^{N+L} in place: the result equals a fresh build of
S^{N+L} bit for bit (canonical order makes S^N its prefix).  proxy_residual on
S^{N+1} with the solution on S^N equals the oracle's proxy error computed over
all of Z^d by exact convolution."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import galerkin as ogal
from oracle import stamp as ostamp
from tests.helpers import rel_l2, stamp_inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2302_00752_gb300 import binding
    return binding


def same_set(s1, s2):
    S1, l1 = s1.export()
    S2, l2 = s2.export()
    return (s1.size == s2.size and s1.nnz == s2.nnz and s1.zero_index == s2.zero_index
            and torch.equal(S1, S2) and torch.equal(l1, l2))


@pytest.mark.parametrize("seed,N,L", [(0, 1, 1), (1, 1, 2), (2, 2, 1), (3, 0, 3)])
def test_extend_equals_fresh_build(B, seed, N, L):
    inst = W.make_tiny(seed, d=2 + seed % 2, n_cos=2, n_u=2, N=N, manufactured_u=False)
    _, af, av, ff, _ = stamp_inputs(inst)
    with B.stamp_build(af, av, ff, N) as s, B.stamp_build(af, av, ff, N + L) as fresh:
        s.extend(L)
        assert same_set(s, fresh)
        S, lvl = s.export()
        S_ref, l_ref = ostamp.stamp_bfs(af, ff, N + L)
        assert np.array_equal(S.cpu().numpy(), S_ref) and np.array_equal(lvl.cpu().numpy(), l_ref)
        rng = np.random.default_rng(seed)
        u = torch.as_tensor(rng.standard_normal(s.size) + 1j * rng.standard_normal(s.size)).cuda()
        assert torch.equal(B.galerkin_apply(s, u), B.galerkin_apply(fresh, u))


def test_extend_widens_the_key_layout(B):
    # coordinates of S^{N+1} fit 5-bit fields at N = 1; N = 6 needs wider ones
    A = np.array([[-3, 0], [0, -3], [0, 0], [0, 3], [3, 0]])
    av = np.array([0.1, 0.1, 1.0, 0.1, 0.1], complex)
    F = np.array([[4, 1], [-4, -1]])
    with B.stamp_build(A, av, F, 1) as s, B.stamp_build(A, av, F, 6) as fresh:
        s.extend(5)
        assert same_set(s, fresh)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_solve_after_extend(B, prec):
    inst, af, av, ff, fv = stamp_inputs("cfg1")
    with B.stamp_build(af, av, ff, 1) as s, B.stamp_build(af, av, ff, 2) as fresh:
        f1, _ = s.scatter(ff, fv)
        B.solve(s, f1, 1e-12, 500, prec)          # a solve before the extension
        s.extend(1)
        f2, _ = s.scatter(ff, fv)
        u, st = B.solve(s, f2, 1e-12, 500, prec)
        u_ref, _ = B.solve(fresh, f2, 1e-12, 500, prec)
        assert st["status"] == "SS_OK"
        assert rel_l2(u.cpu().numpy(), u_ref.cpu().numpy()) < 1e-10


@pytest.mark.parametrize("name,N", [("tiny", 1), ("tiny", 2), ("cfg3", 2)])
def test_proxy_matches_oracle(B, name, N):
    # the same seeded u on S^N on both sides (any u: the proxy is a residual)
    inst = W.make_tiny(5, d=3, n_cos=2, n_u=2, N=N, manufactured_u=False) if name == "tiny" else W.make_cfg3()
    _, af, av, ff, fv = stamp_inputs(inst)
    S, _ = ostamp.stamp_bfs(af, ff, N)
    rng = np.random.default_rng(N)
    u = rng.standard_normal(len(S)) + 1j * rng.standard_normal(len(S))
    u[~S.any(axis=1)] = 0.0                 # the solver's pinned mean
    with B.stamp_build(af, av, ff, N) as s:
        s.extend(1)
        f1, outside = s.scatter(ff, fv)
        assert outside == 0
        num, den = B.proxy_residual(s, torch.as_tensor(u), f1)
    got = np.sqrt(num / den)
    want = ogal.proxy_error(af, av, S, u, ff, fv)
    assert abs(got - want) <= 1e-12 * want


def test_proxy_decays_with_stamping_level(B):
    # Section "Low sparsity": the error converges exponentially in N
    inst = W.make_one_term(6, seed=3, kmax=50)
    _, af, av, ff, fv = stamp_inputs(inst)
    errs = []
    with B.stamp_build(af, av, ff, 1) as s:
        for N in range(1, 5):
            f_on, _ = s.scatter(ff, fv)
            u, _ = B.solve(s, f_on, 1e-13, 1000, "fp64")
            s.extend(1)
            f1, _ = s.scatter(ff, fv)
            num, den = B.proxy_residual(s, u, f1)
            errs.append(np.sqrt(num / den))
    assert all(b < 0.5 * a for a, b in zip(errs, errs[1:])), errs
