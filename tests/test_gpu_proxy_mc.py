"""Monte Carlo proxy (Lemma ProxyError; Section "Code and testing overview").

Per point, r(x) = f(x) - f^{s,N}(x) and f(x) from proxy_mc equal the oracle's
values on the same seeded points and the same seeded u.  Tolerance, from the
arithmetic: every term is a product of double-float values (a 2^-44 relative
bound per product, five products per term) and table entries rounded to
double-float (2^-48 relative), so |error| <= 1e-12 * (sum_t |c_t|) with the sum
over all terms of f and of f^{s,N} (2^-44 * 8 terms of slack * 10 ~ 5e-12
relative to the largest term, well inside the bound summed over terms).

The estimate sqrt(sum r^2 / sum f^2) agrees with the exact proxy (proxy_residual,
Lemma ProxyError) to within the Monte Carlo standard error."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import galerkin as ogal
from oracle import stamp as ostamp
from oracle.stamp import index_map
from tests.helpers import stamp_inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2302_00752_gb300 import binding
    return binding


def hermitian_random(S, seed):
    """Seeded u on S with u_{-k} = conj(u_k) where -k is in S (a real function)."""
    rng = np.random.default_rng(seed)
    u = rng.standard_normal(len(S)) + 1j * rng.standard_normal(len(S))
    idx = index_map(S)
    out = u.copy()
    for i, k in enumerate(np.asarray(S).tolist()):
        j = idx.get(tuple(-x for x in k))
        if j is not None:
            out[i] = (u[i] + np.conj(u[j])) / 2
    return out


def l1_terms(af, av, S, u, f_coef):
    _, gv = ogal.convolve(af, av, S, u)
    return float(np.abs(gv).sum() + np.abs(np.asarray(f_coef)).sum())


CASES = [
    ("tiny2", lambda: W.make_tiny(7, d=2, n_cos=2, n_u=2, N=1, manufactured_u=False), 1, 257),
    ("tiny3", lambda: W.make_tiny(8, d=3, n_cos=2, n_u=2, N=2, manufactured_u=False), 2, 1000),
    ("d5", lambda: W.make_tiny(9, d=5, n_cos=2, n_u=3, N=1, manufactured_u=False), 1, 700),
    ("d8", lambda: W.make_tiny(10, d=8, n_cos=3, n_u=2, N=1, manufactured_u=False), 1, 1),
    ("cfg3", lambda: W.make_cfg3(), 1, 300),
    ("mid4", lambda: W.make_tiny(12, d=4, n_cos=4, n_u=4, N=3, manufactured_u=False), 3, 1000),
    ("onet64", lambda: W.make_one_term(64, seed=2, kmax=500), 3, 513),
]


@pytest.mark.parametrize("name,make,N,Q", CASES, ids=[c[0] for c in CASES])
def test_point_values_match_oracle(B, name, make, N, Q):
    inst = make()
    _, af, av, ff, fv = stamp_inputs(inst)
    S, _ = ostamp.stamp_bfs(af, ff, N)
    u = hermitian_random(S, 100 + N)
    X = W.mc_points(3, Q, S.shape[1])
    r_ref, f_ref = ogal.proxy_mc(af, av, S, u, inst.f.freq, inst.f.coef, X)
    with B.stamp_build(af, av, ff, N) as s:
        s.extend(1)
        r, f = B.proxy_mc(s, torch.as_tensor(u), inst.f.freq, inst.f.coef, X)
    tol = 1e-12 * l1_terms(af, av, S, u, inst.f.coef)
    assert np.max(np.abs(f.cpu().numpy() - f_ref)) <= tol
    assert np.max(np.abs(r.cpu().numpy() - r_ref)) <= tol


def test_no_points_and_no_forcing_terms(B):
    inst = W.make_tiny(11, d=2, n_cos=2, n_u=2, N=1, manufactured_u=False)
    _, af, av, ff, fv = stamp_inputs(inst)
    S, _ = ostamp.stamp_bfs(af, ff, 1)
    u = hermitian_random(S, 5)
    with B.stamp_build(af, av, ff, 1) as s:
        s.extend(1)
        r, f = B.proxy_mc(s, torch.as_tensor(u), inst.f.freq, inst.f.coef, np.zeros((0, 2), np.uint32))
        assert r.numel() == 0 and f.numel() == 0
        # f = 0: r = -f^{s,N}
        X = W.mc_points(4, 64, 2)
        r, f = B.proxy_mc(s, torch.as_tensor(u), np.zeros((0, 2), np.int32), np.zeros(0, complex), X)
    r_ref, _ = ogal.proxy_mc(af, av, S, u, np.zeros((0, 2), np.int64), np.zeros(0, complex), X)
    assert torch.count_nonzero(f).item() == 0
    assert np.max(np.abs(r.cpu().numpy() - r_ref)) <= 1e-12 * l1_terms(af, av, S, u, [])


@pytest.mark.parametrize("d,seed", [(1, 0), (16, 1), (64, 2)])
def test_estimate_tracks_exact_proxy(B, d, seed):
    # Section "Low sparsity": one-term a and f, N = 1..4; with 4000 points the
    # Monte Carlo estimate stays within a few standard errors of the exact value
    inst = W.make_one_term(d, seed=seed, kmax=500)
    _, af, av, ff, fv = stamp_inputs(inst)
    X = W.mc_points(seed, 4000, d)
    with B.stamp_build(af, av, ff, 1) as s:
        for N in range(1, 5):
            f_on, _ = s.scatter(ff, fv)
            u, st = B.solve(s, f_on, 1e-13, 1000, "fp64")
            s.extend(1)
            f1, _ = s.scatter(ff, fv)
            num, den = B.proxy_residual(s, u, f1)
            exact = np.sqrt(num / den)
            r, f = B.proxy_mc(s, u, inst.f.freq, inst.f.coef, X)
            r2 = r.cpu().numpy() ** 2
            f2 = f.cpu().numpy() ** 2
            est2 = r2.mean() / f2.mean()
            # delta-method standard error of the ratio of means
            se2 = np.sqrt(np.var(r2 - est2 * f2) / len(r2)) / f2.mean()
            assert abs(est2 - exact ** 2) <= 5 * se2 + 1e-20, (N, est2, exact ** 2, se2)
