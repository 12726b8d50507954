"""Advection-diffusion-reaction operator (Remark ADR) through the C ABI.

Stamping set and levels bit-exact against the oracle's breadth-first
construction with the union step set; the FP64 operator against the oracle's
explicit matrix (relative l2 1e-13); BiCGStab solutions against the oracle's
direct solve and against manufactured solutions (relative l2 1e-10); the
exact proxy against the oracle's convolution; extension equal to a fresh
build; the paths that do not take ADR stamps fail cleanly."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import adr as oadr
from oracle import stamp as ostamp
from oracle.sft import true_coefficients
from tests.helpers import rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2302_00752_gb300 import binding
    return binding


def coeffs(trig):
    dct = true_coefficients(trig.freq, trig.coef)
    keys = sorted(dct)
    return np.array(keys, np.int64).reshape(len(keys), -1), np.array([dct[k] for k in keys], np.complex128)


def data(inst):
    a, c = coeffs(inst.a), coeffs(inst.c)
    b = [coeffs(t) for t in inst.b]
    if inst.f is not None:
        f = coeffs(inst.f)
    else:
        f = oadr.convolve(a, b, c, inst.u_freq, inst.u_val)
    return a, b, c, f


def build(B, a, b, c, f, N):
    return B.stamp_build_adr(a[0], a[1], b, c[0], c[1], f[0], N)


def scatter_rhs(s, f):
    f_on, outside = s.scatter(f[0], f[1])
    return f_on, outside


SMALL = dict(n_a=1, n_bc=2)


@pytest.mark.parametrize("seed,N,kw", [(0, 1, {}), (1, 2, SMALL), (2, 0, {})])
def test_stamp_matches_oracle(B, seed, N, kw):
    inst = W.make_adr(seed, N=N, **kw)
    a, b, c, f = data(inst)
    U, _, _, _ = oadr.coefficient_maps(a, b, c)
    S_ref, l_ref = ostamp.stamp_bfs(U, f[0], N)
    with build(B, a, b, c, f, N) as s:
        S, lvl = s.export()
        assert np.array_equal(S.cpu().numpy(), S_ref)
        assert np.array_equal(lvl.cpu().numpy(), l_ref)
        _, nnz = oadr.adr_matrix(S_ref, a, b, c)
        assert s.nnz == nnz


@pytest.mark.parametrize("seed,N,kw", [(3, 1, {}), (4, 2, SMALL)])
def test_apply_matches_oracle(B, seed, N, kw):
    inst = W.make_adr(seed, N=N, **kw)
    a, b, c, f = data(inst)
    with build(B, a, b, c, f, N) as s:
        S = s.export()[0].cpu().numpy()
        rng = np.random.default_rng(seed)
        u = rng.standard_normal(len(S)) + 1j * rng.standard_normal(len(S))
        y = B.galerkin_apply(s, torch.as_tensor(u).cuda()).cpu().numpy()
    L, _ = oadr.adr_matrix(S, a, b, c)
    assert rel_l2(y, L @ u) < 1e-13


@pytest.mark.parametrize("seed,N,kw", [(5, 1, {}), (6, 1, {}), (7, 2, SMALL)])
def test_solve_matches_oracle(B, seed, N, kw):
    inst = W.make_adr(seed, N=N, **kw)
    a, b, c, f = data(inst)
    with build(B, a, b, c, f, N) as s:
        f_on, outside = scatter_rhs(s, f)
        assert outside == 0
        u, st = B.solve(s, f_on, 1e-12, 2000, "fp64")
        S = s.export()[0].cpu().numpy()
    assert st["status"] == "SS_OK" and st["rel_residual"] <= 1e-11
    u_ref, _ = oadr.solve(S, a, b, c, *f)
    assert rel_l2(u.cpu().numpy(), u_ref) < 1e-10


@pytest.mark.parametrize("N,n_u,kw", [(1, 3, {}), (2, 1, SMALL)])
def test_manufactured_solution(B, N, n_u, kw):
    # f = L u over Z^d with u on level 0: the Galerkin solution on S^N is u
    inst = W.make_adr(8, N=N, manufactured_u=n_u, **kw)
    a, b, c, f = data(inst)
    with build(B, a, b, c, f, N) as s:
        f_on, _ = scatter_rhs(s, f)
        u, st = B.solve(s, f_on, 1e-13, 2000, "fp64")
        want, outside = s.scatter(inst.u_freq, inst.u_val)
        assert outside == 0
    assert st["status"] == "SS_OK"
    assert rel_l2(u.cpu().numpy(), want.cpu().numpy()) < 1e-10


def test_nonzero_mean_forcing(B):
    # the reaction term determines u_hat_0: f_hat_0 != 0 and 0 in F are allowed
    inst = W.make_adr(9, N=1)
    a, b, c, f = data(inst)
    f = (np.vstack([np.zeros((1, 3), np.int64), f[0]]), np.concatenate([[0.7 + 0j], f[1]]))
    with build(B, a, b, c, f, 1) as s:
        z = s.zero_index
        f_on, _ = scatter_rhs(s, f)
        u, st = B.solve(s, f_on, 1e-12, 2000, "fp64")
        S = s.export()[0].cpu().numpy()
    assert z >= 0 and not S[z].any()
    u_ref, _ = oadr.solve(S, a, b, c, *f)
    assert st["status"] == "SS_OK"
    assert rel_l2(u.cpu().numpy(), u_ref) < 1e-10
    assert abs(u_ref[z]) > 1e-3


def test_exact_proxy_matches_oracle(B):
    inst = W.make_adr(10, N=1)
    a, b, c, f = data(inst)
    U, _, _, _ = oadr.coefficient_maps(a, b, c)
    S, _ = ostamp.stamp_bfs(U, f[0], 1)
    rng = np.random.default_rng(10)
    u = rng.standard_normal(len(S)) + 1j * rng.standard_normal(len(S))
    with build(B, a, b, c, f, 1) as s:
        s.extend(1)
        f1, _ = s.scatter(*f)
        num, den = B.proxy_residual(s, torch.as_tensor(u), f1)
    want = oadr.proxy_error(a, b, c, S, u, *f)
    assert abs(np.sqrt(num / den) - want) <= 1e-12 * want


def test_extend_equals_fresh_build(B):
    inst = W.make_adr(11, N=1, **SMALL)
    a, b, c, f = data(inst)
    with build(B, a, b, c, f, 1) as s, build(B, a, b, c, f, 2) as fresh:
        s.extend(1)
        assert s.size == fresh.size and s.nnz == fresh.nnz
        assert torch.equal(s.export()[0], fresh.export()[0])
        rng = np.random.default_rng(2)
        u = torch.as_tensor(rng.standard_normal(s.size) + 1j * rng.standard_normal(s.size)).cuda()
        assert torch.equal(B.galerkin_apply(s, u), B.galerkin_apply(fresh, u))


def test_paths_without_adr_support_refuse(B):
    inst = W.make_adr(12, N=1, **SMALL)
    a, b, c, f = data(inst)
    with build(B, a, b, c, f, 1) as s:
        f_on, _ = scatter_rhs(s, f)
        for call in (lambda: B.solve(s, f_on, 1e-12, 100, "fp32"),
                     lambda: B.galerkin_apply(s, f_on.to(torch.complex64), "fp32"),
                     lambda: B.solve_noalloc(s, f_on, torch.empty_like(f_on)),
                     lambda: B.Batch([s])):
            with pytest.raises(B.SSError) as e:
                call()
            assert e.value.args[0] == 1 or "SS_ERR_INVALID" in str(e.value)
        # and the stamp is still usable
        u, st = B.solve(s, f_on, 1e-12, 2000, "fp64")
        assert st["status"] == "SS_OK"


def test_pipeline_recovers_and_solves(B):
    # Remark ADR's pipeline: lattice for the union of the supports, SFT of
    # a, b_1..b_d, c and f, union stamp, BiCGStab; against the oracle's direct
    # solve on the exact coefficients
    from paper_2302_00752_gb300 import pipeline as gp
    inst = W.make_adr(13, N=1)
    a, b, c, f = data(inst)
    res = gp.run_adr(inst)
    try:
        S = res.stamp.export()[0].cpu().numpy()
        U, _, _, _ = oadr.coefficient_maps(a, b, c)
        S_ref, _ = ostamp.stamp_bfs(U, f[0], 1)
        assert np.array_equal(S, S_ref)
        u_ref, _ = oadr.solve(S, a, b, c, *f)
        assert res.stats["status"] == "SS_OK"
        assert rel_l2(res.u.cpu().numpy(), u_ref) < 1e-10
    finally:
        res.stamp.destroy()


def test_monte_carlo_proxy_matches_oracle(B):
    from oracle import galerkin as ogal
    inst = W.make_adr(14, N=1, **SMALL)
    a, b, c, f = data(inst)
    U, _, _, _ = oadr.coefficient_maps(a, b, c)
    S, _ = ostamp.stamp_bfs(U, f[0], 1)
    rng = np.random.default_rng(14)
    u = rng.standard_normal(len(S)) + 1j * rng.standard_normal(len(S))
    X = W.mc_points(5, 300, 3)
    with build(B, a, b, c, f, 1) as s:
        s.extend(1)
        r, fx = B.proxy_mc(s, torch.as_tensor(u), inst.f.freq, inst.f.coef, X)
    gf, gv = oadr.convolve(a, b, c, S, u)
    f_ref = ogal.trig_at(inst.f.freq, inst.f.coef, X)
    r_ref = f_ref - ogal.trig_at(gf, gv, X)
    tol = 1e-12 * (np.abs(gv).sum() + np.abs(inst.f.coef).sum())
    assert np.max(np.abs(fx.cpu().numpy() - f_ref)) <= tol
    assert np.max(np.abs(r.cpu().numpy() - r_ref)) <= tol


def test_repeated_solves_identical(B):
    # every partial sum a BiCGStab phase reads is written by the phase before
    # it: a second solve on the same stamp reuses the workspace the first one
    # left behind and must return the same bits
    inst = W.make_adr(15, N=1)
    a, b, c, f = data(inst)
    with build(B, a, b, c, f, 1) as s:
        f_on, _ = scatter_rhs(s, f)
        u1, st1 = B.solve(s, f_on, 1e-12, 2000, "fp64")
        u2, st2 = B.solve(s, f_on, 1e-12, 2000, "fp64")
        S = s.export()[0].cpu().numpy()
    assert st1["status"] == st2["status"] == "SS_OK"
    assert st1["rel_residual"] <= 1e-11 and st2["rel_residual"] <= 1e-11
    assert torch.equal(u1, u2)
    u_ref, _ = oadr.solve(S, a, b, c, *f)
    assert rel_l2(u2.cpu().numpy(), u_ref) < 1e-10
