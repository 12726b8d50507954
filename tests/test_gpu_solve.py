"""solve parity: the GPU solution of L_{N,s} u = f (eq. SparseSpectralSFTEquation)
against the oracle's FP64 PCG (run to 1e-14) on the same recovered data, within
relative l2 1e-10 in both precisions (FP64 CG and FP32-refined); manufactured
solutions and the constant-coefficient closed form pin the absolute answer."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import pipeline as opipe
from oracle import stamp as ostamp
from tests.helpers import rel_l2, stamp_inputs

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def B():
    from paper_2302_00752_gb300 import binding
    return binding


@pytest.fixture(scope="module")
def gp():
    from paper_2302_00752_gb300 import pipeline
    return pipeline


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_constant_coefficient_closed_form(B, prec):
    rng = np.random.default_rng(0)
    d, a0 = 4, 1.7
    q = rng.integers(-5, 6, size=(6, d))
    q = q[q.any(axis=1)]
    F = np.vstack([q, -q])
    fv = rng.standard_normal(len(q)) + 1j * rng.standard_normal(len(q))
    fval = np.concatenate([fv, np.conj(fv)])
    with B.stamp_build(np.zeros((1, d), int), np.array([a0 + 0j]), F, 2) as s:
        f_on, outside = s.scatter(F, fval)
        assert outside == 0
        u, st = B.solve(s, f_on, 1e-13, 100, prec)
        S = s.export()[0].cpu().numpy()
    n2 = (S.astype(np.int64) ** 2).sum(1)
    want = f_on.cpu().numpy() / np.where(n2 == 0, 1, 4 * np.pi ** 2 * a0 * n2)
    assert rel_l2(u.cpu().numpy(), want) < 1e-12
    assert st["status"] == "SS_OK"


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("seed", range(3))
def test_manufactured_tiny(gp, prec, seed):
    inst = W.make_tiny(seed, d=3, n_cos=2, n_u=3, N=2)
    res = gp.run(gp.prepare(inst), tol=1e-12, solve_precision=prec)
    S = res.stamp.export()[0].cpu().numpy()
    idx = ostamp.index_map(S)
    want = np.zeros(len(S), complex)
    for k, v in zip(inst.u_freq.tolist(), inst.u_val):
        want[idx[tuple(k)]] = v
    assert rel_l2(res.u.cpu().numpy(), want) < TOL
    assert res.stats["rel_residual"] <= 1e-12
    res.stamp.destroy()


def oracle_on_same_data(res, N):
    """Oracle solve from the GPU's recovered coefficients (same discrete system)."""
    return opipe.solve_recovered(N, res.a_freq.cpu().numpy(), res.a_val.cpu().numpy(), res.f_freq.cpu().numpy(),
                                 res.f_val.cpu().numpy(), tol=1e-14)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_cfg1_end_to_end(gp, prec):
    inst = W.make_cfg1()
    ref = opipe.run(inst)
    res = gp.run(gp.prepare(inst), tol=1e-12, solve_precision=prec)
    S = res.stamp.export()[0].cpu().numpy()
    assert np.array_equal(S, ref.S)
    assert rel_l2(res.u.cpu().numpy(), ref.u) < TOL
    res.stamp.destroy()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_cfg3_multiscale(gp, prec):
    inst = W.make_cfg3()
    res = gp.run(gp.prepare(inst), tol=1e-12, solve_precision=prec)
    ref = oracle_on_same_data(res, inst.N)
    S = res.stamp.export()[0].cpu().numpy()
    assert np.array_equal(S, ref.S)
    err = rel_l2(res.u.cpu().numpy(), ref.u)
    assert err < TOL, err
    assert res.stats["status"] == "SS_OK"
    # independent of any CG: the FP64 residual with the oracle's explicit
    # L_{N,s} (eq. GF assembled entry by entry) on the recovered data
    from oracle.galerkin import galerkin_matrix
    L, _ = galerkin_matrix(S, res.a_freq.cpu().numpy(), res.a_val.cpu().numpy())
    f, u = res.f_on_S.cpu().numpy(), res.u.cpu().numpy()
    assert np.linalg.norm(f - L @ u) <= 1e-11 * np.linalg.norm(f)
    res.stamp.destroy()


def test_solve_rejects_nonzero_mean(B):
    A = np.array([[-1, 0], [0, 0], [1, 0]])
    av = np.array([0.2, 1.0, 0.2], complex)
    with B.stamp_build(A, av, np.array([[1, 0], [-1, 0]]), 1) as s:
        assert s.zero_index >= 0
        f = torch.zeros(s.size, dtype=torch.complex128, device="cuda")
        f[s.zero_index] = 1.0
        from paper_2302_00752_gb300.binding import SSError
        with pytest.raises(SSError):
            B.solve(s, f, 1e-12, 100, "fp64")


def test_iteration_cap_reports_not_converged(B):
    inst, af, av, ff, fv = stamp_inputs("cfg1")
    with B.stamp_build(af, av, ff, inst.N) as s:
        f_on, _ = s.scatter(ff, fv)
        u, st = B.solve(s, f_on, 1e-14, 2, "fp64", raise_on_error=False)
        assert st["status"] == "SS_ERR_NOT_CONVERGED"
        u, st = B.solve(s, f_on, 1e-12, 500, "fp64")
        assert st["status"] == "SS_OK"


@pytest.mark.parametrize("name", ["cfg1", "cfg3"])
def test_df64_matches_oracle(B, name):
    # the FP64 CG in double-float arithmetic: same answer as the oracle within
    # the FP64 tolerance
    inst, af, av, ff, fv = stamp_inputs(name)
    ref = opipe.solve_recovered(inst.N, af, av, ff, fv, tol=1e-14)
    with B.stamp_build(af, av, ff, inst.N) as s:
        f_on, _ = s.scatter(ff, fv)
        u, st = B.solve(s, f_on, 1e-12, 1000, "df64")
        u64, st64 = B.solve(s, f_on, 1e-12, 1000, "fp64")
        u2, _ = B.solve(s, f_on, 1e-12, 1000, "df64")
    assert st["status"] == "SS_OK" and st["rel_residual"] <= 1e-12
    assert rel_l2(u.cpu().numpy(), ref.u) < TOL
    assert torch.equal(u, u2)                       # deterministic
    assert abs(st["applies"] - st64["applies"]) <= 2  # same recurrences


def test_df64_manufactured_cfg2(B, gp):
    inst = W.make_cfg2()
    res = gp.run(gp.prepare(inst), tol=1e-12, solve=False)
    try:
        u, st = B.solve(res.stamp, res.f_on_S, 1e-12, 1000, "df64")
        want, outside = res.stamp.scatter(inst.u_freq, inst.u_val)
        assert outside == 0 and st["status"] == "SS_OK"
        assert rel_l2(u.cpu().numpy(), want.cpu().numpy()) < TOL
    finally:
        res.stamp.destroy()


@pytest.mark.parametrize("prec", ["fp64", "fp32", "df64"])
def test_nonzero_mean_forcing_is_rejected(B, prec):
    # the diffusion problem is mean-zero: f_hat_0 != 0 on S is SS_ERR_INVALID
    A = np.array([[-1, 0], [0, 0], [1, 0]])
    av = np.array([0.2, 1.0, 0.2], complex)
    F = np.array([[1, 0], [-1, 0], [0, 2], [0, -2]])
    with B.stamp_build(A, av, F, 1) as s:
        assert s.zero_index >= 0
        f_on, _ = s.scatter(F, np.array([1, 1, 0.5, 0.5], complex))
        u, st = B.solve(s, f_on, 1e-12, 100, prec)
        assert st["status"] == "SS_OK"
        f_on[s.zero_index] = 0.25
        with pytest.raises(B.SSError):
            B.solve(s, f_on, 1e-12, 100, prec)
        f_on[s.zero_index] = 0.0
        u, st = B.solve(s, f_on, 1e-12, 100, prec)   # the context is still usable
        assert st["status"] == "SS_OK"
