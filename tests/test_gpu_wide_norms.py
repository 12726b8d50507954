"""Sets whose squared norms pass 2^29: the paper's low-sparsity test (Section
"Low sparsity") at d = 64 with k_a, k_f in [-499, 500]^d and N = 12 (|k|^2 up
to ~8e8), and multiscale data with frequencies up to 2e4 per coordinate
(|k|^2 ~ 1e10).  The FP64 operator stays exact (int64 norms, FP64 entry
coefficients), the FP32 operator forms 2 k.l in FP32; both solves match the
oracle within relative l2 1e-10, and the applies match the oracle's explicit
matrix (FP64 to 1e-13, FP32 to 1e-5 relative l2)."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import galerkin as ogal
from oracle import pipeline as opipe
from tests.helpers import rel_l2, stamp_inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2302_00752_gb300 import binding
    return binding


def one_term(seed=2):
    return W.make_one_term(64, seed=seed, kmax=500)


CASES = {"oneterm64": (lambda: one_term(), 12), "wide4": (lambda: W.make_wide(0), 2),
         "wide6": (lambda: W.make_wide(1, d=6, scale=8000, n_cos=4, n_f=4), 2)}


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("case", list(CASES))
def test_wide_solve_matches_oracle(B, prec, case):
    make, N = CASES[case]
    inst = make()
    _, af, av, ff, fv = stamp_inputs(inst)
    ref = opipe.solve_recovered(N, af, av, ff, fv, tol=1e-14)
    assert (ref.S.astype(np.int64) ** 2).sum(1).max() >= 2 ** 29
    with B.stamp_build(af, av, ff, N) as s:
        f_on, _ = s.scatter(ff, fv)
        u, st = B.solve(s, f_on, 1e-12, 1000, prec)
        S = s.export()[0].cpu().numpy()
    assert np.array_equal(S, ref.S)
    assert st["status"] == "SS_OK"
    assert rel_l2(u.cpu().numpy(), ref.u) < 1e-10


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("fp32", 1e-5)])
@pytest.mark.parametrize("case", list(CASES))
def test_wide_apply_matches_oracle(B, prec, tol, case):
    make, N = CASES[case]
    inst = make()
    _, af, av, ff, fv = stamp_inputs(inst)
    with B.stamp_build(af, av, ff, N) as s:
        S = s.export()[0].cpu().numpy()
        rng = np.random.default_rng(1)
        u = rng.standard_normal(len(S)) + 1j * rng.standard_normal(len(S))
        dt = torch.complex128 if prec == "fp64" else torch.complex64
        y = B.galerkin_apply(s, torch.as_tensor(u).to(dt).cuda(), prec).cpu().numpy()
    L, _ = ogal.galerkin_matrix(S, af, av)
    assert rel_l2(y, L @ u) < tol


def test_extend_across_the_wide_boundary(B):
    # the norm bound d (max |k_c|)^2 is below 2^29 at N = 3 and above it at
    # N = 5: the FP32 norm words change encoding in place
    inst = one_term()
    _, af, av, ff, fv = stamp_inputs(inst)
    with B.stamp_build(af, av, ff, 3) as s, B.stamp_build(af, av, ff, 5) as fresh:
        s.extend(2)
        rng = np.random.default_rng(4)
        u = torch.as_tensor(rng.standard_normal(s.size) + 1j * rng.standard_normal(s.size)).cuda()
        assert torch.equal(B.galerkin_apply(s, u), B.galerkin_apply(fresh, u))
        u32 = u.to(torch.complex64)
        assert torch.equal(B.galerkin_apply(s, u32, "fp32"), B.galerkin_apply(fresh, u32, "fp32"))


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_batch_mixes_wide_and_narrow(B, prec):
    insts = [(one_term(2), 12), (W.make_tiny(3, d=3, n_cos=2, n_u=3, N=2, manufactured_u=False), 2),
             (W.make_wide(2), 2)]
    stamps, fs, refs = [], [], []
    try:
        for inst, N in insts:
            _, af, av, ff, fv = stamp_inputs(inst)
            s = B.stamp_build(af, av, ff, N)
            f_on, _ = s.scatter(ff, fv)
            stamps.append(s)
            fs.append(f_on)
            refs.append(opipe.solve_recovered(N, af, av, ff, fv, tol=1e-14))
        us, stats = B.Batch(stamps).solve(fs, tol=1e-12, max_iter=1000, precision=prec)
        for u, st, ref in zip(us, stats, refs):
            assert st["status"] == "SS_OK"
            assert rel_l2(u.cpu().numpy(), ref.u) < 1e-10
    finally:
        for s in stamps:
            s.destroy()
