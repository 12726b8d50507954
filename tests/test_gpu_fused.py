"""Algorithm 1 in one library call (sparse_spectral_solve) against the same
stages called one by one: the same lattice, the same stamping set and the
same bits of the solution; against the oracle on a small instance; and the
error paths of the one-call form."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import lattice as olat
from oracle import pipeline as opipe
from oracle.solve import rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    from paper_2302_00752_gb300 import binding, pipeline
    return binding, pipeline


def paired(p, M):
    """Whether the one-call form recovers a and f with one complex transform:
    on a 7-smooth M above 2^22 in either precision (the pruned transforms),
    FP64 on a 7-smooth M <= 2^22 (double-float FFT), FP32 on an M that is not
    7-smooth (cuFFT's Bluestein C2C costs about one real transform)."""
    if olat.is_smooth(M) and M > 2 ** 22:
        return True
    if p.sft_precision == "fp64":
        return olat.is_smooth(M)
    return not olat.is_smooth(M)


def fp32_cfg1():
    inst = W.make_cfg1()          # M = 1089 = 3^2 11^2: not 7-smooth
    inst.sft_precision = "fp32"
    return inst


@pytest.mark.parametrize("make,prec", [(lambda: W.make_tiny(3, d=3, n_cos=2, n_u=3, N=2), "fp64"),
                                       (fp32_cfg1, "fp64"), (W.make_cfg5, "fp32_refined"),
                                       (W.make_cfg1, "fp64"), (W.make_cfg1, "fp32_refined"),
                                       (W.make_cfg2, "fp64"), (lambda: W.make_cfg5(smooth=True), "fp32_refined")])
def test_fused_equals_staged(mods, make, prec):
    B, gp = mods
    inst = make()
    p = gp.prepare(inst)
    staged = gp.run(p, solve_precision=prec)
    z, M = p.z.copy(), p.M
    fused = gp.run_fused(p, solve_precision=prec)
    try:
        assert np.array_equal(fused.z, z) and fused.M == M
        assert fused.stamp.size == staged.stamp.size and fused.stamp.nnz == staged.stamp.nnz
        assert torch.equal(fused.stamp.export()[0], staged.stamp.export()[0])
        assert fused.stats["status"] == staged.stats["status"] == "SS_OK"
        if paired(p, M):
            # the fused call transforms a and f together (one complex transform
            # of s_a + i s_f), the staged calls one at a time: the same support
            # and stamp, the values within the transform's rounding
            assert abs(fused.stats["applies"] - staged.stats["applies"]) <= 1
            tol = 1e-12 if p.sft_precision == "fp64" else 1e-5
            assert rel_l2(fused.u.cpu().numpy(), staged.u.cpu().numpy()) < tol
        else:
            assert fused.stats["applies"] == staged.stats["applies"]
            assert torch.equal(fused.u, staged.u)
    finally:
        fused.stamp.destroy()
        staged.stamp.destroy()


def test_fused_into_caller_buffer(mods):
    B, gp = mods
    p = gp.prepare(W.make_cfg1())
    plain = gp.run_fused(p)
    buf = torch.full((plain.stamp.size + 7,), 3.0 + 1j, dtype=torch.complex128, device="cuda")
    small = torch.zeros(plain.stamp.size - 1, dtype=torch.complex128, device="cuda")
    into = gp.run_fused(p, out=buf)
    too_small = gp.run_fused(p, out=small)
    try:
        assert into.u.data_ptr() == buf.data_ptr() and torch.equal(into.u, plain.u)
        assert torch.all(buf[plain.stamp.size:] == 3.0 + 1j)
        assert torch.equal(too_small.u, plain.u) and not small.any()
    finally:
        for r in (plain, into, too_small):
            r.stamp.destroy()


def test_fused_matches_oracle(mods):
    B, gp = mods
    inst = W.make_tiny(5, d=3, n_cos=2, n_u=3, N=2)
    ref = opipe.run(inst)
    res = gp.run_fused(gp.prepare(inst))
    try:
        S = res.stamp.export()[0].cpu().numpy()
        assert np.array_equal(S, ref.S)
        assert rel_l2(res.u.cpu().numpy(), ref.u) < 1e-10
    finally:
        res.stamp.destroy()


def test_fused_errors_leave_no_stamp(mods):
    B, gp = mods
    inst = W.make_tiny(6, d=3, n_cos=2, n_u=3, N=1)
    p = gp.prepare(inst)
    # a box lattice that is not reconstructing for the candidate set
    bad = {"kind": "box", "z": np.ones(3, np.int64), "M": 5}
    with pytest.raises(B.SSError) as e:
        B.sparse_spectral_solve(bad, p.a_freq, p.a_coef, p.f_freq, p.f_coef, p.cand, 1)
    assert e.value.status in (1, 4)
    # and a good call afterwards works
    stamp, u, st, z, M = B.sparse_spectral_solve(p.extra["lattice"], p.a_freq, p.a_coef, p.f_freq, p.f_coef, p.cand,
                                                 1)
    try:
        assert st["status"] == "SS_OK" and u.shape[0] == stamp.size
    finally:
        stamp.destroy()
