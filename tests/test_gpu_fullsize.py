"""Parity at the full sizes of the d = 10, batched and d = 100 workloads, each
through the C ABI and against the oracle only:

* the d = 10 CBC lattice (M = 10^6, |I| = 861) equals the oracle's search;
* d = 100, FP64 path: the GPU stamping set equals the oracle's BFS, and the
  FP64 solution satisfies the oracle's operator - f_hat - L u evaluated row by
  row with the oracle's eq. GF on 2000 random rows plus every row of f's
  support, with the exact coefficients of a and f (no CG involved);
* d = 100, FP32 path: samples at 10^4 random lattice indices;
* batched: instances of the 512-instance workload spanning |S| = 10^3..10^5,
  solved in one graph-replayed persistent launch, element by element against
  the oracle's PCG."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import galerkin as ogal
from oracle import lattice as olat
from oracle import pipeline as opipe
from oracle import sft as osft
from oracle import stamp as ostamp
from tests.helpers import rel_l2, stamp_inputs, true_a, true_f

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2302_00752_gb300 import binding
    return binding


def test_cfg2_cbc_lattice_matches_oracle(B):
    inst = W.make_cfg2()
    ff, _ = opipe.forcing(inst)
    cand = opipe.candidates(inst, ff)
    assert inst.d == 10 and len(cand) > 800
    z, M = olat.cbc_lattice(cand, inst.lattice)
    gz, gM = B.lattice_cbc(cand, inst.lattice["raw"], inst.lattice["M_min"])
    assert gM == M == 10 ** 6
    assert np.array_equal(np.asarray(gz), np.asarray(z))
    assert olat.is_reconstructing(cand, z, M)


def test_cfg5_fp64_residual_with_oracle_operator(B):
    from paper_2302_00752_gb300 import pipeline as gp
    inst = W.make_cfg5(smooth=True)
    p = gp.prepare(inst)
    p.sft_precision = "fp64"
    r = gp.run_fused(p, tol=1e-12, max_iter=1000, tau=1e-9, solve_precision="fp64")
    assert r.stats["status"] == "SS_OK" and r.M == 2 ** 26
    S_gpu, _ = r.stamp.export()
    S_gpu = S_gpu.cpu().numpy()
    u = r.u.cpu().numpy()
    r.stamp.destroy()
    af, av = true_a(inst)
    ff, fv = true_f(inst)
    S, _ = ostamp.stamp_bfs(af, ff, inst.N)
    assert len(S) == 1152100 and np.array_equal(S_gpu, S)
    b = opipe.rhs_on(S, ff, fv)
    rng = np.random.default_rng(0)
    rows = np.unique(np.concatenate([np.flatnonzero(b), rng.choice(len(S), 2000, replace=False)]))
    res = b[rows] - ogal.apply_rows(S, af, av, u, rows)
    # the solve stops at ||f - L u||_2 <= 1e-12 ||f||_2; each row's residual
    # is bounded by that norm, plus the recovery's rounding (1e-13 of the
    # coefficients' l1 norms) carried through L
    assert np.abs(res).max() <= 1e-11 * np.linalg.norm(b)


@pytest.mark.parametrize("smooth", [False, True])
def test_cfg5_fp32_samples(B, smooth):
    inst = W.make_cfg5(smooth=smooth)
    cand = opipe.candidates(inst, inst.f.freq)
    z, M, _ = olat.random_lattice(cand, inst.lattice)
    js = np.unique(np.concatenate([[0, 1, M - 1, M // 2], np.random.default_rng(9).integers(0, M, 10000)]))
    for trig in (inst.a, inst.f):
        g = B.lattice_sample(z, M, trig.freq, trig.coef, "fp32").double().cpu().numpy()[js]
        ref = osft.sample(trig.freq, trig.coef, z, M, js)
        assert np.abs(g - ref).max() <= 2e-6 * np.abs(trig.coef).sum()


def _spread_instances(n=8, pool=64):
    """n members of the 512-instance workload (seed 0) whose generic stamp
    sizes spread over its range, smallest to largest."""
    insts = [W.make_batch_instance(0, i) for i in range(pool)]
    size = [W.generic_stamp_count(2 * len(inst.f.freq), 2 * len(inst.a.freq) + 1, inst.N) for inst in insts]
    order = np.argsort(size, kind="stable")
    pick = order[np.linspace(0, pool - 1, n).round().astype(int)]
    return [insts[i] for i in pick]


def test_batch_full_range_matches_oracle(B):
    insts = _spread_instances()
    stamps, fs, refs = [], [], []
    try:
        for inst in insts:
            _, af, av, ff, fv = stamp_inputs(inst)
            s = B.stamp_build(af, av, ff, inst.N)
            stamps.append(s)
            fs.append(s.scatter(ff, fv)[0])
            refs.append(opipe.solve_recovered(inst.N, af, av, ff, fv, tol=1e-14))
        sizes = [s.size for s in stamps]
        assert min(sizes) >= 1000 and max(sizes) >= 50000 and max(sizes) <= 100000
        batch = B.Batch(stamps)
        for prec in ("fp32", "fp64"):
            us, stats = batch.solve(fs, tol=1e-12, max_iter=1000, precision=prec, use_graph=True)
            for u, st, ref in zip(us, stats, refs):
                assert st["status"] == "SS_OK"
                u = u.cpu().numpy()
                assert np.array_equal(np.asarray(ref.S).shape, (len(u), ref.S.shape[1]))
                assert rel_l2(u, ref.u) <= 1e-10
                assert np.abs(u - ref.u).max() <= 1e-10 * np.abs(ref.u).max()
        batch.destroy()
    finally:
        for s in stamps:
            s.destroy()
