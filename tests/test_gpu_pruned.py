"""FP64 recovery on long 7-smooth lattices (M above 2^22): the sparse
evaluation that samples a trigonometric sum and the pruned forward transform
that reads the candidates' bins, both in double-float arithmetic.

Expected values come from the oracle only: the closed-form coefficients
(cosine c -> c/2 at +-p, sine -> -+ i c/2, the mean at 0), the direct evaluation
of the sum at chosen lattice indices, and the plain DFT of arbitrary samples
at the candidates' bins.  Tolerances: samples 1e-13 sum|c|, coefficients
1e-12 sum|c| (the double-float rounding, about 2^-47 per operation, over a
few dozen operations per value)."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import lattice as olat
from oracle import pipeline as opipe
from oracle import sft as osft
from tests.helpers import rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2302_00752_gb300 import binding
    return binding


# 7-smooth lengths above 2^22 with different prime factors, so that the
# length-P column transforms run radix 8/4/2, 3, 5, 7 and mixed passes
SIZES = [2 ** 23,                # P, Q powers of two
         3 ** 15,                # radix 3 only
         5 ** 10,                # radix 5 only
         7 ** 9,                 # radix 7 only
         2 ** 16 * 3 ** 3 * 35]  # every radix


def _instance(M, n_terms, seed, d=3, span=40):
    rng = np.random.default_rng([M % 1000003, seed])
    freq = rng.integers(-span, span + 1, size=(n_terms, d))
    freq[0] = 0                                   # the mean (residue 0)
    freq[2] = -freq[1]                            # a +-p pair merged into one term
    coef = rng.standard_normal(n_terms) + 1j * rng.standard_normal(n_terms)
    extra = rng.integers(-span, span + 1, size=(n_terms, d))
    I = np.unique(np.vstack([freq, -freq, extra, -extra]), axis=0)
    for _ in range(200):
        z = rng.integers(1, M, size=d)
        if olat.is_reconstructing(I, z, M):
            break
    assert olat.is_reconstructing(I, z, M)
    return freq, coef, I, z


def _check_coefficients(gf, gv, freq, coef, tol=1e-12, tau=1e-9):
    # kept: |g_k| > tau max |g| (coefficients within rounding of the cut may go
    # either way), values within tol sum|c| of the closed form
    want = osft.true_coefficients(freq, coef)
    got = {tuple(k): v for k, v in zip(gf.cpu().numpy().tolist(), gv.cpu().numpy())}
    scale = np.abs(coef).sum()
    vmax = max(abs(v) for v in want.values())
    assert {k for k, v in want.items() if abs(v) > 2 * tau * vmax} <= set(got)
    assert set(got) <= {k for k, v in want.items() if abs(v) > 0.5 * tau * vmax}
    err = max(abs(v - want[k]) for k, v in got.items())
    assert err <= tol * scale, err


# tolerances per precision: samples, coefficients (of sum|c|), threshold
TOLS = {"fp64": (1e-13, 1e-12, 1e-9), "fp32": (2e-6, 1e-5, 1e-4)}


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("M", SIZES)
def test_sampling_and_recovery(B, M, prec):
    tol_s, tol_c, tau = TOLS[prec]
    freq, coef, I, z = _instance(M, 40, 0)
    scale = np.abs(coef).sum()
    # samples by the sparse evaluation, against the direct sum at chosen and
    # random indices (tile and column boundaries included)
    s = B.lattice_sample(z, M, freq, coef, prec)
    assert s.dtype == (torch.float64 if prec == "fp64" else torch.float32) and s.numel() == M
    rng = np.random.default_rng(1)
    js = np.unique(np.concatenate([[0, 1, 2, M - 1, M - 2, M // 2, M // 3, M // 7],
                                   [M // q * t for q in (8, 27, 125, 343) for t in (1, 2)],
                                   rng.integers(0, M, 3000)]))
    ref = osft.sample(freq, coef, z, M, js)
    got = s.double().cpu().numpy()[js]
    assert np.abs(got - ref).max() <= tol_s * scale
    # recovery through the library (sampling + pruned transform) and from the
    # samples above (pruned transform of real input)
    gf, gv = B.sft_recover(z, M, freq, coef, I, tau=tau, precision=prec)
    _check_coefficients(gf, gv, freq, coef, tol_c, tau)
    gf2, gv2 = B.sft_recover_samples(z, M, s, I, tau=tau, precision=prec)
    _check_coefficients(gf2, gv2, freq, coef, tol_c, tau)


def test_many_terms_and_buckets(B):
    # 300 terms: the entries come in several rounds of the evaluation and
    # many share a bucket (r mod P); a frequency k and its negative both given
    M = 2 ** 23
    freq, coef, I, z = _instance(M, 300, 7, d=4, span=25)
    freq[10] = -freq[11]
    freq[12] = freq[13]                           # a repeated frequency (summed)
    I = np.unique(np.vstack([I, freq, -freq]), axis=0)
    assert olat.is_reconstructing(I, z, M)
    scale = np.abs(coef).sum()
    s = B.lattice_sample(z, M, freq, coef, "fp64").cpu().numpy()
    js = np.random.default_rng(2).integers(0, M, 2000)
    assert np.abs(s[js] - osft.sample(freq, coef, z, M, js)).max() <= 1e-13 * scale
    gf, gv = B.sft_recover(z, M, freq, coef, I, tau=1e-9)
    _check_coefficients(gf, gv, freq, coef)


def test_half_lattice_residue(B):
    # a term whose residue is M/2 (a real sample sign (-1)^j): sampled exactly
    M = 2 ** 23
    z = np.array([1, 3, 5])
    freq = np.array([[M // 2, 0, 0], [1, 2, 3], [0, 0, 0]])
    coef = np.array([0.75 - 0.5j, 1.0 + 2.0j, 0.25])
    s = B.lattice_sample(z, M, freq, coef, "fp64").cpu().numpy()
    js = np.concatenate([np.arange(64), np.random.default_rng(3).integers(0, M, 1000)])
    assert np.abs(s[js] - osft.sample(freq, coef, z, M, js)).max() <= 1e-13 * np.abs(coef).sum()


@pytest.mark.parametrize("M", [3 * 2 ** 22, 7 ** 9])
def test_forward_transform_of_arbitrary_samples(B, M):
    # the pruned transform of dense random samples (no sparse structure)
    # against the oracle's plain DFT at the candidates' bins
    rng = np.random.default_rng(11)
    I = np.array([[1, 0], [-1, 0], [3, -2], [-3, 2], [0, 5], [0, -5]])
    z = np.array([1, 1 + int(rng.integers(1, M - 1))])
    assert olat.is_reconstructing(I, z, M)
    x = rng.standard_normal(M)
    gf, gv = B.sft_recover_samples(z, M, torch.as_tensor(x).cuda(), I, tau=0.0)
    kf, kv = osft.recover_known(x, I, z, M, tau=0.0)
    assert np.array_equal(gf.cpu().numpy(), kf)
    assert np.abs(gv.cpu().numpy() - kv).max() <= 1e-13 * np.abs(x).mean()


def test_cfg5_fp64_recovery_closed_form(B):
    # the d = 100 data (a: 41 coefficients, f: 100) on its 7-smooth lattice
    # M = 2^26, recovered in FP64 against the exact coefficients
    from paper_2302_00752_gb300 import pipeline as gp
    inst = W.make_cfg5(smooth=True)
    cand = opipe.candidates(inst, inst.f.freq)
    L = inst.lattice
    M = olat.next_smooth(int(max(np.ceil(len(cand) ** 2 / L["sigma"]), olat.expansion(cand) + 1, L["M_min"])))
    gz, gM, gatt = B.lattice_random(cand, L["raw"], L["sigma"], L["M_min"], smooth=True)
    assert gM == M == 2 ** 26
    # the first reconstructing draw of the stream, as the oracle checks it
    for a in range(gatt + 1):
        z = olat.z_from_raw(L["raw"][a], M)
        assert olat.is_reconstructing(cand, z, M) == (a == gatt)
    assert np.array_equal(gz, z)
    for trig in (inst.a, inst.f):
        gf, gv = B.sft_recover(z, M, trig.freq, trig.coef, cand, tau=1e-9)
        _check_coefficients(gf, gv, trig.freq, trig.coef)
    # FP64 samples at 10^4 random lattice indices against the direct sum
    s = B.lattice_sample(z, M, inst.f.freq, inst.f.coef, "fp64").cpu().numpy()
    js = np.random.default_rng(5).integers(0, M, 10000)
    assert np.abs(s[js] - osft.sample(inst.f.freq, inst.f.coef, z, M, js)).max() <= 1e-13 * np.abs(inst.f.coef).sum()
    del s
    # one-call path: a and f share one evaluation and one pruned transform;
    # the FP64 solution equals the staged one (separate recoveries)
    p = gp.prepare(inst)
    p.sft_precision = "fp64"
    r = gp.run_fused(p, tol=1e-12, max_iter=1000, tau=1e-9, solve_precision="fp64")
    assert r.stats["status"] == "SS_OK"
    staged = gp.run(p, tol=1e-12, tau=1e-9, solve_precision="fp64", lattice=False)
    S1, _ = r.stamp.export()
    S2, _ = staged.stamp.export()
    assert torch.equal(S1, S2)
    assert rel_l2(r.u.cpu().numpy(), staged.u.cpu().numpy()) <= 1e-11
    r.stamp.destroy()
    staged.stamp.destroy()


def test_cfg5_fp32_pair_recovery(B):
    # the d = 100 data as configured (FP32 samples and FFT) on M = 2^26: a and
    # f share one FP32 evaluation and one pruned FP32 transform in the one-call
    # path; each sum recovered alone against the closed form, and the one-call
    # solution against the staged one (same S, u within the FP32 recovery's
    # rounding)
    from paper_2302_00752_gb300 import pipeline as gp
    inst = W.make_cfg5(smooth=True)
    cand = opipe.candidates(inst, inst.f.freq)
    L = inst.lattice
    z, M, _ = B.lattice_random(cand, L["raw"], L["sigma"], L["M_min"], smooth=True)
    assert M == 2 ** 26
    for trig in (inst.a, inst.f):
        gf, gv = B.sft_recover(z, M, trig.freq, trig.coef, cand, tau=1e-4, precision="fp32")
        _check_coefficients(gf, gv, trig.freq, trig.coef, 1e-5, 1e-4)
    p = gp.prepare(inst)
    r = gp.run_fused(p, tol=1e-12, max_iter=1000, solve_precision="fp32_refined")
    assert r.stats["status"] == "SS_OK" and p.M == 2 ** 26
    staged = gp.run(p, tol=1e-12, solve_precision="fp32_refined", lattice=False)
    S1, _ = r.stamp.export()
    S2, _ = staged.stamp.export()
    assert torch.equal(S1, S2)
    assert rel_l2(r.u.cpu().numpy(), staged.u.cpu().numpy()) <= 1e-5
    r.stamp.destroy()
    staged.stamp.destroy()
