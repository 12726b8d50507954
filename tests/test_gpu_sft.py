"""Lattice choice, lattice sampling and coefficient recovery against the oracle.
Integer results (M, z, attempt, residues, kept support) match exactly; FP64
values within 1e-12 sum|c| (FFT rounding, O(log M) eps), FP32 within 1e-5 sum|c|."""
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


def test_lattice_check(B):
    from paper_2302_00752_gb300.binding import SSError
    g = np.arange(-16, 17)
    box = np.stack(np.meshgrid(g, g, indexing="ij"), -1).reshape(-1, 2)
    B.lattice_check([1, 33], 1089, box)
    with pytest.raises(SSError) as e:
        B.lattice_check([1, 33], 1089, np.vstack([box, [[17, 0]]]))
    assert e.value.name == "SS_ERR_NOT_RECONSTRUCTING"
    with pytest.raises(SSError) as e:
        B.lattice_check([1, 33], 1089, np.vstack([box, [[3, 3]]]))
    assert e.value.name == "SS_ERR_INVALID"


def test_random_lattice_matches_oracle(B):
    inst = W.make_cfg3()
    cand = opipe.candidates(inst, inst.f.freq)
    z, M, att = olat.random_lattice(cand, inst.lattice)
    gz, gM, gatt = B.lattice_random(cand, inst.lattice["raw"], inst.lattice["sigma"], inst.lattice["M_min"])
    assert (gM, gatt) == (M, att) and np.array_equal(gz, z)


def test_random_lattice_retries(B):
    # a deliberately tiny M forces failed attempts; both sides agree on which succeeds
    rng = np.random.default_rng(4)
    cand = np.unique(rng.integers(-3, 4, size=(20, 3)), axis=0)
    draws = {"kind": "random", "raw": rng.integers(0, 2**62, size=(40, 3)), "M_min": 0, "sigma": 1.0}
    z, M, att = olat.random_lattice(cand, draws)
    gz, gM, gatt = B.lattice_random(cand, draws["raw"], 1.0, 0)
    assert (gM, gatt) == (M, att) and np.array_equal(gz, z)


def test_cbc_lattice_matches_oracle(B):
    rng = np.random.default_rng(5)
    I = np.unique(rng.integers(-8, 9, size=(300, 6)), axis=0)
    I = np.unique(np.vstack([I, -I]), axis=0)
    draws = {"raw": rng.integers(0, 2**62, size=(6, 32)), "M_min": 200003}
    z, M = olat.cbc_lattice(I, draws)
    gz, gM = B.lattice_cbc(I, draws["raw"], draws["M_min"])
    assert gM == M and np.array_equal(gz, z)


@pytest.mark.parametrize("seed,M_min,n_cand", [(6, 5000, 48), (7, 3000, 64), (8, 20000, 8)])
def test_cbc_lattice_later_candidates(B, seed, M_min, n_cand):
    # M close to |I|^2 / 2: many candidates collide, so the first passing one
    # is often not the first drawn (the pick that every block of the
    # one-launch search must agree on)
    rng = np.random.default_rng(seed)
    I = np.unique(rng.integers(-9, 10, size=(120, 5)), axis=0)
    I = np.unique(np.vstack([I, -I]), axis=0)
    draws = {"raw": rng.integers(0, 2**62, size=(5, n_cand)), "M_min": M_min}
    M = olat.next_smooth(max(M_min, olat.expansion(I) + 1))
    try:
        z, Mo = olat.cbc_lattice(I, draws)
    except ValueError:
        with pytest.raises(B.SSError) as e:
            B.lattice_cbc(I, draws["raw"], draws["M_min"])
        assert e.value.status == 4
        return
    gz, gM = B.lattice_cbc(I, draws["raw"], draws["M_min"])
    assert gM == Mo == M and np.array_equal(gz, z)


def test_cbc_lattice_no_candidate(B):
    rng = np.random.default_rng(9)
    I = np.unique(rng.integers(-9, 10, size=(200, 4)), axis=0)
    I = np.unique(np.vstack([I, -I]), axis=0)
    draws = {"raw": rng.integers(0, 2**62, size=(4, 2)), "M_min": 400}
    with pytest.raises(ValueError):
        olat.cbc_lattice(I, draws)
    with pytest.raises(B.SSError) as e:
        B.lattice_cbc(I, draws["raw"], draws["M_min"])
    assert e.value.status == 4


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("fp32", 2e-6)])
def test_sampling_matches_oracle(B, prec, tol):
    rng = np.random.default_rng(1)
    d, M = 4, 100003
    z = rng.integers(1, M, size=d)
    freq = rng.integers(-30, 31, size=(37, d))
    coef = rng.standard_normal(37) + 1j * rng.standard_normal(37)
    g = B.lattice_sample(z, M, freq, coef, prec).double().cpu().numpy()
    js = np.concatenate([np.arange(0, M, 7), [M - 1]])
    ref = osft.sample(freq, coef, z, M, js)
    scale = np.abs(coef).sum()
    assert np.abs(g[js] - ref).max() <= tol * scale


@pytest.mark.parametrize("M,n_terms", [(2 ** 5 * 3 ** 4 * 5 ** 2 * 7, 300), (100003, 700)])
def test_many_term_sampling_matches_oracle(B, M, n_terms):
    # many terms: the FP64 samples come from one inverse FFT of the binned
    # terms; residue collisions are planted (a frequency aliasing to bin 0,
    # one on bin M/2 when M is even, pairs sharing a residue or its negative)
    rng = np.random.default_rng(2)
    d = 4
    z = np.concatenate([[1], rng.integers(1, M, size=d - 1)])
    freq = rng.integers(-40, 41, size=(n_terms, d))
    e1 = np.array([M, 0, 0, 0])
    freq[1] = e1
    freq[2] = freq[10] + e1
    freq[3] = e1 - freq[11]
    freq[4] = -freq[12] - e1
    if M % 2 == 0:
        freq[5] = [M // 2, 0, 0, 0]
        freq[6] = [-M // 2, 0, 0, 0]
    freq[7] = freq[13]            # a repeated frequency
    freq[8] = -freq[14]           # and its negative
    coef = rng.standard_normal(n_terms) + 1j * rng.standard_normal(n_terms)
    g = B.lattice_sample(z, M, freq, coef, "fp64").double().cpu().numpy()
    js = np.concatenate([np.arange(0, M, 11), [M // 2, M - 1]])
    ref = osft.sample(freq, coef, z, M, js)
    assert np.abs(g[js] - ref).max() <= 1e-13 * np.abs(coef).sum()


@pytest.mark.parametrize("M,d,span", [(453600, 3, 12),   # 672 x 675: radices 8 4 3 7 | 5 5 3 3 3
                                      (18816, 3, 6),     # 128 x 147: radices 8 8 2 | 3 7 7
                                      (48, 1, 3),        # 6 x 8: radices 2 3 | 8
                                      (14, 1, 3),        # 2 x 7
                                      (2 ** 20, 2, 20)])  # 1024 x 1024: radices 8 8 8 2
def test_recover_smooth_sizes_matches_oracle(B, M, d, span):
    # FP64 recovery on 7-smooth M runs the double-float transform (two
    # launches of per-block Stockham passes): every radix and uneven factor
    # pairs, against the exact coefficients and the oracle's plain DFT
    rng = np.random.default_rng(M)
    n_terms = 40 if d > 1 else 3
    freq = rng.integers(-span, span + 1, size=(n_terms, d))
    if d == 1:
        freq = np.array([[0], [1], [3]])
    coef = rng.standard_normal(n_terms) + 1j * rng.standard_normal(n_terms)
    extra = rng.integers(-span, span + 1, size=(2 * n_terms, d))
    I = np.unique(np.vstack([freq, -freq, extra, -extra]), axis=0)
    for _ in range(200):
        z = rng.integers(1, M, size=d) if d > 1 else np.array([1])
        if olat.is_reconstructing(I, z, M):
            break
    assert olat.is_reconstructing(I, z, M)
    gf, gv = B.sft_recover(z, M, freq, coef, I, tau=1e-9)
    want = osft.true_coefficients(freq, coef)
    got = {tuple(k): v for k, v in zip(gf.cpu().numpy().tolist(), gv.cpu().numpy())}
    scale = np.abs(coef).sum()
    assert set(got) == {k for k, v in want.items() if abs(v) > 1e-9 * scale}
    for k, v in got.items():
        assert abs(v - want[k]) <= 1e-12 * scale
    if M <= 20000:   # the plain DFT costs M |I| exponentials
        kf, kv = osft.recover_known(osft.sample(freq, coef, z, M), I, z, M, tau=1e-9)
        assert np.array_equal(gf.cpu().numpy(), kf)
        assert np.abs(gv.cpu().numpy() - kv).max() <= 1e-12 * scale


def test_recover_cfg2_full_size_closed_form(B):
    # the d = 10 forcing (840 terms) on its CBC lattice, M >= 10^6 (7-smooth:
    # the double-float transform), against the exact coefficients
    from paper_2302_00752_gb300 import pipeline as gp
    inst = W.make_cfg2()
    p = gp.prepare(inst)
    z, M = gp.choose_lattice(p.extra["lattice"], p.cand)
    assert olat.is_smooth(M) and M <= 2 ** 22
    ff, fc = p.f_freq.cpu().numpy(), p.f_coef.cpu().numpy()
    gf, gv = B.sft_recover(z, M, ff, fc, p.cand, tau=1e-9)
    want = osft.true_coefficients(ff, fc)
    got = {tuple(k): v for k, v in zip(gf.cpu().numpy().tolist(), gv.cpu().numpy())}
    scale = np.abs(fc).sum()
    assert set(got) == {k for k, v in want.items() if abs(v) > 1e-9 * scale}
    assert max(abs(v - want[k]) for k, v in got.items()) <= 1e-12 * scale


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_recover_cfg1_matches_oracle(B, prec, tol):
    inst = W.make_cfg1()
    z, M = inst.lattice["z"], inst.lattice["M"]
    samples = osft.sample(inst.a.freq, inst.a.coef, z, M)
    kf, kv = osft.recover_known(samples, inst.cand, z, M, tau=1e-9 if prec == "fp64" else 1e-4)
    gf, gv = B.sft_recover(z, M, inst.a.freq, inst.a.coef, inst.cand, tau=1e-9 if prec == "fp64" else 1e-4,
                           precision=prec)
    assert np.array_equal(gf.cpu().numpy(), kf)
    scale = np.abs(inst.a.coef).sum()
    assert np.abs(gv.cpu().numpy() - kv).max() <= tol * scale


def test_recover_closed_form_and_forcing(B):
    # cfg3: a (cosines) and f (cosines and sines) recovered on the random lattice;
    # closed form: c/2 at +-p, -i c/2 / +i c/2 for sines, the mean at 0
    inst = W.make_cfg3()
    cand = opipe.candidates(inst, inst.f.freq)
    z, M, _ = olat.random_lattice(cand, inst.lattice)
    for trig in (inst.a, inst.f):
        want = osft.true_coefficients(trig.freq, trig.coef)
        gf, gv = B.sft_recover(z, M, trig.freq, trig.coef, cand, tau=1e-9)
        got = {tuple(k): v for k, v in zip(gf.cpu().numpy().tolist(), gv.cpu().numpy())}
        assert set(got) == {k for k, v in want.items() if abs(v) > 0}
        scale = np.abs(trig.coef).sum()
        for k, v in got.items():
            assert abs(v - want[k]) <= 1e-12 * scale


def test_recover_from_samples_and_cap(B):
    from paper_2302_00752_gb300.binding import SSError
    inst = W.make_cfg1()
    z, M = inst.lattice["z"], inst.lattice["M"]
    s = B.lattice_sample(z, M, inst.a.freq, inst.a.coef, "fp64")
    gf, gv = B.sft_recover_samples(z, M, s, inst.cand, tau=1e-9)
    assert len(gf) == 9
    with pytest.raises(SSError):
        B.sft_recover_samples(z, M, s, inst.cand, s_max=5, tau=1e-9)
    with pytest.raises(SSError) as e:
        B.sft_recover_samples(z, M, s, inst.cand[:-1], tau=1e-9)     # not closed under negation
    assert e.value.name == "SS_ERR_INVALID"


def test_recover_cfg5_fp32_sampled(B):
    # M = smallest prime >= 2^26, FP32 samples and FP32 FFT, d = 100
    inst = W.make_cfg5()
    cand = opipe.candidates(inst, inst.f.freq)
    z, M, att = olat.random_lattice(cand, inst.lattice)
    gz, gM, gatt = B.lattice_random(cand, inst.lattice["raw"], inst.lattice["sigma"], inst.lattice["M_min"])
    assert gM == M == 2**26 + 15 and np.array_equal(gz, z)
    for trig in (inst.a, inst.f):
        want = osft.true_coefficients(trig.freq, trig.coef)
        gf, gv = B.sft_recover(z, M, trig.freq, trig.coef, cand, tau=1e-4, precision="fp32")
        got = {tuple(k): v for k, v in zip(gf.cpu().numpy().tolist(), gv.cpu().numpy())}
        assert set(got) == {k for k, v in want.items() if abs(v) > 0}
        scale = np.abs(trig.coef).sum()
        err = max(abs(v - want[k]) for k, v in got.items())
        assert err <= 1e-5 * scale, err
    # a few FP32 samples against the oracle's direct evaluation
    js = np.array([0, 1, 12345, M // 2, M - 1])
    g = B.lattice_sample(z, M, inst.a.freq, inst.a.coef, "fp32").double().cpu().numpy()
    ref = osft.sample(inst.a.freq, inst.a.coef, z, M, js)
    assert np.abs(g[js] - ref).max() <= 2e-6 * np.abs(inst.a.coef).sum()


def test_random_lattice_smooth_size(B):
    # 7-smooth M >= the Lemma's bound, reconstructing (exact check) for I
    from oracle import lattice as olat
    inst = W.make_cfg3()
    rng = np.random.default_rng(3)
    I = np.unique(rng.integers(-40, 41, size=(60, 3)), axis=0)
    I = np.unique(np.vstack([I, -I]), axis=0)
    raw = rng.integers(0, 2**62, size=(16, 3), dtype=np.int64)
    z, M, att = B.lattice_random(I, raw, sigma=0.05, M_min=1000, smooth=True)
    assert olat.is_smooth(M) and M >= max(len(I) ** 2 / 0.05, 1000)
    assert M == olat.next_smooth(int(max(np.ceil(len(I) ** 2 / 0.05), olat.expansion(I) + 1, 1000)))
    assert olat.is_reconstructing(I, z, M)
    assert np.array_equal(z, 1 + raw[att] % (M - 1))
