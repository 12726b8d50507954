"""stamp_build / stamp_lookup parity with the oracle: the stamping set, its
canonical order, levels and the frequency -> index map are integers and must
match bit for bit (eq. StampSet; canonical-order reading in oracle.stamp)."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import galerkin as ogal
from oracle import stamp as ostamp
from tests.golden.loader import stamp_cases
from tests.helpers import stamp_inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2302_00752_gb300 import binding
    return binding


def check_set(B, af, av, F, N, with_nnz=True):
    S_ref, lvl_ref = ostamp.stamp_bfs(af, F, N)
    with B.stamp_build(af, av, F, N) as s:
        S, lvl = s.export()
        S, lvl = S.cpu().numpy(), lvl.cpu().numpy()
        assert s.size == len(S_ref)
        assert np.array_equal(S, S_ref), "stamping set or canonical order differs"
        assert np.array_equal(lvl, lvl_ref)
        z = np.flatnonzero(~S_ref.any(axis=1))
        assert s.zero_index == (int(z[0]) if len(z) else -1)
        if with_nnz:
            assert s.nnz == ogal.nnz_count(S_ref, af)
        # lookups: every member maps to its index; shifted copies mostly do not
        idx = s.lookup(S_ref).cpu().numpy()
        assert np.array_equal(idx, np.arange(len(S_ref)))
        rng = np.random.default_rng(0)
        q = S_ref[rng.integers(0, len(S_ref), 200)] + rng.integers(-3, 4, size=(200, S_ref.shape[1]))
        got = s.lookup(q).cpu().numpy()
        im = ostamp.index_map(S_ref)
        want = np.array([im.get(tuple(int(x) for x in k), -1) for k in q])
        assert np.array_equal(got, want)


@pytest.mark.parametrize("case", stamp_cases(), ids=lambda c: c["name"])
def test_hand_worked_cases(B, case):
    A = case["A"]
    av = np.where(~A.any(axis=1), 1.0, 0.1).astype(complex)
    check_set(B, A, av, case["F"], case["N"])


@pytest.mark.parametrize("seed", range(6))
def test_tiny_random(B, seed):
    inst = W.make_tiny(seed, d=int(1 + seed % 3), n_cos=2, n_u=3, N=int(1 + seed % 4))
    _, af, av, ff, _ = stamp_inputs(inst)
    check_set(B, af, av, ff, inst.N)


@pytest.mark.parametrize("name", ["cfg1", "cfg3"])
def test_configs(B, name):
    inst, af, av, ff, _ = stamp_inputs(name)
    check_set(B, af, av, ff, inst.N)


def test_cfg2_full_size(B):
    inst, af, av, ff, _ = stamp_inputs("cfg2")
    check_set(B, af, av, ff, inst.N, with_nnz=False)


def test_cfg5_full_size_properties(B):
    # |S| = 1.15e6 in d = 100: the count of Lemma StampSetCardinality is attained
    # (no coincidences), levels have the per-level counts, S = -S, and level-1
    # elements are exactly F + p, checked against the oracle's own level 0..1.
    inst, af, av, ff, _ = stamp_inputs("cfg5")
    with B.stamp_build(af, av, ff, inst.N) as s:
        S, lvl = s.export()
        S, lvl = S.cpu().numpy(), lvl.cpu().numpy()
        assert s.size == ostamp.cardinality_bound(len(ff), len(af), inst.N)
        counts = np.bincount(lvl, minlength=inst.N + 1)
        for n in range(inst.N + 1):
            assert counts[n] == ostamp.cardinality_bound(len(ff), len(af), n) - (
                ostamp.cardinality_bound(len(ff), len(af), n - 1) if n else 0)
        neg = s.lookup(-S[::97]).cpu().numpy()
        assert (neg >= 0).all()
        S1, l1 = ostamp.stamp_bfs(af, ff, 1)
        assert np.array_equal(S[: len(S1)], S1) and np.array_equal(lvl[: len(S1)], l1)


def test_errors(B):
    from paper_2302_00752_gb300.binding import SSError
    A = np.array([[-1, 0], [0, 0], [1, 0]])
    av = np.array([0.2, 1.0, 0.2], complex)
    with pytest.raises(SSError) as e:
        B.stamp_build(A, av, np.array([[1, 1], [1, 1]]), 1)
    assert e.value.name == "SS_ERR_INVALID"
    with pytest.raises(SSError) as e:
        B.stamp_build(A, np.array([0.6, 1.0, 0.6], complex), np.array([[1, 1]]), 1)
    assert e.value.name == "SS_ERR_NOT_ELLIPTIC"
    with pytest.raises(SSError) as e:
        B.stamp_build(A[:2], av[:2], np.array([[1, 1]]), 1)
    assert e.value.name == "SS_ERR_INVALID"
    with pytest.raises(SSError) as e:
        B.stamp_build(A, av, np.array([[0, 0], [1, 1]]), 1)
    assert e.value.name == "SS_ERR_INVALID"
    with pytest.raises(SSError) as e:
        B.stamp_build(A, np.array([0.2, 1.0, 0.2 + 0.1j], complex), np.array([[1, 1]]), 1)
    assert e.value.name == "SS_ERR_INVALID"
