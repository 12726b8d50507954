"""Failure paths, each provoked from the host and ending in a status, never in
a GPU fault, trap or hang: a device-side wait that gives up (SS_ERR_TIMEOUT),
an exhausted frequency hash table (SS_ERR_HASH_FULL) and frequencies too large
for the packed key or the exact norms (SS_ERR_KEY_RANGE).  After each, the
library keeps working: the same stamp solves (bit for bit as before), and new
stamps build."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import stamp as ostamp
from tests.helpers import stamp_inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2302_00752_gb300 import binding
    return binding


def test_solver_wait_timeout_then_recovers(B):
    # a zero wait bound makes the first grid barrier of the persistent solver
    # give up: every block returns and the solve reports SS_ERR_TIMEOUT
    inst, af, av, ff, fv = stamp_inputs("cfg3")          # 86,272 rows: a full grid of blocks
    with B.stamp_build(af, av, ff, inst.N) as s:
        f_on, _ = s.scatter(ff, fv)
        ref, st = B.solve(s, f_on, 1e-12, 1000, "fp64")
        assert st["status"] == "SS_OK"
        s.set_wait_limit(0)
        for prec in ("fp64", "fp32", "df64"):
            _, st = B.solve(s, f_on, 1e-12, 1000, prec, raise_on_error=False)
            assert st["status"] == "SS_ERR_TIMEOUT", prec
        s.set_symmetry(False)                            # the full system's launch as well
        _, st = B.solve(s, f_on, 1e-12, 1000, "fp64", raise_on_error=False)
        assert st["status"] == "SS_ERR_TIMEOUT"
        s.set_symmetry(True)
        s.set_wait_limit(2_000_000_000)
        u, st = B.solve(s, f_on, 1e-12, 1000, "fp64")
        assert st["status"] == "SS_OK"
        assert torch.equal(u, ref)                       # deterministic solver, same bits


def test_exhausted_hash_table(B):
    from paper_2302_00752_gb300.binding import SSError
    inst, af, av, ff, fv = stamp_inputs("cfg1")          # |S| = 571
    want = ostamp.stamp_bfs(af, ff, inst.N)[0]
    B.set_table_limit(256)                               # fewer slots than frequencies
    try:
        with pytest.raises(SSError) as e:
            B.stamp_build(af, av, ff, inst.N)
        assert e.value.name == "SS_ERR_HASH_FULL"
        # a set that fits under the same bound still builds, and equals the oracle's
        tiny = W.make_tiny(2, d=2, n_cos=1, n_u=2, N=1)
        _, taf, tav, tff, tfv = stamp_inputs(tiny)
        tw = ostamp.stamp_bfs(taf, tff, tiny.N)[0]
        assert len(tw) < 128
        with B.stamp_build(taf, tav, tff, tiny.N) as t:
            S, _ = t.export()
            assert np.array_equal(S.cpu().numpy(), tw)
    finally:
        B.set_table_limit(0)
    with B.stamp_build(af, av, ff, inst.N) as s:
        S, _ = s.export()
        assert np.array_equal(S.cpu().numpy(), want)


def _one_cos(d, p, c=0.2):
    p = np.asarray(p, np.int64)
    af = np.array([np.zeros(d, np.int64), p, -p])
    av = np.array([1.0, c / 2, c / 2], np.complex128)
    return af, av


def test_key_range(B):
    from paper_2302_00752_gb300.binding import SSError
    # d = 100, coordinates up to 2 10^4: 16 bits each, more key words than supported
    d = 100
    p = np.zeros(d, np.int64)
    p[:3] = [20000, -7, 3]
    af, av = _one_cos(d, p)
    F = np.zeros((2, d), np.int64)
    F[0, 5], F[1, 5] = 1, -1
    with pytest.raises(SSError) as e:
        B.stamp_build(af, av, F, 2)
    assert e.value.name == "SS_ERR_KEY_RANGE"
    # d = 3, |k|^2 beyond 2^51: the exact FP64 entry coefficients would round
    af, av = _one_cos(3, [2 ** 26, 2 ** 26, 0])
    F = np.array([[0, 0, 1], [0, 0, -1]])
    with pytest.raises(SSError) as e:
        B.stamp_build(af, av, F, 2)
    assert e.value.name == "SS_ERR_KEY_RANGE"
    # the library still builds and solves after both
    inst, af, av, ff, fv = stamp_inputs("cfg1")
    with B.stamp_build(af, av, ff, inst.N) as s:
        f_on, _ = s.scatter(ff, fv)
        _, st = B.solve(s, f_on, 1e-12, 500, "fp64")
        assert st["status"] == "SS_OK"
