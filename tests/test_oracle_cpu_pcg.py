"""The multi-core C PCG baseline follows oracle.solve.pcg (same recurrences):
the same iteration count and solution to rounding, and the manufactured
solution reproduced."""
import numpy as np
import pytest

import workloads as W
from oracle import cpu_pcg, galerkin, solve, stamp
from tests.helpers import stamp_inputs


@pytest.mark.parametrize("seed", range(3))
def test_c_pcg_matches_python_pcg(seed):
    inst = W.make_tiny(seed, d=3, n_cos=2, n_u=3, N=2)
    _, af, av, ff, fv = stamp_inputs(inst)
    S, _ = stamp.stamp_bfs(af, ff, 2)
    L, _ = galerkin.galerkin_matrix(S, af, av)
    idx = stamp.index_map(S)
    b = np.zeros(len(S), complex)
    for k, v in zip(ff.tolist(), fv):
        b[idx[tuple(k)]] = v
    D = solve.jacobi_diag(S, av[~af.any(axis=1)][0])
    x_py, it_py, _ = solve.pcg(L, b, D, 1e-12)
    x_c, it_c = cpu_pcg.pcg(L, b, D, 1e-12, n_threads=2)
    assert abs(it_c - it_py) <= 1
    assert np.linalg.norm(x_c - x_py) <= 1e-10 * np.linalg.norm(x_py)
    want = np.zeros(len(S), complex)
    for k, v in zip(inst.u_freq.tolist(), inst.u_val):
        want[idx[tuple(k)]] = v
    assert np.linalg.norm(x_c - want) <= 1e-10 * np.linalg.norm(want)


def test_zero_rhs_returns_zero():
    inst = W.make_tiny(0, d=2, n_cos=2, n_u=2, N=1)
    _, af, av, ff, _ = stamp_inputs(inst)
    S, _ = stamp.stamp_bfs(af, ff, 1)
    L, _ = galerkin.galerkin_matrix(S, af, av)
    D = solve.jacobi_diag(S, av[~af.any(axis=1)][0])
    x, it = cpu_pcg.pcg(L, np.zeros(len(S), complex), D)
    assert it == 0 and not x.any()
