"""Real coefficients.  For an even a (every a_hat_p real) every entry
coefficient 2 pi^2 (|k|^2 + |l|^2 - |p|^2) a_hat_p of eq. GF is real and the
FP64 and double-float operators take two multiply-adds per nonzero.  A cosine
a takes that form, a with a sine term does not, and an a_hat whose imaginary
parts are of rounding size (1e-15 of the largest) takes it with those parts
dropped.  In every case the solution matches the oracle's, which keeps the
complex arithmetic, within 1e-10 relative l2 in all three precisions."""
import numpy as np
import pytest

from oracle import pipeline as opipe
from tests.helpers import rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2302_00752_gb300 import binding
    return binding


def data(sine, noise, seed=4):
    rng = np.random.default_rng(seed)
    p = np.array([[1, 0, 0], [0, 2, 1], [1, -1, 2]])
    c = np.array([0.2, 0.15, 0.1])
    s = np.array([0.1, 0.0, 0.05]) * sine
    e = noise * rng.standard_normal(3)
    ap = c / 2 - 0.5j * s + 1j * e           # a_hat_p; a_hat_{-p} is its conjugate
    a_freq = np.vstack([np.zeros((1, 3), int), p, -p])
    a_val = np.concatenate([[1.5 + 0j], ap, np.conj(ap)])
    q = rng.integers(-4, 5, size=(5, 3))
    q = np.unique(q[q.any(axis=1)], axis=0)
    q = q[[tuple(k) not in {tuple(-x) for x in q[:i]} for i, k in enumerate(q)]]
    fv = rng.standard_normal(len(q)) + 1j * rng.standard_normal(len(q))
    F = np.vstack([q, -q])
    return a_freq, a_val, F, np.concatenate([fv, np.conj(fv)])


@pytest.mark.parametrize("prec", ["fp64", "df64", "fp32"])
@pytest.mark.parametrize("sine,noise,real", [(0.0, 0.0, True), (1.0, 0.0, False), (0.0, 1e-15 * 0.1, True),
                                              (0.0, 1e-9, False)])
def test_real_coefficients_match_oracle(B, prec, sine, noise, real):
    a_freq, a_val, F, fval = data(sine, noise)
    ref = opipe.solve_recovered(2, a_freq, a_val, F, fval, tol=1e-14)
    with B.stamp_build(a_freq, a_val, F, 2) as s:
        assert s.real_coefficients == real
        f_on, _ = s.scatter(F, fval)
        u, st = B.solve(s, f_on, 1e-13, 500, prec)
        S = s.export()[0].cpu().numpy()
    assert np.array_equal(S, ref.S)
    assert st["status"] == "SS_OK"
    if prec != "fp32":
        assert st["real_coefficients"] == real
    assert rel_l2(u.cpu().numpy(), ref.u) < 1e-10


def test_real_coefficients_operator_matches_oracle(B):
    # the FP64 operator on a random (non-Hermitian) vector, real and complex a
    import torch
    from oracle.galerkin import galerkin_matrix
    rng = np.random.default_rng(1)
    for sine in (0.0, 1.0):
        a_freq, a_val, F, fval = data(sine, 0.0)
        with B.stamp_build(a_freq, a_val, F, 2) as s:
            S = s.export()[0].cpu().numpy()
            x = rng.standard_normal(len(S)) + 1j * rng.standard_normal(len(S))
            y = B.galerkin_apply(s, torch.tensor(x, device="cuda"), "fp64").cpu().numpy()
        L, _ = galerkin_matrix(S, a_freq, a_val)
        want = L @ x
        assert np.linalg.norm(y - want) <= 1e-14 * np.linalg.norm(want)
