"""Solving L_{N,s} u_hat = f_hat (oracle; test infrastructure only).

Algorithm 1 ends with a direct solve of eq. SparseSpectralSFTEquation.  The
matrix is Hermitian positive definite on mean-zero vectors (Proposition
GalerkinBilinearForm with coercivity, Proposition ExistenceUniquenessStability;
a_hat is Hermitian because a is real), so the solution is unique and any
correct solver reaches it up to rounding.  Provided here:

  pcg          Jacobi-preconditioned conjugate gradients in complex128.  The
               preconditioner is the diagonal of L, D_k = 4 pi^2 Re(a_hat_0)|k|^2,
               the denominator of the diagonal rearrangement in the proof of
               Proposition SolutionSupport (1 on the pinned zero row).
  dense_solve  LAPACK LU with partial pivoting (numpy.linalg.solve).
  thomas       the textbook tridiagonal elimination, for the chain systems of
               the one-term problem (Section "Low sparsity").
  is_elliptic  the positivity check of the Remark after Corollary
               SpectralConvergenceNoSFT:  ||a_hat - a_hat_0||_1 < |a_hat_0|.

Pins: closed form u_hat_k = f_hat_k / (4 pi^2 a_0 |k|^2) for constant a;
manufactured solutions reproduced exactly; PCG against dense LU; the chain
solve against the general solver (tests/test_oracle_solve.py).
"""
from __future__ import annotations

import numpy as np

FOUR_PI_SQ = 4.0 * np.pi ** 2


def jacobi_diag(S, a0):
    """D_k = 4 pi^2 Re(a0) |k|^2, and 1 for k = 0."""
    n2 = (np.asarray(S, np.int64) ** 2).sum(axis=1).astype(np.float64)
    D = FOUR_PI_SQ * float(np.real(a0)) * n2
    D[n2 == 0] = 1.0
    return D


def pcg(L, b, D, tol=1e-14, max_iter=10000, x0=None):
    """Preconditioned CG for Hermitian positive definite L; stops when
    ||b - L x|| <= tol ||b|| (recursive residual).  Returns (x, iterations,
    relative residual history)."""
    b = np.asarray(b, np.complex128)
    x = np.zeros_like(b) if x0 is None else np.array(x0, np.complex128)
    r = b - L @ x
    bnorm = np.linalg.norm(b)
    if bnorm == 0:
        return x, 0, [0.0]
    z = r / D
    p = z.copy()
    rho = np.vdot(r, z).real
    hist = [np.linalg.norm(r) / bnorm]
    it = 0
    while hist[-1] > tol and it < max_iter:
        q = L @ p
        alpha = rho / np.vdot(p, q).real
        x += alpha * p
        r -= alpha * q
        it += 1
        hist.append(np.linalg.norm(r) / bnorm)
        z = r / D
        rho_new = np.vdot(r, z).real
        p = z + (rho_new / rho) * p
        rho = rho_new
    return x, it, hist


def dense_solve(L, b):
    """LU with partial pivoting on the assembled matrix."""
    A = L.toarray() if hasattr(L, "toarray") else np.asarray(L)
    return np.linalg.solve(A, np.asarray(b, np.complex128))


def thomas(lower, diag, upper, rhs):
    """Tridiagonal elimination: lower[i] multiplies x[i-1] in row i (lower[0]
    unused), upper[i] multiplies x[i+1] (upper[-1] unused)."""
    n = len(diag)
    c = np.zeros(n, np.complex128)
    g = np.zeros(n, np.complex128)
    c[0] = upper[0] / diag[0] if n > 1 else 0
    g[0] = rhs[0] / diag[0]
    for i in range(1, n):
        den = diag[i] - lower[i] * c[i - 1]
        c[i] = upper[i] / den if i < n - 1 else 0
        g[i] = (rhs[i] - lower[i] * g[i - 1]) / den
    x = np.zeros(n, np.complex128)
    x[-1] = g[-1]
    for i in range(n - 2, -1, -1):
        x[i] = g[i] - c[i] * x[i + 1]
    return x


def is_elliptic(a_freq, a_val):
    """||a_hat - a_hat_0||_1 < |a_hat_0| (sufficient for a > 0)."""
    a_freq = np.asarray(a_freq)
    a_val = np.asarray(a_val)
    zero = ~a_freq.any(axis=1)
    if not zero.any():
        return False
    a0 = abs(a_val[zero][0])
    return float(np.abs(a_val[~zero]).sum()) < a0


def rel_l2(x, ref):
    """||x - ref||_2 / ||ref||_2."""
    x = np.asarray(x)
    ref = np.asarray(ref)
    den = np.linalg.norm(ref)
    return float(np.linalg.norm(x - ref) / (den if den > 0 else 1.0))
