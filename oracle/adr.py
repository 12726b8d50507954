"""Advection-diffusion-reaction operator (oracle; test infrastructure only).

Remark ADR extends the method to
    -div(a grad u) + b . grad u + c u = f   on T^d
with real a, c and a real vector field b = (b_1, ..., b_d).  In Fourier
variables (the Fourier coefficient definition of Section 2, with
grad e_l = 2 pi i l e_l and products becoming convolutions):
    (L u)_k = sum_l [ 4 pi^2 (k.l) a_hat_{k-l} + 2 pi i (l . b_hat_{k-l}) + c_hat_{k-l} ] u_hat_l,
where b_hat_p = (b_hat_{1,p}, ..., b_hat_{d,p}).  The stamp of Remark ADR
adds, at every level, the supports of a_hat, of each b_hat_j and of c_hat.
Reading: the step set is their union U (the operator couples k and l exactly
when k - l lies in U; a Minkowski sum of all the supports would be a superset
whose extra members carry no coupling).  Unlike eq. GF the zero frequency is
an ordinary row and column here: c_hat_0 makes u_hat_0 part of the solution.

Functions: the union step set, the explicit sparse operator on S, the exact
convolution over Z^d (manufactured data, proxy error) and a direct sparse
solve (SuperLU through scipy; the paper uses a dense direct solve).

Pins (tests/test_oracle_adr.py): the convolution against -div(a grad u) +
b.grad u + c u evaluated pointwise on a grid and transformed by numpy's FFT
(trapezoidal rule, exact for these trigonometric polynomials); with b = 0 and
c = 0 the operator equals eq. GF's; the matrix applied to u equals the
convolution restricted to S when supp u and its neighbours lie in S;
manufactured solutions reproduced by the direct solve.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .stamp import index_map, lex_order

FOUR_PI_SQ = 4.0 * np.pi ** 2
TWO_PI = 2.0 * np.pi


def _dict(freq, val):
    return {tuple(int(x) for x in k): complex(v) for k, v in zip(np.asarray(freq), np.asarray(val))}


def coefficient_maps(a, b, c):
    """a, c: (freq, val); b: list of d (freq, val), one per component.
    Returns (U sorted lexicographically, {p: a_hat_p}, {p: b_hat_p vector}, {p: c_hat_p})."""
    A = _dict(*a)
    C = _dict(*c)
    d = np.asarray(a[0]).shape[1]
    Bv = {}
    for j, (bf, bv) in enumerate(b):
        for k, v in _dict(bf, bv).items():
            Bv.setdefault(k, np.zeros(d, np.complex128))[j] += v
    keys = set(A) | set(C) | set(Bv)
    U = np.array(sorted(keys), np.int64).reshape(len(keys), d)
    U = U[lex_order(U)]
    return U, A, Bv, C


def entry(k, l, A, Bv, C):
    """Coefficient of u_hat_l in (L u)_k (the bracket above), p = k - l."""
    p = tuple(x - y for x, y in zip(k, l))
    v = 0j
    if p in A:
        v += FOUR_PI_SQ * sum(x * y for x, y in zip(k, l)) * A[p]
    if p in Bv:
        v += TWO_PI * 1j * complex(np.dot(np.asarray(l, np.float64), Bv[p]))
    if p in C:
        v += C[p]
    return v


def adr_matrix(S, a, b, c):
    """Explicit operator on the set S (scipy CSR) and its stored-entry count:
    every (k, l) with k, l in S and k - l in U."""
    S = np.asarray(S, np.int64)
    idx = index_map(S)
    U, A, Bv, C = coefficient_maps(a, b, c)
    rows, cols, vals = [], [], []
    for i, k in enumerate(S.tolist()):
        for p in U.tolist():
            l = tuple(x - y for x, y in zip(k, p))
            j = idx.get(l)
            if j is None:
                continue
            rows.append(i); cols.append(j); vals.append(entry(k, l, A, Bv, C))
    n = len(S)
    L = sp.csr_matrix((np.array(vals, np.complex128), (rows, cols)), shape=(n, n))
    return L, len(vals)


def convolve(a, b, c, u_freq, u_val):
    """L u over all of Z^d: (freq [n, d], val [n]) in signed lexicographic order,
    every k = l + p (l in supp u, p in U) listed."""
    U, A, Bv, C = coefficient_maps(a, b, c)
    out = {}
    for l, ul in zip(np.asarray(u_freq, np.int64).tolist(), np.asarray(u_val)):
        for p in U.tolist():
            k = tuple(x + y for x, y in zip(l, p))
            out[k] = out.get(k, 0j) + entry(k, tuple(l), A, Bv, C) * ul
    keys = sorted(out)
    return np.array(keys, np.int64).reshape(len(keys), -1), np.array([out[k] for k in keys], np.complex128)


def solve(S, a, b, c, f_freq, f_val):
    """Direct solve of the Galerkin system on S (f_hat scattered onto S)."""
    S = np.asarray(S, np.int64)
    idx = index_map(S)
    rhs = np.zeros(len(S), np.complex128)
    for k, v in zip(np.asarray(f_freq, np.int64).tolist(), np.asarray(f_val)):
        j = idx.get(tuple(k))
        if j is not None:
            rhs[j] += v
    L, _ = adr_matrix(S, a, b, c)
    return spla.spsolve(L.tocsc(), rhs), rhs


def proxy_error(a, b, c, u_freq, u_val, f_freq, f_val):
    """Lemma ProxyError's relative form for the ADR operator, over Z^d."""
    Lf, Lv = convolve(a, b, c, u_freq, u_val)
    r = {tuple(int(x) for x in k): v for k, v in zip(Lf.tolist(), Lv)}
    for k, v in zip(np.asarray(f_freq, np.int64).tolist(), np.asarray(f_val)):
        r[tuple(k)] = r.get(tuple(k), 0j) - v
    return float(np.sqrt(sum(abs(v) ** 2 for v in r.values())) / np.linalg.norm(np.asarray(f_val)))
