"""The Galerkin operator (oracle; test infrastructure only).

eq. GF:   (L[a_hat] u_hat)_k = sum_l (2 pi)^2 (l.k) a_hat_{k-l} u_hat_l.
eq. FiniteGalerkinOperator / the operator L_{N,s}: the same sum with k and l
restricted to the stamping set S^N and a_hat replaced by its recovered
coefficients.

Written out here as an explicit sparse matrix: for every row k in S and every
p in supp(a_hat) with l = k - p in S, the entry (k, l) is 4 pi^2 (k.l) a_hat_p,
the dot product taken in exact integers.

Zero frequency (the paper's system is mean-zero, Section 2 and Proposition
ExistenceUniquenessStability; row and column 0 of eq. GF vanish because of the
factor l.k): when 0 is in S its row is replaced by the identity row, which
pins u_hat_0 = 0 given f_hat_0 = 0.  Column-0 entries are zero and are not
stored; neither the identity row nor zero-column entries count as nonzeros.

The exact proxy error of Lemma ProxyError, ||f_hat - L[a_hat] u_hat||_2 /
||f_hat||_2, is evaluated over all of Z^d by the same convolution (``proxy_error``).
Its Monte Carlo form, ||f - f^{s,N}||_{L2} / ||f||_{L2} estimated from point
values at uniform random points of T^d (Section "Code and testing overview"),
is ``proxy_mc``: points on the grid (2^-32 Z)^d, so that every phase k.x mod 1
is an exact integer fraction.

Pins: the Monte Carlo values against closed-form sines at chosen points and,
averaged over a reconstructing power-of-two rank-1 lattice, against the exact
proxy (Parseval); the bilinear-form identity (Proposition GalerkinBilinearForm) against
trapezoidal quadrature of  integral a grad u . conj(grad v)  on a grid; the
manufactured f_hat against the Fourier coefficients of -div(a grad u) computed
pointwise; Hermitian symmetry; the constant-coefficient diagonal; the level
structure of Proposition LExpansion (tests/test_oracle_galerkin.py).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .stamp import index_map

FOUR_PI_SQ = 4.0 * np.pi ** 2


def _a_dict(a_freq, a_val):
    return {tuple(int(x) for x in p): complex(v) for p, v in zip(np.asarray(a_freq), np.asarray(a_val))}


def galerkin_matrix(S, a_freq, a_val):
    """Explicit L_{N,s} on S (scipy CSR, complex128) and its nonzero count."""
    S = np.asarray(S, np.int64)
    idx = index_map(S)
    a = _a_dict(a_freq, a_val)
    rows, cols, vals = [], [], []
    nnz = 0
    for i, k in enumerate(S.tolist()):
        if not any(k):
            rows.append(i); cols.append(i); vals.append(1.0)
            continue
        for p, ap in a.items():
            l = tuple(x - y for x, y in zip(k, p))
            j = idx.get(l)
            if j is None or not any(l):
                continue
            kl = sum(x * y for x, y in zip(k, l))
            rows.append(i); cols.append(j); vals.append(FOUR_PI_SQ * kl * ap)
            nnz += 1
    n = len(S)
    L = sp.csr_matrix((np.array(vals, np.complex128), (rows, cols)), shape=(n, n))
    return L, nnz


def apply_rows(S, a_freq, a_val, u, rows, idx=None):
    """(L u)_k for the selected row indices only (same entries as
    ``galerkin_matrix``), for spot checks on sets too large to assemble.
    ``idx`` may pass ``index_map(S)`` when several calls share one set."""
    S = np.asarray(S, np.int64)
    if idx is None:
        idx = index_map(S)
    a = _a_dict(a_freq, a_val)
    out = np.zeros(len(rows), np.complex128)
    for o, i in enumerate(rows):
        k = S[i].tolist()
        if not any(k):
            out[o] = u[i]
            continue
        acc = 0j
        for p, ap in a.items():
            l = tuple(x - y for x, y in zip(k, p))
            j = idx.get(l)
            if j is None or not any(l):
                continue
            acc += FOUR_PI_SQ * sum(x * y for x, y in zip(k, l)) * ap * u[j]
        out[o] = acc
    return out


def convolve(a_freq, a_val, u_freq, u_val):
    """f_hat = L[a_hat] u_hat over all of Z^d (eq. GF summed directly over the
    pairs (p, l) in supp a_hat x supp u_hat with k = l + p).  Returns
    (freq [n, d], val [n]) in signed lexicographic order, every k = l + p
    listed even where the sum vanishes."""
    out = {}
    for p, ap in _a_dict(a_freq, a_val).items():
        for l, ul in zip(np.asarray(u_freq, np.int64).tolist(), np.asarray(u_val)):
            k = tuple(x + y for x, y in zip(l, p))
            kl = sum(x * y for x, y in zip(k, l))
            out[k] = out.get(k, 0j) + FOUR_PI_SQ * kl * ap * ul
    keys = sorted(out)
    return np.array(keys, np.int64).reshape(len(keys), -1), np.array([out[k] for k in keys], np.complex128)


def nnz_count(S, a_freq):
    """#{(k, p): k in S\\{0}, p in supp a_hat, k - p in S\\{0}}."""
    idx = index_map(S)
    A = [tuple(int(x) for x in p) for p in np.asarray(a_freq)]
    n = 0
    for k in idx:
        if not any(k):
            continue
        for p in A:
            l = tuple(x - y for x, y in zip(k, p))
            if any(l) and l in idx:
                n += 1
    return n


def proxy_error(a_freq, a_val, u_freq, u_val, f_freq, f_val):
    """Lemma ProxyError: ||f_hat - L[a_hat] u_hat||_2 / ||f_hat||_2 over Z^d,
    with L[a_hat] u_hat from ``convolve`` (exact support)."""
    Lf, Lv = convolve(a_freq, a_val, u_freq, u_val)
    r = {tuple(int(x) for x in k): v for k, v in zip(Lf.tolist(), Lv)}
    for k, v in zip(np.asarray(f_freq, np.int64).tolist(), np.asarray(f_val)):
        r[tuple(k)] = r.get(tuple(k), 0j) - v
    num = np.sqrt(sum(abs(v) ** 2 for v in r.values()))
    den = np.linalg.norm(np.asarray(f_val))
    return float(num / den)


MC_GRID = 1 << 32


def trig_at(freq, coef, X):
    """sum_t Re(coef_t exp(2 pi i freq_t.x)) at the points x = X / 2^32
    (X: integer [Q, d] in [0, 2^32)); the phase freq_t.X mod 2^32 is formed in
    exact integers before the exponential."""
    X = np.asarray(X, np.int64)
    out = np.zeros(len(X), np.float64)
    for k, c in zip(np.asarray(freq, np.int64).tolist(), np.asarray(coef, np.complex128)):
        ph = (X @ np.array(k, np.int64)) % MC_GRID   # int64 wrap-around is harmless: 2^32 divides 2^64
        out += (c * np.exp(2j * np.pi * (ph / MC_GRID))).real
    return out


def proxy_mc(a_freq, a_val, u_freq, u_val, f_freq, f_coef, X):
    """Point values for the Monte Carlo proxy of Lemma ProxyError:
    r(x) = f(x) - f^{s,N}(x) and f(x) at x = X / 2^32, where f is the trig sum
    (f_freq, f_coef) and f^{s,N} = L[a_hat] u^{s,N} is taken on its exact
    support (``convolve``).  The estimate is sqrt(sum r^2 / sum f^2)."""
    g_freq, g_val = convolve(a_freq, a_val, u_freq, u_val)
    fx = trig_at(f_freq, f_coef, X)
    return fx - trig_at(g_freq, g_val, X), fx


def mc_estimate(r, fx):
    return float(np.sqrt(np.sum(np.square(r)) / np.sum(np.square(fx))))
