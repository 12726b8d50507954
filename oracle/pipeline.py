"""Algorithm 1 end to end on the CPU (oracle; test infrastructure only).

Algorithm 1 (Sparse spectral method): recover a_hat^s and f_hat^s from lattice
samples, build S^N[a_hat^s](supp f_hat^s), assemble L_{N,s} and solve
L_{N,s} u = f_hat^s.  Manufactured instances first build f_hat = L[a_hat] u_hat
over all of Z^d by exact convolution (eq. GF) and sample f through that
trigonometric sum.

The candidate set for known-support recovery is the union of the supports of
a and f (closed under negation), unless the workload prescribes one (the
bijective box lattice).  Its lattice is the workload's box lattice, a CBC
lattice or a random lattice (Lemma RandomRank1Lattice), chosen by ``lattice``.

Parity: pinned through the pins of the modules it strings together and by
manufactured solutions, whose Galerkin solution on S equals u_hat exactly
(supp u_hat lies in S, and the solution is unique).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import lattice as lat
from .galerkin import convolve, galerkin_matrix
from .sft import recover_known, sample, true_coefficients
from .solve import jacobi_diag, pcg
from .stamp import stamp_bfs


@dataclass
class OracleResult:
    z: np.ndarray
    M: int
    a_freq: np.ndarray
    a_val: np.ndarray
    f_freq: np.ndarray
    f_val: np.ndarray
    S: np.ndarray
    level: np.ndarray
    nnz: int
    u: np.ndarray          # solution on S (canonical order)
    iters: int
    f_on_S: np.ndarray


def forcing(inst):
    """f as a trigonometric sum: the workload's own, or the exact convolution
    L[a_hat] u_hat for manufactured instances."""
    if inst.f is not None:
        return np.asarray(inst.f.freq, np.int64), np.asarray(inst.f.coef, np.complex128)
    a = true_coefficients(inst.a.freq, inst.a.coef)
    af = np.array(list(a.keys()), np.int64)
    av = np.array(list(a.values()), np.complex128)
    return convolve(af, av, inst.u_freq, inst.u_val)


def support_of(freq):
    """Support of sum_t Re(c_t e_{p_t}): every p_t and -p_t."""
    f = np.asarray(freq, np.int64)
    return np.unique(np.vstack([f, -f]), axis=0)


def candidates(inst, f_freq):
    if inst.cand is not None:
        return np.asarray(inst.cand, np.int64)
    return np.unique(np.vstack([support_of(inst.a.freq), support_of(f_freq)]), axis=0)


def choose_lattice(inst, cand):
    L = inst.lattice
    if L["kind"] == "box":
        return np.asarray(L["z"], np.int64), int(L["M"])
    if L["kind"] == "cbc":
        return lat.cbc_lattice(cand, L)
    z, M, _ = lat.random_lattice(cand, L)
    return z, M


def run(inst, tol=1e-14, tau=1e-9, max_iter=10000):
    f_freq, f_coef = forcing(inst)
    cand = candidates(inst, f_freq)
    z, M = choose_lattice(inst, cand)
    ga = sample(inst.a.freq, inst.a.coef, z, M)
    gf = sample(f_freq, f_coef, z, M)
    a_freq, a_val = recover_known(ga, cand, z, M, tau)
    f_freq_s, f_val_s = recover_known(gf, cand, z, M, tau)
    return solve_recovered(inst.N, a_freq, a_val, f_freq_s, f_val_s, tol, max_iter, z, M)


def solve_recovered(N, a_freq, a_val, f_freq, f_val, tol=1e-14, max_iter=10000, z=None, M=0):
    """Steps 3-5 of Algorithm 1 from given recovered coefficients."""
    S, level = stamp_bfs(a_freq, f_freq, N)
    L, nnz = galerkin_matrix(S, a_freq, a_val)
    b = rhs_on(S, f_freq, f_val)
    a0 = a_val[~np.asarray(a_freq).any(axis=1)][0]
    u, it, _ = pcg(L, b, jacobi_diag(S, a0), tol, max_iter)
    return OracleResult(z, M, np.asarray(a_freq), np.asarray(a_val), np.asarray(f_freq),
                        np.asarray(f_val), S, level, nnz, u, it, b)


def rhs_on(S, f_freq, f_val):
    """f_hat scattered onto S (zero where f_hat has no entry)."""
    idx = {tuple(int(x) for x in k): i for i, k in enumerate(np.asarray(S))}
    b = np.zeros(len(S), np.complex128)
    for k, v in zip(np.asarray(f_freq, np.int64).tolist(), np.asarray(f_val)):
        b[idx[tuple(k)]] = v
    return b
