"""Algorithm 1 of the paper (sparse spectral method) driven through the C ABI.

Every numerical step runs in the library's kernels: lattice choice and its
reconstructing check, lattice sampling, the FFT-based recovery of a_hat and
f_hat, the stamping set, the right-hand side on S and the solve.  Python only
chooses which frequencies to look at (the candidate set I of Theorem
SFTRecovery: the supports of the given trigonometric data, closed under
negation) and moves handles between calls.

Manufactured instances (u_hat given) first build f_hat = L[a_hat] u_hat on
S^1[a_hat](supp u_hat), which holds its whole support (eq. GF), with the same
stamping and operator kernels; a_hat for that step is recovered on a lattice of
its own.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import torch

from . import binding as B


def support_of(freq):
    """Support of sum_t Re(c_t e_{p_t}): every p_t and -p_t (planning only)."""
    f = np.asarray(freq, np.int64)
    return np.unique(np.vstack([f, -f]), axis=0)


@dataclass
class Prepared:
    """Device-side inputs of one instance: the data as trigonometric sums, the
    candidate set and the lattice."""
    d: int
    N: int
    a_freq: torch.Tensor
    a_coef: torch.Tensor
    f_freq: torch.Tensor
    f_coef: torch.Tensor
    cand: torch.Tensor
    z: np.ndarray = None
    M: int = 0
    sft_precision: str = "fp64"
    solve_precision: str = "fp64"
    extra: dict = field(default_factory=dict)


def choose_lattice(lat_spec, cand):
    """a1: box lattice as given, or CBC / random lattice chosen on the GPU."""
    if lat_spec["kind"] == "box":
        return np.asarray(lat_spec["z"], np.int64), int(lat_spec["M"])
    if lat_spec["kind"] == "cbc":
        return B.lattice_cbc(cand, lat_spec["raw"], lat_spec["M_min"])
    z, M, _ = B.lattice_random(cand, lat_spec["raw"], lat_spec["sigma"], lat_spec["M_min"],
                               smooth=lat_spec.get("smooth", False))
    return z, M


def manufacture_forcing(inst, tau=1e-9):
    """f_hat = L[a_hat] u_hat on S^1[a_hat](supp u_hat) (device tensors)."""
    cand_a = np.asarray(inst.cand, np.int64) if inst.cand is not None else support_of(inst.a.freq)
    z, M = choose_lattice(inst.lattice, cand_a)
    af, av = B.sft_recover(z, M, inst.a.freq, inst.a.coef, cand_a, tau=tau)
    with B.stamp_build(af, av, inst.u_freq, 1) as s1:
        u_on, _ = s1.scatter(inst.u_freq, inst.u_val)
        fval = B.galerkin_apply(s1, u_on)
        ffreq, _ = s1.export()
    return ffreq, fval


def prepare(inst):
    """Inputs of the timed path: a and f as trigonometric sums on the device
    and the candidate set I."""
    d = inst.d
    a_freq = torch.as_tensor(np.asarray(inst.a.freq, np.int32)).cuda()
    a_coef = torch.as_tensor(np.asarray(inst.a.coef, np.complex128)).cuda()
    if inst.f is not None:
        f_freq = torch.as_tensor(np.asarray(inst.f.freq, np.int32)).cuda()
        f_coef = torch.as_tensor(np.asarray(inst.f.coef, np.complex128)).cuda()
        f_sup = support_of(inst.f.freq)
    else:
        f_freq, f_coef = manufacture_forcing(inst)
        f_sup = f_freq.cpu().numpy()
    if inst.cand is not None:
        cand = np.asarray(inst.cand, np.int64)
    else:
        cand = np.unique(np.vstack([support_of(inst.a.freq), support_of(f_sup)]), axis=0)
    cand_t = torch.as_tensor(cand.astype(np.int32)).cuda()
    return Prepared(d, inst.N, a_freq, a_coef, f_freq, f_coef, cand_t, sft_precision=inst.sft_precision,
                    solve_precision=inst.solve_precision, extra={"lattice": inst.lattice})


@dataclass
class Result:
    z: np.ndarray
    M: int
    a_freq: torch.Tensor
    a_val: torch.Tensor
    f_freq: torch.Tensor
    f_val: torch.Tensor
    stamp: B.Stamp
    f_on_S: torch.Tensor
    u: torch.Tensor
    stats: dict


def run(p: Prepared, tol=1e-12, max_iter=1000, tau=None, solve_precision=None, lattice=True, solve=True):
    """Algorithm 1: lattice, sft_recover(a), sft_recover(f), stamp_build, solve
    (solve=False stops after the right-hand side on S)."""
    if lattice or p.z is None:
        p.z, p.M = choose_lattice(p.extra["lattice"], p.cand)
    tau = (1e-9 if p.sft_precision == "fp64" else 1e-4) if tau is None else tau
    af, av = B.sft_recover(p.z, p.M, p.a_freq, p.a_coef, p.cand, tau=tau, precision=p.sft_precision)
    ff, fv = B.sft_recover(p.z, p.M, p.f_freq, p.f_coef, p.cand, tau=tau, precision=p.sft_precision)
    stamp = B.stamp_build(af, av, ff, p.N)
    f_on, _ = stamp.scatter(ff, fv, count_outside=False)
    if not solve:
        return Result(p.z, p.M, af, av, ff, fv, stamp, f_on, None, {})
    u, stats = B.solve(stamp, f_on, tol, max_iter, solve_precision or p.solve_precision)
    return Result(p.z, p.M, af, av, ff, fv, stamp, f_on, u, stats)


def run_fused(p: Prepared, tol=1e-12, max_iter=1000, tau=None, solve_precision=None, out=None):
    """Algorithm 1 through the single library call sparse_spectral_solve: the
    same stages as run(), without returning to Python between them.  The
    recovered coefficient lists and the right-hand side stay inside the
    library (None here)."""
    tau = (1e-9 if p.sft_precision == "fp64" else 1e-4) if tau is None else tau
    stamp, u, stats, p.z, p.M = B.sparse_spectral_solve(
        p.extra["lattice"], p.a_freq, p.a_coef, p.f_freq, p.f_coef, p.cand, p.N, tau=tau,
        sft_precision=p.sft_precision, solve_precision=solve_precision or p.solve_precision, tol=tol,
        max_iter=max_iter, out=out)
    return Result(p.z, p.M, None, None, None, None, stamp, None, u, stats)


def proxy_errors(res: Result, p: Prepared, X=None):
    """Lemma ProxyError after a solve: extends res.stamp by one level (S^{N+1}
    holds the support of L[a_hat] u^{s,N}, Proposition LExpansion) and returns
    the exact relative proxy ||f_hat - L u||_2 / ||f_hat||_2 and, given
    Monte Carlo points X (uint32 [Q, d], x = X / 2^32), its Monte Carlo
    estimate from the point values of f (the input trigonometric sum) and of
    f^{s,N}.  The stamp is left at level N + 1."""
    n_u = res.stamp.size
    res.stamp.extend(1)
    f1, _ = res.stamp.scatter(res.f_freq, res.f_val)
    num, den = B.proxy_residual(res.stamp, res.u.to(torch.complex128), f1)
    out = {"exact": float(np.sqrt(num / den)), "n_u": n_u, "size": res.stamp.size}
    if X is not None:
        r, fx = B.proxy_mc(res.stamp, res.u.to(torch.complex128), p.f_freq, p.f_coef, X)
        out["mc"] = float(torch.sqrt((r * r).sum() / (fx * fx).sum()))
    return out


def run_adr(inst, tol=1e-12, max_iter=2000, tau=1e-9):
    """Algorithm 1 with the modifications of Remark ADR: one reconstructing
    lattice for the union of the data's supports, sft_recover of a, of every
    component of b, of c and of f, stamp_build_adr (union step set) and the
    FP64 BiCGStab solve."""
    funcs = [inst.a, *inst.b, inst.c, inst.f]
    cand = np.unique(np.vstack([support_of(g.freq) for g in funcs]), axis=0)
    z, M = choose_lattice(inst.lattice, cand)
    rec = [B.sft_recover(z, M, g.freq, g.coef, cand, tau=tau) for g in funcs]
    a, c, f = rec[0], rec[-2], rec[-1]
    stamp = B.stamp_build_adr(a[0], a[1], rec[1:-2], c[0], c[1], f[0], inst.N)
    f_on, _ = stamp.scatter(*f)
    u, stats = B.solve(stamp, f_on, tol, max_iter, "fp64")
    return Result(z, M, a[0], a[1], f[0], f[1], stamp, f_on, u, stats)
