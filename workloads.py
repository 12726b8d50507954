"""Seeded synthetic workloads for the sparse spectral method of Gross & Iwen
(arXiv 2302.00752) for -div(a grad u) = f on the d-torus.

This module only *draws*: integer frequency vectors, real and complex
coefficients, and raw random integers from which a rank-1 lattice generator is
picked.  It holds none of the method's arithmetic (no lattice residues, no
Fourier coefficients, no stamping, no Galerkin operator); both the CUDA path
and the CPU oracle consume its output and compute everything else on their
own.

Function data is a real trigonometric sum

    g(x) = sum_t Re( coef[t] * exp(2 pi i freq[t] . x) ),

so a cosine term c cos(2 pi p.x) is (p, c), a sine term c sin(2 pi p.x) is
(p, -i c) and the mean is (0, a0).  A manufactured solution is given by its
Fourier coefficients directly (both halves of each +-q pair).

Workload shapes follow the paper's exactly sparse experiments (Section
"Multivariate exactly sparse": one cosine term in a with a0 = 4; 25 cosine
terms with frequencies uniform in a box) scaled to the five configurations the
benchmarks use:

  cfg1  d=2,   s_a=9,  manufactured u (5 pairs in [-6,6]^2), N=2, box lattice
  cfg2  d=10,  s_a=21, manufactured u (20 pairs in [-8,8]^10), N=3, CBC lattice (M >= 1e6)
  cfg3  d=3,   multiscale a (scales 1, 2^6, 2^10), 8 f pairs, N=4
  cfg4  512 instances, d in 6..30, s_a odd in 5..41, 5..30 f pairs, N in {2,3}
  cfg5  d=100, s_a=41, 50 f pairs, 3 nonzero coordinates per frequency, N=3
"""
from __future__ import annotations

from dataclasses import dataclass, field
from math import comb

import numpy as np


@dataclass
class TrigSum:
    """g(x) = sum_t Re(coef[t] exp(2 pi i freq[t].x)); freq int32 [T, d]."""
    freq: np.ndarray
    coef: np.ndarray

    @property
    def d(self) -> int:
        return int(self.freq.shape[1])


@dataclass
class Instance:
    name: str
    d: int
    N: int                      # stamping level
    a: TrigSum                  # diffusion coefficient
    f: TrigSum | None = None    # forcing (None: manufactured from u)
    u_freq: np.ndarray | None = None   # manufactured solution support [n, d]
    u_val: np.ndarray | None = None    # its Fourier coefficients (Hermitian)
    lattice: dict = field(default_factory=dict)
    solve_precision: str = "fp64"      # "fp64" or "fp32_refined"
    sft_precision: str = "fp64"        # "fp64" or "fp32" samples + FFT
    cand: np.ndarray | None = None     # explicit candidate set (box lattice)
    seed: tuple = ()


# --------------------------------------------------------------------------
# draws


def _key(v):
    return tuple(int(x) for x in v)


def draw_freqs(rng, n, d, lo, hi, taken=None):
    """n integer vectors uniform in [lo, hi]^d, nonzero, no duplicate and no
    pair q, -q among themselves or with the vectors already in ``taken``."""
    taken = set() if taken is None else taken
    out = []
    while len(out) < n:
        v = rng.integers(lo, hi + 1, size=d)
        k = _key(v)
        if not any(k) or k in taken or _key(-v) in taken:
            continue
        taken.add(k)
        out.append(v)
    return np.array(out, dtype=np.int32).reshape(n, d), taken


def draw_sparse_freqs(rng, n, d, nnz, lo, hi, taken=None):
    """n vectors with ``nnz`` distinct nonzero coordinates, each uniform in
    [lo, hi] \\ {0}; no duplicates and no +-pairs (as ``draw_freqs``)."""
    taken = set() if taken is None else taken
    vals = np.array([x for x in range(lo, hi + 1) if x != 0])
    out = []
    while len(out) < n:
        v = np.zeros(d, dtype=np.int64)
        pos = rng.choice(d, size=nnz, replace=False)
        v[pos] = rng.choice(vals, size=nnz)
        k = _key(v)
        if k in taken or _key(-v) in taken:
            continue
        taken.add(k)
        out.append(v)
    return np.array(out, dtype=np.int32).reshape(n, d), taken


def draw_l1_coefs(rng, n, total):
    """n coefficients uniform in [-1, 1], rescaled so that sum |c| = total."""
    c = rng.uniform(-1.0, 1.0, size=n)
    return c * (total / np.abs(c).sum())


def cosine_sum(d, a0, freqs, coefs):
    """a0 + sum_j c_j cos(2 pi p_j.x) as a TrigSum (mean first)."""
    freq = np.vstack([np.zeros((1, d), np.int32), np.asarray(freqs, np.int32).reshape(-1, d)])
    coef = np.concatenate([[a0], np.asarray(coefs, np.float64)]).astype(np.complex128)
    return TrigSum(freq, coef)


def random_cos_sin(rng, freqs):
    """Each frequency gets amplitude U[-1,1] on a cosine or a sine (coin flip)."""
    n = len(freqs)
    amp = rng.uniform(-1.0, 1.0, size=n)
    is_sin = rng.integers(0, 2, size=n).astype(bool)
    coef = np.where(is_sin, -1j * amp, amp + 0j)
    return TrigSum(np.asarray(freqs, np.int32), coef.astype(np.complex128))


def manufactured(rng, qs):
    """Hermitian coefficients on +-q: re, im ~ N(0,1), u_{-q} = conj(u_q)."""
    n, d = qs.shape
    w = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    freq = np.empty((2 * n, d), np.int32)
    val = np.empty(2 * n, np.complex128)
    freq[0::2], freq[1::2] = qs, -qs
    val[0::2], val[1::2] = w, np.conj(w)
    return freq, val


def random_lattice_draws(rng, d, attempts=8, M_min=0, sigma=0.05):
    """Raw integers for a random rank-1 lattice (z_j uniform in 1..M-1 after
    M is chosen); ``attempts`` independent vectors, used in order until one
    is reconstructing."""
    raw = rng.integers(0, 2**62, size=(attempts, d), dtype=np.int64)
    return {"kind": "random", "raw": raw, "M_min": int(M_min), "sigma": float(sigma)}


def cbc_lattice_draws(rng, d, n_cand=64, M_min=10**6):
    """Raw candidate stream for a component-by-component lattice: row j holds
    the candidates tried, in order, for z_j (z_1 = 1)."""
    raw = rng.integers(0, 2**62, size=(d, n_cand), dtype=np.int64)
    return {"kind": "cbc", "raw": raw, "M_min": int(M_min)}


def generic_stamp_count(n_f, s_a, N):
    """Number of frequencies reachable from n_f starting points with at most N
    non-cancelling steps from (s_a-1)/2 +- pairs, with no coincidences.  Only
    used to shape the batched workload into its stated |S| range."""
    A = (s_a - 1) // 2
    tot = 0
    for n in range(N + 1):
        for t in range(0, min(n, A) + 1):
            c = 1 if (n == 0 and t == 0) else (comb(n - 1, t - 1) if t >= 1 else 0)
            tot += (2 ** t) * comb(A, t) * c
    return n_f * tot


# --------------------------------------------------------------------------
# configurations


def make_cfg1(seed=0):
    """d=2, 4 cosines (p in [-4,4]^2, sum|c| = 0.5), u with 10 nonzero
    coefficients in [-6,6]^2, N=2, box lattice z=(1,33), M=33^2 over [-16,16]^2."""
    rng = np.random.default_rng(seed)
    d = 2
    p, taken = draw_freqs(rng, 4, d, -4, 4)
    a = cosine_sum(d, 1.0, p, draw_l1_coefs(rng, 4, 0.5))
    q, _ = draw_freqs(rng, 5, d, -6, 6)
    uf, uv = manufactured(rng, q)
    g = np.arange(-16, 17)
    cand = np.stack(np.meshgrid(g, g, indexing="ij"), -1).reshape(-1, 2).astype(np.int32)
    lat = {"kind": "box", "z": np.array([1, 33], np.int64), "M": 33 * 33}
    return Instance("cfg1_d2_fp64", d, 2, a, None, uf, uv, lat, "fp64", "fp64", cand, (seed,))


def make_cfg2(seed=0):
    """d=10, 10 cosines in [-8,8]^10 (sum|c| = 0.5), u with 20 +-pairs in
    [-8,8]^10, N=3, CBC lattice with M >= 1e6."""
    rng = np.random.default_rng(seed)
    d = 10
    p, _ = draw_freqs(rng, 10, d, -8, 8)
    a = cosine_sum(d, 1.0, p, draw_l1_coefs(rng, 10, 0.5))
    q, _ = draw_freqs(rng, 20, d, -8, 8)
    uf, uv = manufactured(rng, q)
    lat = cbc_lattice_draws(rng, d, 64, 10**6)
    return Instance("cfg2_d10_fp64", d, 3, a, None, uf, uv, lat, "fp64", "fp64", None, (seed,))


def make_cfg3(seed=0):
    """d=3 multiscale: 1 + .25cos(2pi x1) + .15cos(2pi 2^6 x2) + .1cos(2pi 2^10 x3)
    plus 6 cosines in [-2^10,2^10]^3 with sum|c| = 0.25; f has 8 +-pairs whose
    j-th vector is drawn from the box of scale (1, 2^6, 2^10)[j mod 3]; N=4."""
    rng = np.random.default_rng(seed)
    d = 3
    fixed = np.array([[1, 0, 0], [0, 64, 0], [0, 0, 1024]], np.int32)
    taken = {_key(v) for v in fixed}
    extra, taken = draw_freqs(rng, 6, d, -1024, 1024, taken)
    a = cosine_sum(d, 1.0, np.vstack([fixed, extra]),
                   np.concatenate([[0.25, 0.15, 0.10], draw_l1_coefs(rng, 6, 0.25)]))
    scales = (1, 64, 1024)
    qs, ftaken = [], set()
    for j in range(8):
        s = scales[j % 3]
        v, ftaken = draw_freqs(rng, 1, d, -s, s, ftaken)
        qs.append(v[0])
    f = random_cos_sin(rng, np.array(qs, np.int32))
    lat = random_lattice_draws(rng, d)
    return Instance("cfg3_d3_multiscale_fp32ir", d, 4, a, f, None, None, lat,
                    "fp32_refined", "fp64", None, (seed,))


def make_cfg5(seed=0, smooth=False):
    """d=100, 20 cosines with 3 nonzero coordinates in [-4,4] (sum|c| = 0.5),
    f with 50 +-pairs of the same form, N=3, random lattice with M the
    smallest prime >= 2^26 (smooth=True: the smallest 7-smooth M >= 2^26, i.e.
    2^26), FP32 samples and FFT, FP32-refined solve."""
    rng = np.random.default_rng(seed)
    d = 100
    p, _ = draw_sparse_freqs(rng, 20, d, 3, -4, 4)
    a = cosine_sum(d, 1.0, p, draw_l1_coefs(rng, 20, 0.5))
    q, _ = draw_sparse_freqs(rng, 50, d, 3, -4, 4)
    f = random_cos_sin(rng, q)
    lat = random_lattice_draws(rng, d, M_min=2**26)
    lat["smooth"] = bool(smooth)
    return Instance("cfg5_d100_fp32ir", d, 3, a, f, None, None, lat,
                    "fp32_refined", "fp32", None, (seed,))


def make_batch_instance(seed, inst, lo=10**3, hi=10**5):
    """One instance of the batched workload (substream [seed, inst, attempt]);
    redrawn until the no-coincidence stamp size lies in [lo, hi]."""
    for attempt in range(1000):
        rng = np.random.default_rng([seed, inst, attempt])
        d = int(rng.integers(6, 31))
        s_a = int(rng.choice(np.arange(5, 42, 2)))
        n_fp = int(rng.integers(5, 31))
        N = int(rng.integers(2, 4))
        if not lo <= generic_stamp_count(2 * n_fp, s_a, N) <= hi:
            continue
        A = (s_a - 1) // 2
        p, _ = draw_freqs(rng, A, d, -8, 8)
        a = cosine_sum(d, 1.0, p, draw_l1_coefs(rng, A, 0.5))
        q, _ = draw_freqs(rng, n_fp, d, -8, 8)
        f = random_cos_sin(rng, q)
        lat = random_lattice_draws(rng, d)
        return Instance(f"batch{inst}_d{d}_s{s_a}_n{n_fp}_N{N}", d, N, a, f, None, None, lat,
                        "fp32_refined", "fp64", None, (seed, inst, attempt))
    raise RuntimeError("no instance in range")


def make_cfg4(seed=0, n=512):
    """512 independent instances of uneven size for the batched solve."""
    return [make_batch_instance(seed, i) for i in range(n)]


def make_one_term(d, seed=0, kmax=500, a0=4.0, c=None):
    """The paper's low-sparsity test: a = a0 + c cos(2 pi k_a.x), f = sin(2 pi k_f.x),
    k_a, k_f uniform in [-(kmax-1), kmax]^d."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(-1, 1) if c is None else c
    ka, taken = draw_freqs(rng, 1, d, -(kmax - 1), kmax)
    kf, _ = draw_freqs(rng, 1, d, -(kmax - 1), kmax, taken)
    a = cosine_sum(d, a0, ka, [c])
    f = TrigSum(kf.astype(np.int32), np.array([-1j], np.complex128))
    return Instance(f"oneterm_d{d}", d, 1, a, f, None, None, random_lattice_draws(rng, d),
                    "fp64", "fp64", None, (seed,))


def make_wide(seed=0, d=4, scale=20000, n_cos=3, n_f=3, N=2):
    """Multiscale data with large frequencies (|k|^2 ~ 1e10, past the int32
    norm range): a = 2 + n_cos cosines with sum |c| = 0.8, f = n_f cos/sin
    terms, all frequencies uniform in [-scale, scale]^d."""
    rng = np.random.default_rng([seed, 0x77])
    pa, taken = draw_freqs(rng, n_cos, d, -scale, scale)
    a = cosine_sum(d, 2.0, pa, draw_l1_coefs(rng, n_cos, 0.8))
    pf, _ = draw_freqs(rng, n_f, d, -scale, scale, taken)
    return Instance(f"wide_d{d}", d, N, a, random_cos_sin(rng, pf), None, None, random_lattice_draws(rng, d),
                    "fp64", "fp64", None, (seed,))


@dataclass
class AdrInstance:
    """Data of -div(a grad u) + b.grad u + c u = f (Remark ADR)."""
    name: str
    d: int
    N: int
    a: TrigSum
    b: list                     # d TrigSums, one per component of b
    c: TrigSum
    f: TrigSum | None = None
    u_freq: np.ndarray | None = None
    u_val: np.ndarray | None = None
    seed: tuple = ()
    lattice: dict = field(default_factory=dict)


def _sin_cos(rng, n_sin, n_cos, d, lo, hi, amp_lo, amp_hi):
    freq, _ = draw_freqs(rng, n_sin + n_cos, d, lo, hi)
    amp = rng.uniform(amp_lo, amp_hi, size=n_sin + n_cos)
    coef = np.concatenate([-1j * amp[:n_sin], amp[n_sin:] + 0j])
    return freq, coef.astype(np.complex128), amp


def make_adr(seed=0, N=1, d=3, kmax=50, n_a=2, n_bc=5, n_f=(2, 3), manufactured_u=None):
    """The three-dimensional exactly sparse ADR data of Section "Three-dimensional
    exactly sparse advection-diffusion-reaction equation": a = a0 + 2 sines + 2
    cosines (amplitudes U[-1,1]), each b_j and c (minus its mean) 5 sines + 5
    cosines (amplitudes U[0,1]), f = 2 sines + 3 cosines (U[-1,1]); every
    frequency uniform in [-(kmax-1), kmax]^d; a0 and c0 are 4 ceil(l2 norm of
    the other amplitudes).  manufactured_u = n draws a Hermitian u with n pairs
    in the same box instead of f (f then follows from the operator)."""
    rng = np.random.default_rng([seed, 0xadc])
    lo, hi = -(kmax - 1), kmax
    fa, ca, amp_a = _sin_cos(rng, n_a, n_a, d, lo, hi, -1.0, 1.0)
    a = TrigSum(np.vstack([np.zeros((1, d), np.int32), fa]).astype(np.int32),
                np.concatenate([[4.0 * np.ceil(np.linalg.norm(amp_a))], ca]).astype(np.complex128))
    b = []
    for _ in range(d):
        fb, cb, _ = _sin_cos(rng, n_bc, n_bc, d, lo, hi, 0.0, 1.0)
        b.append(TrigSum(fb.astype(np.int32), cb))
    fc, cc, amp_c = _sin_cos(rng, n_bc, n_bc, d, lo, hi, 0.0, 1.0)
    c = TrigSum(np.vstack([np.zeros((1, d), np.int32), fc]).astype(np.int32),
                np.concatenate([[4.0 * np.ceil(np.linalg.norm(amp_c))], cc]).astype(np.complex128))
    if manufactured_u:
        qs, _ = draw_freqs(rng, manufactured_u, d, lo, hi)
        uf, uv = manufactured(rng, qs)
        return AdrInstance(f"adr_d{d}_N{N}_u", d, N, a, b, c, None, uf, uv, (seed,), random_lattice_draws(rng, d))
    ff, cf, _ = _sin_cos(rng, n_f[0], n_f[1], d, lo, hi, -1.0, 1.0)
    return AdrInstance(f"adr_d{d}_N{N}", d, N, a, b, c, TrigSum(ff.astype(np.int32), cf), None, None, (seed,),
                       random_lattice_draws(rng, d))


def make_tiny(seed=0, d=2, n_cos=2, n_u=2, N=2, box=3, ubox=4, manufactured_u=True):
    """Small instances for brute-force checks (d <= 3, few terms)."""
    rng = np.random.default_rng(seed)
    p, _ = draw_freqs(rng, n_cos, d, -box, box)
    a = cosine_sum(d, 1.0, p, draw_l1_coefs(rng, n_cos, 0.5))
    q, _ = draw_freqs(rng, n_u, d, -ubox, ubox)
    if manufactured_u:
        uf, uv = manufactured(rng, q)
        return Instance(f"tiny{seed}", d, N, a, None, uf, uv, random_lattice_draws(rng, d),
                        "fp64", "fp64", None, (seed,))
    f = random_cos_sin(rng, q)
    return Instance(f"tiny{seed}", d, N, a, f, None, None, random_lattice_draws(rng, d),
                    "fp64", "fp64", None, (seed,))


CONFIGS = {
    "cfg1": make_cfg1,
    "cfg2": make_cfg2,
    "cfg3": make_cfg3,
    "cfg5": make_cfg5,
}


def mc_points(seed, Q, d):
    """Q uniform random points of T^d on the grid (2^-32 Z)^d, as the integer
    numerators X (uint32 [Q, d]); x = X / 2^32 (Monte Carlo proxy draws)."""
    rng = np.random.default_rng([seed, 0x6d63])
    return rng.integers(0, 1 << 32, size=(Q, d), dtype=np.uint64).astype(np.uint32)
