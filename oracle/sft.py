"""Lattice sampling and Fourier-coefficient recovery (oracle; test
infrastructure only).

Section 2 (Definition of Fourier coefficients): g_hat_k = integral of
g(x) exp(-2 pi i k.x) over the torus.  On a rank-1 lattice, x_j = (j z / M) mod 1
and k.x_j = j (k.z) / M (mod 1), so the univariate samples t -> g(t z) hold
the coefficient of k in DFT bin (k.z mod M):

    g_hat_k = (1/M) sum_{j<M} g(x_j) exp(-2 pi i j (k.z mod M) / M)

exactly, whenever g's support is a subset of a set I on which the lattice is
reconstructing (Section "Previous results on SFTs", the reconstructing
property).  This module evaluates that sum directly (no FFT).

Known-support recovery (the premise of Theorem SFTRecovery that a
reconstructing lattice for I is known): read the bins of the candidates k in
I, symmetrise g_hat_k := (g_hat_k + conj(g_hat_{-k}))/2 (a real g has
Hermitian coefficients), and keep |g_hat_k| > tau * max |g_hat| (the paper
gives no threshold: tau is a parameter, 1e-9 in FP64 by default).  More than
``s_max`` survivors is an error (the paper's SFT returns at most 2s terms).

Support identification (no candidate set; the paper delegates it to the SFT
of its reference [gross_sparse_2021], which is not available, so this is the
reading used here): sample g also on the d shifted lattices x_j + e_i / P with
P a prime above 2 max |k_i|.  g(. + e_i/P) has coefficients
g_hat_k exp(2 pi i k_i / P), so in every bin b that holds a frequency k the
ratio X_i[b] / X_0[b] of the shifted to the plain spectrum is
exp(2 pi i k_i / P) and k_i = round(P arg(ratio) / (2 pi)) taken in
(-P/2, P/2].  The bins kept are those of the half spectrum 0 <= b <= M/2 with
|X_0[b]| > tau max |X_0|; a bin whose identified k does not satisfy
k.z = b (mod M) betrays a collision.  Values g_hat_k = X_0[b] / M; -k gets the
conjugate.  The spectra are numpy FFTs of the samples (a library step).

Pins: closed forms of cosine, sine and constant terms; equality with a full
length-M FFT from numpy when I is a bijective box; direct evaluation of g at
floating-point lattice points; exact support and values identified for
random sparse sums; the shifted-spectrum ratio of a single term in closed form
(tests/test_oracle_sft.py).
"""
from __future__ import annotations

import numpy as np

from .lattice import residues, is_reconstructing


def sample(freq, coef, z, M, js=None):
    """g(x_j) for g(x) = sum_t Re(coef_t exp(2 pi i freq_t.x)), at lattice
    indices ``js`` (all j < M by default).  The phase of term t at x_j is
    2 pi (j q_t mod M)/M with q_t = freq_t.z mod M, in exact integers."""
    M = int(M)
    js = np.arange(M, dtype=np.int64) if js is None else np.asarray(js, dtype=np.int64)
    q = residues(freq, z, M)
    g = np.zeros(len(js), dtype=np.float64)
    for qt, ct in zip(q, np.asarray(coef, np.complex128)):
        r = (js * int(qt)) % M
        g += (ct * np.exp(2j * np.pi * (r / M))).real
    return g


def dft_bins(samples, bins, M, chunk=1 << 14):
    """(1/M) sum_j samples[j] exp(-2 pi i j b / M) for each bin b (plain DFT)."""
    M = int(M)
    samples = np.asarray(samples)
    bins = np.asarray(bins, dtype=np.int64)
    out = np.zeros(len(bins), dtype=np.complex128)
    for j0 in range(0, M, chunk):
        j = np.arange(j0, min(M, j0 + chunk), dtype=np.int64)
        r = (j[:, None] * bins[None, :]) % M
        out += samples[j0:j0 + len(j)] @ np.exp(-2j * np.pi * (r / M))
    return out / M


def recover_known(samples, cand, z, M, tau=1e-9, s_max=None):
    """Known-support recovery from lattice samples.

    Returns (freq, val) of the kept candidates, in candidate order.  Raises if
    the lattice is not reconstructing for ``cand``, if ``cand`` is not closed
    under negation, or if more than ``s_max`` candidates survive."""
    cand = np.asarray(cand, np.int64)
    M = int(M)
    keys = {tuple(int(x) for x in row) for row in cand}
    if len(keys) != len(cand):
        raise ValueError("duplicate candidates")
    if any(tuple(-x for x in k) not in keys for k in keys):
        raise ValueError("candidate set is not symmetric")
    if not is_reconstructing(cand, z, M):
        raise ValueError("lattice is not reconstructing for the candidates")
    b = residues(cand, z, M)
    bneg = (M - b) % M
    ghat = dft_bins(samples, np.concatenate([b, bneg]), M)
    n = len(cand)
    val = 0.5 * (ghat[:n] + np.conj(ghat[n:]))
    mag = np.abs(val)
    keep = mag > tau * mag.max() if n else np.zeros(0, bool)
    if s_max is not None and keep.sum() > s_max:
        raise ValueError("more terms above threshold than s_max")
    return cand[keep].astype(np.int32), val[keep]


def true_coefficients(freq, coef):
    """Fourier coefficients of sum_t Re(c_t e_{p_t}) from the definition:
    Re(c e_p) = (c e_p + conj(c) e_{-p})/2, so p gets c/2 and -p gets conj(c)/2
    (p = 0 gets Re(c)).  Returns a dict {k: value}."""
    out = {}
    for p, c in zip(np.asarray(freq, np.int64), np.asarray(coef, np.complex128)):
        k = tuple(int(x) for x in p)
        mk = tuple(-x for x in k)
        if not any(k):
            out[k] = out.get(k, 0) + c.real
        else:
            out[k] = out.get(k, 0) + c / 2
            out[mk] = out.get(mk, 0) + np.conj(c) / 2
    return out


def sample_shifted(freq, coef, z, M, P, i):
    """g(x_j + e_i / P) for j < M: the phase p.x_j + p_i / P is the exact
    rational ((j q mod M) P + p_i M) / (M P) mod 1, q = p.z mod M."""
    M, P = int(M), int(P)
    js = np.arange(M, dtype=np.int64)
    q = residues(freq, z, M)
    out = np.zeros(M, np.float64)
    for qt, pt, ct in zip(q, np.asarray(freq, np.int64), np.asarray(coef, np.complex128)):
        num = (((js * int(qt)) % M) * P + int(pt[i]) * M) % (M * P)
        out += (ct * np.exp(2j * np.pi * (num / (M * P)))).real
    return out


def identify_samples(samples, z, M, P, tau=1e-9, s_max=None, keep=None, robust=False):
    """Support identification from given samples: row 0 of ``samples`` holds
    g(x_j), row i holds g(x_j + e_i / P) (i = 1..d).  Bins: the half
    spectrum 0 <= b <= M/2 with |X_0[b]| > tau max |X_0|; with ``keep``, at
    most that many, namely those strictly larger than the (keep+1)-th largest
    magnitude (compressible data, Section "Compressible"-type inputs).
    ``robust``: a bin whose identified k does not map back to it (aliasing of
    the neglected tail, or a collision) is dropped instead of raising."""
    M, P = int(M), int(P)
    samples = np.asarray(samples, np.float64)
    d = samples.shape[0] - 1
    X0 = np.fft.fft(samples[0])
    mag = np.abs(X0[: M // 2 + 1])
    bins = np.nonzero(mag > tau * mag.max())[0]
    if keep is not None and len(bins) > keep:
        cut = np.sort(mag[bins])[::-1][keep]
        bins = bins[mag[bins] > cut]
    ks = np.zeros((len(bins), d), np.int64)
    for i in range(d):
        Xi = np.fft.fft(samples[i + 1])
        ang = np.angle(Xi[bins] / X0[bins])
        k = np.rint(P * ang / (2 * np.pi)).astype(np.int64) % P
        ks[:, i] = np.where(k > P // 2, k - P, k)
    ok = residues(ks, z, M) == bins if len(bins) else np.zeros(0, bool)
    if not robust and not np.all(ok):
        raise ValueError("identified frequency does not sit in its bin (collision)")
    bins, ks = bins[ok], ks[ok]
    out_f, out_v = [], []
    for b, k in zip(bins.tolist(), ks):
        v = X0[b] / M
        out_f.append(k)
        out_v.append(v)
        if b != 0:
            out_f.append(-k)
            out_v.append(np.conj(v))
    if s_max is not None and len(out_f) > s_max:
        raise ValueError("more terms above threshold than s_max")
    return np.array(out_f, np.int32).reshape(len(out_f), d), np.array(out_v, np.complex128)


def identify(freq, coef, z, M, P, tau=1e-9, s_max=None):
    """Support identification of g = sum_t Re(c_t e_{p_t}) (see the module
    header).  Returns (freq [n, d] int32, val [n]) with every kept bin's k
    followed by -k (bin 0 alone), bins ascending."""
    d = np.asarray(freq).shape[1]
    rows = [sample(freq, coef, z, M)] + [sample_shifted(freq, coef, z, M, P, i) for i in range(d)]
    return identify_samples(np.stack(rows), z, M, P, tau=tau, s_max=s_max)
