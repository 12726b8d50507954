/*
 * sparse_spectral.h - C ABI of a single-GPU (sm_103a) implementation of the
 * sparse spectral method of Gross & Iwen (arXiv 2302.00752) for the periodic
 * elliptic problem  -div(a grad u) = f  on the d-dimensional torus.
 *
 * The method (Algorithm 1 of the paper) is:
 *   1. recover the Fourier coefficients a_hat, f_hat of the data by sampling
 *      on a rank-1 lattice and taking a length-M one-dimensional FFT
 *      (sft_recover; Section "Previous results on SFTs", Theorem SFTRecovery);
 *   2. build the stamping set S^N[a_hat](supp f_hat) (stamp_build; eq. StampSet);
 *   3. apply the finite Galerkin operator (galerkin_apply; eq. GF,
 *      eq. FiniteGalerkinOperator);
 *   4. solve L_{N,s} u_hat = f_hat on S^N (solve, batch_solve;
 *      eq. SparseSpectralSFTEquation).
 *
 * Conventions shared by every call
 *   - Plain C types only.  "device" pointers are CUDA device memory owned by
 *     the caller; the library never frees them.  "host" pointers are read
 *     during the call only.
 *   - Complex values are interleaved (re, im): 2*n doubles for FP64, 2*n
 *     floats for FP32.  Frequencies are int32, row-major [n][d].
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Work is
 *     enqueued on it.  Calls that must return a size or a status computed on
 *     the GPU synchronise that stream once before returning (stated per call).
 *   - Every call returns SS_OK or an error status; ss_last_error() then holds
 *     a message for the calling thread.  On error, outputs are unspecified and
 *     handles stay valid to destroy.
 *   - Fourier convention (Section 2): g_hat_k = integral g(x) exp(-2 pi i k.x) dx.
 *   - A "trigonometric sum" is g(x) = sum_t Re(c_t exp(2 pi i p_t . x)): a
 *     cosine c cos(2 pi p.x) is (p, c), a sine c sin(2 pi p.x) is (p, -i c).
 */
#ifndef SPARSE_SPECTRAL_H
#define SPARSE_SPECTRAL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SS_OK = 0,
    SS_ERR_INVALID = 1,            /* bad argument (sizes, duplicates, f_hat_0 != 0, ...) */
    SS_ERR_OOM = 2,                /* device allocation failed */
    SS_ERR_CUDA = 3,               /* CUDA runtime or cuFFT error */
    SS_ERR_NOT_RECONSTRUCTING = 4, /* two candidates share a lattice residue */
    SS_ERR_HASH_FULL = 5,          /* frequency hash table exhausted */
    SS_ERR_NOT_ELLIPTIC = 6,       /* ||a_hat - a_hat_0||_1 >= |a_hat_0| */
    SS_ERR_NOT_CONVERGED = 7,      /* iteration cap reached before the tolerance */
    SS_ERR_TIMEOUT = 8,            /* a bounded device-side wait gave up */
    SS_ERR_KEY_RANGE = 9           /* frequencies too large for the packed key / index */
} ss_status;

typedef enum {
    SS_FP64 = 0,   /* FP64 samples and FFT; FP64 operator; plain FP64 CG */
    SS_FP32 = 1,   /* FP32 samples and FFT; FP32 operator; FP32 CG inside FP64 iterative refinement */
    SS_DF64 = 2    /* solve only: the FP64 CG in double-float arithmetic (float pairs, ~2^-48 relative per
                      operation) on the FP32 pipes, FP64 scalars and final residual */
} ss_precision;

/* Rank-1 lattice Lambda(z, M) = { (j z / M) mod 1 : j < M } (Section "Previous
 * results on SFTs", Definition of the rank-1 lattice).  z: host, d entries in
 * [1, M-1]; 2 <= M < 2^31. */
typedef struct { int32_t d; int64_t M; const int64_t* z; } ss_lattice;

/* Trigonometric sum: freq device int32 [n_terms][d], coef device FP64 complex
 * [n_terms]. */
typedef struct { int32_t d; int64_t n_terms; const int32_t* freq; const double* coef; } ss_trig;

/* Sparse coefficient list: freq device int32 [n][d], val device FP64 complex [n]. */
typedef struct { int32_t d; int64_t n; const int32_t* freq; const double* val; } ss_sparse;

/* Opaque stamping set: owns its hash table, packed keys, levels, neighbour
 * table and operator scratch until stamp_destroy. */
typedef struct ss_stamp_s* ss_stamp;

/* Opaque batch of stamping sets prepared for one persistent solve. */
typedef struct ss_batch_s* ss_batch;

typedef struct {
    int32_t status;        /* ss_status of this solve */
    int32_t outer_iters;   /* refinement steps (FP32 mode), 1 in FP64 mode */
    int32_t inner_iters;   /* CG iterations in total */
    int32_t applies;       /* operator applications (FP64 + FP32) */
    double rel_residual;   /* ||f - L u||_2 / ||f||_2 in FP64 at exit */
    double kernel_ms;      /* duration of the persistent solver launch (CUDA events on the stream) */
    int32_t half_system;   /* 1 when the Hermitian half system was solved (see solve) */
    int32_t real_coefficients;   /* 1 when a_hat was real and the operator's entry
                                    coefficients real (two FP64 FMAs per nonzero; see stamp_build) */
} ss_solve_stats;

const char* ss_last_error(void);
const char* ss_version(void);

/* Number of allocation calls the library has made in this process so far:
 * device memory (stream-ordered pool, cuFFT plans) and pinned host staging
 * blocks.  A diagnostic with no counterpart in the paper: a caller can check
 * that a stretch of calls (e.g. solve_noalloc) allocated nothing.  Host. */
int64_t ss_alloc_count(void);

/* Kernel timing, a diagnostic with no counterpart in the paper.  With on = 1
 * the library brackets its main kernels (the recovery transforms, the
 * neighbour lookups, the operator and the solver) with CUDA events on the
 * stream each is launched on - except while that stream is being captured
 * into a graph - and accumulates launches and device time per kernel name;
 * on = 2 brackets every kernel and stage that has a bracket (more event
 * records on the host); on = 0 stops.  Every call resets the totals and the
 * trace.  Host. */
ss_status ss_profile(int32_t on);

/* Totals of entry i (0-based, in name order): the kernel name (NUL-terminated,
 * truncated to name_cap bytes; name may be NULL), its launches and total
 * milliseconds.  Waits for the events still pending.  *n_out (may be NULL)
 * receives the number of entries; SS_ERR_INVALID when i is out of range. */
ss_status ss_profile_entry(int32_t i, char* name, int32_t name_cap, int64_t* launches, double* total_ms,
                           int32_t* n_out);

/* Trace entry i of the current profiling session: the bracket's name and its
 * start and end in ms relative to the session's first bracket start (device
 * time, in the order the brackets were resolved, at most 65536 entries).
 * n_out (nullable) receives the entry count.  Waits for the brackets queued
 * so far.  SS_ERR_INVALID for an index out of range. */
ss_status ss_profile_trace(int32_t i, char* name, int32_t name_cap, double* t0_ms, double* t1_ms, int32_t* n_out);

/* ---------------------------------------------------------------- lattice */

/* Lemma RandomRank1Lattice: smallest prime > max(K, n_I^2 / sigma) and
 * >= M_min.  Host arithmetic only.  K = expansion of the frequency set (side of
 * the smallest cube holding it). */
ss_status lattice_size(int64_t K, int64_t n_I, double sigma, int64_t M_min, int64_t* M_out);

/* Reconstructing property (Definition after the rank-1 lattice): checks
 * k.z != l.z (mod M) for all distinct rows of `freq` (device [n][d]).
 * Returns SS_ERR_NOT_RECONSTRUCTING on a collision and SS_ERR_INVALID on a
 * duplicate row.  Synchronises `stream`. */
ss_status lattice_check(const ss_lattice* lat, const int32_t* freq, int64_t n, void* stream);

/* Random lattice of Lemma RandomRank1Lattice for the frequency set `freq`
 * (device [n][d], distinct rows): M = lattice_size(K, n, sigma, M_min) and, for
 * attempt a = 0.., z_j = 1 + raw[a][j] mod (M-1) (raw: host [attempts][d],
 * non-negative); the first reconstructing attempt is returned in z_out (host,
 * d entries), M_out, attempt_out.  SS_ERR_NOT_RECONSTRUCTING if none is.
 * Synchronises `stream`. */
ss_status lattice_random(const int32_t* freq, int64_t n, int32_t d, double sigma, int64_t M_min,
                         const int64_t* raw, int32_t attempts, int64_t* z_out, int64_t* M_out,
                         int32_t* attempt_out, void* stream);

/* lattice_random with an FFT-friendly size: M = the smallest 7-smooth integer
 * (prime factors 2, 3, 5, 7) >= max(K + 1, |I|^2 / sigma, M_min), then the
 * same draws.  Lemma RandomRank1Lattice's probability bound is for prime M;
 * here the exact reconstructing check of every draw stands in for it (a draw
 * that fails is skipped), so the result is as reliable and the length-M FFT
 * needs no Bluestein chirp. */
ss_status lattice_random_smooth(const int32_t* freq, int64_t n, int32_t d, double sigma, int64_t M_min,
                                const int64_t* raw, int32_t attempts, int64_t* z_out, int64_t* M_out,
                                int32_t* attempt_out, void* stream);

/* Component-by-component lattice (named in Section "Improvements with
 * randomized lattices"; criterion not given by the paper): M = smallest
 * 7-smooth integer (prime factors 2, 3, 5, 7: a mixed-radix FFT length)
 * >= max(M_min, K + 1), z_1 = 1, and for j >= 2 the first candidate
 * 1 + raw[j][c] mod (M-1) (raw: host [d][n_cand]) under which the distinct
 * projections of `freq` onto coordinates 1..j have distinct residues.
 * Synchronises `stream`. */
ss_status lattice_cbc(const int32_t* freq, int64_t n, int32_t d, int64_t M_min, const int64_t* raw,
                      int32_t n_cand, int64_t* z_out, int64_t* M_out, void* stream);

/* -------------------------------------------------------------------- SFT */

/* Lattice sampling: samples[j] = g(x_j), x_j = (j z / M) mod 1, j < M, with the
 * phase of each term taken from the exact residue (j (p.z mod M)) mod M.
 * Terms are evaluated directly, O(M T).  An FP64 sum with many terms (at
 * least 64 on a 7-smooth M up to 2^25, at least 512 on another M) is instead
 * evaluated as the length-M inverse DFT of its terms binned by residue; a
 * residue shared by several terms is summed in term order.
 * samples: device, M doubles (SS_FP64) or M floats (SS_FP32). */
ss_status lattice_sample(const ss_lattice* lat, const ss_trig* g, ss_precision prec, void* samples,
                         void* stream);

/* Known-support recovery from lattice samples (Theorem SFTRecovery with a
 * reconstructing lattice for the candidate set I given): one real-to-complex
 * FFT of length M (cuFFT), then for every candidate k in I (device [n_cand][d],
 * closed under negation, lattice reconstructing for I):
 *   g_hat_k = (X[k.z mod M] + conj(X[-k.z mod M])) / (2M),
 * kept when |g_hat_k| > tau * max_I |g_hat|.  Kept frequencies and values are
 * written in candidate order to freq_out (device [n_cand][d]) and val_out
 * (device FP64 complex [n_cand]); their number to *n_out.  More than s_max
 * survivors is SS_ERR_INVALID.  samples: device, M reals in `prec`.
 * Synchronises `stream`. */
ss_status sft_recover_samples(const ss_lattice* lat, const void* samples, ss_precision prec,
                              const int32_t* cand, int64_t n_cand, int64_t s_max, double tau,
                              int32_t* freq_out, double* val_out, int64_t* n_out, void* stream);

/* lattice_sample followed by sft_recover_samples (library-owned sample and
 * FFT buffers).  In FP64 on a 7-smooth M up to 2^22 both transforms (the
 * inverse one that samples g and the forward one that recovers it) run in the
 * library's double-float FFT instead of cuFFT.  That FFT rounds at about
 * 2^-46 relative.  The thresholding and output are as in sft_recover_samples.
 * Synchronises `stream`. */
ss_status sft_recover(const ss_lattice* lat, const ss_trig* g, ss_precision prec, const int32_t* cand,
                      int64_t n_cand, int64_t s_max, double tau, int32_t* freq_out, double* val_out,
                      int64_t* n_out, void* stream);

/* Support identification when no candidate set is known (the paper delegates
 * it to the SFT of its reference [gross_sparse_2021]; this is the reading
 * used here).  Samples g on the lattice and on the d shifted lattices
 * x_j + e_i / P (P > 2 max |k_i|, e.g. the smallest prime above 2K + 1 for
 * bandwidth K): the shifted sum has the coefficients g_hat_k exp(2 pi i k_i / P),
 * so in each kept bin b (0 <= b <= M/2, |X_0[b]| > tau max |X_0|) the ratio of
 * the shifted to the plain spectrum gives k_i = round(P arg(X_i[b] / X_0[b]) / (2 pi))
 * in (-P/2, P/2].  g_hat_k = X_0[b] / M; -k gets the conjugate.  Output in
 * increasing bin order, each k followed by -k (k = 0 alone): freq_out device
 * [s_max][d], val_out device FP64 complex [s_max], the count in *n_out; more
 * than s_max terms is SS_ERR_INVALID; a k that does not map back to its bin
 * (k.z mod M != b: the lattice is not reconstructing for the support) is
 * SS_ERR_NOT_RECONSTRUCTING.  Costs d + 1 samplings and FFTs of length M.
 * Synchronises `stream`. */
ss_status sft_identify(const ss_lattice* lat, const ss_trig* g, ss_precision prec, int32_t P, int64_t s_max,
                       double tau, int32_t* freq_out, double* val_out, int64_t* n_out, void* stream);

/* The same from given samples (black-box access to g):
 * samples: device, (d + 1) rows of M reals in `prec`, row 0 = g(x_j), row i =
 * g(x_j + e_i / P).  For compressible (not exactly sparse) data, keep > 0
 * limits the bins to the keep largest magnitudes above the threshold (exact
 * selection: values strictly above the (keep+1)-th largest, found by radix
 * passes over their bit patterns), and robust != 0 drops the bins whose
 * identified k does not map back to them (aliasing of the neglected tail)
 * instead of failing.  keep = 0, robust = 0 is sft_identify's behaviour. */
ss_status sft_identify_samples(const ss_lattice* lat, int32_t P, const void* samples, ss_precision prec,
                               int64_t s_max, double tau, int64_t keep, int32_t robust, int32_t* freq_out,
                               double* val_out, int64_t* n_out, void* stream);

/* ------------------------------------------------------------------ stamp */

/* S^N[a_hat](F) of eq. StampSet with F = f_freq (device [n_f][d], distinct,
 * nonzero) and supp a_hat from a_hat (closed under negation, containing 0,
 * Hermitian values).  Canonical order: level 0 is F in signed lexicographic
 * order; level n lists new frequencies in order of first discovery over the
 * parents of level n-1 (index order) and the nonzero p of supp a_hat in
 * signed lexicographic order.  Also builds the neighbour table of the
 * operator.  Rejects a_hat that fails the positivity check
 * ||a_hat - a_hat_0||_1 < |a_hat_0| (Remark after Corollary
 * SpectralConvergenceNoSFT) with SS_ERR_NOT_ELLIPTIC.  Synchronises `stream`
 * once per level. */
ss_status stamp_build(const ss_sparse* a_hat, const int32_t* f_freq, int64_t n_f, int32_t N,
                      ss_stamp* out, void* stream);

/* Stamping set and operator of the advection-diffusion-reaction problem
 * -div(a grad u) + b.grad u + c u = f (Remark ADR).  a_hat and c_hat as in
 * stamp_build's a_hat; b_hat: host array of d sparse lists, component j of
 * the vector field b (device frequencies and values, possibly empty).  All
 * Hermitian (real data); a_hat must pass the positivity check.  The step set
 * of eq. StampSet is the union U of supp a_hat, supp b_hat_j and supp c_hat
 * (their Minkowski sum would add frequencies with no coupling); the canonical
 * order is stamp_build's with U in place of supp a_hat.  The operator entry
 * of row k and l = k - p, p in U, is
 *   4 pi^2 (k.l) a_hat_p + 2 pi i (l . b_hat_p) + c_hat_p
 * (b_hat_p = (b_hat_{1,p}, ..., b_hat_{d,p})); k = 0 is an ordinary row and
 * column, and F may contain 0.  Solved by solve in SS_FP64 (BiCGStab);
 * galerkin_apply, proxy_residual, proxy_mc and stamp_extend apply; the FP32
 * operator, solve_noalloc and batches do not (SS_ERR_INVALID).  d <= 64. */
ss_status stamp_build_adr(const ss_sparse* a_hat, const ss_sparse* b_hat, const ss_sparse* c_hat,
                          const int32_t* f_freq, int64_t n_f, int32_t N, ss_stamp* out, void* stream);

/* |S|, operator nonzeros #{(k,p): k in S\{0}, k-p in S\{0}}, the canonical
 * index of k = 0 (-1 if absent), and the number of levels (N + 1).  Host. */
ss_status stamp_info(ss_stamp s, int64_t* size, int64_t* nnz, int64_t* zero_index, int32_t* n_levels);

/* *real = 1 when the stamp's a_hat was taken as real: a even, every
 * |Im a_hat_p| <= 1e-13 max |a_hat| (below an FP64 recovery's rounding), the
 * imaginary parts dropped at build.  Every entry coefficient
 * 2 pi^2 (|k|^2 + |l|^2 - |p|^2) a_hat_p is then real and the FP64 and
 * double-float operators take two multiply-adds per nonzero instead of four.
 * Never for an ADR stamp.  Host. */
ss_status stamp_real_coefficients(ss_stamp s, int32_t* real);

/* Frequencies (device int32 [|S|][d]) and levels (device int8 [|S|]) in
 * canonical order; either output may be NULL. */
ss_status stamp_export(ss_stamp s, int32_t* freq_out, int8_t* level_out, void* stream);

/* Canonical index of each query frequency (device [n][d]) into idx_out
 * (device int64 [n]), -1 when absent. */
ss_status stamp_lookup(ss_stamp s, const int32_t* freq, int64_t n, int64_t* idx_out, void* stream);

/* Scatter a sparse list onto S: out (device FP64 complex [|S|]) is zeroed,
 * then out[index(k)] = val for every entry whose k lies in S; *n_outside
 * (host) receives the number of entries that do not, and the call then
 * synchronises `stream`; with n_outside NULL it stays asynchronous. */
ss_status stamp_scatter(ss_stamp s, const ss_sparse* g, double* out, int64_t* n_outside, void* stream);

/* Grow S^N to S^{N+levels} in place (eq. StampSet applied `levels` more times;
 * the paper re-solves on successive stamping levels, Section "Low
 * sparsity").  Canonical indices of the existing frequencies do not change: a
 * vector on S^N is the prefix of the same vector on S^{N+levels}.  The key
 * layout is widened when the new levels need it; the neighbour table is
 * rebuilt.  Synchronises `stream` once per new level.  On error the stamp may
 * only be destroyed. */
ss_status stamp_extend(ss_stamp s, int32_t levels, void* stream);

/* Upper bound on the slots of the frequency hash table of every stamping set
 * built or extended after this call (rounded down to a power of two, at least
 * 16; 0 = no bound, the default).  A set whose frequencies do not fit makes
 * stamp_build / stamp_extend return SS_ERR_HASH_FULL (every probe sequence is
 * bounded by the table size, so an exhausted table ends the build with that
 * status instead of waiting).  For capping the table's device memory, and for
 * exercising the exhausted-table path.  Process-wide; host. */
ss_status stamp_set_table_limit(int64_t max_slots);

void stamp_destroy(ss_stamp s);

/* -------------------------------------------------------------- operator */

/* y = L_{N,s} u on S (eq. FiniteGalerkinOperator):
 *   y_k = sum_{p in supp a_hat, k-p in S} 4 pi^2 (k.(k-p)) a_hat_p u_{k-p},
 * the integer k.(k-p) formed exactly as (|k|^2 + |k-p|^2 - |p|^2)/2; the row of
 * k = 0 is the identity (pins u_hat_0).  ADR stamps: the entries of
 * stamp_build_adr, no identity row, SS_FP64 only.  u, y: device complex [|S|], FP64 or
 * FP32 per `prec` (FP32: FP32 values, FP32 accumulation).  Uses the stamp's
 * scratch: concurrent calls on one stamp must be on one stream. */
ss_status galerkin_apply(ss_stamp s, const void* u, void* y, ss_precision prec, void* stream);

/* Exact proxy error of Lemma ProxyError: with u given on the first n_u
 * frequencies of S (u_prefix: device FP64 complex [n_u], zero elsewhere) and
 * f_on_S (device FP64 complex [|S|]), writes out2[0] = ||f - L u||_2^2 and
 * out2[1] = ||f||_2^2 over S (host, 2 doubles).  When S = S^{N+1} and u solves
 * on S^N, L[a_hat] u is supported in S^{N+1} (Proposition LExpansion), so the
 * sum is exact.  FP64 operator; deterministic reduction; synchronises `stream`. */
ss_status proxy_residual(ss_stamp s, const double* u_prefix, int64_t n_u, const double* f_on_S, double* out2,
                         void* stream);

/* Monte Carlo proxy error (Lemma ProxyError; Section "Code and testing
 * overview"): point values at x_q = X[q] / 2^32 (X: device uint32 [Q][d], the
 * caller's uniform random draws on the grid (2^-32 Z)^d):
 *   f_out[q] = f(x_q) = sum_t Re(f.coef[t] exp(2 pi i f.freq[t] . x_q)),
 *   r_out[q] = f(x_q) - f^{s,N}(x_q),  f^{s,N}(x) = sum_{k in S} (L u)_k exp(2 pi i k.x),
 * with u on the first n_u frequencies of S (u_prefix: device FP64 complex
 * [n_u], zero elsewhere) and L the operator on S's rows ((L u)_0 = 0 for the
 * diffusion operator; an ordinary row for ADR stamps).  When
 * S = S^{N+1} and u solves on S^N, f^{s,N} = L[a_hat] u is exact (Proposition
 * LExpansion).  The estimate of ||f - f^{s,N}||_{L2} / ||f||_{L2} is
 * sqrt(sum r^2 / sum f^2).  Phases k.X mod 2^32 are exact integers; each
 * term is evaluated in double-float arithmetic (about 1e-13 of |coef| per
 * term).  r_out, f_out: device FP64 [Q].  Deterministic; asynchronous on
 * `stream`; uses the stamp's operator scratch. */
ss_status proxy_mc(ss_stamp s, const double* u_prefix, int64_t n_u, const ss_trig* f, const uint32_t* X, int64_t Q,
                   double* r_out, double* f_out, void* stream);

/* ----------------------------------------------------------------- solve */

/* Solve L_{N,s} u = f on S (eq. SparseSpectralSFTEquation) by Jacobi-
 * preconditioned CG (D_k = 4 pi^2 Re(a_hat_0) |k|^2, the denominator of the
 * diagonal rearrangement in the proof of Proposition SolutionSupport):
 *   SS_FP64  plain FP64 CG until ||f - L u||_2 <= tol ||f||_2;
 *   SS_FP32  FP32-operator CG (FP64 vectors and scalars) inside FP64 iterative
 *            refinement whose residual f - L u is formed with the FP64 operator.
 * f_on_S, u_on_S: device FP64 complex [|S|].  One persistent cooperative
 * launch.  Writes stats (host, may be NULL) and synchronises `stream`.
 * f_hat_0 must be 0 (SS_ERR_INVALID otherwise).  ADR stamps (stamp_build_adr)
 * take SS_FP64 only and are solved by BiCGStab with the operator's complex
 * diagonal as right Jacobi preconditioner, to the same stopping rule; f_hat_0
 * is unrestricted there. */
ss_status solve(ss_stamp s, const double* f_on_S, double* u_on_S, double tol, int32_t max_iter,
                ss_precision prec, ss_solve_stats* stats, void* stream);

/* Hermitian half system (no counterpart in the paper, which solves the full
 * system): for real data - F = -F and a_hat_{-p} = conj(a_hat_p) bit for bit,
 * which stamp_build detects - S is symmetric and L maps Hermitian vectors
 * (u_{-k} = conj(u_k)) to Hermitian vectors, so for a Hermitian f the rows
 * k >lex 0 carry the whole solution.  solve (every precision; not ADR stamps)
 * then runs the same solver on those rows only, reading a neighbour l <lex 0 as conj(u_{-l}) (half the
 * rows and half the stored nonzeros per application; CG scalars and the
 * residual ratio are those of the full system up to rounding), and unfolds u
 * over S; stats->half_system = 1.  An f that is not Hermitian bit for bit
 * falls back to the full system within the same call.  use_half = 0 always
 * solves the full system (default 1). */
ss_status solve_set_symmetry(ss_stamp s, int32_t use_half);

/* Bound on every device-side wait of this stamp's persistent solver (the grid
 * barrier between CG phases): a wait longer than ns nanoseconds ends the
 * launch - every block returns - and solve reports SS_ERR_TIMEOUT, leaving
 * the stamp usable for the next solve.  ns = 0 gives up at the first poll of
 * a wait (always a timeout on a launch of more than one block).  Default
 * 2 s.  Takes effect at the next solve. */
ss_status solve_set_wait_limit(ss_stamp s, int64_t ns);

/* Tile shape of this stamp's persistent solve: threads per block (128, 256,
 * 512 or 1024), resident blocks per SM (0 = as many as fit) and static work
 * chunks per block.  Takes effect at the next solve.  Default 1024, 1, 1. */
ss_status solve_set_config(ss_stamp s, int32_t block, int32_t blocks_per_sm, int32_t chunks_per_block);

/* Allocation-free variant of solve() (the paper has no counterpart: this is a
 * deployment convenience).  For callers that may not allocate device memory
 * while they run - plug-ins inside a host application that owns all device
 * memory, latency-bound loops that must not stall on cudaMalloc (which
 * synchronises the device), or processes with a device-memory budget fixed at
 * start-up.
 * The caller passes f_on_S and u_on_S exactly as for solve(); all workspace
 * comes from one file-scope device array of about 7.4 MB that every GPU which
 * loads the library holds until exit, sized for a stamping set of at most
 * 32,768 padded rows (|S| <= 32,768, rounded up to whole 32-row slices);
 * larger sets return SS_ERR_INVALID.  It calls no allocating routine.
 * Set-up: the first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current and keeps it for the life of
 * the process; make that first call before any stream capture.  The kept
 * address does not survive cudaDeviceReset (or any other teardown of the
 * device's primary context): do not call solve_noalloc on a device after
 * resetting it.  Unlike solve() it always solves the full system (never the
 * Hermitian half system), with the work split solve() uses for the full
 * system at its default tile shape.  Every call uses the whole array and leaves its contents
 * there (the next call re-initialises what must start at zero), so calls whose
 * GPU work overlaps - on different streams or threads - race and must be
 * serialised by the caller.  Synchronises `stream`; stats as solve() (without
 * kernel_ms). */
ss_status solve_noalloc(ss_stamp s, const double* f_on_S, double* u_on_S, double tol, int32_t max_iter,
                        ss_precision prec, ss_solve_stats* stats, void* stream);

/* Many instances in one persistent launch: the rows of all instances are
 * concatenated, every CG phase runs over all of them with per-instance scalars,
 * and converged instances drop out.  batch_create copies the instances'
 * operators into one layout (the stamps may be destroyed afterwards);
 * tile shapes come from the autotuner (batch_autotune) when it has run. */
ss_status batch_create(int32_t n_inst, const ss_stamp* stamps, ss_batch* out, void* stream);

/* f[i], u[i]: device FP64 complex [|S_i|].  use_graph != 0 captures the
 * launch sequence in a CUDA graph on first use and replays it while the
 * pointers are unchanged.  stats: host array [n_inst] (may be NULL).
 * Synchronises `stream`. */
ss_status batch_solve(ss_batch b, const double* const* f, double* const* u, double tol,
                      int32_t max_iter, ss_precision prec, int32_t use_graph,
                      ss_solve_stats* stats, void* stream);

/* Times the persistent solve over candidate tile shapes (warps per block,
 * blocks per SM) for this batch and keeps the fastest.  best_ms (host, may be
 * NULL) receives its time.  Synchronises `stream`. */
ss_status batch_autotune(ss_batch b, const double* const* f, double* const* u, double tol,
                         int32_t max_iter, ss_precision prec, double* best_ms, void* stream);

/* Current tile shape and work split of the batch (any output may be NULL). */
ss_status batch_config(ss_batch b, int32_t* block, int32_t* blocks_per_sm, int32_t* chunks_per_block,
                       int32_t* grid, int32_t* n_chunks);

/* Set the tile shape: block in {128, 256, 512, 1024} threads, blocks_per_sm
 * (0 = as many as fit), chunks_per_block >= 1 (static work units per block). */
ss_status batch_set_config(ss_batch b, int32_t block, int32_t blocks_per_sm, int32_t chunks_per_block);

/* When every stamp of the batch has a Hermitian half system (see
 * solve_set_symmetry), batch_create also builds the batch of the half systems
 * and batch_solve runs it: the callers' f are gathered onto the compact rows
 * (and checked to be Hermitian bit for bit), the half batch is solved, and
 * every u is unfolded over its S; stats[i].half_system = 1.  A non-Hermitian
 * f makes the call solve the full batch instead.  use_half = 0 always solves
 * the full batch (default 1).  batch_autotune and batch_config act on the
 * batch that batch_solve runs. */
ss_status batch_set_symmetry(ss_batch b, int32_t use_half);

void batch_destroy(ss_batch b);

/* ------------------------------------------------------ the whole method */

/* How sparse_spectral_solve picks its rank-1 lattice. */
typedef enum {
    SS_LATTICE_GIVEN = 0,          /* z and M as given */
    SS_LATTICE_CBC = 1,            /* lattice_cbc(cand, M_min, raw [d][n_raw]) */
    SS_LATTICE_RANDOM = 2,         /* lattice_random(cand, sigma, M_min, raw [n_raw][d]) */
    SS_LATTICE_RANDOM_SMOOTH = 3   /* lattice_random_smooth, same arguments */
} ss_lattice_kind;

typedef struct {
    int32_t kind;          /* ss_lattice_kind */
    int32_t d;
    const int64_t* z;      /* GIVEN: host [d] */
    int64_t M;             /* GIVEN */
    const int64_t* raw;    /* CBC, RANDOM*: host draws (layouts above), non-negative */
    int32_t n_raw;         /* CBC: candidates per coordinate; RANDOM*: attempts */
    int64_t M_min;         /* CBC, RANDOM* */
    double sigma;          /* RANDOM* */
} ss_lattice_spec;

/* Algorithm 1 (Section "Sparse spectral method", Algorithm SparseSFT) in one
 * call: the lattice for the candidate set `cand` (device int32 [n_cand][d],
 * the frequency set I of Theorem SFTRecovery), a_hat = SFT(a) and
 * f_hat = SFT(f) on it (sft_recover with threshold tau, precision sft_prec),
 * S^N[a_hat](supp f_hat) (stamp_build), f_hat scattered onto S and the solve
 * of L_{N,s} u = f_hat (solve with tol, max_iter, solve_prec).  a and f
 * share one complex transform in two cases: FP64 on a 7-smooth M up to 2^22,
 * where sft_recover takes the double-float FFT and one transform runs each
 * way; and FP32 on an M that is not 7-smooth, where cuFFT takes Bluestein's
 * method and one forward C2C carries s_a / s_a' + i s_f / s_f'.  The scales
 * s_a', s_f' (and their FP64 counterparts) are powers of two near the two
 * sums' l1 norms.  In both cases f_hat agrees with two separate sft_recover
 * calls to within the transform's rounding, not bit for bit.  The stages
 * run back to back on `stream` without returning to the caller in between;
 * each synchronises where its own entry point does.  Outputs: the lattice
 * (z_out host [d], M_out), the stamping set (*stamp_out, caller destroys it;
 * the solution is kept in it, see stamp_solution), the solution copied into
 * u_out (device FP64 complex, capacity u_cap rows; skipped when u_out is
 * NULL or |S| > u_cap) and the solve statistics (stats, host, may be NULL).
 * Returns the first failing stage's status;
 * SS_ERR_NOT_CONVERGED still returns the stamp, any other error destroys it
 * and leaves *stamp_out NULL. */
ss_status sparse_spectral_solve(const ss_lattice_spec* lat, const ss_trig* a, const ss_trig* f,
                                const int32_t* cand, int64_t n_cand, int32_t N, double tau,
                                ss_precision sft_prec, ss_precision solve_prec, double tol, int32_t max_iter,
                                int64_t* z_out, int64_t* M_out, ss_stamp* stamp_out, double* u_out, int64_t u_cap,
                                ss_solve_stats* stats, void* stream);

/* Copy the solution that sparse_spectral_solve left in the stamp into u_out
 * (device FP64 complex, as many rows as S had at the solve: after
 * stamp_extend it is the prefix of the extended set).  Asynchronous. */
ss_status stamp_solution(ss_stamp s, double* u_out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SPARSE_SPECTRAL_H */
