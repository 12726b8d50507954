// Pruned DFTs of a 7-smooth length M for the coefficient recovery on long
// lattices (FP64: double-float arithmetic, beyond the full transform of
// fft_df.cu; FP32: FP32 arithmetic)
// (Section "Previous results on SFTs": one length-M 1D FFT of the lattice
// samples; only the bins k.z mod M of the candidate set are read).
//
// Both directions use the four-step split M = P Q (j = q + Q p, r = k + P m):
//   w^{j r} = w^{q r} w_P^{p k},   w = exp(2 pi i / M), w_P = w^Q.
// * Evaluation (sampling a trigonometric sum: s[j] = sum_e v_e w^{j r_e} over a
//   few entries (r_e, v_e)): for every column q, C[k][q] = sum_{e : r_e = k mod P}
//   v_e w^{q r_e} (the entries bucketed by r_e mod P), then one length-P
//   transform over k gives s[q + Q p] for all p.  Cost O(M log P + Q n_e).
// * Pruned forward transform (X[b] = sum_j s[j] w^{-j b} at n_out bins): one
//   length-P transform over p per column q gives Y[k][q]; then
//   X[b] = sum_q Y[b mod P][q] w^{-q b}.  Cost O(M log P + Q n_out).
// Blocks take tiles of W consecutive columns (W P = kPrTile values in shared
// memory), so global reads and writes of s run along q and are coalesced.
// Twiddles come from the two-level double-float table
// w^r = T1[r >> b] T0[r & (2^b - 1)].
#pragma once

#include "fft_df.cuh"
#include "ss_internal.cuh"

namespace ss {

// exp(2 pi i r / M) = t1[r >> b] * t0[r & (2^b - 1)], double-float float4
// (re.hi, re.lo, im.hi, im.lo); b = ceil(log2(M) / 2).
struct TwoLevelTable {
  int64_t M = 0;
  int b = 0;
  DevBuf<float4> t0, t1;
};
ss_status two_level_table(int64_t M, TwoLevelTable* T, cudaStream_t st);

// Split M = P Q for a pruned transform that touches n sparse bins (entries
// or outputs): P the divisor of M (prime factors 2, 3, 5, 7; at most 1024)
// that minimises log2 P + n / P, and W the largest power of two with
// W P <= tile.  False when M has no such divisor (then the pruned transforms
// do not apply).
struct PrunedSplit {
  int P = 0;
  int64_t Q = 0;
  int W = 0;   // columns per tile
  DfRadices rad;
};
bool pruned_split(int64_t M, int64_t n, PrunedSplit* out, int tile = 2048);

// True when M is 7-smooth and a split exists for a handful of bins.
bool pruned_supported(int64_t M);

// Layout of the sample vector s of the pruned transforms.
enum class PrunedFormat {
  kDfComplex,   // double-float complex (float4 per node): FP64 recovery of two sums
  kF64Real,     // FP64 real (double per node)
  kF32Complex,  // FP32 complex (float2 per node): FP32 recovery of two sums
  kF32Real      // FP32 real (float per node)
};

// Samples of s_a / scale[0] + i s_f / scale[1] at the M lattice nodes, where
// s_a(j) = sum_t Re(ca_t w^{j qa_t}) over na (device count, at most na_max)
// merged terms and likewise s_f, in the layout fmt (the real formats hold the
// real parts; f must then be empty).  Double-float arithmetic for the FP64
// formats, FP32 for the FP32 ones.  scale: device [2] (powers of two) or null
// (1).  Asynchronous on st.
ss_status pruned_eval_pair(const TwoLevelTable& T, const int64_t* qa, const double2* ca, const int64_t* na_dev,
                           int64_t na_max, const int64_t* qf, const double2* cf, const int64_t* nf_dev,
                           int64_t nf_max, const double* scale, void* out, PrunedFormat fmt, cudaStream_t st);

// X[o] = sum_{j < M} s[j] exp(-2 pi i j bins[o] / M) for o < n_out (host count),
// s in the layout fmt (double-float or FP32 arithmetic accordingly; the sum
// over the blocks in FP64).  X: device double-float complex [n_out].
// Deterministic (fixed summation order).  Asynchronous on st.
ss_status pruned_forward(const TwoLevelTable& T, const void* s, PrunedFormat fmt, const int64_t* bins, int64_t n_out,
                         float4* X, cudaStream_t st);

}  // namespace ss
