// Complex length-M DFT in double-float arithmetic (FP32 pipes) for the FP64
// coefficient recovery (Section "Previous results on SFTs": one length-M 1D
// FFT of the lattice samples).  Values are float4 (re.hi, re.lo, im.hi, im.lo).
#pragma once

#include "ss_internal.cuh"

namespace ss {

constexpr int kDfFftMaxL = 4096;     // longest factor transformed in one block
constexpr int kDfFftMaxPasses = 16;

struct DfRadices {
  int n = 0;
  int r[kDfFftMaxPasses] = {};
};

// M = L1 L2 with L1, L2 <= kDfFftMaxL and every prime factor in {2, 3, 5, 7}.
struct DfFftPlan {
  int64_t M = 0;
  int L1 = 1, L2 = 1;
  DfRadices rad1, rad2;
};

// Radices of a self-sorting transform of length L (odd radices first, then
// 8, 4, 2); n = -1 when L has a prime factor above 7.
DfRadices df_radices(int L);

// False when M has a prime factor above 7 or no factor pair fits.
bool df_fft_plan(int64_t M, DfFftPlan* out);

// out[k] = sum_j in[j] exp(sign 2 pi i j k / M) (no scaling), sign = +1 or -1;
// tab[r] = exp(2 pi i r / M) for r < M in double-float form.  tmp holds M
// values; out may alias in.  Two launches on st.
ss_status df_fft(const DfFftPlan& F, const float4* tab, const float4* in, float4* tmp, float4* out, int sign,
                 cudaStream_t st);

}  // namespace ss
