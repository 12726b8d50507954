// Double-float complex FFT of a 7-smooth length M on the FP32 pipes.
//
// Four-step split M = L1 L2 (j = j1 L2 + j2, k = k1 + L1 k2):
//   X[k1 + L1 k2] = sum_{j2} w_{L2}^{j2 k2} w_M^{j2 k1} sum_{j1} w_{L1}^{j1 k1} x[j1 L2 + j2],
// w_n = exp(sign 2 pi i / n).  Launch A runs one block per column j2 (length
// L1 transform of the stride-L2 column, then the w_M^{j2 k1} twist, written to
// T[k1 L2 + j2]); launch B one block per row k1 (length L2 transform of the
// contiguous row of T, written to X[k1 + L1 k2]).  Inside a block the length-L
// transform is a self-sorting (Stockham) sequence of radix-R passes in shared
// memory (two buffers): with Ns the product of the radices already applied,
// butterfly j < L/R takes in[j + r L/R], turns input r by w_{Ns R}^{(j mod Ns) r},
// applies the R-point DFT and writes output r to out[(j / Ns) Ns R + j mod Ns + r Ns]
// (the Stockham autosort formulation, e.g. Govindaraju et al., SC 2008).
// Radices 8, 4, 2 use the usual split forms; 3, 5 and 7 the symmetric form
// y_s = v_0 + sum_r cos(2 pi r s / R) (v_r + v_{R-r}) + sign i sin(2 pi r s / R) (v_r - v_{R-r}).
// Every twiddle and constant is an entry of the double-float table
// exp(2 pi i r / M), conjugated for sign = -1; a block stages the L-th roots
// exp(2 pi i m / L) = tab[m M / L] it uses in shared memory.
//
// On this part an FP64 instruction issues at 1/64 of the FP32 rate; a
// double-float operation costs 7 to 19 FP32 instructions, so the transform
// runs several times faster than in FP64 at ~2^-46 relative rounding.
#include "dfc.cuh"
#include "fft_df.cuh"

namespace ss {
namespace {

using namespace dfc;

// tw[m] = exp(2 pi i m / L), m < L, in shared memory.
template <int R, int SIGN>
__device__ __forceinline__ void pass(const float4* __restrict__ a, float4* __restrict__ b, int L, int Ns,
                                     const float4* __restrict__ tw) {
  constexpr int NC = R == 8 ? 1 : (R - 1) / 2;
  C4 cs[NC > 0 ? NC : 1];
#pragma unroll
  for (int m = 0; m < NC; ++m) cs[m] = ld(tw[(L / R) * (m + 1)]);
  const int nb = L / R;
  const int tstride = L / (Ns * R);
  for (int j = threadIdx.x; j < nb; j += blockDim.x) {
    const int k = j % Ns;
    C4 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = ld(a[j + r * nb]);
    if (Ns > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        const C4 w = ld(tw[tstride * (k * r)]);
        v[r] = cmul(v[r], SIGN > 0 ? w : C4{w.re, df_neg(w.im)});
      }
    }
    dft<R, SIGN>(v, cs);
    const int base = (j / Ns) * Ns * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) b[base + r * Ns] = st4(v[r]);
  }
}

// SECOND = false: launch A (block = column j2 < L2, transform length L = L1);
// SECOND = true: launch B (block = row k1 < L1, transform length L = L2).
template <int SIGN, bool SECOND>
__global__ void k_fft_df(const float4* __restrict__ in, float4* __restrict__ out, const float4* __restrict__ tab,
                         int64_t M, int L1, int L2, DfRadices rad) {
  extern __shared__ __align__(16) float4 sbuf[];
  const int L = SECOND ? L2 : L1;
  float4* a = sbuf;
  float4* b = sbuf + L;
  float4* tw = sbuf + 2 * L;
  const int64_t blk = blockIdx.x;
  const int64_t tstep = M / L;
  for (int i = threadIdx.x; i < L; i += blockDim.x) {
    a[i] = SECOND ? in[blk * L2 + i] : in[(int64_t)i * L2 + blk];
    tw[i] = __ldg(tab + tstep * i);
  }
  __syncthreads();
  int Ns = 1;
  for (int p = 0; p < rad.n; ++p) {
    const int R = rad.r[p];
    switch (R) {
      case 8: pass<8, SIGN>(a, b, L, Ns, tw); break;
      case 4: pass<4, SIGN>(a, b, L, Ns, tw); break;
      case 2: pass<2, SIGN>(a, b, L, Ns, tw); break;
      case 5: pass<5, SIGN>(a, b, L, Ns, tw); break;
      case 3: pass<3, SIGN>(a, b, L, Ns, tw); break;
      default: pass<7, SIGN>(a, b, L, Ns, tw); break;
    }
    __syncthreads();
    float4* t = a;
    a = b;
    b = t;
    Ns *= R;
  }
  if (SECOND) {
    for (int i = threadIdx.x; i < L; i += blockDim.x) out[blk + (int64_t)L1 * i] = a[i];
  } else {
    // twist by w_M^{j2 k1} (j2 k1 < M)
    for (int i = threadIdx.x; i < L; i += blockDim.x)
      out[(int64_t)i * L2 + blk] = st4(cmul(ld(a[i]), twiddle<SIGN>(tab, blk * (int64_t)i)));
  }
}

int min_radix(const DfRadices& d) {
  int m = 8;
  for (int p = 0; p < d.n; ++p) m = d.r[p] < m ? d.r[p] : m;
  return m;
}

template <int SIGN, bool SECOND>
ss_status launch(const DfFftPlan& F, const float4* tab, const float4* in, float4* out, cudaStream_t st) {
  const int L = SECOND ? F.L2 : F.L1;
  const DfRadices& rad = SECOND ? F.rad2 : F.rad1;
  const size_t sm = 3 * (size_t)L * sizeof(float4);
  int threads = (L / min_radix(rad) + 31) / 32 * 32;
  threads = threads < 64 ? 64 : (threads > 512 ? 512 : threads);
  if (sm > 48 * 1024)
    SS_CUDA(cudaFuncSetAttribute(k_fft_df<SIGN, SECOND>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  ProfScope prof_("k_fft_df", st, true);
  k_fft_df<SIGN, SECOND><<<SECOND ? F.L1 : F.L2, threads, sm, st>>>(in, out, tab, F.M, F.L1, F.L2, rad);
  SS_LAUNCH_CHECK();
  return SS_OK;
}

}  // namespace

DfRadices df_radices(int L) {
  DfRadices d;
  // odd radices first: the first pass (Ns = 1) writes at stride R, free of
  // shared-memory bank conflicts for odd R
  for (int R : {7, 5, 3, 8, 4, 2})
    while (L > 1 && L % R == 0 && d.n < kDfFftMaxPasses) {
      d.r[d.n++] = R;
      L /= R;
    }
  if (L != 1) d.n = -1;
  return d;
}

bool df_fft_plan(int64_t M, DfFftPlan* out) {
  if (M < 1) return false;
  int64_t best = -1;
  for (int64_t l1 = 1; l1 <= kDfFftMaxL && l1 <= M; ++l1) {
    if (M % l1 || M / l1 > kDfFftMaxL) continue;
    const int64_t l2 = M / l1;
    if (best < 0 || (l1 > l2 ? l1 - l2 : l2 - l1) < (best > M / best ? best - M / best : M / best - best)) best = l1;
  }
  if (best < 0) return false;
  DfFftPlan F;
  F.M = M;
  F.L1 = (int)best;
  F.L2 = (int)(M / best);
  F.rad1 = df_radices(F.L1);
  F.rad2 = df_radices(F.L2);
  if (F.rad1.n < 0 || F.rad2.n < 0) return false;
  *out = F;
  return true;
}

ss_status df_fft(const DfFftPlan& F, const float4* tab, const float4* in, float4* tmp, float4* out, int sign,
                 cudaStream_t st) {
  if (sign > 0) {
    SS_TRY((launch<1, false>(F, tab, in, tmp, st)));
    return launch<1, true>(F, tab, tmp, out, st);
  }
  SS_TRY((launch<-1, false>(F, tab, in, tmp, st)));
  return launch<-1, true>(F, tab, tmp, out, st);
}

}  // namespace ss
