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
#include "df.cuh"
#include "fft_df.cuh"

namespace ss {
namespace {

struct C4 {
  DF re, im;
};

__device__ __forceinline__ C4 ld(const float4 v) { return C4{DF{v.x, v.y}, DF{v.z, v.w}}; }
__device__ __forceinline__ float4 st4(const C4 c) { return make_float4(c.re.hi, c.re.lo, c.im.hi, c.im.lo); }
__device__ __forceinline__ C4 cadd(const C4 a, const C4 b) { return C4{df_add(a.re, b.re), df_add(a.im, b.im)}; }
__device__ __forceinline__ C4 csub(const C4 a, const C4 b) { return C4{df_sub(a.re, b.re), df_sub(a.im, b.im)}; }
// a * w
__device__ __forceinline__ C4 cmul(const C4 a, const C4 w) {
  return C4{df_dot2(a.re, w.re, df_neg(a.im), w.im), df_dot2(a.re, w.im, a.im, w.re)};
}
// a * (sign i)
template <int SIGN>
__device__ __forceinline__ C4 mul_si(const C4 a) {
  return SIGN > 0 ? C4{df_neg(a.im), a.re} : C4{a.im, df_neg(a.re)};
}

// exp(sign 2 pi i m / M) from the table of exp(+2 pi i r / M)
template <int SIGN>
__device__ __forceinline__ C4 twiddle(const float4* __restrict__ tab, int64_t m) {
  const float4 e = __ldg(tab + m);
  return SIGN > 0 ? C4{DF{e.x, e.y}, DF{e.z, e.w}} : C4{DF{e.x, e.y}, DF{-e.z, -e.w}};
}

template <int SIGN>
__device__ __forceinline__ void dft4(C4& v0, C4& v1, C4& v2, C4& v3) {
  const C4 t0 = cadd(v0, v2), t1 = csub(v0, v2), t2 = cadd(v1, v3), t3 = mul_si<SIGN>(csub(v1, v3));
  v0 = cadd(t0, t2);
  v2 = csub(t0, t2);
  v1 = cadd(t1, t3);
  v3 = csub(t1, t3);
}

// R-point DFT in place; cs[m - 1] = exp(2 pi i m / R) (unconjugated), m <= (R - 1) / 2,
// and for R = 8 cs[0] = exp(2 pi i / 8).
template <int R, int SIGN>
__device__ __forceinline__ void dft(C4 (&v)[R], const C4* cs) {
  if constexpr (R == 2) {
    const C4 a = v[0];
    v[0] = cadd(a, v[1]);
    v[1] = csub(a, v[1]);
  } else if constexpr (R == 4) {
    dft4<SIGN>(v[0], v[1], v[2], v[3]);
  } else if constexpr (R == 8) {
    C4 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6], o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    dft4<SIGN>(e0, e1, e2, e3);
    dft4<SIGN>(o0, o1, o2, o3);
    // w8 = c (1 + sign i), w8^2 = sign i, w8^3 = c (-1 + sign i), c = cos(pi / 4)
    const DF c = cs[0].re;
    const DF sg1 = SIGN > 0 ? o1.re : df_neg(o1.re);   // sign * x of o1
    const DF sh1 = SIGN > 0 ? o1.im : df_neg(o1.im);   // sign * y of o1
    o1 = C4{df_mul(c, df_sub(o1.re, sh1)), df_mul(c, df_add(o1.im, sg1))};
    o2 = mul_si<SIGN>(o2);
    const DF sg3 = SIGN > 0 ? o3.re : df_neg(o3.re);
    const DF sh3 = SIGN > 0 ? o3.im : df_neg(o3.im);
    o3 = C4{df_mul(c, df_neg(df_add(o3.re, sh3))), df_mul(c, df_sub(sg3, o3.im))};
    v[0] = cadd(e0, o0);
    v[4] = csub(e0, o0);
    v[1] = cadd(e1, o1);
    v[5] = csub(e1, o1);
    v[2] = cadd(e2, o2);
    v[6] = csub(e2, o2);
    v[3] = cadd(e3, o3);
    v[7] = csub(e3, o3);
  } else {
    constexpr int H = (R - 1) / 2;
    C4 a[H], b[H];
#pragma unroll
    for (int r = 1; r <= H; ++r) {
      a[r - 1] = cadd(v[r], v[R - r]);
      b[r - 1] = csub(v[r], v[R - r]);
    }
    const C4 v0 = v[0];
    C4 y0 = v0;
#pragma unroll
    for (int r = 0; r < H; ++r) y0 = cadd(y0, a[r]);
#pragma unroll
    for (int s = 1; s <= H; ++s) {
      C4 A = v0, B{DF{0.f, 0.f}, DF{0.f, 0.f}};
#pragma unroll
      for (int r = 1; r <= H; ++r) {
        const int m = (r * s) % R;
        // cos and sin of 2 pi m / R from the entry of min(m, R - m)
        const int mm = m <= H ? m : R - m;
        const DF cm = cs[mm - 1].re;
        const DF sm = m <= H ? cs[mm - 1].im : df_neg(cs[mm - 1].im);
        df_fma(A.re, cm, a[r - 1].re);
        df_fma(A.im, cm, a[r - 1].im);
        df_fma(B.re, sm, b[r - 1].re);
        df_fma(B.im, sm, b[r - 1].im);
      }
      const C4 iB = mul_si<SIGN>(B);
      v[s] = cadd(A, iB);
      v[R - s] = csub(A, iB);
    }
    v[0] = y0;
  }
}

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

DfRadices radices(int L) {
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
  k_fft_df<SIGN, SECOND><<<SECOND ? F.L1 : F.L2, threads, sm, st>>>(in, out, tab, F.M, F.L1, F.L2, rad);
  SS_LAUNCH_CHECK();
  return SS_OK;
}

}  // namespace

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
  F.rad1 = radices(F.L1);
  F.rad2 = radices(F.L2);
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
