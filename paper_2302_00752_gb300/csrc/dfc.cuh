// Complex double-float values and the small DFT kernels shared by the
// double-float transforms (fft_df.cu: full length-M transform; fft_pruned.cu:
// sparse-input evaluation and pruned-output transform).  A value is
// (re, im) with each part an unevaluated float pair (df.cuh).
#pragma once

#include "df.cuh"

namespace ss {
namespace dfc {

struct C4 {
  DF re, im;
};

__device__ __forceinline__ C4 ld(const float4 v) { return C4{DF{v.x, v.y}, DF{v.z, v.w}}; }
__device__ __forceinline__ float4 st4(const C4 c) { return make_float4(c.re.hi, c.re.lo, c.im.hi, c.im.lo); }
__device__ __forceinline__ C4 cadd(const C4 a, const C4 b) { return C4{df_add(a.re, b.re), df_add(a.im, b.im)}; }
__device__ __forceinline__ C4 csub(const C4 a, const C4 b) { return C4{df_sub(a.re, b.re), df_sub(a.im, b.im)}; }
// the same without renormalisation (inner butterfly levels; see df_add_nr)
__device__ __forceinline__ C4 cadd_nr(const C4 a, const C4 b) {
  return C4{df_add_nr(a.re, b.re), df_add_nr(a.im, b.im)};
}
__device__ __forceinline__ C4 csub_nr(const C4 a, const C4 b) {
  return C4{df_sub_nr(a.re, b.re), df_sub_nr(a.im, b.im)};
}
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

// 4-point DFT; the first level's sums are left unnormalised, the outputs are
// renormalised unless LAZY (then the caller's next level renormalises).
template <int SIGN, bool LAZY = false>
__device__ __forceinline__ void dft4(C4& v0, C4& v1, C4& v2, C4& v3) {
  const C4 t0 = cadd_nr(v0, v2), t1 = csub_nr(v0, v2), t2 = cadd_nr(v1, v3), t3 = mul_si<SIGN>(csub_nr(v1, v3));
  if (LAZY) {
    v0 = cadd_nr(t0, t2);
    v2 = csub_nr(t0, t2);
    v1 = cadd_nr(t1, t3);
    v3 = csub_nr(t1, t3);
  } else {
    v0 = cadd(t0, t2);
    v2 = csub(t0, t2);
    v1 = cadd(t1, t3);
    v3 = csub(t1, t3);
  }
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
    dft4<SIGN, true>(e0, e1, e2, e3);
    dft4<SIGN, true>(o0, o1, o2, o3);
    // w8 = c (1 + sign i), w8^2 = sign i, w8^3 = c (-1 + sign i), c = cos(pi / 4)
    const DF c = cs[0].re;
    const DF sg1 = SIGN > 0 ? o1.re : df_neg(o1.re);   // sign * x of o1
    const DF sh1 = SIGN > 0 ? o1.im : df_neg(o1.im);   // sign * y of o1
    o1 = C4{df_mul(c, df_sub_nr(o1.re, sh1)), df_mul(c, df_add_nr(o1.im, sg1))};
    o2 = mul_si<SIGN>(o2);
    const DF sg3 = SIGN > 0 ? o3.re : df_neg(o3.re);
    const DF sh3 = SIGN > 0 ? o3.im : df_neg(o3.im);
    o3 = C4{df_mul(c, df_neg(df_add_nr(o3.re, sh3))), df_mul(c, df_sub_nr(sg3, o3.im))};
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
      a[r - 1] = cadd_nr(v[r], v[R - r]);
      b[r - 1] = csub_nr(v[r], v[R - r]);
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


}  // namespace dfc
}  // namespace ss
