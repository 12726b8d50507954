// Double-float arithmetic shared by the lattice sampler and the Monte Carlo
// proxy: FP64-accurate sums of products on the FP32 pipe, which on this part
// issues far more operations per clock than the FP64 pipe.
#pragma once

namespace ss {

// Double-float arithmetic (an unevaluated sum hi + lo of two floats, ~48-bit
// significand) from the error-free transformations TwoSum (Knuth) and the
// FMA-based TwoProd (Ogita, Rump and Oishi, "Accurate sum and dot product",
// 2005).  The _rn intrinsics keep the compiler from contracting or reordering.
struct DF {
  float hi, lo;
};

__device__ __forceinline__ DF df_split(double x) {
  const float h = (float)x;
  return DF{h, (float)(x - (double)h)};
}

// acc += a * b with a, b double-float; the product error and the sum error are
// kept exactly (up to the dropped lo*lo term), then acc is renormalised.
__device__ __forceinline__ void df_fma(DF& acc, const DF a, const DF b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  const float s = __fadd_rn(acc.hi, p);
  const float bb = __fsub_rn(s, acc.hi);
  const float t = __fadd_rn(__fsub_rn(acc.hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  const float lo = __fadd_rn(__fadd_rn(acc.lo, t), e);
  const float hi = __fadd_rn(s, lo);
  acc.lo = __fsub_rn(lo, __fsub_rn(hi, s));
  acc.hi = hi;
}

}  // namespace ss
