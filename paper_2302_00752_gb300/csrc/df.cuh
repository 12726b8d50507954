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

// a + b (TwoSum of the high parts, the low parts added, renormalised).
__device__ __forceinline__ DF df_add(const DF a, const DF b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bb = __fsub_rn(s, a.hi);
  const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  const float lo = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  const float hi = __fadd_rn(s, lo);
  return DF{hi, __fsub_rn(lo, __fsub_rn(hi, s))};
}

// a + b without the final renormalisation: the high part is the rounded sum
// of the high parts, the low part their exact rounding error plus the low
// parts, so hi + lo carries the same ~48-bit accuracy while |lo| may exceed
// half an ulp of hi by a few ulps.  Such a pair is a valid input to df_add,
// df_mul, df_dot2 and df_fma (their TwoSum and TwoProd act on the high parts
// exactly; the low parts enter as FP32 corrections), which renormalise.  Used
// for the inner levels of the small DFT kernels.
__device__ __forceinline__ DF df_add_nr(const DF a, const DF b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bb = __fsub_rn(s, a.hi);
  const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  return DF{s, __fadd_rn(e, __fadd_rn(a.lo, b.lo))};
}

__device__ __forceinline__ DF df_neg(const DF a) { return DF{-a.hi, -a.lo}; }

__device__ __forceinline__ DF df_sub_nr(const DF a, const DF b) { return df_add_nr(a, DF{-b.hi, -b.lo}); }

__device__ __forceinline__ DF df_sub(const DF a, const DF b) { return df_add(a, df_neg(b)); }

// a * b (TwoProd of the high parts plus the cross terms, renormalised).
__device__ __forceinline__ DF df_mul(const DF a, const DF b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  const float hi = __fadd_rn(p, e);
  return DF{hi, __fsub_rn(e, __fsub_rn(hi, p))};
}

// a1 b1 + a2 b2: both TwoProds, one TwoSum of the products, the errors added.
__device__ __forceinline__ DF df_dot2(const DF a1, const DF b1, const DF a2, const DF b2) {
  const float p1 = __fmul_rn(a1.hi, b1.hi);
  float e1 = __fmaf_rn(a1.hi, b1.hi, -p1);
  e1 = __fmaf_rn(a1.hi, b1.lo, e1);
  e1 = __fmaf_rn(a1.lo, b1.hi, e1);
  const float p2 = __fmul_rn(a2.hi, b2.hi);
  float e2 = __fmaf_rn(a2.hi, b2.hi, -p2);
  e2 = __fmaf_rn(a2.hi, b2.lo, e2);
  e2 = __fmaf_rn(a2.lo, b2.hi, e2);
  const float s = __fadd_rn(p1, p2);
  const float bb = __fsub_rn(s, p1);
  const float t = __fadd_rn(__fsub_rn(p1, __fsub_rn(s, bb)), __fsub_rn(p2, bb));
  const float lo = __fadd_rn(t, __fadd_rn(e1, e2));
  const float hi = __fadd_rn(s, lo);
  return DF{hi, __fsub_rn(lo, __fsub_rn(hi, s))};
}

__device__ __forceinline__ double df_to_double(const DF a) { return (double)a.hi + (double)a.lo; }

// Sum over the warp (fixed butterfly; every lane gets the result).
__device__ __forceinline__ DF df_warp_sum(DF v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
    v = df_add(v, DF{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)});
  return v;
}

// Complex double-float values as float4 (re.hi, re.lo, im.hi, im.lo).
__device__ __forceinline__ DF re_of(const float4 a) { return DF{a.x, a.y}; }
__device__ __forceinline__ DF im_of(const float4 a) { return DF{a.z, a.w}; }
__device__ __forceinline__ float4 cdf(const DF re, const DF im) { return make_float4(re.hi, re.lo, im.hi, im.lo); }

}  // namespace ss
