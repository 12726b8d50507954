// Row kernels of the finite Galerkin operator (eq. FiniteGalerkinOperator),
// shared by the standalone apply and the persistent solver.
//
// For a row k and a stored neighbour l = k - p_j:
//     4 pi^2 (k.l) a_hat_j u_l = 2 pi^2 (|k|^2 + |l|^2 - |p_j|^2) a_hat_j u_l,
// the integer (|k|^2 + |l|^2 - |p_j|^2) = 2 k.l is formed exactly in int64 for
// the FP64 operator, which reads the product with ca_j = 2 pi^2 a_hat_j,
// precomputed per entry, beside the index stream.  The FP32 operator forms
// the coefficient on the fly from the gathered norm word (FP32 arithmetic is
// cheap): exact in int32 when every |k|^2 < 2^29, else in FP32 (norm_word).
//
// Gather source ("records"): FP32  float4 (re, im, norm word of |l|^2, 0);
//                            FP64  two double2 (re, im), (|l|^2 as int64 bits, 0),
// so one 16- or 32-byte sector brings both the value and the norm.
#pragma once

#include "df.cuh"
#include "ss_internal.cuh"

namespace ss {

// Loads of gather data: CG = true reads through L2 only (data written by other
// blocks of a persistent kernel), false uses the read-only path.
template <bool CG, typename T>
__device__ __forceinline__ T ldv(const T* p) {
  if constexpr (CG) return __ldcg(p);
  else return __ldg(p);
}

struct OpView {
  const int32_t* woff;     // slice offsets in units of 32 entries
  const uint32_t* ent;     // col | (j << colbits)
  const double2* ecoef;    // FP64 coefficient of every entry (realc: one double per entry, same index)
  const float4* ecoefdf;   // the same as double-float (re.hi, re.lo, im.hi, im.lo), or null
  int colbits;
  uint32_t colmask;
  bool conj = false;       // half system: entry bit 31 set = the neighbour's value is conjugated
  uint32_t jmask = 0xffffffffu;   // step index = (entry >> colbits) & jmask
  bool realc = false;      // every entry coefficient has imaginary part exactly 0 (real a_hat)
};

// Imaginary part of a gathered value, negated (the value conjugated) when the
// table is a half-system table and the entry's bit 31 is set: a sign flip on
// the integer pipe.
__device__ __forceinline__ double conj_if(double y, bool conj, uint32_t ent) {
  const unsigned long long m = conj ? (unsigned long long)(ent >> 31) << 63 : 0ull;
  return __longlong_as_double(__double_as_longlong(y) ^ (long long)m);
}

__device__ __forceinline__ float conj_if(float y, bool conj, uint32_t ent) {
  const uint32_t m = conj ? (ent & 0x80000000u) : 0u;
  return __uint_as_float(__float_as_uint(y) ^ m);
}

// Accumulate row `row` (lane of slice s) of L u in FP64 from the stored entry
// coefficients: four FP64 FMAs per nonzero, two when the coefficients are real
// (REAL: their imaginary parts are exactly 0, so the two dropped products add
// exact zeros).  GB300 issues one FP64 FMA per SM clock, so the FP64 operator
// counts its FP64 instructions.
template <bool CG, bool REAL>
__device__ __forceinline__ double2 row_apply64_t(const OpView& op, int64_t s, int lane,
                                                 const double2* __restrict__ rec) {
  const int32_t w0 = __ldg(op.woff + s), w1 = __ldg(op.woff + s + 1);
  const int64_t base = (int64_t)w0 * kSlice + lane;
  const uint32_t* e = op.ent + base;
  const double2* cf = op.ecoef + base;
  const double* cfr = reinterpret_cast<const double*>(op.ecoef) + base;   // real coefficients
  double ar = 0.0, ai = 0.0;
  int t = 0;
  const int w = w1 - w0;
  for (; t + 4 <= w; t += 4) {
    uint32_t ee[4];
    double2 c[4], v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      ee[q] = __ldg(e + (int64_t)(t + q) * kSlice);
      if constexpr (REAL) c[q].x = __ldg(cfr + (int64_t)(t + q) * kSlice);
      else c[q] = __ldg(cf + (int64_t)(t + q) * kSlice);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      v[q] = ldv<CG>(rec + (ee[q] & op.colmask));
      v[q].y = conj_if(v[q].y, op.conj, ee[q]);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if constexpr (REAL) {
        ar = fma(c[q].x, v[q].x, ar);
        ai = fma(c[q].x, v[q].y, ai);
      } else {
        ar = fma(c[q].x, v[q].x, ar); ar = fma(-c[q].y, v[q].y, ar);
        ai = fma(c[q].x, v[q].y, ai); ai = fma(c[q].y, v[q].x, ai);
      }
    }
  }
  for (; t < w; ++t) {
    const uint32_t ee = __ldg(e + (int64_t)t * kSlice);
    double2 v = ldv<CG>(rec + (ee & op.colmask));
    v.y = conj_if(v.y, op.conj, ee);
    if constexpr (REAL) {
      const double c = __ldg(cfr + (int64_t)t * kSlice);
      ar = fma(c, v.x, ar);
      ai = fma(c, v.y, ai);
    } else {
      const double2 c = __ldg(cf + (int64_t)t * kSlice);
      ar = fma(c.x, v.x, ar); ar = fma(-c.y, v.y, ar);
      ai = fma(c.x, v.y, ai); ai = fma(c.y, v.x, ai);
    }
  }
  return make_double2(ar, ai);
}

template <bool CG = false>
__device__ __forceinline__ double2 row_apply64(const OpView& op, int64_t s, int lane,
                                               const double2* __restrict__ rec) {
  return op.realc ? row_apply64_t<CG, true>(op, s, lane, rec) : row_apply64_t<CG, false>(op, s, lane, rec);
}

// Same in double-float (DF64 mode): the FP64 entry coefficient and u_l as
// unevaluated float pairs, four double-float multiply-adds per nonzero on the
// FP32 pipe (about 2^-48 relative per operation).  rec: float4 per column.
template <bool CG, bool REAL>
__device__ __forceinline__ float4 row_applydf_t(const OpView& op, int64_t s, int lane,
                                                const float4* __restrict__ rec) {
  const int32_t w0 = __ldg(op.woff + s), w1 = __ldg(op.woff + s + 1);
  const int64_t base = (int64_t)w0 * kSlice + lane;
  const uint32_t* e = op.ent + base;
  const float4* cf = op.ecoefdf + base;
  DF ar{0.f, 0.f}, ai{0.f, 0.f};
  int t = 0;
  const int w = w1 - w0;
  for (; t + 4 <= w; t += 4) {
    uint32_t ee[4];
    float4 c[4], v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      ee[q] = __ldg(e + (int64_t)(t + q) * kSlice);
      if constexpr (REAL) {
        const float2 h = __ldg(reinterpret_cast<const float2*>(cf + (int64_t)(t + q) * kSlice));
        c[q] = make_float4(h.x, h.y, 0.f, 0.f);
      } else {
        c[q] = __ldg(cf + (int64_t)(t + q) * kSlice);
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      v[q] = ldv<CG>(rec + (ee[q] & op.colmask));
      v[q].z = conj_if(v[q].z, op.conj, ee[q]);
      v[q].w = conj_if(v[q].w, op.conj, ee[q]);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      df_fma(ar, re_of(c[q]), re_of(v[q]));
      df_fma(ai, re_of(c[q]), im_of(v[q]));
      if constexpr (!REAL) {
        df_fma(ar, df_neg(im_of(c[q])), im_of(v[q]));
        df_fma(ai, im_of(c[q]), re_of(v[q]));
      }
    }
  }
  for (; t < w; ++t) {
    const uint32_t ee = __ldg(e + (int64_t)t * kSlice);
    float4 v = ldv<CG>(rec + (ee & op.colmask));
    v.z = conj_if(v.z, op.conj, ee);
    v.w = conj_if(v.w, op.conj, ee);
    float4 c;
    if constexpr (REAL) {
      const float2 h = __ldg(reinterpret_cast<const float2*>(cf + (int64_t)t * kSlice));
      c = make_float4(h.x, h.y, 0.f, 0.f);
    } else {
      c = __ldg(cf + (int64_t)t * kSlice);
    }
    df_fma(ar, re_of(c), re_of(v));
    df_fma(ai, re_of(c), im_of(v));
    if constexpr (!REAL) {
      df_fma(ar, df_neg(im_of(c)), im_of(v));
      df_fma(ai, im_of(c), re_of(v));
    }
  }
  return cdf(ar, ai);
}

template <bool CG = false>
__device__ __forceinline__ float4 row_applydf(const OpView& op, int64_t s, int lane, const float4* __restrict__ rec) {
  return op.realc ? row_applydf_t<CG, true>(op, s, lane, rec) : row_applydf_t<CG, false>(op, s, lane, rec);
}

// Same in FP32 (FP32 values, FP32 accumulation).  nk, the records' third
// word and pn are FP32 norm words (norm_word): int32 norms, or FP32 values
// when WIDE.
template <bool WIDE>
__device__ __forceinline__ float entry_scale(int32_t nk, float rec_z, int32_t pnj) {
  if constexpr (WIDE) return (__int_as_float(nk) + rec_z) - __int_as_float(pnj);
  else return (float)(nk + __float_as_int(rec_z) - pnj);
}

// U index words per lane are loaded before their U gathers are issued, so a
// row of width <= U costs one index round trip and one gather round trip.
template <bool CG, bool WIDE, int U>
__device__ __forceinline__ float2 row_apply32_t(const OpView& op, int64_t s, int lane, int32_t nk,
                                                const float4* __restrict__ rec, const float2* ca,
                                                const int32_t* pn) {
  const int32_t w0 = __ldg(op.woff + s), w1 = __ldg(op.woff + s + 1);
  const uint32_t* e = op.ent + (int64_t)w0 * kSlice + lane;
  float ar = 0.f, ai = 0.f;
  const int w = w1 - w0;
  for (int t = 0; t < w; t += U) {
    uint32_t ee[U];
    float4 v[U];
#pragma unroll
    for (int q = 0; q < U; ++q) ee[q] = t + q < w ? __ldg(e + (int64_t)(t + q) * kSlice) : 0u;
#pragma unroll
    for (int q = 0; q < U; ++q) {
      v[q] = t + q < w ? ldv<CG>(rec + (ee[q] & op.colmask)) : make_float4(0.f, 0.f, 0.f, 0.f);
      v[q].y = conj_if(v[q].y, op.conj, ee[q]);
    }
#pragma unroll
    for (int q = 0; q < U; ++q) {
      if (t + q < w) {
        const int j = (int)((ee[q] >> op.colbits) & op.jmask);
        const float sc = entry_scale<WIDE>(nk, v[q].z, pn[j]);
        const float2 a = ca[j];
        const float tr = sc * a.x, ti = sc * a.y;
        ar = fmaf(tr, v[q].x, ar); ar = fmaf(-ti, v[q].y, ar);
        ai = fmaf(tr, v[q].y, ai); ai = fmaf(ti, v[q].x, ai);
      }
    }
  }
  return make_float2(ar, ai);
}

// Standalone FP32 operator on the caller's u: the value u_l and the norm word
// of |l|^2 are two gathers (u from the caller's array, guarded because padding
// entries name column rows_pad, one past any row of u; the norm word from the
// stamp's nw32).  No packing step rewrites u first.
template <bool WIDE, int U>
__device__ __forceinline__ float2 row_apply32_direct(const OpView& op, int64_t s, int lane, int32_t nk, int64_t size,
                                                     const float2* __restrict__ u, const int32_t* __restrict__ nw,
                                                     const float2* __restrict__ ca, const int32_t* __restrict__ pn) {
  const int32_t w0 = __ldg(op.woff + s), w1 = __ldg(op.woff + s + 1);
  const uint32_t* e = op.ent + (int64_t)w0 * kSlice + lane;
  float ar = 0.f, ai = 0.f;
  const int w = w1 - w0;
  for (int t = 0; t < w; t += U) {
    uint32_t ee[U];
    float2 v[U];
    int32_t nl[U];
#pragma unroll
    for (int q = 0; q < U; ++q) ee[q] = t + q < w ? __ldg(e + (int64_t)(t + q) * kSlice) : 0u;
#pragma unroll
    for (int q = 0; q < U; ++q) {
      const uint32_t c = ee[q] & op.colmask;
      const bool ok = t + q < w && (int64_t)c < size;
      v[q] = ok ? __ldg(u + c) : make_float2(0.f, 0.f);
      nl[q] = ok ? __ldg(nw + c) : 0;
    }
#pragma unroll
    for (int q = 0; q < U; ++q) {
      if (t + q < w) {
        const int j = (int)((ee[q] >> op.colbits) & op.jmask);
        const float sc = entry_scale<WIDE>(nk, __int_as_float(nl[q]), __ldg(pn + j));
        const float2 a = __ldg(ca + j);
        const float tr = sc * a.x, ti = sc * a.y;
        ar = fmaf(tr, v[q].x, ar); ar = fmaf(-ti, v[q].y, ar);
        ai = fmaf(tr, v[q].y, ai); ai = fmaf(ti, v[q].x, ai);
      }
    }
  }
  return make_float2(ar, ai);
}

template <bool CG = false, int U = 4>
__device__ __forceinline__ float2 row_apply32(const OpView& op, int64_t s, int lane, int64_t nk, bool wide,
                                              const float4* __restrict__ rec, const float2* ca,
                                              const int32_t* pn) {
  return wide ? row_apply32_t<CG, true, U>(op, s, lane, norm_word(nk, true), rec, ca, pn)
              : row_apply32_t<CG, false, U>(op, s, lane, norm_word(nk, false), rec, ca, pn);
}

}  // namespace ss
