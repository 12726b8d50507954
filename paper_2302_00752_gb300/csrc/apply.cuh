// Row kernels of the finite Galerkin operator (eq. FiniteGalerkinOperator),
// shared by the standalone apply and the persistent solver.
//
// For a row k and a stored neighbour l = k - p_j:
//     4 pi^2 (k.l) a_hat_j u_l = 2 pi^2 (|k|^2 + |l|^2 - |p_j|^2) a_hat_j u_l,
// the integer (|k|^2 + |l|^2 - |p_j|^2) = 2 k.l is exact in int32 (|k|^2 < 2^29
// is checked when the set is built) and ca_j = 2 pi^2 a_hat_j is tabulated.
//
// Gather source ("records"): FP32  float4 (re, im, |l|^2 as int bits, 0);
//                            FP64  two double2 (re, im), (|l|^2 as int64 bits, 0),
// so one 16- or 32-byte sector brings both the value and the norm.
#pragma once

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
  int colbits;
  uint32_t colmask;
};

// Accumulate row `row` (lane of slice s) of L u in FP64.
template <bool CG = false>
__device__ __forceinline__ double2 row_apply64(const OpView& op, int64_t s, int lane, int32_t nk,
                                               const double2* __restrict__ rec, const double2* ca,
                                               const int32_t* pn) {
  const int32_t w0 = __ldg(op.woff + s), w1 = __ldg(op.woff + s + 1);
  const uint32_t* e = op.ent + (int64_t)w0 * kSlice + lane;
  double ar = 0.0, ai = 0.0;
  int t = 0;
  const int w = w1 - w0;
  for (; t + 2 <= w; t += 2) {
    const uint32_t e0 = __ldg(e + (int64_t)t * kSlice), e1 = __ldg(e + (int64_t)(t + 1) * kSlice);
    const uint32_t c0 = e0 & op.colmask, c1 = e1 & op.colmask;
    const int j0 = (int)(e0 >> op.colbits), j1 = (int)(e1 >> op.colbits);
    const double2 v0 = ldv<CG>(rec + 2 * (int64_t)c0), v1 = ldv<CG>(rec + 2 * (int64_t)c1);
    const int32_t n0 = (int32_t)__double_as_longlong(ldv<CG>(rec + 2 * (int64_t)c0 + 1).x);
    const int32_t n1 = (int32_t)__double_as_longlong(ldv<CG>(rec + 2 * (int64_t)c1 + 1).x);
    const double s0 = (double)(nk + n0 - pn[j0]), s1 = (double)(nk + n1 - pn[j1]);
    const double2 a0 = ca[j0], a1 = ca[j1];
    const double tr0 = s0 * a0.x, ti0 = s0 * a0.y, tr1 = s1 * a1.x, ti1 = s1 * a1.y;
    ar = fma(tr0, v0.x, ar); ar = fma(-ti0, v0.y, ar);
    ai = fma(tr0, v0.y, ai); ai = fma(ti0, v0.x, ai);
    ar = fma(tr1, v1.x, ar); ar = fma(-ti1, v1.y, ar);
    ai = fma(tr1, v1.y, ai); ai = fma(ti1, v1.x, ai);
  }
  if (t < w) {
    const uint32_t e0 = __ldg(e + (int64_t)t * kSlice);
    const uint32_t c0 = e0 & op.colmask;
    const int j0 = (int)(e0 >> op.colbits);
    const double2 v0 = ldv<CG>(rec + 2 * (int64_t)c0);
    const int32_t n0 = (int32_t)__double_as_longlong(ldv<CG>(rec + 2 * (int64_t)c0 + 1).x);
    const double s0 = (double)(nk + n0 - pn[j0]);
    const double2 a0 = ca[j0];
    const double tr0 = s0 * a0.x, ti0 = s0 * a0.y;
    ar = fma(tr0, v0.x, ar); ar = fma(-ti0, v0.y, ar);
    ai = fma(tr0, v0.y, ai); ai = fma(ti0, v0.x, ai);
  }
  return make_double2(ar, ai);
}

// Same in FP32 (FP32 values, FP32 accumulation).
template <bool CG = false>
__device__ __forceinline__ float2 row_apply32(const OpView& op, int64_t s, int lane, int32_t nk,
                                              const float4* __restrict__ rec, const float2* ca,
                                              const int32_t* pn) {
  const int32_t w0 = __ldg(op.woff + s), w1 = __ldg(op.woff + s + 1);
  const uint32_t* e = op.ent + (int64_t)w0 * kSlice + lane;
  float ar = 0.f, ai = 0.f;
  int t = 0;
  const int w = w1 - w0;
  for (; t + 4 <= w; t += 4) {
    uint32_t ee[4];
    float4 v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) ee[q] = __ldg(e + (int64_t)(t + q) * kSlice);
#pragma unroll
    for (int q = 0; q < 4; ++q) v[q] = ldv<CG>(rec + (ee[q] & op.colmask));
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int j = (int)(ee[q] >> op.colbits);
      const float sc = (float)(nk + __float_as_int(v[q].z) - pn[j]);
      const float2 a = ca[j];
      const float tr = sc * a.x, ti = sc * a.y;
      ar = fmaf(tr, v[q].x, ar); ar = fmaf(-ti, v[q].y, ar);
      ai = fmaf(tr, v[q].y, ai); ai = fmaf(ti, v[q].x, ai);
    }
  }
  for (; t < w; ++t) {
    const uint32_t ee = __ldg(e + (int64_t)t * kSlice);
    const float4 v = ldv<CG>(rec + (ee & op.colmask));
    const int j = (int)(ee >> op.colbits);
    const float sc = (float)(nk + __float_as_int(v.z) - pn[j]);
    const float2 a = ca[j];
    const float tr = sc * a.x, ti = sc * a.y;
    ar = fmaf(tr, v.x, ar); ar = fmaf(-ti, v.y, ar);
    ai = fmaf(tr, v.y, ai); ai = fmaf(ti, v.x, ai);
  }
  return make_float2(ar, ai);
}

}  // namespace ss
