// Packed frequency keys and the open-addressing frequency -> index table.
#pragma once

#include "ss_internal.cuh"

namespace ss {

// Parameters of the packed layout, passed by value to kernels.
struct KeyParams {
  int d, b, fb, fpw, WT;
  int64_t bias_val;                 // 2^(b-1)
  uint64_t fieldmask;               // 2^b - 1
  uint64_t bias[kMaxWords];         // packed bias of every word
  uint64_t lin_bias;                // key_lin of the packed bias (the linear form of frequency 0)
};

inline KeyParams make_key_params(const KeyLayout& L) {
  KeyParams P{};
  P.d = L.d;
  P.b = L.b;
  P.fb = L.fb;
  P.fpw = L.fpw;
  P.WT = L.WT;
  P.bias_val = 1ll << (L.b - 1);
  P.fieldmask = (L.b >= 64) ? ~0ull : ((1ull << L.b) - 1);
  for (int w = 0; w < kMaxWords; ++w) P.bias[w] = 0;
  for (int c = 0; c < L.d; ++c) {
    const int w = c / L.fpw, sh = 64 - L.fb * (c % L.fpw + 1);
    P.bias[w] |= (uint64_t)P.bias_val << sh;
  }
  P.lin_bias = 0;
  for (int w = 0; w < L.WT; ++w) P.lin_bias += key_lin_coef(w) * P.bias[w];
  return P;
}

// Pack k (d int32 coordinates).  Returns false when a coordinate is outside
// the layout's range (such a frequency cannot be in the set).
template <int WT>
__device__ __forceinline__ bool pack_key(const int32_t* k, const KeyParams& P, uint64_t* out) {
#pragma unroll
  for (int w = 0; w < WT; ++w) out[w] = 0;
  bool ok = true;
  for (int c = 0; c < P.d; ++c) {
    const int64_t v = (int64_t)k[c] + P.bias_val;
    ok &= (v >= 0) && (v <= (int64_t)P.fieldmask);
    const int w = c / P.fpw, sh = 64 - P.fb * (c % P.fpw + 1);
    // runtime word index into a register array: select with a small loop
#pragma unroll
    for (int q = 0; q < WT; ++q)
      if (q == w) out[q] |= ((uint64_t)v & P.fieldmask) << sh;
  }
  return ok;
}

__device__ __forceinline__ int32_t unpack_coord(const uint64_t* key, const KeyParams& P, int c) {
  const int w = c / P.fpw, sh = 64 - P.fb * (c % P.fpw + 1);
  return (int32_t)((int64_t)((key[w] >> sh) & P.fieldmask) - P.bias_val);
}

// a + b - bias, field by field (valid when every resulting field is in range).
template <int WT>
__device__ __forceinline__ void add_keys(const uint64_t* a, const uint64_t* b, const KeyParams& P,
                                         uint64_t* out) {
#pragma unroll
  for (int w = 0; w < WT; ++w) out[w] = a[w] + b[w] - P.bias[w];
}

template <int WT>
__device__ __forceinline__ void load_key(const uint64_t* __restrict__ base, int64_t idx, uint64_t* out) {
#pragma unroll
  for (int w = 0; w < WT; ++w) out[w] = __ldg(base + idx * WT + w);
}

template <int WT>
__device__ __forceinline__ int64_t key_norm(const uint64_t* key, const KeyParams& P) {
  int64_t s = 0;
#pragma unroll
  for (int w = 0; w < WT; ++w) {
    const uint64_t x = key[w];
    for (int f = 0; f < P.fpw; ++f) {
      const int c = w * P.fpw + f;
      if (c >= P.d) break;
      const int sh = 64 - P.fb * (f + 1);
      const int64_t v = (int64_t)((x >> sh) & P.fieldmask) - P.bias_val;
      s += v * v;
    }
  }
  return s;
}

// Slot words: kEmpty, or [63] pending flag | [62:32] fingerprint | [31:0]
// canonical index (final) or candidate id (pending).  The fingerprint is 31
// bits of the key hash disjoint from the bits that pick the slot, so a probe
// reads a stored key only when the fingerprints agree.
__device__ __forceinline__ uint64_t slot_fp(uint64_t h) { return (h >> 33) & 0x7fffffffull; }
__device__ __forceinline__ uint64_t slot_word(uint64_t fp, uint64_t low) { return (fp << 32) | low; }
__device__ __forceinline__ uint64_t word_fp(uint64_t v) { return (v >> 32) & 0x7fffffffull; }
__device__ __forceinline__ uint64_t word_low(uint64_t v) { return v & 0xffffffffull; }

// Lookup of a finalised key given its hash and linear form: the canonical
// index, or -1.  A slot whose fingerprint agrees is confirmed by eq(o), the
// exact word-by-word comparison with stored key o; when hl (the linear form of
// every stored key) is given, the linear forms are compared first.
template <typename Eq>
__device__ __forceinline__ int64_t table_find_h(const uint64_t* __restrict__ table, uint64_t capmask, uint64_t hh,
                                                const uint64_t* __restrict__ hl, uint64_t lin, Eq eq) {
  const uint64_t fp = slot_fp(hh);
  uint64_t h = hh & capmask;
  for (uint64_t probe = 0; probe <= capmask; ++probe) {
    const uint64_t v = __ldg(table + h);
    if (v == kEmpty) return -1;
    if (word_fp(v) == fp) {
      const int64_t o = (int64_t)word_low(v);
      if ((!hl || __ldg(hl + o) == lin) && eq(o)) return o;
    }
    h = (h + 1) & capmask;
  }
  return -1;
}

// Stored key o equals a + b - bias (packed sum of a frequency and a step), or
// equals m * bias - a (m = 2: the negated frequency) when b is null; the rows
// are read two words at a time when WT is even (16-byte aligned rows).
template <int WT>
__device__ __forceinline__ bool key_eq_sum(const uint64_t* __restrict__ so, const uint64_t* __restrict__ a,
                                           const uint64_t* __restrict__ b, const KeyParams& P) {
  bool e = true;
  if constexpr (WT % 2 == 0) {
#pragma unroll
    for (int w = 0; w < WT; w += 2) {
      const ulonglong2 x = __ldg(reinterpret_cast<const ulonglong2*>(so + w));
      const ulonglong2 y = __ldg(reinterpret_cast<const ulonglong2*>(a + w));
      if (b) {
        const ulonglong2 z = __ldg(reinterpret_cast<const ulonglong2*>(b + w));
        e &= (x.x == y.x + z.x - P.bias[w]) & (x.y == y.y + z.y - P.bias[w + 1]);
      } else {
        e &= (x.x == 2 * P.bias[w] - y.x) & (x.y == 2 * P.bias[w + 1] - y.y);
      }
    }
  } else {
#pragma unroll
    for (int w = 0; w < WT; ++w) {
      const uint64_t x = __ldg(so + w), y = __ldg(a + w);
      e &= b ? (x == y + __ldg(b + w) - P.bias[w]) : (x == 2 * P.bias[w] - y);
    }
  }
  return e;
}

#define SS_DISPATCH_WT(wt, ...)                              \
  switch (wt) {                                              \
    case 1: { constexpr int WT = 1; __VA_ARGS__; } break;    \
    case 2: { constexpr int WT = 2; __VA_ARGS__; } break;    \
    case 4: { constexpr int WT = 4; __VA_ARGS__; } break;    \
    case 8: { constexpr int WT = 8; __VA_ARGS__; } break;    \
    case 12: { constexpr int WT = 12; __VA_ARGS__; } break;  \
    case 16: { constexpr int WT = 16; __VA_ARGS__; } break;  \
    default: SS_FAIL(SS_ERR_KEY_RANGE, "unsupported key width %d", (int)(wt)); \
  }

}  // namespace ss
