// Coefficient recovery by rank-1 lattice sampling and one length-M FFT
// (Section "Previous results on SFTs": samples of t -> g(t z) on j/M carry the
// coefficient of k in DFT bin k.z mod M when the lattice is reconstructing).
//
// lattice_sample evaluates g(x_j) = sum_t Re(c_t exp(2 pi i (j q_t mod M)/M)),
// q_t = p_t.z mod M, with the integer phase kept exact: each thread owns the
// samples j0 + 256 m (m < kSampPerThread), starts from (j0 q_t) mod M and steps
// by (256 q_t) mod M.  exp(2 pi i r/M) is the product of two table entries,
// exp(2 pi i (r >> bl) 2^bl / M) exp(2 pi i (r & (2^bl - 1)) / M), tabulated
// with sincospi and staged in shared memory when they fit.  In FP64 mode, for M
// up to 2^22, one full table exp(2 pi i r / M) (64 MB, L2-resident) replaces the
// product and the sum runs in double-float arithmetic (pairs of floats with
// error-free transformations, ~2^-48 relative) on the FP32 pipes: a term costs
// one 16-byte gather and ~15 (real) or ~30 (complex) FP32 operations instead of
// FP64 instructions, which GB300 issues at one per SM clock.  The samples are
// real, so the FFT is real-to-complex (bins b > M/2 are conj(X[M-b])).
// With many terms (FP64, M up to 2^25) the samples come instead from one
// complex-to-real inverse FFT of the terms binned by residue: evaluation at
// the nodes of a rank-1 lattice is a length-M inverse DFT.
#include <cufft.h>

#include <cstdlib>

#include <list>
#include <memory>
#include <mutex>

#include "df.cuh"
#include "fft_df.cuh"
#include "fft_pruned.cuh"
#include "lattice.cuh"

namespace ss {
namespace {

constexpr int kSampThreads = 256;
constexpr int kSampPerThread = 8;
constexpr int kTermChunk = 256;
constexpr int64_t kFullTableMax = 1ll << 22;   // FP64 full table up to 64 MB (stays in the 126 MB L2)

template <typename R> struct C2;
template <> struct C2<double> { using T = double2; };
template <> struct C2<float> { using T = float2; };

template <typename R>
__global__ void k_twiddles(int64_t M, int bl, int64_t H, typename C2<R>::T* lo, typename C2<R>::T* hi) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t L = 1ll << bl;
  if (i < L) {
    double s, c;
    sincospi(2.0 * (double)i / (double)M, &s, &c);
    lo[i].x = (R)c;
    lo[i].y = (R)s;
  }
  if (i < H) {
    const int64_t r = (i << bl) % M;
    double s, c;
    sincospi(2.0 * (double)r / (double)M, &s, &c);
    hi[i].x = (R)c;
    hi[i].y = (R)s;
  }
}

// Full double-float table (cos_hi, cos_lo, sin_hi, sin_lo)(2 pi r / M), r < M.
__global__ void k_twiddles_df(int64_t M, float4* tab) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= M) return;
  double s, c;
  sincospi(2.0 * (double)r / (double)M, &s, &c);
  const DF cc = df_split(c), ss = df_split(s);
  tab[r] = make_float4(cc.hi, cc.lo, ss.hi, ss.lo);
}

// Per merged term: W_m = exp(2 pi i (m * step mod M) / M), m < kSampPerThread,
// from the double-float table (the phase steps of one thread's samples).
__global__ void k_term_powers(const int64_t* __restrict__ step, const int64_t* __restrict__ n_terms, int64_t M,
                              const float4* __restrict__ tab, float4* W) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= *n_terms) return;
  const uint64_t st = (uint64_t)step[t];
#pragma unroll
  for (int m = 0; m < kSampPerThread; ++m) W[t * kSampPerThread + m] = tab[((uint64_t)m * st) % (uint64_t)M];
}

// FP32 path: W_m = exp(2 pi i (m * step mod M) / M) in FP32 (from FP64 sincospi).
__global__ void k_term_powers32(const int64_t* __restrict__ step, const int64_t* __restrict__ n_terms, int64_t M,
                                float2* W) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= *n_terms) return;
  const uint64_t st = (uint64_t)step[t];
#pragma unroll
  for (int m = 0; m < kSampPerThread; ++m) {
    double s, c;
    sincospi(2.0 * (double)(((uint64_t)m * st) % (uint64_t)M) / (double)M, &s, &c);
    W[t * kSampPerThread + m] = make_float2((float)c, (float)s);
  }
}

// Three-level FP32 tables: exp(2 pi i r / M) = T2[r >> 2b] T1[(r >> b) & m] T0[r & m]
// with b = kT3Bits, each level tabulated from FP64 sincospi.
constexpr int kT3Bits = 9;
constexpr int kT3Size = 1 << kT3Bits;

__global__ void k_twiddles3(int64_t M, int64_t n2, float2* t0, float2* t1, float2* t2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double s, c;
  if (i < kT3Size) {
    sincospi(2.0 * (double)i / (double)M, &s, &c);
    t0[i] = make_float2((float)c, (float)s);
    sincospi(2.0 * (double)((i << kT3Bits) % M) / (double)M, &s, &c);
    t1[i] = make_float2((float)c, (float)s);
  }
  if (i < n2) {
    sincospi(2.0 * (double)((i << (2 * kT3Bits)) % M) / (double)M, &s, &c);
    t2[i] = make_float2((float)c, (float)s);
  }
}

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// FP32 lattice evaluation: B = c exp(2 pi i r0 / M) from the shared-memory
// tables once per term and thread, then Re(B W_m) per sample (W_m broadcast
// from shared memory): two FP32 FMAs per term-sample.
__global__ void __launch_bounds__(kSampThreads) k_sample32(int64_t M, int64_t n2, const float2* __restrict__ t0g,
                                                           const float2* __restrict__ t1g,
                                                           const float2* __restrict__ t2g,
                                                           const int64_t* __restrict__ q,
                                                           const float2* __restrict__ W,
                                                           const double2* __restrict__ coef,
                                                           const int64_t* __restrict__ n_terms_dev, float* out) {
  extern __shared__ __align__(16) unsigned char smem[];
  float2* s_t0 = reinterpret_cast<float2*>(smem);
  float2* s_t1 = s_t0 + kT3Size;
  float2* s_t2 = s_t1 + kT3Size;
  float2* s_w = s_t2 + n2;
  float2* s_c = s_w + kTermChunk * kSampPerThread;
  uint32_t* s_q = reinterpret_cast<uint32_t*>(s_c + kTermChunk);
  for (int i = threadIdx.x; i < kT3Size; i += blockDim.x) {
    s_t0[i] = t0g[i];
    s_t1[i] = t1g[i];
  }
  for (int64_t i = threadIdx.x; i < n2; i += blockDim.x) s_t2[i] = t2g[i];
  const int64_t n_terms = *n_terms_dev;
  const uint32_t mask = kT3Size - 1;
  const int64_t j0 = (int64_t)blockIdx.x * (kSampThreads * kSampPerThread) + threadIdx.x;
  const uint64_t inv = ~0ull / (uint64_t)M;   // once per thread (Barrett constant of mulmod)
  float acc[kSampPerThread];
#pragma unroll
  for (int m = 0; m < kSampPerThread; ++m) acc[m] = 0.f;
  for (int64_t t0 = 0; t0 < n_terms; t0 += kTermChunk) {
    const int tc = (n_terms - t0 < kTermChunk) ? (int)(n_terms - t0) : kTermChunk;
    __syncthreads();
    for (int i = threadIdx.x; i < tc; i += blockDim.x) {
      s_q[i] = (uint32_t)q[t0 + i];
      const double2 c = coef[t0 + i];
      s_c[i] = make_float2((float)c.x, (float)c.y);
    }
    for (int i = threadIdx.x; i < tc * kSampPerThread; i += blockDim.x) s_w[i] = W[t0 * kSampPerThread + i];
    __syncthreads();
    for (int t = 0; t < tc; ++t) {
      const uint32_t r0 = mulmod((uint64_t)j0, s_q[t], (uint64_t)M, inv);
      const float2 e = cmulf(cmulf(s_t2[r0 >> (2 * kT3Bits)], s_t1[(r0 >> kT3Bits) & mask]), s_t0[r0 & mask]);
      const float2 b = cmulf(s_c[t], e);
      const float2* w = s_w + t * kSampPerThread;
#pragma unroll
      for (int m = 0; m < kSampPerThread; ++m) acc[m] = fmaf(b.x, w[m].x, fmaf(-b.y, w[m].y, acc[m]));
    }
  }
#pragma unroll
  for (int m = 0; m < kSampPerThread; ++m) {
    const int64_t j = j0 + (int64_t)m * kSampThreads;
    if (j < M) out[j] = acc[m];
  }
}

// Lattice evaluation in double-float for the FP64 path.  Thread samples are
// j0 + 256 m; with r0 = j0 q mod M and B = c exp(2 pi i r0 / M) (one table
// gather and one double-float complex product per term and thread), sample m
// adds Re(B W_m): two double-float FMAs per term-sample, no further gathers.
__global__ void __launch_bounds__(kSampThreads) k_sample_df(int64_t M, const float4* __restrict__ tab,
                                                            const int64_t* __restrict__ q,
                                                            const float4* __restrict__ W,
                                                            const double2* __restrict__ coef,
                                                            const int64_t* __restrict__ n_terms_dev, double* out) {
  __shared__ uint32_t s_q[kTermChunk];
  __shared__ float4 s_c[kTermChunk];
  __shared__ float4 s_w[kTermChunk * kSampPerThread];
  // blockIdx.y takes the terms [T y / S, T (y+1) / S) (S = gridDim.y); with
  // S > 1 the block writes its partial sums to out + y M
  const int64_t n_all = *n_terms_dev;
  const int64_t tb = n_all * blockIdx.y / gridDim.y, te = n_all * (blockIdx.y + 1) / gridDim.y;
  out += (int64_t)blockIdx.y * M;
  const int64_t j0 = (int64_t)blockIdx.x * (kSampThreads * kSampPerThread) + threadIdx.x;
  const uint64_t inv = ~0ull / (uint64_t)M;   // once per thread (Barrett constant of mulmod)
  DF acc[kSampPerThread];
#pragma unroll
  for (int m = 0; m < kSampPerThread; ++m) acc[m] = DF{0.f, 0.f};
  for (int64_t t0 = tb; t0 < te; t0 += kTermChunk) {
    const int tc = (te - t0 < kTermChunk) ? (int)(te - t0) : kTermChunk;
    __syncthreads();
    for (int i = threadIdx.x; i < tc; i += blockDim.x) {
      s_q[i] = (uint32_t)q[t0 + i];
      const double2 c = coef[t0 + i];
      const DF cx = df_split(c.x), cy = df_split(c.y);
      s_c[i] = make_float4(cx.hi, cx.lo, cy.hi, cy.lo);
    }
    for (int i = threadIdx.x; i < tc * kSampPerThread; i += blockDim.x) s_w[i] = W[t0 * kSampPerThread + i];
    __syncthreads();
    for (int t = 0; t < tc; ++t) {
      const uint32_t r0 = mulmod((uint64_t)j0, s_q[t], (uint64_t)M, inv);
      const float4 e = __ldg(tab + r0);
      const float4 c = s_c[t];
      // B = c e (double-float complex product)
      DF br{0.f, 0.f}, bi{0.f, 0.f};
      df_fma(br, DF{c.x, c.y}, DF{e.x, e.y});
      df_fma(br, DF{-c.z, -c.w}, DF{e.z, e.w});
      df_fma(bi, DF{c.x, c.y}, DF{e.z, e.w});
      df_fma(bi, DF{c.z, c.w}, DF{e.x, e.y});
      const DF nbi{-bi.hi, -bi.lo};
      const float4* w = s_w + t * kSampPerThread;
#pragma unroll
      for (int m = 0; m < kSampPerThread; ++m) {
        const float4 wm = w[m];
        df_fma(acc[m], br, DF{wm.x, wm.y});    // Re(B W_m) = B.re W.re - B.im W.im
        df_fma(acc[m], nbi, DF{wm.z, wm.w});
      }
    }
  }
#pragma unroll
  for (int m = 0; m < kSampPerThread; ++m) {
    const int64_t j = j0 + (int64_t)m * kSampThreads;
    if (j < M) out[j] = (double)acc[m].hi + (double)acc[m].lo;
  }
}

// out[j] = sum_y part[y][j], y in order.
__global__ void k_sum_splits(const double* __restrict__ part, int n_split, int64_t M, double* __restrict__ out) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= M) return;
  double v = 0.0;
  for (int y = 0; y < n_split; ++y) v += part[(int64_t)y * M + j];
  out[j] = v;
}

// Full table exp(2 pi i r / M), r < M (FP64 path, L2-resident for M <= 4M).
__global__ void k_twiddles_full(int64_t M, double2* tab) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= M) return;
  double s, c;
  sincospi(2.0 * (double)r / (double)M, &s, &c);
  tab[r] = make_double2(c, s);
}

// Terms p and -p of a real sum are one term: Re(c e_{-p}) = Re(conj(c) e_p).
// Each term is mapped to the sign representative of its frequency (first
// nonzero coordinate positive) with c or conj(c); equal representatives are
// merged by their first occurrence ("leader"), which sums its group in index
// order (deterministic).  The zero frequency keeps Re(c).

// One warp per term: sgn[t] = sign of the first nonzero coordinate of p_t
// (0 for p_t = 0), 32 coordinates per step.
__global__ void k_term_signs(const int32_t* __restrict__ freq, int64_t n, int d, int32_t* sgn) {
  const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (t >= n) return;   // warp-uniform
  int s = 0;
  for (int c0 = 0; c0 < d && s == 0; c0 += 32) {
    const int32_t v = c0 + lane < d ? freq[t * d + c0 + lane] : 0;
    const unsigned m = __ballot_sync(0xffffffffu, v != 0);
    if (m) s = __shfl_sync(0xffffffffu, v, __ffs(m) - 1) > 0 ? 1 : -1;
  }
  if (lane == 0) sgn[t] = s;
}

// first[t] = smallest u < t with the same representative sgn p (n if none):
// one block per term t, its warps taking u = w, w + 8, ... in increasing
// order and comparing 32 coordinates per step.
constexpr int kMergeWarps = 8;

__global__ void __launch_bounds__(32 * kMergeWarps) k_merge_first(const int32_t* __restrict__ freq, int64_t n, int d,
                                                                   const int32_t* __restrict__ sgn, int32_t* first) {
  __shared__ int32_t s_min[kMergeWarps];
  const int64_t t = blockIdx.x;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int xt = sgn[t] < 0 ? -1 : 1;
  const int32_t* pt = freq + t * d;
  int32_t best = (int32_t)n;
  for (int64_t u = w; u < t; u += kMergeWarps) {
    const int xu = sgn[u] < 0 ? -1 : 1;
    const int32_t* pu = freq + u * d;
    bool diff = false;
    for (int c = lane; c < d; c += 32) diff |= xu * pu[c] != xt * pt[c];
    if (!__any_sync(0xffffffffu, diff)) {
      best = (int32_t)u;
      break;
    }
  }
  if (lane == 0) s_min[w] = best;
  __syncthreads();
  if (threadIdx.x == 0) {
    int32_t m = (int32_t)n;
    for (int q = 0; q < kMergeWarps; ++q) m = min(m, s_min[q]);
    first[t] = m;
  }
}

// Leaders sum their group: one warp per term, lanes take the members in a
// fixed stride, then a fixed butterfly (deterministic).
__global__ void k_merge_sum(const int32_t* __restrict__ sgn, const double2* __restrict__ coef, int64_t n,
                            const int32_t* __restrict__ first, int32_t* leader_flag, double2* merged,
                            int32_t* imag_nonzero) {
  const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (t >= n) return;
  const bool leader = first[t] == (int32_t)n;
  if (lane == 0) leader_flag[t] = leader ? 1 : 0;
  if (!leader) return;
  const int st = sgn[t];
  double re = 0.0, im = 0.0;
  for (int64_t u = t + lane; u < n; u += 32) {
    if (u != t && first[u] != (int32_t)t) continue;
    const int su = sgn[u];
    const double2 c = coef[u];
    re += c.x;
    im += (su == st) ? c.y : -c.y;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    re += __shfl_xor_sync(0xffffffffu, re, o);
    im += __shfl_xor_sync(0xffffffffu, im, o);
  }
  if (lane != 0) return;
  if (st == 0) im = 0.0;
  merged[t] = make_double2(re, im);
  if (im != 0.0) atomicExch(imag_nonzero, 1);
}

// Compact the leaders: residue of the leader's frequency, step and coefficient.
// One warp per term.
__global__ void k_compact_terms(const int32_t* __restrict__ freq, int64_t n, LatticeDev L,
                                const int32_t* __restrict__ flag, const int32_t* __restrict__ pos,
                                const double2* __restrict__ merged, int64_t* q, int64_t* step, double2* coef_out) {
  const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (t >= n || !flag[t]) return;   // warp-uniform
  const int64_t k = pos[t];
  // the merged coefficient is expressed in the leader's own orientation p_t
  const int64_t r = residue_warp(freq + t * L.d, L.d, L);
  if ((threadIdx.x & 31) != 0) return;
  q[k] = r;
  step[k] = (int64_t)(((uint64_t)r * (uint64_t)kSampThreads) % (uint64_t)L.M);
  coef_out[k] = merged[t];
}


// TAB: 0 split tables in shared memory, 1 split tables in global memory,
//      2 one full table exp(2 pi i r / M) in global memory (L2-resident).
template <typename R, int TAB>
__global__ void __launch_bounds__(kSampThreads) k_sample(int64_t M, int bl, int64_t H,
                                                         const typename C2<R>::T* __restrict__ lo_g,
                                                         const typename C2<R>::T* __restrict__ hi_g,
                                                         const int64_t* __restrict__ q, const int64_t* __restrict__ step,
                                                         const double2* __restrict__ coef,
                                                         const int64_t* __restrict__ n_terms_dev, R* out) {
  const int64_t n_terms = *n_terms_dev;
  using T2 = typename C2<R>::T;
  extern __shared__ __align__(16) unsigned char smem[];
  const int64_t L = 1ll << bl;
  T2* s_lo = reinterpret_cast<T2*>(smem);
  T2* s_hi = s_lo + (TAB == 0 ? L : 0);
  int64_t* s_q = reinterpret_cast<int64_t*>(s_hi + (TAB == 0 ? H : 0));
  int64_t* s_step = s_q + kTermChunk;
  T2* s_c = reinterpret_cast<T2*>(s_step + kTermChunk);
  if (TAB == 0) {
    for (int64_t i = threadIdx.x; i < L; i += blockDim.x) s_lo[i] = lo_g[i];
    for (int64_t i = threadIdx.x; i < H; i += blockDim.x) s_hi[i] = hi_g[i];
  }
  const T2* lo = TAB == 0 ? s_lo : lo_g;
  const T2* hi = TAB == 0 ? s_hi : hi_g;
  const uint32_t lmask = (uint32_t)(L - 1);
  const int64_t j0 = (int64_t)blockIdx.x * (kSampThreads * kSampPerThread) + threadIdx.x;
  const uint64_t inv = ~0ull / (uint64_t)M;   // once per thread (Barrett constant of mulmod)
  R acc[kSampPerThread];
#pragma unroll
  for (int m = 0; m < kSampPerThread; ++m) acc[m] = (R)0;
  for (int64_t t0 = 0; t0 < n_terms; t0 += kTermChunk) {
    const int tc = (n_terms - t0 < kTermChunk) ? (int)(n_terms - t0) : kTermChunk;
    __syncthreads();
    for (int i = threadIdx.x; i < tc; i += blockDim.x) {
      s_q[i] = q[t0 + i];
      s_step[i] = step[t0 + i];
      const double2 c = coef[t0 + i];
      s_c[i].x = (R)c.x;
      s_c[i].y = (R)c.y;
    }
    __syncthreads();
    for (int t = 0; t < tc; ++t) {
      const uint32_t st = (uint32_t)s_step[t];
      uint32_t r = mulmod((uint64_t)j0, (uint64_t)s_q[t], (uint64_t)M, inv);
      const T2 c = s_c[t];
      if (TAB == 2) {
        uint32_t rr[kSampPerThread];
#pragma unroll
        for (int m = 0; m < kSampPerThread; ++m) {
          rr[m] = r;
          r += st;
          if (r >= (uint32_t)M) r -= (uint32_t)M;
        }
        T2 e[kSampPerThread];
#pragma unroll
        for (int m = 0; m < kSampPerThread; ++m) e[m] = __ldg(lo + rr[m]);
#pragma unroll
        for (int m = 0; m < kSampPerThread; ++m) acc[m] += c.x * e[m].x - c.y * e[m].y;
      } else {
#pragma unroll
        for (int m = 0; m < kSampPerThread; ++m) {
          const T2 h = hi[r >> bl], l = lo[r & lmask];
          const R er = h.x * l.x - h.y * l.y;   // cos(2 pi r / M)
          const R ei = h.x * l.y + h.y * l.x;   // sin(2 pi r / M)
          acc[m] += c.x * er - c.y * ei;
          r += st;
          if (r >= (uint32_t)M) r -= (uint32_t)M;
        }
      }
    }
  }
#pragma unroll
  for (int m = 0; m < kSampPerThread; ++m) {
    const int64_t j = j0 + (int64_t)m * kSampThreads;
    if (j < M) out[j] = acc[m];
  }
}

template <typename T2>
__device__ __forceinline__ double2 bin(const T2* spec, int64_t M, int64_t b) {
  if (2 * b <= M) return make_double2((double)spec[b].x, (double)spec[b].y);
  const T2 v = spec[M - b];
  return make_double2((double)v.x, -(double)v.y);
}

template <typename T2>
__global__ void k_extract(const int32_t* __restrict__ cand, int64_t n, LatticeDev L, const T2* __restrict__ spec,
                          double2* val, double* mag, unsigned long long* maxbits) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t b = residue_of(cand + i * L.d, L.d, L);
  const int64_t nb = (L.M - b) % L.M;
  const double2 x = bin(spec, L.M, b), y = bin(spec, L.M, nb);
  const double sc = 0.5 / (double)L.M;
  const double2 v = make_double2((x.x + y.x) * sc, (x.y - y.y) * sc);
  val[i] = v;
  const double m = hypot(v.x, v.y);
  mag[i] = m;
  atomicMax(maxbits, (unsigned long long)__double_as_longlong(m));
}

__global__ void k_keep(const double* __restrict__ mag, int64_t n, const unsigned long long* __restrict__ maxbits,
                       double tau, int32_t* flag) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double mx = __longlong_as_double((long long)*maxbits);
  flag[i] = mag[i] > tau * mx ? 1 : 0;
}

__global__ void k_compact(const int32_t* __restrict__ cand, const double2* __restrict__ val, int64_t n, int d,
                          const int32_t* __restrict__ flag, const int32_t* __restrict__ pos, int32_t* fo, double2* vo) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || !flag[i]) return;
  const int64_t p = pos[i];
  for (int c = 0; c < d; ++c) fo[p * d + c] = cand[i * d + c];
  vo[p] = val[i];
}

inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// Per-(M, precision) FFT plan, sample and spectrum buffers and twiddle tables.
struct SftPlan {
  int64_t M = 0;
  ss_precision prec = SS_FP64;
  int bl = 0;
  int64_t H = 0;
  cufftHandle fft = 0;
  bool has_fft = false;
  DevBuf<unsigned char> samples, spectrum, lo, hi, full;   // full: exp(2 pi i r/M), r < M
  DevBuf<float2> t3[3];                                    // FP32 three-level tables
  int64_t n2 = 0;
  bool df = false;                                         // full table in double-float form
  // double-float complex FFT (FP64 recovery of two real sums at once)
  bool has_dff = false;
  DfFftPlan dff;
  DevBuf<float4> dfz, dftmp;
  DevBuf<double> dfscale;   // the two sums' scales of the last round trip
  // pruned transforms (on a 7-smooth M above the full table's limit;
  // double-float arithmetic in FP64, FP32 in FP32): two-level twiddle table,
  // the complex sample vector s_a / sigma_a + i s_f / sigma_f and the two
  // scales
  bool has_pr = false;
  TwoLevelTable prt;
  DevBuf<float4> prz;
  DevBuf<double> prscale;
  // inverse (Z2D) plan of the FFT evaluation path, made on first use
  mutable std::mutex ifft_mu;
  mutable cufftHandle ifft = 0;
  mutable bool has_ifft = false;
  // FP32 on sizes cuFFT transforms by Bluestein's method: a and f share one
  // complex transform (made on first use: plan, f's samples, the packed
  // vector, the two scales)
  mutable cufftHandle c2c = 0;
  mutable bool has_c2c = false;
  mutable DevBuf<float> samples2;
  mutable DevBuf<float2> z32;
  mutable DevBuf<double> scale32;
  ~SftPlan() {
    if (has_fft) cufftDestroy(fft);
    if (has_ifft) cufftDestroy(ifft);
    if (has_c2c) cufftDestroy(c2c);
  }
};

// The FP64 path evaluates samples in double-float on the FP32 pipes (GB300
// issues one FP64 FMA per SM clock, 1/128 of its FP32 rate).  Setting
// SS_NATIVE_FP64_SAMPLING=1 selects native FP64 arithmetic instead.
bool native_fp64_sampling() {
  static const bool v = [] {
    const char* e = getenv("SS_NATIVE_FP64_SAMPLING");
    return e && e[0] == '1';
  }();
  return v;
}

std::mutex g_plan_mu;
std::list<std::shared_ptr<SftPlan>> g_plans;   // most recent first
constexpr size_t kMaxPlans = 4;

ss_status get_plan(int64_t M, ss_precision prec, cudaStream_t st, std::shared_ptr<SftPlan>* out) {
  std::lock_guard<std::mutex> lk(g_plan_mu);
  for (auto it = g_plans.begin(); it != g_plans.end(); ++it) {
    if ((*it)->M == M && (*it)->prec == prec) {
      auto p = *it;
      g_plans.erase(it);
      g_plans.push_front(p);
      *out = p;
      return SS_OK;
    }
  }
  auto p = std::make_shared<SftPlan>();
  p->M = M;
  p->prec = prec;
  int bits = 0;
  while ((1ll << bits) < M) ++bits;
  p->bl = (bits + 1) / 2;
  p->H = (M + (1ll << p->bl) - 1) >> p->bl;
  const size_t real_sz = prec == SS_FP64 ? sizeof(double) : sizeof(float);
  const size_t cplx_sz = 2 * real_sz;
  SS_TRY(p->samples.alloc(M * real_sz, st));
  SS_TRY(p->spectrum.alloc((M / 2 + 1) * cplx_sz, st));
  SS_TRY(p->lo.alloc((1ll << p->bl) * cplx_sz, st));
  SS_TRY(p->hi.alloc(p->H * cplx_sz, st));
  const int64_t nt = std::max<int64_t>(1ll << p->bl, p->H);
  if (prec == SS_FP64)
    k_twiddles<double><<<nblk(nt), 256, 0, st>>>(M, p->bl, p->H, reinterpret_cast<double2*>(p->lo.get()),
                                                 reinterpret_cast<double2*>(p->hi.get()));
  else
    k_twiddles<float><<<nblk(nt), 256, 0, st>>>(M, p->bl, p->H, reinterpret_cast<float2*>(p->lo.get()),
                                                reinterpret_cast<float2*>(p->hi.get()));
  SS_LAUNCH_CHECK();
  if (prec == SS_FP32) {
    p->n2 = (M + (1ll << (2 * kT3Bits)) - 1) >> (2 * kT3Bits);
    SS_TRY(p->t3[0].alloc(kT3Size, st));
    SS_TRY(p->t3[1].alloc(kT3Size, st));
    SS_TRY(p->t3[2].alloc(p->n2, st));
    k_twiddles3<<<nblk(std::max<int64_t>(kT3Size, p->n2)), 256, 0, st>>>(M, p->n2, p->t3[0].get(), p->t3[1].get(),
                                                                         p->t3[2].get());
    SS_LAUNCH_CHECK();
  }
  if (prec == SS_FP64 && M <= kFullTableMax) {
    SS_TRY(p->full.alloc(M * sizeof(double2), st));   // 16 bytes per entry in either form
    if (native_fp64_sampling())
      k_twiddles_full<<<nblk(M), 256, 0, st>>>(M, reinterpret_cast<double2*>(p->full.get()));
    else
      k_twiddles_df<<<nblk(M), 256, 0, st>>>(M, reinterpret_cast<float4*>(p->full.get()));
    SS_LAUNCH_CHECK();
    p->df = !native_fp64_sampling();
    if (p->df && df_fft_plan(M, &p->dff)) {
      SS_TRY(p->dfz.alloc(M, st));
      SS_TRY(p->dftmp.alloc(M, st));
      SS_TRY(p->dfscale.alloc(2, st));
      p->has_dff = true;
    }
  }
  if (M > kFullTableMax && !(prec == SS_FP64 && native_fp64_sampling()) && pruned_supported(M)) {
    SS_TRY(two_level_table(M, &p->prt, st));
    SS_TRY(p->prz.alloc(prec == SS_FP64 ? M : (M + 1) / 2, st));   // float4 or float2 per node
    SS_TRY(p->prscale.alloc(2, st));
    p->has_pr = true;
  }
  note_alloc();   // the plan allocates its work area
  const cufftResult r = cufftPlan1d(&p->fft, (int)M, prec == SS_FP64 ? CUFFT_D2Z : CUFFT_R2C, 1);
  if (r != CUFFT_SUCCESS) SS_FAIL(SS_ERR_CUDA, "cufftPlan1d(%lld) failed: %d", (long long)M, (int)r);
  p->has_fft = true;
  // the plan is cached across calls and streams
  SS_CUDA(cudaStreamSynchronize(st));
  p->samples.settle(); p->spectrum.settle(); p->lo.settle(); p->hi.settle(); p->full.settle();
  p->dfz.settle(); p->dftmp.settle(); p->dfscale.settle();
  p->prt.t0.settle(); p->prt.t1.settle(); p->prz.settle(); p->prscale.settle();
  for (auto& t : p->t3) t.settle();
  g_plans.push_front(p);
  while (g_plans.size() > kMaxPlans) g_plans.pop_back();
  *out = p;
  return SS_OK;
}

// FFT evaluation (FP64): g_j = Re sum_t c_t w^{j r_t}, w = exp(2 pi i / M),
// is the inverse DFT of the Hermitian spectrum X with X_{r_t} += c_t / 2 and
// X_{M - r_t} += conj(c_t) / 2 (bins 0 and M/2 take Re c_t), so one Z2D
// transform of the half spectrum (bins b <= M/2) gives all M samples in
// O(M log M) instead of O(M T).  It pays for many terms on a size cuFFT
// factors into small primes.
constexpr int64_t kFftEvalMaxM = 1ll << 25;
constexpr int64_t kFftEvalTermsSmooth = 64;     // unmerged terms, M 7-smooth
constexpr int64_t kFftEvalTermsOther = 512;     // unmerged terms, other M (Bluestein)

bool smooth7(int64_t M) {
  for (int64_t p : {2, 3, 5, 7})
    while (M % p == 0) M /= p;
  return M == 1;
}

bool use_fft_eval(const SftPlan& P, int64_t n) {
  if (P.prec != SS_FP64 || P.M < 2 || P.M > kFftEvalMaxM) return false;
  return n >= (smooth7(P.M) ? kFftEvalTermsSmooth : kFftEvalTermsOther);
}

// FP32 recovery of two sums by one complex transform: on sizes that cuFFT
// factors into small primes two real transforms cost no more than one complex
// one; on the others (Bluestein) one complex transform costs about one real.
bool use_pair32(const SftPlan& P) { return P.prec == SS_FP32 && !smooth7(P.M); }

ss_status ensure_pair32(const SftPlan& P, cudaStream_t st) {
  std::lock_guard<std::mutex> lk(P.ifft_mu);
  if (P.has_c2c) return SS_OK;
  SS_TRY(P.samples2.alloc(P.M, st));
  SS_TRY(P.z32.alloc(P.M, st));
  SS_TRY(P.scale32.alloc(2, st));
  note_alloc();   // the plan allocates its work area
  const cufftResult r = cufftPlan1d(&P.c2c, (int)P.M, CUFFT_C2C, 1);
  if (r != CUFFT_SUCCESS) SS_FAIL(SS_ERR_CUDA, "cufftPlan1d(%lld, C2C) failed: %d", (long long)P.M, (int)r);
  // the buffers belong to the cached plan and outlive this call
  SS_CUDA(cudaStreamSynchronize(st));
  P.samples2.settle();
  P.z32.settle();
  P.scale32.settle();
  P.has_c2c = true;
  return SS_OK;
}

ss_status ensure_ifft(const SftPlan& P) {
  std::lock_guard<std::mutex> lk(P.ifft_mu);
  if (P.has_ifft) return SS_OK;
  note_alloc();   // the plan allocates its work area
  const cufftResult r = cufftPlan1d(&P.ifft, (int)P.M, CUFFT_Z2D, 1);
  if (r != CUFFT_SUCCESS) SS_FAIL(SS_ERR_CUDA, "cufftPlan1d(%lld, Z2D) failed: %d", (long long)P.M, (int)r);
  P.has_ifft = true;
  return SS_OK;
}

// bins[b] for the b that some compacted term t < *n_dev reaches (the rest
// stay as the caller zeroed them).  One warp per term: a term with an earlier
// term in its bin writes nothing; the first one sums the bin's terms (lanes in
// a fixed stride, then a fixed butterfly: deterministic).
__device__ __forceinline__ int64_t half_bin(int64_t r, int64_t M) { return 2 * r <= M ? r : M - r; }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void k_bin_terms(const int64_t* __restrict__ q, const double2* __restrict__ coef,
                            const int64_t* __restrict__ n_dev, int64_t M, double2* __restrict__ bins) {
  const int64_t n = *n_dev;
  const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (t >= n) return;   // warp-uniform
  const int64_t b = half_bin(q[t], M);
  bool earlier = false;
  for (int64_t u = lane; u < t && !earlier; u += 32) earlier = half_bin(q[u], M) == b;
  if (__any_sync(0xffffffffu, earlier)) return;
  double re = 0.0, im = 0.0;
  for (int64_t u = t + lane; u < n; u += 32) {
    const int64_t r = q[u];
    if (half_bin(r, M) != b) continue;
    const double2 c = coef[u];
    re += c.x;
    im += 2 * r <= M ? c.y : -c.y;
  }
  re = warp_sum(re);
  im = warp_sum(im);
  if (lane) return;
  bins[b] = (b == 0 || 2 * b == M) ? make_double2(re, 0.0) : make_double2(0.5 * re, 0.5 * im);
}

// scale[w] = the power of two at or below sum_t |c_t| of sum w (1 if zero):
// the two sums share one transform at comparable magnitudes, so each keeps its
// own relative rounding error; powers of two scale exactly.
constexpr int kScaleThreads = 512;
__device__ void pair_scale(const double2* const c[2], const int64_t n[2], double* scale) {
  __shared__ double s_part[kScaleThreads];
  for (int w = 0; w < 2; ++w) {
    double acc = 0.0;
    for (int64_t t = threadIdx.x; t < n[w]; t += kScaleThreads) acc += hypot(c[w][t].x, c[w][t].y);
    s_part[threadIdx.x] = acc;
    __syncthreads();
    for (int o = kScaleThreads / 2; o > 0; o >>= 1) {
      if (threadIdx.x < o) s_part[threadIdx.x] += s_part[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) scale[w] = s_part[0] > 0.0 ? ldexp(1.0, ilogb(s_part[0])) : 1.0;
    __syncthreads();
  }
}

// term counts on the device (merged sums)
__global__ void __launch_bounds__(kScaleThreads) k_pair_scale(const double2* __restrict__ ca,
                                                              const int64_t* __restrict__ na_dev,
                                                              const double2* __restrict__ cf,
                                                              const int64_t* __restrict__ nf_dev, double* scale) {
  const double2* c[2] = {ca, cf};
  const int64_t n[2] = {*na_dev, *nf_dev};
  pair_scale(c, n, scale);
}

// term counts from the host (the sums as given)
__global__ void __launch_bounds__(kScaleThreads) k_pair_scale_n(const double2* __restrict__ ca, int64_t na,
                                                                const double2* __restrict__ cf, int64_t nf,
                                                                double* scale) {
  const double2* c[2] = {ca, cf};
  const int64_t n[2] = {na, nf};
  pair_scale(c, n, scale);
}

// z[j] = s_a[j] / scale[0] + i s_f[j] / scale[1] (FP32, exact scaling)
__global__ void k_pack_pair32(const float* __restrict__ sa, const float* __restrict__ sf,
                              const double* __restrict__ scale, int64_t M, float2* __restrict__ z) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= M) return;
  const float ia = (float)(1.0 / scale[0]), jf = (float)(1.0 / scale[1]);
  z[j] = make_float2(sa[j] * ia, sf[j] * jf);
}

// Bins of a (WHICH = 0) and f (WHICH = 1) from the FP32 complex transform of
// s_a / scale[0] + i s_f / scale[1], as in k_extract_pair.
template <int WHICH>
__global__ void k_extract_pair32(const int32_t* __restrict__ cand, int64_t n, LatticeDev L,
                                 const float2* __restrict__ Zh, const double* __restrict__ scale, double2* val,
                                 double* mag, unsigned long long* maxbits) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t b = residue_of(cand + i * L.d, L.d, L);
  const int64_t nb = (L.M - b) % L.M;
  const float2 x = Zh[b], y = Zh[nb];
  const double sc = 0.5 / (double)L.M * scale[WHICH];
  const double2 v = WHICH == 0 ? make_double2(((double)x.x + y.x) * sc, ((double)x.y - y.y) * sc)
                               : make_double2(((double)x.y + y.y) * sc, ((double)y.x - x.x) * sc);
  val[i] = v;
  const double m = hypot(v.x, v.y);
  mag[i] = m;
  atomicMax(maxbits, (unsigned long long)__double_as_longlong(m));
}

// Two real sums a and f at once: Z = S_a + i S_f with S_a, S_f their
// Hermitian spectra (as in k_bin_terms), over the whole length M, so that the
// inverse transform of Z is s_a + i s_f (real and imaginary parts are the two
// sample vectors).  Terms are a's (u < na) then f's; as in k_bin_terms the
// first term of each bin sums the bin's a and f terms and writes Z[b] and
// Z[M - b] (each sum divided by its scale).  Z must be zero on entry.
__global__ void k_bin_pair(const int64_t* __restrict__ qa, const double2* __restrict__ ca,
                           const int64_t* __restrict__ na_dev, const int64_t* __restrict__ qf,
                           const double2* __restrict__ cf, const int64_t* __restrict__ nf_dev,
                           const double* __restrict__ scale, int64_t M, float4* __restrict__ Z) {
  const int64_t na = *na_dev, n = na + *nf_dev;
  const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (t >= n) return;   // warp-uniform
  auto res = [&](int64_t u) { return u < na ? qa[u] : qf[u - na]; };
  const int64_t b = half_bin(res(t), M);
  bool earlier = false;
  for (int64_t u = lane; u < t && !earlier; u += 32) earlier = half_bin(res(u), M) == b;
  if (__any_sync(0xffffffffu, earlier)) return;
  double are = 0.0, aim = 0.0, fre = 0.0, fim = 0.0;
  for (int64_t u = t + lane; u < n; u += 32) {
    const int64_t r = res(u);
    if (half_bin(r, M) != b) continue;
    const bool lo = 2 * r <= M;
    if (u < na) {
      const double2 c = ca[u];
      are += c.x;
      aim += lo ? c.y : -c.y;
    } else {
      const double2 c = cf[u - na];
      fre += c.x;
      fim += lo ? c.y : -c.y;
    }
  }
  are = warp_sum(are);
  aim = warp_sum(aim);
  fre = warp_sum(fre);
  fim = warp_sum(fim);
  if (lane) return;
  const double ia = 1.0 / scale[0], jf = 1.0 / scale[1];   // exact: powers of two
  are *= ia; aim *= ia; fre *= jf; fim *= jf;
  if (b == 0 || 2 * b == M) {
    const DF zr = df_split(are), zi = df_split(fre);
    Z[b] = make_float4(zr.hi, zr.lo, zi.hi, zi.lo);
    return;
  }
  are *= 0.5; aim *= 0.5; fre *= 0.5; fim *= 0.5;
  DF x = df_split(are - fim), y = df_split(aim + fre);
  Z[b] = make_float4(x.hi, x.lo, y.hi, y.lo);
  x = df_split(are + fim);
  y = df_split(fre - aim);
  Z[M - b] = make_float4(x.hi, x.lo, y.hi, y.lo);
}

// Recovery from the forward transform Zh of s_a + i s_f: with x = Zh[b] and
// y = Zh[M - b], the bin of the real sum a is (x + conj(y)) / 2 and that of f
// is (x - conj(y)) / (2 i), each scaled by 1 / M.
template <int WHICH>
__global__ void k_extract_pair(const int32_t* __restrict__ cand, int64_t n, LatticeDev L, const float4* __restrict__ Zh,
                               const double* __restrict__ scale, double2* val, double* mag,
                               unsigned long long* maxbits) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t b = residue_of(cand + i * L.d, L.d, L);
  const int64_t nb = (L.M - b) % L.M;
  const float4 xs = Zh[b], ys = Zh[nb];
  const double xr = (double)xs.x + (double)xs.y, xi = (double)xs.z + (double)xs.w;
  const double yr = (double)ys.x + (double)ys.y, yi = (double)ys.z + (double)ys.w;
  const double sc = 0.5 / (double)L.M * scale[WHICH];
  const double2 v = WHICH == 0 ? make_double2((xr + yr) * sc, (xi - yi) * sc)
                               : make_double2((xi + yi) * sc, (yr - xr) * sc);
  val[i] = v;
  const double m = hypot(v.x, v.y);
  mag[i] = m;
  atomicMax(maxbits, (unsigned long long)__double_as_longlong(m));
}

template <typename R, int TAB>
ss_status launch_sample(const SftPlan& P, unsigned grid, size_t sm, const int64_t* q, const int64_t* step,
                        const double2* coef, const int64_t* n_dev, void* out, cudaStream_t st) {
  using T2 = typename C2<R>::T;
  auto lo = reinterpret_cast<const T2*>(TAB == 2 ? P.full.get() : P.lo.get());
  auto hi = reinterpret_cast<const T2*>(P.hi.get());
  SS_CUDA(cudaFuncSetAttribute(k_sample<R, TAB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  k_sample<R, TAB><<<grid, kSampThreads, sm, st>>>(P.M, P.bl, P.H, lo, hi, q, step, coef, n_dev,
                                                   reinterpret_cast<R*>(out));
  SS_LAUNCH_CHECK();
  return SS_OK;
}

// The merged terms of one real sum: residues q, phase steps, coefficients and
// their count (on the device).
struct Terms {
  DevBuf<int64_t> q, step, total;
  DevBuf<double2> coef;
};

// Merge +-p terms (exact rewrite of the real sum) and compact them; no host
// synchronisation (the merged count stays on the device).
ss_status prep_terms(const LatticeDev& L, const ss_trig* g, Terms* T, cudaStream_t st) {
  ProfScope prof_("prep_terms", st);
  const int64_t n = g->n_terms;
  SS_TRY(T->total.alloc_tmp(1, st));
  if (n == 0) {
    SS_CUDA(cudaMemsetAsync(T->total.get(), 0, sizeof(int64_t), st));
    return SS_OK;
  }
  if (n > 46340) SS_FAIL(SS_ERR_INVALID, "lattice_sample: more than 46340 terms");
  DevBuf<int32_t> flag, pos, imag, first, sgn;
  DevBuf<double2> merged;
  SS_TRY(T->q.alloc_tmp(n, st));
  SS_TRY(T->step.alloc_tmp(n, st));
  SS_TRY(flag.alloc_tmp(n, st));
  SS_TRY(pos.alloc_tmp(n, st));
  SS_TRY(imag.alloc_tmp(1, st));
  SS_TRY(first.alloc_tmp(n, st));
  SS_TRY(merged.alloc_tmp(n, st));
  SS_TRY(T->coef.alloc_tmp(n, st));
  SS_TRY(sgn.alloc_tmp(n, st));
  SS_CUDA(cudaMemsetAsync(imag.get(), 0, sizeof(int32_t), st));
  k_term_signs<<<nblk(n * 32), 256, 0, st>>>(g->freq, n, L.d, sgn.get());
  k_merge_first<<<(unsigned)n, 32 * kMergeWarps, 0, st>>>(g->freq, n, L.d, sgn.get(), first.get());
  k_merge_sum<<<nblk(n * 32), 256, 0, st>>>(sgn.get(), reinterpret_cast<const double2*>(g->coef), n, first.get(),
                                            flag.get(), merged.get(), imag.get());
  SS_LAUNCH_CHECK();
  SS_TRY(exclusive_scan_i32(flag.get(), pos.get(), n, T->total.get(), st));
  k_compact_terms<<<nblk(n * 32), 256, 0, st>>>(g->freq, n, L, flag.get(), pos.get(), merged.get(), T->q.get(),
                                                T->step.get(), T->coef.get());
  SS_LAUNCH_CHECK();
  return SS_OK;
}

// Both sums of a pair with at most kPrepSmall terms each: one launch, one
// block per sum doing every step of prep_terms (signs, first occurrences,
// leader sums in the same order, prefix sum, compaction) in shared memory.
constexpr int kPrepSmall = 1024;

struct PrepArgs {
  const int32_t* freq;
  const double2* coef;
  int64_t n;
  int64_t* q;
  int64_t* step;
  double2* coef_out;
  int64_t* total;
};

__global__ void __launch_bounds__(1024) k_prep_terms_small(PrepArgs A0, PrepArgs A1, LatticeDev L) {
  __shared__ int32_t s_sgn[kPrepSmall], s_first[kPrepSmall], s_pos[kPrepSmall];
  __shared__ double2 s_merged[kPrepSmall];
  __shared__ uint64_t s_hash[kPrepSmall];
  __shared__ int32_t s_wsum[32];
  const PrepArgs& A = blockIdx.x == 0 ? A0 : A1;
  const int n = (int)A.n, d = L.d;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  // signs of the first nonzero coordinates
  for (int t = w; t < n; t += nw) {
    int sg = 0;
    for (int c0 = 0; c0 < d && sg == 0; c0 += 32) {
      const int32_t v = c0 + lane < d ? A.freq[(int64_t)t * d + c0 + lane] : 0;
      const unsigned m = __ballot_sync(0xffffffffu, v != 0);
      if (m) sg = __shfl_sync(0xffffffffu, v, __ffs(m) - 1) > 0 ? 1 : -1;
    }
    // a hash of the representative sgn p: equal representatives, equal hashes
    const int x = sg < 0 ? -1 : 1;
    uint64_t h = 0;
    for (int c = lane; c < d; c += 32)
      h += (uint64_t)(int64_t)(x * A.freq[(int64_t)t * d + c]) * (0x9e3779b97f4a7c15ull ^ ((uint64_t)c << 32 | 1u));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) h += __shfl_xor_sync(0xffffffffu, h, o);
    if (lane == 0) {
      s_sgn[t] = sg;
      s_hash[t] = h;
    }
  }
  __syncthreads();
  // first occurrence of every representative: hashes compared 32 at a time,
  // the coordinates only where they agree
  for (int t = w; t < n; t += nw) {
    const int xt = s_sgn[t] < 0 ? -1 : 1;
    const int32_t* pt = A.freq + (int64_t)t * d;
    const uint64_t ht = s_hash[t];
    int fu = n;
    for (int u0 = 0; u0 < t && fu == n; u0 += 32) {
      unsigned m = __ballot_sync(0xffffffffu, u0 + lane < t && s_hash[u0 + lane] == ht);
      while (m) {
        const int u = u0 + __ffs(m) - 1;
        m &= m - 1;
        const int xu = s_sgn[u] < 0 ? -1 : 1;
        const int32_t* pu = A.freq + (int64_t)u * d;
        bool diff = false;
        for (int c = lane; c < d; c += 32) diff |= xu * pu[c] != xt * pt[c];
        if (!__any_sync(0xffffffffu, diff)) {
          fu = u;
          break;
        }
      }
    }
    if (lane == 0) s_first[t] = fu;
  }
  __syncthreads();
  // leaders sum their groups (lanes in a fixed stride, then a fixed butterfly)
  for (int t = w; t < n; t += nw) {
    const bool leader = s_first[t] == n;
    if (lane == 0) s_pos[t] = leader ? 1 : 0;
    if (!leader) continue;
    const int st = s_sgn[t];
    double re = 0.0, im = 0.0;
    for (int u = t + lane; u < n; u += 32) {
      if (u != t && s_first[u] != t) continue;
      const double2 c = A.coef[u];
      re += c.x;
      im += (s_sgn[u] == st) ? c.y : -c.y;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      re += __shfl_xor_sync(0xffffffffu, re, o);
      im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    if (lane == 0) s_merged[t] = make_double2(re, st == 0 ? 0.0 : im);
  }
  __syncthreads();
  // exclusive prefix sum of the leader flags (n <= blockDim)
  const int t = threadIdx.x;
  const int f = t < n ? s_pos[t] : 0;
  int x = f;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_wsum[w] = x;
  __syncthreads();
  int before = 0, total = 0;
  for (int q = 0; q < nw; ++q) {
    if (q < w) before += s_wsum[q];
    total += s_wsum[q];
  }
  __syncthreads();
  if (t < n) s_pos[t] = f ? before + x - f : -1;
  if (t == 0) *A.total = total;
  __syncthreads();
  // compaction: the residue of every leader by its warp
  for (int u = w; u < n; u += nw) {
    const int k = s_pos[u];
    if (k < 0) continue;
    const int64_t r = residue_warp(A.freq + (int64_t)u * d, d, L);
    if (lane == 0) {
      A.q[k] = r;
      A.step[k] = (int64_t)(((uint64_t)r * (uint64_t)kSampThreads) % (uint64_t)L.M);
      A.coef_out[k] = s_merged[u];
    }
  }
}

// prep_terms of the two sums of a pair (f may have no terms).
ss_status prep_terms_pair(const LatticeDev& L, const ss_trig* a, const ss_trig* f, Terms* Ta, Terms* Tf,
                          cudaStream_t st) {
  if (a->n_terms > kPrepSmall || f->n_terms > kPrepSmall) {
    SS_TRY(prep_terms(L, a, Ta, st));
    return prep_terms(L, f, Tf, st);
  }
  ProfScope prof_("prep_terms", st);
  PrepArgs A[2];
  Terms* T[2] = {Ta, Tf};
  const ss_trig* g[2] = {a, f};
  for (int i = 0; i < 2; ++i) {
    const int64_t n = g[i]->n_terms;
    SS_TRY(T[i]->total.alloc_tmp(1, st));
    SS_TRY(T[i]->q.alloc_tmp(std::max<int64_t>(n, 1), st));
    SS_TRY(T[i]->step.alloc_tmp(std::max<int64_t>(n, 1), st));
    SS_TRY(T[i]->coef.alloc_tmp(std::max<int64_t>(n, 1), st));
    A[i] = PrepArgs{g[i]->freq, reinterpret_cast<const double2*>(g[i]->coef), n, T[i]->q.get(), T[i]->step.get(),
                    T[i]->coef.get(), T[i]->total.get()};
  }
  k_prep_terms_small<<<2, 1024, 0, st>>>(A[0], A[1], L);
  SS_LAUNCH_CHECK();
  return SS_OK;
}

// Evaluate a real sum on the lattice; no host synchronisation.
ss_status sample_into(const SftPlan& P, const LatticeDev& L, const ss_trig* g, void* out, cudaStream_t st) {
  const int64_t n = g->n_terms;
  const int64_t Lsz = 1ll << P.bl;
  const unsigned grid = (unsigned)((P.M + kSampThreads * kSampPerThread - 1) / (kSampThreads * kSampPerThread));
  if (n == 0) {
    SS_CUDA(cudaMemsetAsync(out, 0, P.M * (P.prec == SS_FP64 ? sizeof(double) : sizeof(float)), st));
    return SS_OK;
  }
  Terms T;
  SS_TRY(prep_terms(L, g, &T, st));
  DevBuf<int64_t>& q = T.q;
  DevBuf<int64_t>& step = T.step;
  DevBuf<int64_t>& total = T.total;
  DevBuf<double2>& coef = T.coef;
  if (P.has_pr)   // long 7-smooth lattice: sparse evaluation, the real parts in the plan's precision
    return pruned_eval_pair(P.prt, q.get(), coef.get(), total.get(), n, nullptr, nullptr, nullptr, 0, nullptr, out,
                            P.prec == SS_FP64 ? PrunedFormat::kF64Real : PrunedFormat::kF32Real, st);
  if (use_fft_eval(P, n)) {
    // the spectrum buffer holds the bins; its next reader (the forward
    // transform of recovery) follows in stream order
    SS_TRY(ensure_ifft(P));
    auto bins = reinterpret_cast<double2*>(P.spectrum.get());
    SS_CUDA(cudaMemsetAsync(bins, 0, (P.M / 2 + 1) * sizeof(double2), st));
    k_bin_terms<<<nblk(n * 32), 256, 0, st>>>(q.get(), coef.get(), total.get(), P.M, bins);
    SS_LAUNCH_CHECK();
    cufftResult r = cufftSetStream(P.ifft, st);
    if (r == CUFFT_SUCCESS)
      r = cufftExecZ2D(P.ifft, reinterpret_cast<cufftDoubleComplex*>(bins), reinterpret_cast<cufftDoubleReal*>(out));
    if (r != CUFFT_SUCCESS) SS_FAIL(SS_ERR_CUDA, "cuFFT Z2D exec failed: %d", (int)r);
    return SS_OK;
  }
  if (P.prec == SS_FP64) {
    if (P.full.get() && P.df) {
      auto tab = reinterpret_cast<const float4*>(P.full.get());
      DevBuf<float4> W;
      SS_TRY(W.alloc_tmp(n * kSampPerThread, st));
      k_term_powers<<<nblk(n), 256, 0, st>>>(step.get(), total.get(), P.M, tab, W.get());
      // split the terms over gridDim.y when the sample blocks alone would not
      // fill the SMs several times over (n bounds the merged term count)
      const int64_t want = 8LL * sm_count();
      int n_split = (int)std::min<int64_t>(8, std::max<int64_t>(1, (want + grid - 1) / grid));
      n_split = (int)std::max<int64_t>(1, std::min<int64_t>(n_split, n / 64));
      if (n_split == 1) {
        k_sample_df<<<grid, kSampThreads, 0, st>>>(P.M, tab, q.get(), W.get(), coef.get(), total.get(),
                                                   reinterpret_cast<double*>(out));
      } else {
        DevBuf<double> part;
        SS_TRY(part.alloc_tmp((size_t)n_split * P.M, st));
        k_sample_df<<<dim3(grid, n_split), kSampThreads, 0, st>>>(P.M, tab, q.get(), W.get(), coef.get(),
                                                                  total.get(), part.get());
        k_sum_splits<<<nblk(P.M), 256, 0, st>>>(part.get(), n_split, P.M, reinterpret_cast<double*>(out));
      }
      SS_LAUNCH_CHECK();
      return SS_OK;
    }
    const size_t terms_sm = kTermChunk * (2 * sizeof(int64_t) + sizeof(double2));
    if (P.full.get())
      return launch_sample<double, 2>(P, grid, terms_sm, q.get(), step.get(), coef.get(), total.get(), out, st);
    const size_t tab_sm = (Lsz + P.H) * sizeof(double2);
    const bool smem = tab_sm + terms_sm <= 200 * 1024;
    const size_t sm = (smem ? tab_sm : 0) + terms_sm;
    if (smem) return launch_sample<double, 0>(P, grid, sm, q.get(), step.get(), coef.get(), total.get(), out, st);
    return launch_sample<double, 1>(P, grid, sm, q.get(), step.get(), coef.get(), total.get(), out, st);
  }
  const size_t tab_sm = (2 * kT3Size + P.n2) * sizeof(float2);
  const size_t w_sm = kTermChunk * (kSampPerThread * sizeof(float2) + sizeof(float2) + sizeof(uint32_t));
  if (tab_sm + w_sm <= 200 * 1024) {
    DevBuf<float2> W;
    SS_TRY(W.alloc_tmp(n * kSampPerThread, st));
    k_term_powers32<<<nblk(n), 256, 0, st>>>(step.get(), total.get(), P.M, W.get());
    const size_t sm = tab_sm + w_sm;
    SS_CUDA(cudaFuncSetAttribute(k_sample32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    k_sample32<<<grid, kSampThreads, sm, st>>>(P.M, P.n2, P.t3[0].get(), P.t3[1].get(), P.t3[2].get(), q.get(),
                                               W.get(), coef.get(), total.get(), reinterpret_cast<float*>(out));
    SS_LAUNCH_CHECK();
    return SS_OK;
  }
  const size_t terms_sm = kTermChunk * (2 * sizeof(int64_t) + sizeof(float2));
  return launch_sample<float, 1>(P, grid, terms_sm, q.get(), step.get(), coef.get(), total.get(), out, st);
}

// Bins, threshold and compaction in candidate order; the reconstructing and
// symmetry checks run on the device beside them and are read back with the
// kept count in one synchronisation at the end.
// FP64 plans with the double-float transform: the sums a and f (f may be
// null) are sampled by one inverse transform of Z = S_a + i S_f and the
// samples s_a + i s_f transformed forward again; on return P.dfz holds that
// spectrum (read by k_extract_pair).
ss_status dff_round_trip(const SftPlan& P, const LatticeDev& L, const ss_trig* a, const ss_trig* f, cudaStream_t st) {
  const ss_trig none{L.d, 0, nullptr, nullptr};
  if (!f) f = &none;
  Terms ta, tf;
  SS_TRY(prep_terms_pair(L, a, f, &ta, &tf, st));
  float4* Z = P.dfz.get();
  const float4* tab = reinterpret_cast<const float4*>(P.full.get());
  SS_CUDA(cudaMemsetAsync(Z, 0, P.M * sizeof(float4), st));
  double* scale = P.dfscale.get();
  k_pair_scale<<<1, kScaleThreads, 0, st>>>(ta.coef.get(), ta.total.get(), tf.coef.get(), tf.total.get(), scale);
  SS_LAUNCH_CHECK();
  if (a->n_terms + f->n_terms > 0) {
    k_bin_pair<<<nblk((a->n_terms + f->n_terms) * 32), 256, 0, st>>>(ta.q.get(), ta.coef.get(), ta.total.get(), tf.q.get(),
                                                              tf.coef.get(), tf.total.get(), scale, P.M, Z);
    SS_LAUNCH_CHECK();
  }
  SS_TRY(df_fft(P.dff, tab, Z, P.dftmp.get(), Z, +1, st));
  return df_fft(P.dff, tab, Z, P.dftmp.get(), Z, -1, st);
}

// Pruned path (a 7-smooth M above the full table): the two sums a and f (f
// may be null) sampled at the M lattice nodes by the sparse evaluation of
// their merged terms, as s_a / sigma_a + i s_f / sigma_f in P.prz (double-
// float complex in FP64, FP32 complex in FP32).
ss_status pr_sample_pair(const SftPlan& P, const LatticeDev& L, const ss_trig* a, const ss_trig* f, cudaStream_t st) {
  const ss_trig none{L.d, 0, nullptr, nullptr};
  if (!f) f = &none;
  Terms ta, tf;
  SS_TRY(prep_terms_pair(L, a, f, &ta, &tf, st));
  double* scale = P.prscale.get();
  k_pair_scale<<<1, kScaleThreads, 0, st>>>(ta.coef.get(), ta.total.get(), tf.coef.get(), tf.total.get(), scale);
  SS_LAUNCH_CHECK();
  return pruned_eval_pair(P.prt, ta.q.get(), ta.coef.get(), ta.total.get(), a->n_terms, tf.q.get(), tf.coef.get(),
                          tf.total.get(), f->n_terms, scale, P.prz.get(),
                          P.prec == SS_FP64 ? PrunedFormat::kDfComplex : PrunedFormat::kF32Complex, st);
}

// Output bins of the pruned forward transform: for candidate i, its residue
// b_i (output 2 i) and M - b_i (output 2 i + 1).
__global__ void k_pr_bins(const int64_t* __restrict__ res, int64_t n, int64_t M, int64_t* __restrict__ bins) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  bins[2 * i] = res[i];
  bins[2 * i + 1] = (M - res[i]) % M;
}

// k_extract_pair on the pruned transform's outputs (x = X[2 i], y = X[2 i + 1]);
// scale null: one real sum given as samples (scale 1).
template <int WHICH>
__global__ void k_extract_pr(const int64_t* __restrict__ res, int64_t n, int64_t M, const float4* __restrict__ X,
                             const double* __restrict__ scale, double2* val, double* mag,
                             unsigned long long* maxbits) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float4 xs = X[2 * i], ys = X[2 * i + 1];
  const double xr = (double)xs.x + (double)xs.y, xi = (double)xs.z + (double)xs.w;
  const double yr = (double)ys.x + (double)ys.y, yi = (double)ys.z + (double)ys.w;
  const double sc = 0.5 / (double)M * (scale ? scale[WHICH] : 1.0);
  const double2 v = WHICH == 0 ? make_double2((xr + yr) * sc, (xi - yi) * sc)
                               : make_double2((xi + yi) * sc, (yr - xr) * sc);
  val[i] = v;
  const double m = hypot(v.x, v.y);
  mag[i] = m;
  atomicMax(maxbits, (unsigned long long)__double_as_longlong(m));
}

// Extraction, threshold and compaction of both sums in one launch (block k:
// sum k) for at most kExtractSmall candidates: the same values, the same
// threshold tau max|c| and the same candidate order as k_extract_pr, k_keep,
// the prefix sum and k_compact.
constexpr int kExtractSmall = 1024;

__global__ void __launch_bounds__(1024) k_extract_keep_pr(const int64_t* __restrict__ res, int64_t n, int64_t M,
                                                          const float4* __restrict__ X,
                                                          const double* __restrict__ scale, double tau,
                                                          const int32_t* __restrict__ cand, int d, int32_t* fo0,
                                                          double2* vo0, int32_t* fo1, double2* vo1, int64_t* total) {
  __shared__ double s_max[32];
  __shared__ int32_t s_wsum[32];
  __shared__ int32_t s_pos[kExtractSmall];
  const int k = blockIdx.x;
  const int i = threadIdx.x, lane = i & 31, w = i >> 5, nw = blockDim.x >> 5;
  double2 v = make_double2(0.0, 0.0);
  double m = 0.0;
  if (i < n) {
    const float4 xs = X[2 * i], ys = X[2 * i + 1];
    const double xr = (double)xs.x + (double)xs.y, xi = (double)xs.z + (double)xs.w;
    const double yr = (double)ys.x + (double)ys.y, yi = (double)ys.z + (double)ys.w;
    const double sc = 0.5 / (double)M * scale[k];
    v = k == 0 ? make_double2((xr + yr) * sc, (xi - yi) * sc) : make_double2((xi + yi) * sc, (yr - xr) * sc);
    m = hypot(v.x, v.y);
  }
  double mx = m;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) s_max[w] = mx;
  __syncthreads();
  mx = 0.0;
  for (int q = 0; q < nw; ++q) mx = fmax(mx, s_max[q]);
  const int keep = (i < n && m > tau * mx) ? 1 : 0;
  int x = keep;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_wsum[w] = x;
  __syncthreads();
  int before = 0, tot = 0;
  for (int q = 0; q < nw; ++q) {
    if (q < w) before += s_wsum[q];
    tot += s_wsum[q];
  }
  if (i == 0) total[k] = tot;
  int32_t* fo = k == 0 ? fo0 : fo1;
  double2* vo = k == 0 ? vo0 : vo1;
  if (i < n) s_pos[i] = keep ? before + x - 1 : -1;
  if (keep) vo[before + x - 1] = v;
  __syncthreads();
  // the kept frequencies, one warp per row (coalesced coordinates)
  for (int u = w; u < n; u += nw) {
    const int p = s_pos[u];
    if (p < 0) continue;
    for (int c = lane; c < d; c += 32) fo[(int64_t)p * d + c] = cand[(int64_t)u * d + c];
  }
}

// Pruned forward transform of s (P.prz, or the caller's real samples) at
// the 2 n_cand bins of the candidates' residues; X: device [2 n_cand].
ss_status pr_transform(const SftPlan& P, const void* s, bool real, const int64_t* res, int64_t n_cand, float4* X,
                       cudaStream_t st) {
  DevBuf<int64_t> bins;
  SS_TRY(bins.alloc_tmp(2 * n_cand, st));
  k_pr_bins<<<nblk(n_cand), 256, 0, st>>>(res, n_cand, P.M, bins.get());
  SS_LAUNCH_CHECK();
  const PrunedFormat fmt = P.prec == SS_FP64 ? (real ? PrunedFormat::kF64Real : PrunedFormat::kDfComplex)
                                             : (real ? PrunedFormat::kF32Real : PrunedFormat::kF32Complex);
  return pruned_forward(P.prt, s, fmt, bins.get(), 2 * n_cand, X, st);
}

// zh non-null: the bins come from the double-float spectrum zh (real part
// sum, as left by dff_round_trip) instead of a transform of samples.
// pr != 0: the pruned forward transform of P.prz (pr = 1: complex samples of
// one sum, scale P.prscale) or of the real FP64 samples (pr = 2).
ss_status recover_from(const SftPlan& P, const LatticeDev& L, const void* samples, const int32_t* cand, int64_t n_cand,
                       int64_t s_max, double tau, int32_t* freq_out, double* val_out, int64_t* n_out, cudaStream_t st,
                       const float4* zh = nullptr, int pr = 0) {
  DevBuf<int64_t> res, total;
  DevBuf<unsigned long long> table, maxbits;
  DevBuf<int32_t> flags, flag, pos;
  DevBuf<double2> val;
  DevBuf<double> mag;
  uint64_t cap = 1;
  while (cap < (uint64_t)(2 * n_cand)) cap <<= 1;
  SS_TRY(res.alloc_tmp(n_cand, st));
  SS_TRY(table.alloc_tmp(cap, st));
  SS_TRY(flags.alloc_tmp(4, st));
  SS_TRY(val.alloc_tmp(n_cand, st));
  SS_TRY(mag.alloc_tmp(n_cand, st));
  SS_TRY(maxbits.alloc_tmp(1, st));
  SS_TRY(flag.alloc_tmp(n_cand, st));
  SS_TRY(pos.alloc_tmp(n_cand, st));
  SS_TRY(total.alloc_tmp(1, st));
  SS_TRY(residues(cand, n_cand, L, res.get(), st));
  SS_TRY(check_reconstructing_async(cand, n_cand, L, res.get(), true, table.get(), cap, flags.get(), st));
  DevBuf<float4> X;
  if (pr) {
    SS_TRY(X.alloc_tmp(2 * n_cand, st));
    SS_TRY(pr_transform(P, pr == 1 ? (const void*)P.prz.get() : samples, pr == 2, res.get(), n_cand, X.get(), st));
  } else if (!zh) {
    cufftResult r = cufftSetStream(P.fft, st);
    if (r != CUFFT_SUCCESS) SS_FAIL(SS_ERR_CUDA, "cufftSetStream failed: %d", (int)r);
    if (P.prec == SS_FP64)
      r = cufftExecD2Z(P.fft, reinterpret_cast<cufftDoubleReal*>(const_cast<void*>(samples)),
                       reinterpret_cast<cufftDoubleComplex*>(P.spectrum.get()));
    else
      r = cufftExecR2C(P.fft, reinterpret_cast<cufftReal*>(const_cast<void*>(samples)),
                       reinterpret_cast<cufftComplex*>(P.spectrum.get()));
    if (r != CUFFT_SUCCESS) SS_FAIL(SS_ERR_CUDA, "cuFFT exec failed: %d", (int)r);
  }
  SS_CUDA(cudaMemsetAsync(maxbits.get(), 0, sizeof(unsigned long long), st));
  if (pr)
    k_extract_pr<0><<<nblk(n_cand), 256, 0, st>>>(res.get(), n_cand, L.M, X.get(), pr == 1 ? P.prscale.get() : nullptr,
                                                  val.get(), mag.get(), maxbits.get());
  else if (zh)
    k_extract_pair<0><<<nblk(n_cand), 256, 0, st>>>(cand, n_cand, L, zh, P.dfscale.get(), val.get(), mag.get(),
                                                    maxbits.get());
  else if (P.prec == SS_FP64)
    k_extract<double2><<<nblk(n_cand), 256, 0, st>>>(cand, n_cand, L, reinterpret_cast<const double2*>(P.spectrum.get()),
                                                     val.get(), mag.get(), maxbits.get());
  else
    k_extract<float2><<<nblk(n_cand), 256, 0, st>>>(cand, n_cand, L, reinterpret_cast<const float2*>(P.spectrum.get()),
                                                    val.get(), mag.get(), maxbits.get());
  k_keep<<<nblk(n_cand), 256, 0, st>>>(mag.get(), n_cand, maxbits.get(), tau, flag.get());
  SS_LAUNCH_CHECK();
  SS_TRY(exclusive_scan_i32(flag.get(), pos.get(), n_cand, total.get(), st));
  k_compact<<<nblk(n_cand), 256, 0, st>>>(cand, val.get(), n_cand, L.d, flag.get(), pos.get(), freq_out,
                                          reinterpret_cast<double2*>(val_out));
  SS_LAUNCH_CHECK();
  int64_t kept = 0;
  int32_t hf[4];
  SS_TRY(read_back(st, {{&kept, total.get(), sizeof(int64_t)}, {hf, flags.get(), sizeof(hf)}}));
  SS_TRY(reconstructing_status(hf, L.M));
  if (s_max > 0 && kept > s_max)
    SS_FAIL(SS_ERR_INVALID, "sft_recover: %lld terms above threshold exceed s_max = %lld", (long long)kept,
            (long long)s_max);
  *n_out = kept;
  return SS_OK;
}

// ---------------------------------------------------- support identification
//
// No candidate set: the kept bins are those of the half spectrum with
// |X_0[b]| > tau max |X_0|, and the coordinates of the frequency in bin b come
// from the d shifted lattices x_j + e_i / P: g(. + e_i / P) has the
// coefficients g_hat_k exp(2 pi i k_i / P), i.e. the same trigonometric sum
// with every coefficient c_t turned by exp(2 pi i p_{t,i} / P), so its spectrum
// satisfies X_i[b] / X_0[b] = exp(2 pi i k_i / P) and k_i is the nearest
// integer to P arg(X_i[b] / X_0[b]) / (2 pi), taken in (-P/2, P/2] (P > 2 max |k_i|).

template <typename T2>
__global__ void k_spec_max(const T2* __restrict__ spec, int64_t nh, unsigned long long* maxbits) {
  double m = 0.0;
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nh; b += (int64_t)gridDim.x * blockDim.x)
    m = fmax(m, hypot((double)spec[b].x, (double)spec[b].y));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(maxbits, (unsigned long long)__double_as_longlong(m));
}

template <typename T2>
__global__ void k_spec_keep(const T2* __restrict__ spec, int64_t nh, const unsigned long long* __restrict__ maxbits,
                            double tau, int32_t* flag) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nh) return;
  const double mx = __longlong_as_double((long long)*maxbits);
  flag[b] = hypot((double)spec[b].x, (double)spec[b].y) > tau * mx ? 1 : 0;
}

template <typename T2>
__global__ void k_spec_compact(const T2* __restrict__ spec, int64_t nh, const int32_t* __restrict__ flag,
                               const int32_t* __restrict__ pos, int64_t* bins, double2* x0) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nh || !flag[b]) return;
  bins[pos[b]] = b;
  x0[pos[b]] = make_double2((double)spec[b].x, (double)spec[b].y);
}

// c_t exp(2 pi i p_{t,i} / P)
__global__ void k_rotate_coef(const int32_t* __restrict__ freq, const double2* __restrict__ coef, int64_t n, int d,
                              int i, int P, double2* out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  double sn, cs;
  sincospi(2.0 * (double)freq[t * d + i] / (double)P, &sn, &cs);
  const double2 c = coef[t];
  out[t] = make_double2(c.x * cs - c.y * sn, c.x * sn + c.y * cs);
}

template <typename T2>
__global__ void k_identify_coord(const T2* __restrict__ spec, const int64_t* __restrict__ bins,
                                 const double2* __restrict__ x0, int64_t nb, int d, int i, int P, int32_t* kf) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nb) return;
  const T2 v = spec[bins[t]];
  const double2 a = x0[t];
  // arg(X_i / X_0) = arg(X_i conj(X_0))
  const double re = (double)v.x * a.x + (double)v.y * a.y, im = (double)v.y * a.x - (double)v.x * a.y;
  long long k = llrint((double)P * atan2(im, re) / (2.0 * 3.141592653589793)) % P;
  if (k < 0) k += P;
  if (2 * k > P) k -= P;
  kf[t * d + i] = (int32_t)k;
}

// valid[t]: the identified k reproduces its bin (k.z mod M == b); otherwise
// the bin holds an aliased tail or a collision.
__global__ void k_identify_check(const int32_t* __restrict__ kf, const int64_t* __restrict__ bins, int64_t nb,
                                 LatticeDev L, int32_t* valid, int32_t* err) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nb) return;
  const bool ok = residue_of(kf + t * L.d, L.d, L) == bins[t];
  valid[t] = ok ? 1 : 0;
  if (!ok) atomicExch(err, 1);
}

// Each valid bin's k, then -k (bin 0 alone), in increasing bin order.
__global__ void k_identify_write(const int32_t* __restrict__ kf, const int64_t* __restrict__ bins,
                                 const double2* __restrict__ x0, const int32_t* __restrict__ valid,
                                 const int32_t* __restrict__ vpos, int64_t nb, LatticeDev L, int32_t* fo,
                                 double2* vo) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nb || !valid[t]) return;
  const int d = L.d;
  const int64_t b = bins[t];
  const int64_t z0 = (bins[0] == 0 && valid[0]) ? 1 : 0;
  const int64_t o = b == 0 ? 0 : 2 * (int64_t)vpos[t] - z0;
  const double sc = 1.0 / (double)L.M;
  const double2 v = make_double2(x0[t].x * sc, x0[t].y * sc);
  for (int c = 0; c < d; ++c) fo[o * d + c] = kf[t * d + c];
  vo[o] = v;
  if (b != 0) {
    for (int c = 0; c < d; ++c) fo[(o + 1) * d + c] = -kf[t * d + c];
    vo[o + 1] = make_double2(v.x, -v.y);
  }
}

// Exact selection of the `keep` largest magnitudes among the flagged bins:
// the (keep+1)-th largest value is found digit by digit (eight 8-bit radix
// passes over the magnitudes' bit patterns, which order like the values for
// non-negative doubles), then only values strictly above it stay flagged.
struct RadixState {
  unsigned long long prefix, mask;
  long long k;
};

template <typename T2>
__global__ void k_mag_bits(const T2* __restrict__ spec, int64_t nh, unsigned long long* bits) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nh) return;
  bits[b] = (unsigned long long)__double_as_longlong(hypot((double)spec[b].x, (double)spec[b].y));
}

__global__ void k_radix_hist(const unsigned long long* __restrict__ bits, const int32_t* __restrict__ flag, int64_t nh,
                             const RadixState* __restrict__ st, int shift, unsigned int* hist) {
  __shared__ unsigned int sh[256];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) sh[i] = 0;
  __syncthreads();
  const unsigned long long prefix = st->prefix, mask = st->mask;
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nh; b += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long v = bits[b];
    if (flag[b] && (v & mask) == prefix) atomicAdd(&sh[(v >> shift) & 255u], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 256; i += blockDim.x)
    if (sh[i]) atomicAdd(hist + i, sh[i]);
}

__global__ void k_radix_pick(RadixState* st, int shift, unsigned int* hist) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  long long cum = 0;
  for (int dgt = 255; dgt >= 0; --dgt) {
    if (cum + (long long)hist[dgt] >= st->k) {
      st->prefix |= (unsigned long long)dgt << shift;
      st->mask |= 255ull << shift;
      st->k -= cum;
      break;
    }
    cum += hist[dgt];
  }
  for (int i = 0; i < 256; ++i) hist[i] = 0;
}

__global__ void k_radix_cut(const unsigned long long* __restrict__ bits, int64_t nh, const RadixState* __restrict__ st,
                            int32_t* flag) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nh) return;
  if (flag[b] && bits[b] <= st->prefix) flag[b] = 0;
}

ss_status exec_fft(const SftPlan& P, const void* samples, cudaStream_t st) {
  cufftResult r = cufftSetStream(P.fft, st);
  if (r != CUFFT_SUCCESS) SS_FAIL(SS_ERR_CUDA, "cufftSetStream failed: %d", (int)r);
  if (P.prec == SS_FP64)
    r = cufftExecD2Z(P.fft, reinterpret_cast<cufftDoubleReal*>(const_cast<void*>(samples)),
                     reinterpret_cast<cufftDoubleComplex*>(P.spectrum.get()));
  else
    r = cufftExecR2C(P.fft, reinterpret_cast<cufftReal*>(const_cast<void*>(samples)),
                     reinterpret_cast<cufftComplex*>(P.spectrum.get()));
  if (r != CUFFT_SUCCESS) SS_FAIL(SS_ERR_CUDA, "cuFFT exec failed: %d", (int)r);
  return SS_OK;
}

// Rows of the identification: row(i) leaves the samples of row i (0: the
// lattice, i >= 1: the lattice shifted by e_i / P) in device memory and
// returns them.
template <typename T2, class Rows>
ss_status identify_impl(const SftPlan& P, const LatticeDev& L, Rows row, int Pp, int64_t s_max, int64_t keep,
                        bool robust, double tau, int32_t* freq_out, double* val_out, int64_t* n_out, cudaStream_t st) {
  const int64_t nh = L.M / 2 + 1;
  const T2* spec = reinterpret_cast<const T2*>(P.spectrum.get());
  DevBuf<unsigned long long> maxbits;
  DevBuf<int32_t> flag, pos, err;
  DevBuf<int64_t> total, bins;
  DevBuf<double2> x0;
  SS_TRY(maxbits.alloc(1, st));
  SS_TRY(flag.alloc(nh, st));
  SS_TRY(pos.alloc(nh, st));
  SS_TRY(total.alloc(1, st));
  SS_TRY(err.alloc(1, st));
  const void* r0 = nullptr;
  SS_TRY(row(0, &r0));
  SS_TRY(exec_fft(P, r0, st));
  SS_CUDA(cudaMemsetAsync(maxbits.get(), 0, sizeof(unsigned long long), st));
  SS_CUDA(cudaMemsetAsync(err.get(), 0, sizeof(int32_t), st));
  const unsigned gmax = (unsigned)std::min<int64_t>(nblk(nh), 4 * 152);
  k_spec_max<T2><<<gmax, 256, 0, st>>>(spec, nh, maxbits.get());
  k_spec_keep<T2><<<nblk(nh), 256, 0, st>>>(spec, nh, maxbits.get(), tau, flag.get());
  SS_LAUNCH_CHECK();
  SS_TRY(exclusive_scan_i32(flag.get(), pos.get(), nh, total.get(), st));
  int64_t nb = 0;
  SS_CUDA(cudaMemcpyAsync(&nb, total.get(), sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  SS_CUDA(cudaStreamSynchronize(st));
  if (keep > 0 && nb > keep) {
    DevBuf<unsigned long long> bits;
    DevBuf<unsigned int> hist;
    DevBuf<RadixState> rs;
    SS_TRY(bits.alloc(nh, st));
    SS_TRY(hist.alloc(256, st));
    SS_TRY(rs.alloc(1, st));
    const RadixState init{0ull, 0ull, (long long)keep + 1};
    SS_CUDA(cudaMemcpyAsync(rs.get(), &init, sizeof(init), cudaMemcpyHostToDevice, st));
    SS_CUDA(cudaMemsetAsync(hist.get(), 0, 256 * sizeof(unsigned int), st));
    k_mag_bits<T2><<<nblk(nh), 256, 0, st>>>(spec, nh, bits.get());
    for (int shift = 56; shift >= 0; shift -= 8) {
      k_radix_hist<<<gmax, 256, 0, st>>>(bits.get(), flag.get(), nh, rs.get(), shift, hist.get());
      k_radix_pick<<<1, 32, 0, st>>>(rs.get(), shift, hist.get());
    }
    k_radix_cut<<<nblk(nh), 256, 0, st>>>(bits.get(), nh, rs.get(), flag.get());
    SS_LAUNCH_CHECK();
    SS_TRY(exclusive_scan_i32(flag.get(), pos.get(), nh, total.get(), st));
    SS_CUDA(cudaMemcpyAsync(&nb, total.get(), sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    SS_CUDA(cudaStreamSynchronize(st));
  }
  if (nb == 0) {
    *n_out = 0;
    return SS_OK;
  }
  if (!robust && s_max > 0 && 2 * nb - 1 > s_max)
    SS_FAIL(SS_ERR_INVALID, "sft_identify: at least %lld terms above threshold exceed s_max = %lld",
            (long long)(2 * nb - 1), (long long)s_max);
  SS_TRY(bins.alloc(nb, st));
  SS_TRY(x0.alloc(nb, st));
  k_spec_compact<T2><<<nblk(nh), 256, 0, st>>>(spec, nh, flag.get(), pos.get(), bins.get(), x0.get());
  SS_LAUNCH_CHECK();
  DevBuf<int32_t> kf, valid, vpos;
  SS_TRY(kf.alloc((size_t)nb * L.d, st));
  SS_TRY(valid.alloc(nb, st));
  SS_TRY(vpos.alloc(nb, st));
  for (int i = 0; i < L.d; ++i) {
    const void* ri = nullptr;
    SS_TRY(row(i + 1, &ri));
    SS_TRY(exec_fft(P, ri, st));
    k_identify_coord<T2><<<nblk(nb), 256, 0, st>>>(spec, bins.get(), x0.get(), nb, L.d, i, Pp, kf.get());
    SS_LAUNCH_CHECK();
  }
  k_identify_check<<<nblk(nb), 256, 0, st>>>(kf.get(), bins.get(), nb, L, valid.get(), err.get());
  SS_LAUNCH_CHECK();
  SS_TRY(exclusive_scan_i32(valid.get(), vpos.get(), nb, total.get(), st));
  int64_t nv = 0;
  int32_t herr = 0, z0 = 0;
  int64_t b0 = -1;
  SS_CUDA(cudaMemcpyAsync(&nv, total.get(), sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  SS_CUDA(cudaMemcpyAsync(&herr, err.get(), sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  SS_CUDA(cudaMemcpyAsync(&b0, bins.get(), sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  SS_CUDA(cudaMemcpyAsync(&z0, valid.get(), sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  SS_CUDA(cudaStreamSynchronize(st));
  if (herr && !robust)
    SS_FAIL(SS_ERR_NOT_RECONSTRUCTING, "sft_identify: a bin holds a frequency that does not map to it (collision)");
  const int64_t n = 2 * nv - ((b0 == 0 && z0) ? 1 : 0);
  if (s_max > 0 && n > s_max)
    SS_FAIL(SS_ERR_INVALID, "sft_identify: %lld terms exceed s_max = %lld", (long long)n, (long long)s_max);
  k_identify_write<<<nblk(nb), 256, 0, st>>>(kf.get(), bins.get(), x0.get(), valid.get(), vpos.get(), nb, L, freq_out,
                                             reinterpret_cast<double2*>(val_out));
  SS_LAUNCH_CHECK();
  SS_CUDA(cudaStreamSynchronize(st));
  *n_out = n;
  return SS_OK;
}

ss_status check_trig(const ss_trig* g, int d) {
  if (!g) SS_FAIL(SS_ERR_INVALID, "null trigonometric sum");
  if (g->d != d) SS_FAIL(SS_ERR_INVALID, "trigonometric sum has d = %d, lattice d = %d", g->d, d);
  if (g->n_terms < 0 || (g->n_terms > 0 && (!g->freq || !g->coef))) SS_FAIL(SS_ERR_INVALID, "bad trigonometric sum");
  return SS_OK;
}

}  // namespace

ss_status sft_recover_both(const ss_lattice* lat, const ss_trig* a, const ss_trig* f, ss_precision prec,
                           const int32_t* cand, int64_t n_cand, double tau, int32_t* a_freq, double* a_val,
                           int64_t* n_a, int32_t* f_freq, double* f_val, int64_t* n_f, cudaStream_t st) {
  LatticeDev L;
  SS_TRY(make_lattice_dev(lat, &L));
  SS_TRY(check_trig(a, L.d));
  SS_TRY(check_trig(f, L.d));
  if (!cand || n_cand < 1 || !a_freq || !a_val || !n_a || !f_freq || !f_val || !n_f)
    SS_FAIL(SS_ERR_INVALID, "sft_recover: bad argument");
  if (!(tau >= 0.0)) SS_FAIL(SS_ERR_INVALID, "sft_recover: tau must be >= 0");
  if (prec != SS_FP64 && prec != SS_FP32) SS_FAIL(SS_ERR_INVALID, "sft_recover: bad precision");
  std::shared_ptr<SftPlan> Pp;
  SS_TRY(get_plan(L.M, prec, st, &Pp));
  const SftPlan& P = *Pp;
  DevBuf<int64_t> res, total;
  DevBuf<unsigned long long> table, maxbits;
  DevBuf<int32_t> flags, flag, pos;
  DevBuf<double2> val;
  DevBuf<double> mag;
  uint64_t cap = 1;
  while (cap < (uint64_t)(2 * n_cand)) cap <<= 1;
  SS_TRY(res.alloc_tmp(n_cand, st));
  SS_TRY(table.alloc_tmp(cap, st));
  SS_TRY(flags.alloc_tmp(4, st));
  SS_TRY(val.alloc_tmp(n_cand, st));
  SS_TRY(mag.alloc_tmp(n_cand, st));
  SS_TRY(maxbits.alloc_tmp(2, st));
  SS_TRY(flag.alloc_tmp(n_cand, st));
  SS_TRY(pos.alloc_tmp(n_cand, st));
  SS_TRY(total.alloc_tmp(2, st));
  // one candidate set and one lattice: residues and the check once
  SS_TRY(residues(cand, n_cand, L, res.get(), st));
  SS_TRY(check_reconstructing_async(cand, n_cand, L, res.get(), true, table.get(), cap, flags.get(), st));
  cufftResult r = cufftSetStream(P.fft, st);
  if (r != CUFFT_SUCCESS) SS_FAIL(SS_ERR_CUDA, "cufftSetStream failed: %d", (int)r);
  SS_CUDA(cudaMemsetAsync(maxbits.get(), 0, 2 * sizeof(unsigned long long), st));
  const ss_trig* g[2] = {a, f};
  int32_t* fo[2] = {a_freq, f_freq};
  double* vo[2] = {a_val, f_val};
  if (P.has_pr) {
    // a long 7-smooth lattice: both sums sampled by one sparse evaluation
    // and recovered by one pruned forward transform
    SS_TRY(pr_sample_pair(P, L, a, f, st));
    DevBuf<float4> X;
    SS_TRY(X.alloc_tmp(2 * n_cand, st));
    SS_TRY(pr_transform(P, P.prz.get(), false, res.get(), n_cand, X.get(), st));
    if (n_cand <= kExtractSmall) {
      ProfScope prof_("extract", st);
      k_extract_keep_pr<<<2, 1024, 0, st>>>(res.get(), n_cand, L.M, X.get(), P.prscale.get(), tau, cand, L.d,
                                           fo[0], reinterpret_cast<double2*>(vo[0]), fo[1],
                                           reinterpret_cast<double2*>(vo[1]), total.get());
      SS_LAUNCH_CHECK();
    }
    for (int k = 0; k < 2 && n_cand > kExtractSmall; ++k) {
      if (k == 0)
        k_extract_pr<0><<<nblk(n_cand), 256, 0, st>>>(res.get(), n_cand, L.M, X.get(), P.prscale.get(), val.get(),
                                                      mag.get(), maxbits.get());
      else
        k_extract_pr<1><<<nblk(n_cand), 256, 0, st>>>(res.get(), n_cand, L.M, X.get(), P.prscale.get(), val.get(),
                                                      mag.get(), maxbits.get() + 1);
      k_keep<<<nblk(n_cand), 256, 0, st>>>(mag.get(), n_cand, maxbits.get() + k, tau, flag.get());
      SS_LAUNCH_CHECK();
      SS_TRY(exclusive_scan_i32(flag.get(), pos.get(), n_cand, total.get() + k, st));
      k_compact<<<nblk(n_cand), 256, 0, st>>>(cand, val.get(), n_cand, L.d, flag.get(), pos.get(), fo[k],
                                              reinterpret_cast<double2*>(vo[k]));
      SS_LAUNCH_CHECK();
    }
  }
  if (P.has_dff) {
    // FP64: both sums sampled by one inverse and recovered by one forward
    // double-float transform of length M
    SS_TRY(dff_round_trip(P, L, a, f, st));
    const float4* Z = P.dfz.get();
    for (int k = 0; k < 2; ++k) {
      if (k == 0)
        k_extract_pair<0><<<nblk(n_cand), 256, 0, st>>>(cand, n_cand, L, Z, P.dfscale.get(), val.get(), mag.get(),
                                                        maxbits.get());
      else
        k_extract_pair<1><<<nblk(n_cand), 256, 0, st>>>(cand, n_cand, L, Z, P.dfscale.get(), val.get(), mag.get(),
                                                        maxbits.get() + 1);
      k_keep<<<nblk(n_cand), 256, 0, st>>>(mag.get(), n_cand, maxbits.get() + k, tau, flag.get());
      SS_LAUNCH_CHECK();
      SS_TRY(exclusive_scan_i32(flag.get(), pos.get(), n_cand, total.get() + k, st));
      k_compact<<<nblk(n_cand), 256, 0, st>>>(cand, val.get(), n_cand, L.d, flag.get(), pos.get(), fo[k],
                                              reinterpret_cast<double2*>(vo[k]));
      SS_LAUNCH_CHECK();
    }
  }
  if (!P.has_dff && !P.has_pr && use_pair32(P)) {
    SS_TRY(ensure_pair32(P, st));
    SS_TRY(sample_into(P, L, a, P.samples.get(), st));
    SS_TRY(sample_into(P, L, f, P.samples2.get(), st));
    double* scale = P.scale32.get();
    k_pair_scale_n<<<1, kScaleThreads, 0, st>>>(reinterpret_cast<const double2*>(a->coef), a->n_terms,
                                                reinterpret_cast<const double2*>(f->coef), f->n_terms, scale);
    float2* z = P.z32.get();
    k_pack_pair32<<<nblk(P.M), 256, 0, st>>>(reinterpret_cast<const float*>(P.samples.get()), P.samples2.get(),
                                             scale, P.M, z);
    SS_LAUNCH_CHECK();
    r = cufftSetStream(P.c2c, st);
    if (r == CUFFT_SUCCESS)
      r = cufftExecC2C(P.c2c, reinterpret_cast<cufftComplex*>(z), reinterpret_cast<cufftComplex*>(z), CUFFT_FORWARD);
    if (r != CUFFT_SUCCESS) SS_FAIL(SS_ERR_CUDA, "cuFFT C2C exec failed: %d", (int)r);
    for (int k = 0; k < 2; ++k) {
      if (k == 0)
        k_extract_pair32<0><<<nblk(n_cand), 256, 0, st>>>(cand, n_cand, L, z, scale, val.get(), mag.get(),
                                                          maxbits.get());
      else
        k_extract_pair32<1><<<nblk(n_cand), 256, 0, st>>>(cand, n_cand, L, z, scale, val.get(), mag.get(),
                                                          maxbits.get() + 1);
      k_keep<<<nblk(n_cand), 256, 0, st>>>(mag.get(), n_cand, maxbits.get() + k, tau, flag.get());
      SS_LAUNCH_CHECK();
      SS_TRY(exclusive_scan_i32(flag.get(), pos.get(), n_cand, total.get() + k, st));
      k_compact<<<nblk(n_cand), 256, 0, st>>>(cand, val.get(), n_cand, L.d, flag.get(), pos.get(), fo[k],
                                              reinterpret_cast<double2*>(vo[k]));
      SS_LAUNCH_CHECK();
    }
  }
  for (int k = 0; k < 2 && !P.has_dff && !P.has_pr && !use_pair32(P); ++k) {
    // the plan's sample and spectrum buffers serve both sums in stream order
    SS_TRY(sample_into(P, L, g[k], P.samples.get(), st));
    if (P.prec == SS_FP64)
      r = cufftExecD2Z(P.fft, reinterpret_cast<cufftDoubleReal*>(P.samples.get()),
                       reinterpret_cast<cufftDoubleComplex*>(P.spectrum.get()));
    else
      r = cufftExecR2C(P.fft, reinterpret_cast<cufftReal*>(P.samples.get()),
                       reinterpret_cast<cufftComplex*>(P.spectrum.get()));
    if (r != CUFFT_SUCCESS) SS_FAIL(SS_ERR_CUDA, "cuFFT exec failed: %d", (int)r);
    if (P.prec == SS_FP64)
      k_extract<double2><<<nblk(n_cand), 256, 0, st>>>(cand, n_cand, L,
                                                       reinterpret_cast<const double2*>(P.spectrum.get()), val.get(),
                                                       mag.get(), maxbits.get() + k);
    else
      k_extract<float2><<<nblk(n_cand), 256, 0, st>>>(cand, n_cand, L,
                                                      reinterpret_cast<const float2*>(P.spectrum.get()), val.get(),
                                                      mag.get(), maxbits.get() + k);
    k_keep<<<nblk(n_cand), 256, 0, st>>>(mag.get(), n_cand, maxbits.get() + k, tau, flag.get());
    SS_LAUNCH_CHECK();
    SS_TRY(exclusive_scan_i32(flag.get(), pos.get(), n_cand, total.get() + k, st));
    k_compact<<<nblk(n_cand), 256, 0, st>>>(cand, val.get(), n_cand, L.d, flag.get(), pos.get(), fo[k],
                                            reinterpret_cast<double2*>(vo[k]));
    SS_LAUNCH_CHECK();
  }
  int64_t kept[2] = {0, 0};
  int32_t hf[4];
  SS_TRY(read_back(st, {{kept, total.get(), sizeof(kept)}, {hf, flags.get(), sizeof(hf)}}));
  SS_TRY(reconstructing_status(hf, L.M));
  *n_a = kept[0];
  *n_f = kept[1];
  return SS_OK;
}

}  // namespace ss

using namespace ss;

extern "C" ss_status lattice_sample(const ss_lattice* lat, const ss_trig* g, ss_precision prec, void* samples,
                                    void* stream) {
  LatticeDev L;
  SS_TRY(make_lattice_dev(lat, &L));
  SS_TRY(check_trig(g, L.d));
  if (!samples) SS_FAIL(SS_ERR_INVALID, "lattice_sample: null output");
  if (prec != SS_FP64 && prec != SS_FP32) SS_FAIL(SS_ERR_INVALID, "lattice_sample: bad precision");
  cudaStream_t st = as_stream(stream);
  std::shared_ptr<SftPlan> P;
  SS_TRY(get_plan(L.M, prec, st, &P));
  return sample_into(*P, L, g, samples, st);
}

extern "C" ss_status sft_recover_samples(const ss_lattice* lat, const void* samples, ss_precision prec,
                                         const int32_t* cand, int64_t n_cand, int64_t s_max, double tau,
                                         int32_t* freq_out, double* val_out, int64_t* n_out, void* stream) {
  LatticeDev L;
  SS_TRY(make_lattice_dev(lat, &L));
  if (!samples || !cand || !freq_out || !val_out || !n_out || n_cand < 1)
    SS_FAIL(SS_ERR_INVALID, "sft_recover_samples: bad argument");
  if (!(tau >= 0.0)) SS_FAIL(SS_ERR_INVALID, "sft_recover_samples: tau must be >= 0");
  if (prec != SS_FP64 && prec != SS_FP32) SS_FAIL(SS_ERR_INVALID, "sft_recover_samples: bad precision");
  cudaStream_t st = as_stream(stream);
  std::shared_ptr<SftPlan> P;
  SS_TRY(get_plan(L.M, prec, st, &P));
  if (P->has_pr)
    return recover_from(*P, L, samples, cand, n_cand, s_max, tau, freq_out, val_out, n_out, st, nullptr, 2);
  return recover_from(*P, L, samples, cand, n_cand, s_max, tau, freq_out, val_out, n_out, st);
}

extern "C" ss_status sft_recover(const ss_lattice* lat, const ss_trig* g, ss_precision prec, const int32_t* cand,
                                 int64_t n_cand, int64_t s_max, double tau, int32_t* freq_out, double* val_out,
                                 int64_t* n_out, void* stream) {
  LatticeDev L;
  SS_TRY(make_lattice_dev(lat, &L));
  SS_TRY(check_trig(g, L.d));
  if (!cand || !freq_out || !val_out || !n_out || n_cand < 1) SS_FAIL(SS_ERR_INVALID, "sft_recover: bad argument");
  if (!(tau >= 0.0)) SS_FAIL(SS_ERR_INVALID, "sft_recover: tau must be >= 0");
  if (prec != SS_FP64 && prec != SS_FP32) SS_FAIL(SS_ERR_INVALID, "sft_recover: bad precision");
  cudaStream_t st = as_stream(stream);
  std::shared_ptr<SftPlan> P;
  SS_TRY(get_plan(L.M, prec, st, &P));
  if (P->has_dff) {
    SS_TRY(dff_round_trip(*P, L, g, nullptr, st));
    return recover_from(*P, L, nullptr, cand, n_cand, s_max, tau, freq_out, val_out, n_out, st, P->dfz.get());
  }
  if (P->has_pr) {
    SS_TRY(pr_sample_pair(*P, L, g, nullptr, st));
    return recover_from(*P, L, nullptr, cand, n_cand, s_max, tau, freq_out, val_out, n_out, st, nullptr, 1);
  }
  SS_TRY(sample_into(*P, L, g, P->samples.get(), st));
  return recover_from(*P, L, P->samples.get(), cand, n_cand, s_max, tau, freq_out, val_out, n_out, st);
}

extern "C" ss_status sft_identify(const ss_lattice* lat, const ss_trig* g, ss_precision prec, int32_t P,
                                  int64_t s_max, double tau, int32_t* freq_out, double* val_out, int64_t* n_out,
                                  void* stream) {
  LatticeDev L;
  SS_TRY(make_lattice_dev(lat, &L));
  SS_TRY(check_trig(g, L.d));
  if (!freq_out || !val_out || !n_out || s_max < 1) SS_FAIL(SS_ERR_INVALID, "sft_identify: bad argument");
  if (P < 3) SS_FAIL(SS_ERR_INVALID, "sft_identify: P must be > 2 max |k_i| >= 3");
  if (!(tau >= 0.0)) SS_FAIL(SS_ERR_INVALID, "sft_identify: tau must be >= 0");
  if (prec != SS_FP64 && prec != SS_FP32) SS_FAIL(SS_ERR_INVALID, "sft_identify: bad precision");
  cudaStream_t st = as_stream(stream);
  std::shared_ptr<SftPlan> Pl;
  SS_TRY(get_plan(L.M, prec, st, &Pl));
  DevBuf<double2> rot;
  SS_TRY(rot.alloc(std::max<int64_t>(g->n_terms, 1), st));
  const SftPlan& PP = *Pl;
  // row 0: g on the lattice; row i: the coefficients turned by exp(2 pi i p_i / P)
  auto rows = [&](int i, const void** out) -> ss_status {
    if (i == 0) {
      SS_TRY(sample_into(PP, L, g, PP.samples.get(), st));
    } else {
      k_rotate_coef<<<nblk(g->n_terms), 256, 0, st>>>(g->freq, reinterpret_cast<const double2*>(g->coef),
                                                      g->n_terms, L.d, i - 1, P, rot.get());
      SS_LAUNCH_CHECK();
      const ss_trig gi{g->d, g->n_terms, g->freq, reinterpret_cast<const double*>(rot.get())};
      SS_TRY(sample_into(PP, L, &gi, PP.samples.get(), st));
    }
    *out = PP.samples.get();
    return SS_OK;
  };
  if (prec == SS_FP64)
    return identify_impl<double2>(PP, L, rows, P, s_max, 0, false, tau, freq_out, val_out, n_out, st);
  return identify_impl<float2>(PP, L, rows, P, s_max, 0, false, tau, freq_out, val_out, n_out, st);
}

extern "C" ss_status sft_identify_samples(const ss_lattice* lat, int32_t P, const void* samples, ss_precision prec,
                                          int64_t s_max, double tau, int64_t keep, int32_t robust, int32_t* freq_out,
                                          double* val_out, int64_t* n_out, void* stream) {
  LatticeDev L;
  SS_TRY(make_lattice_dev(lat, &L));
  if (!samples || !freq_out || !val_out || !n_out || s_max < 1 || keep < 0)
    SS_FAIL(SS_ERR_INVALID, "sft_identify_samples: bad argument");
  if (P < 3) SS_FAIL(SS_ERR_INVALID, "sft_identify_samples: P must be > 2 max |k_i| >= 3");
  if (!(tau >= 0.0)) SS_FAIL(SS_ERR_INVALID, "sft_identify_samples: tau must be >= 0");
  if (prec != SS_FP64 && prec != SS_FP32) SS_FAIL(SS_ERR_INVALID, "sft_identify_samples: bad precision");
  cudaStream_t st = as_stream(stream);
  std::shared_ptr<SftPlan> Pl;
  SS_TRY(get_plan(L.M, prec, st, &Pl));
  const size_t es = prec == SS_FP64 ? sizeof(double) : sizeof(float);
  // rows are copied into the plan's aligned sample buffer (cuFFT's real input
  // wants more than element alignment, and row i starts at i * M elements)
  auto rows = [&](int i, const void** out) -> ss_status {
    SS_CUDA(cudaMemcpyAsync(Pl->samples.get(), static_cast<const unsigned char*>(samples) + (size_t)i * (size_t)L.M * es,
                            (size_t)L.M * es, cudaMemcpyDeviceToDevice, st));
    *out = Pl->samples.get();
    return SS_OK;
  };
  if (prec == SS_FP64)
    return identify_impl<double2>(*Pl, L, rows, P, s_max, keep, robust != 0, tau, freq_out, val_out, n_out, st);
  return identify_impl<float2>(*Pl, L, rows, P, s_max, keep, robust != 0, tau, freq_out, val_out, n_out, st);
}
