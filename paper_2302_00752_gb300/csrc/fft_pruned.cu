// Pruned DFTs of a 7-smooth length M (the split, the index maps and the cost
// are stated in fft_pruned.cuh), in double-float arithmetic (the FP64
// recovery) or in FP32 (the FP32 recovery).
//
// Inside a block a tile holds W columns of length P in shared memory, column c
// at c (P + 1) (one element of padding: threads that share a row offset and
// differ in the column hit distinct banks).  The length-P transforms run as
// self-sorting (Stockham) radix passes over all W columns at once, thread u
// taking column u mod W, butterfly u / W, with the P-th roots staged in
// shared memory.  The arithmetic is a policy (ArDF: complex double-float
// values as float4 and the butterflies of dfc.cuh; ArF32: float2).  All sums
// run in a fixed order, so results are bit-reproducible.
#include <algorithm>
#include <cmath>

#include "dfc.cuh"
#include "fft_pruned.cuh"

namespace ss {
namespace {

using namespace dfc;

constexpr int kPrTile = 2048;      // complex values of one tile (W columns x P rows), forward transform
constexpr int kPrEvalTile = 2048;  // the same for the evaluation
constexpr int kPrEvalStage = 1024; // step powers (entries x W) staged in shared memory up to this count
constexpr int kPrThreads = 256;
constexpr int kPrChunk = 256;      // entries staged in shared memory per round of the evaluation
constexpr int kPrMaxOut = 1024;    // outputs per forward launch (accumulators in shared memory)
constexpr int kPrMaxP = 1024;

inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

__device__ __forceinline__ C4 conj4(const C4 a) { return C4{a.re, df_neg(a.im)}; }
__device__ __forceinline__ C4 zero4() { return C4{DF{0.f, 0.f}, DF{0.f, 0.f}}; }

// exp(sign 2 pi i r / M), r < M, from the two-level double-float table
template <int SIGN>
__device__ __forceinline__ C4 tw2(const float4* __restrict__ t0, const float4* __restrict__ t1, int b, uint64_t r) {
  const C4 w = cmul(ld(__ldg(t1 + (r >> b))), ld(__ldg(t0 + (r & ((1ull << b) - 1)))));
  return SIGN > 0 ? w : conj4(w);
}

// ------------------------------------------------------------ FP32 complex

__device__ __forceinline__ float2 fadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 fsub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 fmul(float2 a, float2 w) {
  return make_float2(fmaf(a.x, w.x, -a.y * w.y), fmaf(a.x, w.y, a.y * w.x));
}
__device__ __forceinline__ float2 fconj(float2 a) { return make_float2(a.x, -a.y); }
template <int SIGN>
__device__ __forceinline__ float2 fmul_si(float2 a) {   // a * (sign i)
  return SIGN > 0 ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

template <int SIGN>
__device__ __forceinline__ void fdft4(float2& v0, float2& v1, float2& v2, float2& v3) {
  const float2 t0 = fadd(v0, v2), t1 = fsub(v0, v2), t2 = fadd(v1, v3), t3 = fmul_si<SIGN>(fsub(v1, v3));
  v0 = fadd(t0, t2);
  v2 = fsub(t0, t2);
  v1 = fadd(t1, t3);
  v3 = fsub(t1, t3);
}

// R-point DFT in place, the same forms as dfc.cuh's: cs[m - 1] =
// exp(2 pi i m / R), m <= (R - 1) / 2; for R = 8, cs[0] = exp(2 pi i / 8).
template <int R, int SIGN>
__device__ __forceinline__ void fdft(float2 (&v)[R], const float2* cs) {
  if constexpr (R == 2) {
    const float2 a = v[0];
    v[0] = fadd(a, v[1]);
    v[1] = fsub(a, v[1]);
  } else if constexpr (R == 4) {
    fdft4<SIGN>(v[0], v[1], v[2], v[3]);
  } else if constexpr (R == 8) {
    float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6], o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    fdft4<SIGN>(e0, e1, e2, e3);
    fdft4<SIGN>(o0, o1, o2, o3);
    const float c = cs[0].x;   // cos(pi / 4)
    const float sg1 = SIGN > 0 ? o1.x : -o1.x, sh1 = SIGN > 0 ? o1.y : -o1.y;
    o1 = make_float2(c * (o1.x - sh1), c * (o1.y + sg1));
    o2 = fmul_si<SIGN>(o2);
    const float sg3 = SIGN > 0 ? o3.x : -o3.x, sh3 = SIGN > 0 ? o3.y : -o3.y;
    o3 = make_float2(-c * (o3.x + sh3), c * (sg3 - o3.y));
    v[0] = fadd(e0, o0);
    v[4] = fsub(e0, o0);
    v[1] = fadd(e1, o1);
    v[5] = fsub(e1, o1);
    v[2] = fadd(e2, o2);
    v[6] = fsub(e2, o2);
    v[3] = fadd(e3, o3);
    v[7] = fsub(e3, o3);
  } else {
    constexpr int H = (R - 1) / 2;
    float2 a[H], b[H];
#pragma unroll
    for (int r = 1; r <= H; ++r) {
      a[r - 1] = fadd(v[r], v[R - r]);
      b[r - 1] = fsub(v[r], v[R - r]);
    }
    const float2 v0 = v[0];
    float2 y0 = v0;
#pragma unroll
    for (int r = 0; r < H; ++r) y0 = fadd(y0, a[r]);
#pragma unroll
    for (int s = 1; s <= H; ++s) {
      float2 A = v0, Bv = make_float2(0.f, 0.f);
#pragma unroll
      for (int r = 1; r <= H; ++r) {
        const int m = (r * s) % R;
        const int mm = m <= H ? m : R - m;
        const float cm = cs[mm - 1].x;
        const float sm = m <= H ? cs[mm - 1].y : -cs[mm - 1].y;
        A.x = fmaf(cm, a[r - 1].x, A.x);
        A.y = fmaf(cm, a[r - 1].y, A.y);
        Bv.x = fmaf(sm, b[r - 1].x, Bv.x);
        Bv.y = fmaf(sm, b[r - 1].y, Bv.y);
      }
      const float2 iB = fmul_si<SIGN>(Bv);
      v[s] = fadd(A, iB);
      v[R - s] = fsub(A, iB);
    }
    v[0] = y0;
  }
}

// 16-point DFT as dft16 below, on FP32 complex values; output X[k1 + 4 k2]
// at v[4 k1 + k2].
template <int SIGN>
__device__ __forceinline__ void fdft16(float2 (&v)[16], const float2 w1, const float2 w2, const float2 w3) {
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) fdft4<SIGN>(v[n2], v[n2 + 4], v[n2 + 8], v[n2 + 12]);
  auto tw = [](const float2 a, const float2 w) { return fmul(a, SIGN > 0 ? w : fconj(w)); };
  v[5] = tw(v[5], w1);
  v[9] = tw(v[9], w2);
  v[13] = tw(v[13], w3);
  v[6] = tw(v[6], w2);
  v[10] = fmul_si<SIGN>(v[10]);
  v[14] = fmul_si<SIGN>(tw(v[14], w2));
  v[7] = tw(v[7], w3);
  v[11] = fmul_si<SIGN>(tw(v[11], w2));
  {
    const float2 t = tw(v[15], w1);
    v[15] = make_float2(-t.x, -t.y);
  }
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) fdft4<SIGN>(v[4 * k1], v[4 * k1 + 1], v[4 * k1 + 2], v[4 * k1 + 3]);
}

// 16-point DFT in place (SIGN: exponent sign), natural input order; the
// output X[k1 + 4 k2] ends at v[4 k1 + k2].  w1, w2, w3 = exp(2 pi i j / 16).
// Four 4-point transforms (stride 4), the twiddles w16^(n2 k1), four more.
template <int SIGN>
__device__ __forceinline__ void dft16(C4 (&v)[16], const C4 w1, const C4 w2, const C4 w3) {
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) dft4<SIGN>(v[n2], v[n2 + 4], v[n2 + 8], v[n2 + 12]);
  auto tw = [](const C4 a, const C4 w) { return cmul(a, SIGN > 0 ? w : conj4(w)); };
  v[5] = tw(v[5], w1);
  v[9] = tw(v[9], w2);
  v[13] = tw(v[13], w3);
  v[6] = tw(v[6], w2);
  v[10] = mul_si<SIGN>(v[10]);
  v[14] = mul_si<SIGN>(tw(v[14], w2));   // w16^6 = i w16^2
  v[7] = tw(v[7], w3);
  v[11] = mul_si<SIGN>(tw(v[11], w2));
  {
    const C4 t = tw(v[15], w1);   // w16^9 = -w16^1
    v[15] = C4{df_neg(t.re), df_neg(t.im)};
  }
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) dft4<SIGN>(v[4 * k1], v[4 * k1 + 1], v[4 * k1 + 2], v[4 * k1 + 3]);
}

// ------------------------------------------------------- arithmetic policies

// Double-float complex values stored as float4 (re.hi, re.lo, im.hi, im.lo).
struct ArDF {
  using V = float4;
  using C = C4;
  static constexpr int kMinBlocks16 = 2;   // resident blocks per SM of the 4096-value-tile kernels
  static __device__ __forceinline__ C ld(const V v) { return dfc::ld(v); }
  static __device__ __forceinline__ V st(const C c) { return st4(c); }
  static __device__ __forceinline__ C add(const C a, const C b) { return cadd(a, b); }
  static __device__ __forceinline__ C mul(const C a, const C b) { return cmul(a, b); }
  static __device__ __forceinline__ C conj(const C a) { return conj4(a); }
  static __device__ __forceinline__ C zero() { return zero4(); }
  // a double-float table or entry value
  static __device__ __forceinline__ C from_df(const float4 v) { return dfc::ld(v); }
  template <int SIGN>
  static __device__ __forceinline__ C root(const float4* t0, const float4* t1, int b, uint64_t r) {
    return tw2<SIGN>(t0, t1, b, r);
  }
  template <int R, int SIGN>
  static __device__ __forceinline__ void dft(C (&v)[R], const C* cs) {
    dfc::dft<R, SIGN>(v, cs);
  }
  template <int SIGN>
  static __device__ __forceinline__ void dft16(C (&v)[16], const C w1, const C w2, const C w3) {
    ss::dft16<SIGN>(v, w1, w2, w3);
  }
  static __device__ __forceinline__ double2 to_double2(const V v) {
    return make_double2((double)v.x + (double)v.y, (double)v.z + (double)v.w);
  }
  using Real = double;   // real samples: FP64
  static __device__ __forceinline__ C from_real(const double x) { return C4{df_split(x), DF{0.f, 0.f}}; }
  static __device__ __forceinline__ double real_out(const V v) { return (double)v.x + (double)v.y; }
};

// FP32 complex values (the high words of the double-float tables and entries).
struct ArF32 {
  using V = float2;
  using C = float2;
  static constexpr int kMinBlocks16 = 3;
  static __device__ __forceinline__ C ld(const V v) { return v; }
  static __device__ __forceinline__ V st(const C c) { return c; }
  static __device__ __forceinline__ C add(const C a, const C b) { return fadd(a, b); }
  static __device__ __forceinline__ C mul(const C a, const C b) { return fmul(a, b); }
  static __device__ __forceinline__ C conj(const C a) { return fconj(a); }
  static __device__ __forceinline__ C zero() { return make_float2(0.f, 0.f); }
  static __device__ __forceinline__ C from_df(const float4 v) { return make_float2(v.x, v.z); }
  template <int SIGN>
  static __device__ __forceinline__ C root(const float4* t0, const float4* t1, int b, uint64_t r) {
    const float4 u = __ldg(t1 + (r >> b)), l = __ldg(t0 + (r & ((1ull << b) - 1)));
    const float2 w = fmul(make_float2(u.x, u.z), make_float2(l.x, l.z));
    return SIGN > 0 ? w : fconj(w);
  }
  template <int R, int SIGN>
  static __device__ __forceinline__ void dft(C (&v)[R], const C* cs) {
    fdft<R, SIGN>(v, cs);
  }
  template <int SIGN>
  static __device__ __forceinline__ void dft16(C (&v)[16], const C w1, const C w2, const C w3) {
    fdft16<SIGN>(v, w1, w2, w3);
  }
  static __device__ __forceinline__ double2 to_double2(const V v) { return make_double2(v.x, v.y); }
  using Real = float;    // real samples: FP32
  static __device__ __forceinline__ C from_real(const float x) { return make_float2(x, 0.f); }
  static __device__ __forceinline__ float real_out(const V v) { return v.x; }
};

__global__ void k_tl_table(int64_t M, int b, int64_t n1, float4* t0, float4* t1) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double s, c;
  if (i < (1ll << b)) {
    sincospi(2.0 * (double)i / (double)M, &s, &c);
    const DF cc = df_split(c), sn = df_split(s);
    t0[i] = make_float4(cc.hi, cc.lo, sn.hi, sn.lo);
  }
  if (i < n1) {
    sincospi(2.0 * (double)(i << b) / (double)M, &s, &c);
    const DF cc = df_split(c), sn = df_split(s);
    t1[i] = make_float4(cc.hi, cc.lo, sn.hi, sn.lo);
  }
}

// One radix-R Stockham pass over the W = 2^wsh columns (length P, column
// stride CS).  j / Ns is formed as umulhi(j, ceil(2^32 / Ns)), exact for
// j, Ns < 2^16.
template <class A, int R, int SIGN>
__device__ __forceinline__ void mpass(const typename A::V* __restrict__ a, typename A::V* __restrict__ b, int P,
                                      int wsh, int CS, int Ns, const typename A::V* __restrict__ tw) {
  using C = typename A::C;
  constexpr int NC = R == 8 ? 1 : (R - 1) / 2;
  C cs[NC > 0 ? NC : 1];
#pragma unroll
  for (int m = 0; m < NC; ++m) cs[m] = A::ld(tw[(P / R) * (m + 1)]);
  const int nb = P / R;
  const int tstride = P / (Ns * R);
  const int total = nb << wsh;
  const unsigned wmask = (1u << wsh) - 1u;
  const unsigned nsm = Ns > 1 ? 0xffffffffu / (unsigned)Ns + 1u : 0u;
  for (int u = threadIdx.x; u < total; u += blockDim.x) {
    const int c = (int)((unsigned)u & wmask), j = u >> wsh;
    const typename A::V* ac = a + c * CS;
    typename A::V* bc = b + c * CS;
    const int jq = Ns > 1 ? (int)__umulhi((unsigned)j, nsm) : j;   // j / Ns
    const int k = j - jq * Ns;
    C v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = A::ld(ac[j + r * nb]);
    if (Ns > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        const C w = A::ld(tw[tstride * (k * r)]);
        v[r] = A::mul(v[r], SIGN > 0 ? w : A::conj(w));
      }
    }
    A::template dft<R, SIGN>(v, cs);
    const int base = jq * Ns * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) bc[base + r * Ns] = A::st(v[r]);
  }
}

// Length-P transforms of the W columns in `a` (b: the other buffer); returns
// the buffer that holds the result.  Ends with a block barrier.
template <class A, int SIGN>
__device__ typename A::V* columns_dft(typename A::V* a, typename A::V* b, int P, int wsh, int CS,
                                      const DfRadices& rad, const typename A::V* __restrict__ tw) {
  int Ns = 1;
  for (int p = 0; p < rad.n; ++p) {
    const int R = rad.r[p];
    switch (R) {
      case 8: mpass<A, 8, SIGN>(a, b, P, wsh, CS, Ns, tw); break;
      case 4: mpass<A, 4, SIGN>(a, b, P, wsh, CS, Ns, tw); break;
      case 2: mpass<A, 2, SIGN>(a, b, P, wsh, CS, Ns, tw); break;
      case 5: mpass<A, 5, SIGN>(a, b, P, wsh, CS, Ns, tw); break;
      case 3: mpass<A, 3, SIGN>(a, b, P, wsh, CS, Ns, tw); break;
      default: mpass<A, 7, SIGN>(a, b, P, wsh, CS, Ns, tw); break;
    }
    __syncthreads();
    typename A::V* t = a;
    a = b;
    b = t;
    Ns *= R;
  }
  return a;
}

// Entries of the spectrum Z = S_a / scale[0] + i S_f / scale[1] (S_a, S_f the
// Hermitian spectra of the two real sums: a term (r, c) puts c / 2 at r and
// conj(c) / 2 at M - r, or Re c at r when r = 0 or 2 r = M), bucketed by
// r mod P in term order (a's terms, then f's; r before M - r).  One block;
// boff[k] = first entry of bucket k, boff[P] = the number of entries.
// kq: scratch of 2 (na + nf) int32 (the two buckets of every term).
__global__ void k_pr_entries(const int64_t* __restrict__ qa, const double2* __restrict__ ca,
                             const int64_t* __restrict__ na_dev, const int64_t* __restrict__ qf,
                             const double2* __restrict__ cf, const int64_t* __restrict__ nf_dev,
                             const double* __restrict__ scale, int64_t M, int P, int32_t* kq_g, int64_t* er,
                             float4* ev, int32_t* boff, int kq_smem) {
  extern __shared__ int32_t cnt[];   // P + 1, then the buckets of the entries when 2 n <= kq_smem
  const int64_t na = *na_dev, nf = nf_dev ? *nf_dev : 0, n = na + nf;
  int32_t* kq = 2 * n <= kq_smem ? cnt + P + 1 : kq_g;
  auto res = [&](int64_t u) { return u < na ? qa[u] : qf[u - na]; };
  for (int k = threadIdx.x; k <= P; k += blockDim.x) cnt[k] = 0;
  __syncthreads();
  for (int64_t u = threadIdx.x; u < n; u += blockDim.x) {
    const int64_t r = res(u);
    const bool one = r == 0 || 2 * r == M;
    const int32_t k0 = (int32_t)(r % P), k1 = one ? -1 : (int32_t)((M - r) % P);
    kq[2 * u] = k0;
    kq[2 * u + 1] = k1;
    atomicAdd(cnt + k0, 1);
    if (k1 >= 0) atomicAdd(cnt + k1, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int s = 0;
    for (int k = 0; k < P; ++k) {
      const int c = cnt[k];
      cnt[k] = s;
      s += c;
    }
    cnt[P] = s;
  }
  __syncthreads();
  for (int k = threadIdx.x; k <= P; k += blockDim.x) boff[k] = cnt[k];
  const double ia = scale ? 1.0 / scale[0] : 1.0, jf = scale ? 1.0 / scale[1] : 1.0;   // exact: powers of two
  // stable placement: entry v goes after the earlier entries of its bucket
  for (int64_t v = threadIdx.x; v < 2 * n; v += blockDim.x) {
    const int32_t k = kq[v];
    if (k < 0) continue;
    int pos = cnt[k];
    for (int64_t w = 0; w < v; ++w) pos += kq[w] == k;
    const int64_t u = v >> 1;
    const bool neg = v & 1;
    const int64_t r = res(u);
    const bool one = r == 0 || 2 * r == M;
    double x, y;
    if (u < na) {
      const double2 c = ca[u];
      if (one) {
        x = c.x * ia;
        y = 0.0;
      } else {
        x = 0.5 * c.x * ia;
        y = (neg ? -0.5 : 0.5) * c.y * ia;
      }
    } else {
      const double2 c = cf[u - na];
      if (one) {
        x = 0.0;
        y = c.x * jf;
      } else {
        x = (neg ? 0.5 : -0.5) * c.y * jf;
        y = 0.5 * c.x * jf;
      }
    }
    const DF dx = df_split(x), dy = df_split(y);
    er[pos] = neg ? M - r : r;
    ev[pos] = make_float4(dx.hi, dx.lo, dy.hi, dy.lo);
  }
}

// tab[e][i] = exp(sign 2 pi i (i r_e mod M) / M) for e < n (device count n_dev
// when given, else n_host), i < W.
template <int SIGN>
__global__ void k_pr_steps(const int64_t* __restrict__ r, const int32_t* __restrict__ n_dev, int64_t n_host, int W,
                           int64_t M, const float4* __restrict__ t0, const float4* __restrict__ t1, int b,
                           float4* tab) {
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n = n_dev ? *n_dev : n_host;
  const int64_t e = id / W;
  const int i = (int)(id % W);
  if (e >= n) return;
  const uint64_t idx = ((uint64_t)i * (uint64_t)r[e]) % (uint64_t)M;
  tab[id] = st4(tw2<SIGN>(t0, t1, b, idx));
}

// Output bins: bucket b mod P of every output.
__global__ void k_pr_kout(const int64_t* __restrict__ bins, int64_t n, int P, int32_t* kout) {
  const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (o < n) kout[o] = (int32_t)(bins[o] % P);
}

// Evaluation: s[q + Q p] for every tile of W columns (grid-stride over tiles).
template <class A, bool OUT_REAL>
__global__ void __launch_bounds__(kPrThreads) k_pr_eval(int64_t M, int P, int64_t Q, int wsh, DfRadices rad,
                                                        const float4* __restrict__ t0, const float4* __restrict__ t1,
                                                        int b, const int64_t* __restrict__ er,
                                                        const float4* __restrict__ ev,
                                                        const int32_t* __restrict__ boff_g,
                                                        const float4* __restrict__ estep, int n_stage,
                                                        int64_t n_tiles, void* __restrict__ out) {
  using V = typename A::V;
  using C = typename A::C;
  extern __shared__ __align__(16) float4 sm4[];
  const int CS = P + 1, W = 1 << wsh;
  const unsigned wmask = (unsigned)W - 1u;
  V* Av = reinterpret_cast<V*>(sm4);
  V* Bf = Av + W * CS;
  V* tw = Bf + W * CS;
  V* base = tw + P;
  V* es = base + kPrChunk;                          // staged step powers (n_stage > 0)
  int32_t* boff = reinterpret_cast<int32_t*>(es + n_stage);
  const uint64_t Mu = (uint64_t)M, inv = ~0ull / Mu;
  for (int m = threadIdx.x; m < P; m += blockDim.x)
    tw[m] = A::st(A::template root<1>(t0, t1, b, (uint64_t)m * (uint64_t)Q));
  for (int k = threadIdx.x; k <= P; k += blockDim.x) boff[k] = boff_g[k];
  __syncthreads();
  const int ne = boff[P];
  // the step powers exp(2 pi i i r_e / M) are the same for every tile
  if (n_stage > 0) {
    for (int x = threadIdx.x; x < ne * W; x += blockDim.x) es[x] = A::st(A::from_df(__ldg(estep + x)));
    __syncthreads();
  }
  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int64_t q0 = tile * W;
    // C[k][i] = sum_{e in bucket k} v_e w^{(q0 + i) r_e}, in chunks of entries
    int e0 = 0;
    do {
      const int e1 = min(ne, e0 + kPrChunk);
      for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x)
        base[e - e0] = A::st(A::mul(A::from_df(__ldg(ev + e)),
                                    A::template root<1>(t0, t1, b, mulmod((uint64_t)q0, (uint64_t)er[e], Mu, inv))));
      __syncthreads();
#pragma unroll 4
      for (int u = threadIdx.x; u < P * W; u += blockDim.x) {
        const int i = (int)((unsigned)u & wmask), k = u >> wsh;
        const int lo = max(boff[k], e0), hi = min(boff[k + 1], e1);
        C s = e0 == 0 ? A::zero() : A::ld(Av[i * CS + k]);
        if (n_stage > 0) {
          for (int e = lo; e < hi; ++e) s = A::add(s, A::mul(A::ld(base[e - e0]), A::ld(es[e * W + i])));
        } else {
          for (int e = lo; e < hi; ++e)
            s = A::add(s, A::mul(A::ld(base[e - e0]), A::from_df(__ldg(estep + (int64_t)e * W + i))));
        }
        Av[i * CS + k] = A::st(s);
      }
      __syncthreads();
      e0 += kPrChunk;
    } while (e0 < ne);
    // s[q0 + i + Q p] = sum_k w_P^{p k} C[k][i]
    const V* res = columns_dft<A, 1>(Av, Bf, P, wsh, CS, rad, tw);
    for (int u = threadIdx.x; u < P * W; u += blockDim.x) {
      const int i = (int)((unsigned)u & wmask), p = u >> wsh;
      const int64_t q = q0 + i;
      if (q >= Q) continue;
      if (OUT_REAL)
        static_cast<typename A::Real*>(out)[q + Q * p] = A::real_out(res[i * CS + p]);
      else
        static_cast<V*>(out)[q + Q * p] = res[i * CS + p];
    }
    __syncthreads();
  }
}

// Pruned forward transform: per tile the length-P transforms of the W
// columns, then every output o accumulates
//   w^{-q0 b_o} sum_i Y[b_o mod P][q0 + i] z_o^i,   z_o = w^{-b_o},
// the sum over the tile's columns by Horner's scheme (thread o mod blockDim
// owns output o for the whole launch).
template <class A, bool IN_REAL>
__global__ void __launch_bounds__(kPrThreads) k_pr_fwd(int64_t M, int P, int64_t Q, int wsh, DfRadices rad,
                                                       const float4* __restrict__ t0, const float4* __restrict__ t1,
                                                       int b, const void* __restrict__ in,
                                                       const int64_t* __restrict__ ob,
                                                       const int32_t* __restrict__ kout, int n_out,
                                                       const float4* __restrict__ oz, int64_t n_tiles,
                                                       typename A::V* __restrict__ partial) {
  using V = typename A::V;
  using C = typename A::C;
  extern __shared__ __align__(16) float4 sm4[];
  const int CS = P + 1, W = 1 << wsh;
  const unsigned wmask = (unsigned)W - 1u;
  V* Av = reinterpret_cast<V*>(sm4);
  V* Bf = Av + W * CS;
  V* tw = Bf + W * CS;
  V* acc = tw + P;
  const uint64_t Mu = (uint64_t)M, inv = ~0ull / Mu;
  for (int m = threadIdx.x; m < P; m += blockDim.x)
    tw[m] = A::st(A::template root<1>(t0, t1, b, (uint64_t)m * (uint64_t)Q));
  for (int o = threadIdx.x; o < n_out; o += blockDim.x) acc[o] = A::st(A::zero());
  __syncthreads();
  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int64_t q0 = tile * W;
    for (int u = threadIdx.x; u < P * W; u += blockDim.x) {
      const int i = (int)((unsigned)u & wmask), p = u >> wsh;
      const int64_t q = q0 + i;
      C v = A::zero();
      if (q < Q) {
        if (IN_REAL) v = A::from_real(__ldg(static_cast<const typename A::Real*>(in) + q + Q * p));
        else v = A::ld(__ldg(static_cast<const V*>(in) + q + Q * p));
      }
      Av[i * CS + p] = A::st(v);
    }
    __syncthreads();
    const V* res = columns_dft<A, -1>(Av, Bf, P, wsh, CS, rad, tw);
    const int wl = Q - q0 < (int64_t)W ? (int)(Q - q0) : W;
    for (int o = threadIdx.x; o < n_out; o += blockDim.x) {
      const int k = kout[o];
      const C w = A::template root<-1>(t0, t1, b, mulmod((uint64_t)q0, (uint64_t)ob[o], Mu, inv));
      const C z = A::from_df(__ldg(oz + 2 * o));   // oz: stride 2 (the step table of width 2, entry 1)
      C s = A::ld(res[(wl - 1) * CS + k]);
      for (int i = wl - 2; i >= 0; --i) s = A::add(A::mul(s, z), A::ld(res[i * CS + k]));
      acc[o] = A::st(A::add(A::ld(acc[o]), A::mul(s, w)));
    }
    __syncthreads();
  }
  for (int o = threadIdx.x; o < n_out; o += blockDim.x) partial[(int64_t)blockIdx.x * n_out + o] = acc[o];
}

// ------------------------------------------- 4096-value tiles, radix 16
//
// Double-float transforms with P = 128 or 256: tiles of W = 4096 / P columns,
// the column transforms as two in-place Stockham passes, a radix-16 one and
// one of radix P / 16.  Every thread holds one radix-16 butterfly (or two
// radix-8 ones) in registers between a read phase and a write phase, so one
// shared buffer serves both passes (two barriers per pass).  The forward
// kernel's first pass reads the samples straight from global memory and the
// evaluation's second pass writes them straight there.
constexpr int kPr16Tile = 4096;
constexpr int kPr16Threads = 256;   // butterflies of a radix-16 pass over a tile

__host__ __device__ constexpr bool pr16_supported(int P) { return P == 128 || P == 256; }

// Second pass (Ns = 16) of one column in place: butterflies k (and k + 8 when
// the radix is 8) read k + 16 r, take the twiddles w_P^(SIGN k r) and write
// output r at k + 16 r.  out(p, value) receives the outputs (position p in the
// column); with IN_PLACE the block synchronises between reads and writes.
template <class A, int P, int SIGN, bool IN_PLACE, class Out>
__device__ __forceinline__ void pr16_pass2(const typename A::V* col, int k, const typename A::V* tw,
                                           const typename A::C w1, const typename A::C w2, const typename A::C w3,
                                           Out out) {
  using C = typename A::C;
  if constexpr (P == 256) {
    C v[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) v[r] = A::ld(col[k + 16 * r]);
    if (IN_PLACE) __syncthreads();
#pragma unroll
    for (int r = 1; r < 16; ++r) {
      const C w = A::ld(tw[k * r]);
      v[r] = A::mul(v[r], SIGN > 0 ? w : A::conj(w));
    }
    A::template dft16<SIGN>(v, w1, w2, w3);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
      for (int k2 = 0; k2 < 4; ++k2) out(k + 16 * (k1 + 4 * k2), v[4 * k1 + k2]);
  } else {   // P = 128: radix 8, butterflies k and k + 8
    C v[2][8];
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int r = 0; r < 8; ++r) v[h][r] = A::ld(col[k + 8 * h + 16 * r]);
    if (IN_PLACE) __syncthreads();
    const C cs[1] = {w2};   // exp(2 pi i / 8)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int kk = k + 8 * h;
#pragma unroll
      for (int r = 1; r < 8; ++r) {
        const C w = A::ld(tw[kk * r]);
        v[h][r] = A::mul(v[h][r], SIGN > 0 ? w : A::conj(w));
      }
      A::template dft<8, SIGN>(v[h], cs);
#pragma unroll
      for (int r = 0; r < 8; ++r) out(kk + 16 * r, v[h][r]);
    }
  }
}

// Evaluation with 4096-value tiles (see above); the bucket phase as k_pr_eval.
template <class A, int P, bool OUT_REAL>
__global__ void __launch_bounds__(kPr16Threads, A::kMinBlocks16) k_pr_eval16(int64_t M, int64_t Q, const float4* __restrict__ t0,
                                                               const float4* __restrict__ t1, int b,
                                                               const int64_t* __restrict__ er,
                                                               const float4* __restrict__ ev,
                                                               const int32_t* __restrict__ boff_g,
                                                               const float4* __restrict__ estep, int n_stage,
                                                               int64_t n_tiles, void* __restrict__ out) {
  using V = typename A::V;
  using C = typename A::C;
  constexpr int W = kPr16Tile / P, CS = P + 1, R2 = P / 16;
  extern __shared__ __align__(16) float4 sm4[];
  V* tl = reinterpret_cast<V*>(sm4);
  V* tw = tl + W * CS;
  V* base = tw + P;
  V* es = base + kPrChunk;
  int32_t* boff = reinterpret_cast<int32_t*>(es + n_stage);
  const uint64_t Mu = (uint64_t)M, inv = ~0ull / Mu;
  for (int m = threadIdx.x; m < P; m += blockDim.x)
    tw[m] = A::st(A::template root<1>(t0, t1, b, (uint64_t)m * (uint64_t)Q));
  for (int k = threadIdx.x; k <= P; k += blockDim.x) boff[k] = boff_g[k];
  __syncthreads();
  const int ne = boff[P];
  if (n_stage > 0) {
    for (int x = threadIdx.x; x < ne * W; x += blockDim.x) es[x] = A::st(A::from_df(__ldg(estep + x)));
    __syncthreads();
  }
  const C w1 = A::ld(tw[P / 16]), w2 = A::ld(tw[2 * P / 16]), w3 = A::ld(tw[3 * P / 16]);
  const int u = threadIdx.x;
  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int64_t q0 = tile * W;
    // C[k][i] = sum_{e in bucket k} v_e w^{(q0 + i) r_e}, in chunks of entries
    int e0 = 0;
    do {
      const int e1 = min(ne, e0 + kPrChunk);
      for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x)
        base[e - e0] = A::st(A::mul(A::from_df(__ldg(ev + e)),
                                    A::template root<1>(t0, t1, b, mulmod((uint64_t)q0, (uint64_t)er[e], Mu, inv))));
      __syncthreads();
      for (int x = threadIdx.x; x < P * W; x += blockDim.x) {
        const int i = x % W, k = x / W;
        const int lo = max(boff[k], e0), hi = min(boff[k + 1], e1);
        C sum = e0 == 0 ? A::zero() : A::ld(tl[i * CS + k]);
        for (int e = lo; e < hi; ++e) {
          const C st = n_stage > 0 ? A::ld(es[e * W + i]) : A::from_df(__ldg(estep + (int64_t)e * W + i));
          sum = A::add(sum, A::mul(A::ld(base[e - e0]), st));
        }
        tl[i * CS + k] = A::st(sum);
      }
      __syncthreads();
      e0 += kPrChunk;
    } while (e0 < ne);
    // pass 1 (radix 16, Ns = 1): butterfly j of column c reads j + R2 r, writes 16 j + r
    {
      const int c = u % W, j = u / W;
      V* col = tl + c * CS;
      C v[16];
#pragma unroll
      for (int r = 0; r < 16; ++r) v[r] = A::ld(col[j + R2 * r]);
      __syncthreads();
      A::template dft16<1>(v, w1, w2, w3);
#pragma unroll
      for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) col[16 * j + k1 + 4 * k2] = A::st(v[4 * k1 + k2]);
    }
    __syncthreads();
    // pass 2 straight to the samples s[q0 + c + Q p]
    {
      const int c = u % W, k = u / W;
      const int64_t q = q0 + c;
      pr16_pass2<A, P, 1, false>(tl + c * CS, k, tw, w1, w2, w3, [&](int p, const C val) {
        if (q >= Q) return;
        if (OUT_REAL)
          static_cast<typename A::Real*>(out)[q + Q * p] = A::real_out(A::st(val));
        else
          static_cast<V*>(out)[q + Q * p] = A::st(val);
      });
    }
    __syncthreads();
  }
}

// Pruned forward transform with 4096-value tiles (see above); the Horner
// phase as k_pr_fwd.
template <class A, int P, bool IN_REAL>
__global__ void __launch_bounds__(kPr16Threads, A::kMinBlocks16) k_pr_fwd16(int64_t M, int64_t Q, const float4* __restrict__ t0,
                                                              const float4* __restrict__ t1, int b,
                                                              const void* __restrict__ in,
                                                              const int64_t* __restrict__ ob,
                                                              const int32_t* __restrict__ kout, int n_out,
                                                              const float4* __restrict__ oz, int64_t n_tiles,
                                                              typename A::V* __restrict__ partial) {
  using V = typename A::V;
  using C = typename A::C;
  constexpr int W = kPr16Tile / P, CS = P + 1, R2 = P / 16;
  extern __shared__ __align__(16) float4 sm4[];
  V* tl = reinterpret_cast<V*>(sm4);
  V* tw = tl + W * CS;
  V* acc = tw + P;
  const uint64_t Mu = (uint64_t)M, inv = ~0ull / Mu;
  for (int m = threadIdx.x; m < P; m += blockDim.x)
    tw[m] = A::st(A::template root<1>(t0, t1, b, (uint64_t)m * (uint64_t)Q));
  for (int o = threadIdx.x; o < n_out; o += blockDim.x) acc[o] = A::st(A::zero());
  __syncthreads();
  const C w1 = A::ld(tw[P / 16]), w2 = A::ld(tw[2 * P / 16]), w3 = A::ld(tw[3 * P / 16]);
  const int u = threadIdx.x;
  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int64_t q0 = tile * W;
    // pass 1 (radix 16, Ns = 1) from the samples: butterfly j of column c
    // reads p = j + R2 r, writes 16 j + r
    {
      const int c = u % W, j = u / W;
      const int64_t q = q0 + c;
      C v[16];
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        const int64_t p = j + R2 * r;
        if (q >= Q) v[r] = A::zero();
        else if (IN_REAL) v[r] = A::from_real(__ldg(static_cast<const typename A::Real*>(in) + q + Q * p));
        else v[r] = A::ld(__ldg(static_cast<const V*>(in) + q + Q * p));
      }
      A::template dft16<-1>(v, w1, w2, w3);
      V* col = tl + c * CS;
#pragma unroll
      for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) col[16 * j + k1 + 4 * k2] = A::st(v[4 * k1 + k2]);
    }
    __syncthreads();
    {
      const int c = u % W, k = u / W;
      V* col = tl + c * CS;
      pr16_pass2<A, P, -1, true>(col, k, tw, w1, w2, w3, [&](int p, const C val) { col[p] = A::st(val); });
    }
    __syncthreads();
    const int wl = Q - q0 < (int64_t)W ? (int)(Q - q0) : W;
    for (int o = threadIdx.x; o < n_out; o += blockDim.x) {
      const int k = kout[o];
      const C w = A::template root<-1>(t0, t1, b, mulmod((uint64_t)q0, (uint64_t)ob[o], Mu, inv));
      const C z = A::from_df(__ldg(oz + 2 * o));
      C sum = A::ld(tl[(wl - 1) * CS + k]);
      for (int i = wl - 2; i >= 0; --i) sum = A::add(A::mul(sum, z), A::ld(tl[i * CS + k]));
      acc[o] = A::st(A::add(A::ld(acc[o]), A::mul(sum, w)));
    }
    __syncthreads();
  }
  for (int o = threadIdx.x; o < n_out; o += blockDim.x) partial[(int64_t)blockIdx.x * n_out + o] = acc[o];
}

// X[o] = sum over blocks of partial[blk][o] in FP64: one warp per output,
// lanes in a fixed stride, then a fixed butterfly; written as double-float.
template <class A>
__global__ void k_pr_reduce(const typename A::V* __restrict__ partial, int nb, int n_out, float4* __restrict__ X) {
  const int64_t o = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (o >= n_out) return;   // warp-uniform
  double sr = 0.0, si = 0.0;
  for (int blk = lane; blk < nb; blk += 32) {
    const double2 v = A::to_double2(partial[(int64_t)blk * n_out + o]);
    sr += v.x;
    si += v.y;
  }
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) {
    sr += __shfl_xor_sync(0xffffffffu, sr, m);
    si += __shfl_xor_sync(0xffffffffu, si, m);
  }
  if (lane == 0) {
    const DF r = df_split(sr), i = df_split(si);
    X[o] = make_float4(r.hi, r.lo, i.hi, i.lo);
  }
}

template <class A>
size_t eval_smem(const PrunedSplit& S, int64_t n_stage) {
  return (size_t)(2 * S.W * (S.P + 1) + S.P + kPrChunk + n_stage) * sizeof(typename A::V) +
         (size_t)(S.P + 1) * sizeof(int32_t);
}

template <class A>
size_t fwd_smem(const PrunedSplit& S, int n_out) {
  return (size_t)(2 * S.W * (S.P + 1) + S.P + n_out) * sizeof(typename A::V);
}

template <typename K>
ss_status grid_for(K kernel, size_t smem, int64_t n_tiles, int* grid) {
  SS_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  SS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kPrThreads, smem));
  if (per_sm < 1) SS_FAIL(SS_ERR_CUDA, "pruned transform: a block of %zu bytes of shared memory does not fit", smem);
  *grid = (int)std::max<int64_t>(1, std::min<int64_t>(n_tiles, (int64_t)per_sm * sm_count()));
  return SS_OK;
}

template <class A, bool OUT_REAL>
ss_status launch_eval(const TwoLevelTable& T, const PrunedSplit& S, int wsh, const int64_t* er, const float4* ev,
                      const int32_t* boff, const float4* estep, int64_t n_stage, void* out, cudaStream_t st) {
  const int64_t n_tiles = (S.Q + S.W - 1) / S.W;
  const size_t smem = eval_smem<A>(S, n_stage);
  int grid = 0;
  SS_TRY(grid_for(k_pr_eval<A, OUT_REAL>, smem, n_tiles, &grid));
  k_pr_eval<A, OUT_REAL><<<grid, kPrThreads, smem, st>>>(T.M, S.P, S.Q, wsh, S.rad, T.t0.get(), T.t1.get(), T.b, er,
                                                         ev, boff, estep, (int)n_stage, n_tiles, out);
  SS_LAUNCH_CHECK();
  return SS_OK;
}

template <class A, int P, bool OUT_REAL>
ss_status launch_eval16(const TwoLevelTable& T, const PrunedSplit& S, const int64_t* er, const float4* ev,
                        const int32_t* boff, const float4* estep, int64_t n_stage, void* out, cudaStream_t st) {
  constexpr int W = kPr16Tile / P;
  const int64_t n_tiles = (S.Q + W - 1) / W;
  const size_t smem =
      (size_t)(W * (P + 1) + P + kPrChunk + n_stage) * sizeof(typename A::V) + (P + 1) * sizeof(int32_t);
  int grid = 0;
  SS_TRY(grid_for(k_pr_eval16<A, P, OUT_REAL>, smem, n_tiles, &grid));
  k_pr_eval16<A, P, OUT_REAL><<<grid, kPr16Threads, smem, st>>>(T.M, S.Q, T.t0.get(), T.t1.get(), T.b, er, ev, boff,
                                                                 estep, (int)n_stage, n_tiles, out);
  SS_LAUNCH_CHECK();
  return SS_OK;
}

template <class A, bool OUT_REAL>
ss_status launch_eval16_p(const TwoLevelTable& T, const PrunedSplit& S, const int64_t* er, const float4* ev,
                          const int32_t* boff, const float4* estep, int64_t n_stage, void* out, cudaStream_t st) {
  if (S.P == 256) return launch_eval16<A, 256, OUT_REAL>(T, S, er, ev, boff, estep, n_stage, out, st);
  return launch_eval16<A, 128, OUT_REAL>(T, S, er, ev, boff, estep, n_stage, out, st);
}

template <class A, int P, bool IN_REAL>
ss_status launch_fwd16(const TwoLevelTable& T, const PrunedSplit& S, const void* in, const int64_t* ob,
                       const int32_t* kout, int nc, const float4* oz, float4* X, cudaStream_t st) {
  constexpr int W = kPr16Tile / P;
  const int64_t n_tiles = (S.Q + W - 1) / W;
  const size_t smem = (size_t)(W * (P + 1) + P + nc) * sizeof(typename A::V);
  int grid = 0;
  SS_TRY(grid_for(k_pr_fwd16<A, P, IN_REAL>, smem, n_tiles, &grid));
  DevBuf<typename A::V> partial;
  SS_TRY(partial.alloc_tmp((size_t)grid * nc, st));
  {
    ProfScope prof_("k_pr_fwd", st, true);
    k_pr_fwd16<A, P, IN_REAL><<<grid, kPr16Threads, smem, st>>>(T.M, S.Q, T.t0.get(), T.t1.get(), T.b, in, ob, kout,
                                                                 nc, oz, n_tiles, partial.get());
    SS_LAUNCH_CHECK();
  }
  k_pr_reduce<A><<<nblk((int64_t)nc * 32), 256, 0, st>>>(partial.get(), grid, nc, X);
  SS_LAUNCH_CHECK();
  return SS_OK;
}

template <class A, bool IN_REAL>
ss_status launch_fwd16_p(const TwoLevelTable& T, const PrunedSplit& S, const void* in, const int64_t* ob,
                         const int32_t* kout, int nc, const float4* oz, float4* X, cudaStream_t st) {
  if (S.P == 256) return launch_fwd16<A, 256, IN_REAL>(T, S, in, ob, kout, nc, oz, X, st);
  return launch_fwd16<A, 128, IN_REAL>(T, S, in, ob, kout, nc, oz, X, st);
}

template <class A, bool IN_REAL>
ss_status launch_fwd(const TwoLevelTable& T, const PrunedSplit& S, int wsh, const void* in, const int64_t* ob,
                     const int32_t* kout, int nc, const float4* oz, float4* X, cudaStream_t st) {
  const int64_t n_tiles = (S.Q + S.W - 1) / S.W;
  const size_t smem = fwd_smem<A>(S, nc);
  int grid = 0;
  SS_TRY(grid_for(k_pr_fwd<A, IN_REAL>, smem, n_tiles, &grid));
  DevBuf<typename A::V> partial;
  SS_TRY(partial.alloc_tmp((size_t)grid * nc, st));
  {
    ProfScope prof_("k_pr_fwd", st, true);
    k_pr_fwd<A, IN_REAL><<<grid, kPrThreads, smem, st>>>(T.M, S.P, S.Q, wsh, S.rad, T.t0.get(), T.t1.get(), T.b, in,
                                                         ob, kout, nc, oz, n_tiles, partial.get());
    SS_LAUNCH_CHECK();
  }
  k_pr_reduce<A><<<nblk((int64_t)nc * 32), 256, 0, st>>>(partial.get(), grid, nc, X);
  SS_LAUNCH_CHECK();
  return SS_OK;
}

}  // namespace

ss_status two_level_table(int64_t M, TwoLevelTable* T, cudaStream_t st) {
  int bits = 0;
  while ((1ll << bits) < M) ++bits;
  T->M = M;
  T->b = (bits + 1) / 2;
  const int64_t n0 = 1ll << T->b, n1 = (M + n0 - 1) >> T->b;
  SS_TRY(T->t0.alloc(n0, st));
  SS_TRY(T->t1.alloc(n1, st));
  k_tl_table<<<nblk(std::max(n0, n1)), 256, 0, st>>>(M, T->b, n1, T->t0.get(), T->t1.get());
  SS_LAUNCH_CHECK();
  return SS_OK;
}

bool pruned_split(int64_t M, int64_t n, PrunedSplit* out, int tile) {
  // cost per point ~ log2 P (the transform) + n / P (the sparse side)
  double best = 1e300;
  PrunedSplit S;
  for (int P = 8; P <= kPrMaxP; ++P) {
    if (M % P || M / P < 2) continue;
    const DfRadices r = df_radices(P);
    if (r.n < 0) continue;
    const double c = std::log2((double)P) + (double)std::max<int64_t>(n, 1) / P;
    if (c < best) {
      best = c;
      S.P = P;
      S.Q = M / P;
      S.W = 1;
      while (2 * S.W * P <= tile) S.W *= 2;   // W: a power of two, W P <= tile
      S.rad = r;
    }
  }
  if (S.P == 0) return false;
  *out = S;
  return true;
}

bool pruned_supported(int64_t M) {
  int64_t m = M;
  for (int64_t p : {2, 3, 5, 7})
    while (m % p == 0) m /= p;
  PrunedSplit S;
  return m == 1 && M < (1ll << 31) && pruned_split(M, 2, &S) && S.P >= 8;
}

ss_status pruned_eval_pair(const TwoLevelTable& T, const int64_t* qa, const double2* ca, const int64_t* na_dev,
                           int64_t na_max, const int64_t* qf, const double2* cf, const int64_t* nf_dev,
                           int64_t nf_max, const double* scale, void* out, PrunedFormat fmt, cudaStream_t st) {
  const int64_t M = T.M;
  if (!qf) nf_max = 0;
  const int64_t ne_max = std::max<int64_t>(1, 2 * (na_max + nf_max));
  if (ne_max > (1ll << 30)) SS_FAIL(SS_ERR_INVALID, "pruned evaluation: too many terms");
  PrunedSplit S;
  if (!pruned_split(M, ne_max, &S, kPrEvalTile))
    SS_FAIL(SS_ERR_INVALID, "pruned evaluation: M = %lld has no split", (long long)M);
  // P = 128 or 256: 4096-value tiles (k_pr_eval16)
  const bool t16 = pr16_supported(S.P);
  const int Wt = t16 ? kPr16Tile / S.P : S.W;
  DevBuf<int64_t> er;
  DevBuf<float4> ev, estep;
  DevBuf<int32_t> boff, kq;
  SS_TRY(er.alloc_tmp(ne_max, st));
  SS_TRY(ev.alloc_tmp(ne_max, st));
  SS_TRY(boff.alloc_tmp(S.P + 1, st));
  SS_TRY(kq.alloc_tmp(ne_max, st));
  SS_TRY(estep.alloc_tmp((size_t)ne_max * Wt, st));
  {
    ProfScope prof_setup("pr_setup", st);
    const int eb = std::min(1024, (S.P + 31) / 32 * 32);
    // the entries' buckets in shared memory when they fit (48 KB with the counts)
    const int kq_smem = (int)std::min<int64_t>(ne_max, 12288 - (S.P + 1));
    k_pr_entries<<<1, eb, (S.P + 1 + kq_smem) * sizeof(int32_t), st>>>(qa, ca, na_dev, qf, cf, qf ? nf_dev : nullptr,
                                                                        scale, M,
                                                                        S.P, kq.get(), er.get(), ev.get(),
                                                                        boff.get(), kq_smem);
    SS_LAUNCH_CHECK();
    k_pr_steps<1><<<nblk(ne_max * Wt), 256, 0, st>>>(er.get(), boff.get() + S.P, 0, Wt, M, T.t0.get(), T.t1.get(),
                                                     T.b, estep.get());
    SS_LAUNCH_CHECK();
  }
  int wsh = 0;
  while ((1 << wsh) < S.W) ++wsh;
  // the entries' step powers go to shared memory once per block when they fit
  const int64_t n_stage = ne_max * Wt <= kPrEvalStage ? ne_max * Wt : 0;
  ProfScope prof_("k_pr_eval", st, true);
  if (t16) {
    switch (fmt) {
      case PrunedFormat::kDfComplex:
        return launch_eval16_p<ArDF, false>(T, S, er.get(), ev.get(), boff.get(), estep.get(), n_stage, out, st);
      case PrunedFormat::kF64Real:
        return launch_eval16_p<ArDF, true>(T, S, er.get(), ev.get(), boff.get(), estep.get(), n_stage, out, st);
      case PrunedFormat::kF32Complex:
        return launch_eval16_p<ArF32, false>(T, S, er.get(), ev.get(), boff.get(), estep.get(), n_stage, out, st);
      default:
        return launch_eval16_p<ArF32, true>(T, S, er.get(), ev.get(), boff.get(), estep.get(), n_stage, out, st);
    }
  }
  switch (fmt) {
    case PrunedFormat::kDfComplex:
      return launch_eval<ArDF, false>(T, S, wsh, er.get(), ev.get(), boff.get(), estep.get(), n_stage, out, st);
    case PrunedFormat::kF64Real:
      return launch_eval<ArDF, true>(T, S, wsh, er.get(), ev.get(), boff.get(), estep.get(), n_stage, out, st);
    case PrunedFormat::kF32Complex:
      return launch_eval<ArF32, false>(T, S, wsh, er.get(), ev.get(), boff.get(), estep.get(), n_stage, out, st);
    default:
      return launch_eval<ArF32, true>(T, S, wsh, er.get(), ev.get(), boff.get(), estep.get(), n_stage, out, st);
  }
}

ss_status pruned_forward(const TwoLevelTable& T, const void* s, PrunedFormat fmt, const int64_t* bins, int64_t n_out,
                         float4* X, cudaStream_t st) {
  const int64_t M = T.M;
  if (n_out < 1) return SS_OK;
  PrunedSplit S;
  if (!pruned_split(M, n_out, &S)) SS_FAIL(SS_ERR_INVALID, "pruned transform: M = %lld has no split", (long long)M);
  int wsh = 0;
  while ((1 << wsh) < S.W) ++wsh;
  for (int64_t o0 = 0; o0 < n_out; o0 += kPrMaxOut) {
    const int nc = (int)std::min<int64_t>(kPrMaxOut, n_out - o0);
    DevBuf<int32_t> kout;
    DevBuf<float4> oz;
    SS_TRY(kout.alloc_tmp(nc, st));
    SS_TRY(oz.alloc_tmp((size_t)nc * 2, st));
    k_pr_kout<<<nblk(nc), 256, 0, st>>>(bins + o0, nc, S.P, kout.get());
    // oz[2 o + 1] = exp(-2 pi i b_o / M): the Horner root of output o
    k_pr_steps<-1><<<nblk((int64_t)nc * 2), 256, 0, st>>>(bins + o0, nullptr, nc, 2, M, T.t0.get(), T.t1.get(), T.b,
                                                          oz.get());
    SS_LAUNCH_CHECK();
    const float4* z = oz.get() + 1;
    const bool t16 = pr16_supported(S.P);   // 4096-value tiles
    switch (fmt) {
      case PrunedFormat::kDfComplex:
        if (t16) SS_TRY((launch_fwd16_p<ArDF, false>(T, S, s, bins + o0, kout.get(), nc, z, X + o0, st)));
        else SS_TRY((launch_fwd<ArDF, false>(T, S, wsh, s, bins + o0, kout.get(), nc, z, X + o0, st)));
        break;
      case PrunedFormat::kF64Real:
        if (t16) SS_TRY((launch_fwd16_p<ArDF, true>(T, S, s, bins + o0, kout.get(), nc, z, X + o0, st)));
        else SS_TRY((launch_fwd<ArDF, true>(T, S, wsh, s, bins + o0, kout.get(), nc, z, X + o0, st)));
        break;
      case PrunedFormat::kF32Complex:
        if (t16) SS_TRY((launch_fwd16_p<ArF32, false>(T, S, s, bins + o0, kout.get(), nc, z, X + o0, st)));
        else SS_TRY((launch_fwd<ArF32, false>(T, S, wsh, s, bins + o0, kout.get(), nc, z, X + o0, st)));
        break;
      default:
        if (t16) SS_TRY((launch_fwd16_p<ArF32, true>(T, S, s, bins + o0, kout.get(), nc, z, X + o0, st)));
        else SS_TRY((launch_fwd<ArF32, true>(T, S, wsh, s, bins + o0, kout.get(), nc, z, X + o0, st)));
        break;
    }
  }
  return SS_OK;
}

}  // namespace ss
