// Pruned double-float DFTs of a 7-smooth length M (the split, the index maps
// and the cost are stated in fft_pruned.cuh).
//
// Inside a block a tile holds W columns of length P in shared memory, column c
// at c (P + 1) (one float4 of padding: threads that share a row offset and
// differ in the column hit distinct banks).  The length-P transforms run as
// self-sorting (Stockham) radix passes over all W columns at once, thread u
// taking column u mod W, butterfly u / W, with the butterflies of dfc.cuh and
// the P-th roots staged in shared memory.  All sums run in a fixed order, so
// results are bit-reproducible.
#include <algorithm>
#include <cmath>

#include "dfc.cuh"
#include "fft_pruned.cuh"

namespace ss {
namespace {

using namespace dfc;

constexpr int kPrTile = 2048;      // complex values of one tile (W columns x P rows)
constexpr int kPrThreads = 256;
constexpr int kPrChunk = 256;      // entries staged in shared memory per round of the evaluation
constexpr int kPrMaxOut = 1024;    // outputs per forward launch (accumulators in shared memory)
constexpr int kPrMaxP = 1024;

inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

__device__ __forceinline__ C4 conj4(const C4 a) { return C4{a.re, df_neg(a.im)}; }
__device__ __forceinline__ C4 zero4() { return C4{DF{0.f, 0.f}, DF{0.f, 0.f}}; }

// exp(sign 2 pi i r / M), r < M, from the two-level table
template <int SIGN>
__device__ __forceinline__ C4 tw2(const float4* __restrict__ t0, const float4* __restrict__ t1, int b, uint64_t r) {
  const C4 w = cmul(ld(__ldg(t1 + (r >> b))), ld(__ldg(t0 + (r & ((1ull << b) - 1)))));
  return SIGN > 0 ? w : conj4(w);
}

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
template <int R, int SIGN>
__device__ __forceinline__ void mpass(const float4* __restrict__ a, float4* __restrict__ b, int P, int wsh, int CS,
                                      int Ns, const float4* __restrict__ tw) {
  constexpr int NC = R == 8 ? 1 : (R - 1) / 2;
  C4 cs[NC > 0 ? NC : 1];
#pragma unroll
  for (int m = 0; m < NC; ++m) cs[m] = ld(tw[(P / R) * (m + 1)]);
  const int nb = P / R;
  const int tstride = P / (Ns * R);
  const int total = nb << wsh;
  const unsigned wmask = (1u << wsh) - 1u;
  const unsigned nsm = Ns > 1 ? 0xffffffffu / (unsigned)Ns + 1u : 0u;
  for (int u = threadIdx.x; u < total; u += blockDim.x) {
    const int c = (int)((unsigned)u & wmask), j = u >> wsh;
    const float4* ac = a + c * CS;
    float4* bc = b + c * CS;
    const int jq = Ns > 1 ? (int)__umulhi((unsigned)j, nsm) : j;   // j / Ns
    const int k = j - jq * Ns;
    C4 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = ld(ac[j + r * nb]);
    if (Ns > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        const C4 w = ld(tw[tstride * (k * r)]);
        v[r] = cmul(v[r], SIGN > 0 ? w : conj4(w));
      }
    }
    dft<R, SIGN>(v, cs);
    const int base = jq * Ns * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) bc[base + r * Ns] = st4(v[r]);
  }
}

// Length-P transforms of the W columns in `a` (b: the other buffer); returns
// the buffer that holds the result.  Ends with a block barrier.
template <int SIGN>
__device__ float4* columns_dft(float4* a, float4* b, int P, int wsh, int CS, const DfRadices& rad,
                               const float4* __restrict__ tw) {
  int Ns = 1;
  for (int p = 0; p < rad.n; ++p) {
    const int R = rad.r[p];
    switch (R) {
      case 8: mpass<8, SIGN>(a, b, P, wsh, CS, Ns, tw); break;
      case 4: mpass<4, SIGN>(a, b, P, wsh, CS, Ns, tw); break;
      case 2: mpass<2, SIGN>(a, b, P, wsh, CS, Ns, tw); break;
      case 5: mpass<5, SIGN>(a, b, P, wsh, CS, Ns, tw); break;
      case 3: mpass<3, SIGN>(a, b, P, wsh, CS, Ns, tw); break;
      default: mpass<7, SIGN>(a, b, P, wsh, CS, Ns, tw); break;
    }
    __syncthreads();
    float4* t = a;
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
                             const double* __restrict__ scale, int64_t M, int P, int32_t* kq, int64_t* er,
                             float4* ev, int32_t* boff) {
  extern __shared__ int32_t cnt[];   // P + 1
  const int64_t na = *na_dev, nf = nf_dev ? *nf_dev : 0, n = na + nf;
  auto res = [&](int64_t u) { return u < na ? qa[u] : qf[u - na]; };
  for (int64_t u = threadIdx.x; u < n; u += blockDim.x) {
    const int64_t r = res(u);
    const bool one = r == 0 || 2 * r == M;
    kq[2 * u] = (int32_t)(r % P);
    kq[2 * u + 1] = one ? -1 : (int32_t)((M - r) % P);
  }
  __syncthreads();
  for (int k = threadIdx.x; k < P; k += blockDim.x) {
    int c = 0;
    for (int64_t v = 0; v < 2 * n; ++v) c += kq[v] == k;
    cnt[k] = c;
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
  for (int k = threadIdx.x; k < P; k += blockDim.x) {
    int pos = cnt[k];
    for (int64_t v = 0; v < 2 * n; ++v) {
      if (kq[v] != k) continue;
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
      ++pos;
    }
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
template <bool OUT_REAL>
__global__ void __launch_bounds__(kPrThreads) k_pr_eval(int64_t M, int P, int64_t Q, int wsh, DfRadices rad,
                                                        const float4* __restrict__ t0, const float4* __restrict__ t1,
                                                        int b, const int64_t* __restrict__ er,
                                                        const float4* __restrict__ ev,
                                                        const int32_t* __restrict__ boff_g,
                                                        const float4* __restrict__ estep, int64_t n_tiles,
                                                        void* __restrict__ out) {
  extern __shared__ __align__(16) float4 sm[];
  const int CS = P + 1, W = 1 << wsh;
  const unsigned wmask = (unsigned)W - 1u;
  float4* A = sm;
  float4* Bf = A + W * CS;
  float4* tw = Bf + W * CS;
  float4* base = tw + P;
  int32_t* boff = reinterpret_cast<int32_t*>(base + kPrChunk);
  const uint64_t Mu = (uint64_t)M, inv = ~0ull / Mu;
  for (int m = threadIdx.x; m < P; m += blockDim.x) tw[m] = st4(tw2<1>(t0, t1, b, (uint64_t)m * (uint64_t)Q));
  for (int k = threadIdx.x; k <= P; k += blockDim.x) boff[k] = boff_g[k];
  __syncthreads();
  const int ne = boff[P];
  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int64_t q0 = tile * W;
    // C[k][i] = sum_{e in bucket k} v_e w^{(q0 + i) r_e}, in chunks of entries
    int e0 = 0;
    do {
      const int e1 = min(ne, e0 + kPrChunk);
      for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x)
        base[e - e0] = st4(cmul(ld(__ldg(ev + e)), tw2<1>(t0, t1, b, mulmod((uint64_t)q0, (uint64_t)er[e], Mu, inv))));
      __syncthreads();
      for (int u = threadIdx.x; u < P * W; u += blockDim.x) {
        const int i = (int)((unsigned)u & wmask), k = u >> wsh;
        const int lo = max(boff[k], e0), hi = min(boff[k + 1], e1);
        C4 s = e0 == 0 ? zero4() : ld(A[i * CS + k]);
        for (int e = lo; e < hi; ++e) s = cadd(s, cmul(ld(base[e - e0]), ld(__ldg(estep + (int64_t)e * W + i))));
        A[i * CS + k] = st4(s);
      }
      __syncthreads();
      e0 += kPrChunk;
    } while (e0 < ne);
    // s[q0 + i + Q p] = sum_k w_P^{p k} C[k][i]
    const float4* res = columns_dft<1>(A, Bf, P, wsh, CS, rad, tw);
    for (int u = threadIdx.x; u < P * W; u += blockDim.x) {
      const int i = (int)((unsigned)u & wmask), p = u >> wsh;
      const int64_t q = q0 + i;
      if (q >= Q) continue;
      const float4 v = res[i * CS + p];
      if (OUT_REAL)
        static_cast<double*>(out)[q + Q * p] = (double)v.x + (double)v.y;
      else
        static_cast<float4*>(out)[q + Q * p] = v;
    }
    __syncthreads();
  }
}

// Pruned forward transform: per tile the length-P transforms of the W
// columns, then every output o accumulates
//   w^{-q0 b_o} sum_i Y[b_o mod P][q0 + i] w^{-i b_o}
// (thread o mod blockDim owns output o for the whole launch).
template <bool IN_REAL>
__global__ void __launch_bounds__(kPrThreads) k_pr_fwd(int64_t M, int P, int64_t Q, int wsh, DfRadices rad,
                                                       const float4* __restrict__ t0, const float4* __restrict__ t1,
                                                       int b, const void* __restrict__ in,
                                                       const int64_t* __restrict__ ob,
                                                       const int32_t* __restrict__ kout, int n_out,
                                                       const float4* __restrict__ ostep, int64_t n_tiles,
                                                       float4* __restrict__ partial) {
  extern __shared__ __align__(16) float4 sm[];
  const int CS = P + 1, W = 1 << wsh;
  const unsigned wmask = (unsigned)W - 1u;
  float4* A = sm;
  float4* Bf = A + W * CS;
  float4* tw = Bf + W * CS;
  float4* acc = tw + P;
  const uint64_t Mu = (uint64_t)M, inv = ~0ull / Mu;
  for (int m = threadIdx.x; m < P; m += blockDim.x) tw[m] = st4(tw2<1>(t0, t1, b, (uint64_t)m * (uint64_t)Q));
  for (int o = threadIdx.x; o < n_out; o += blockDim.x) acc[o] = make_float4(0.f, 0.f, 0.f, 0.f);
  __syncthreads();
  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int64_t q0 = tile * W;
    for (int u = threadIdx.x; u < P * W; u += blockDim.x) {
      const int i = (int)((unsigned)u & wmask), p = u >> wsh;
      const int64_t q = q0 + i;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (q < Q) {
        if (IN_REAL) {
          const DF x = df_split(__ldg(static_cast<const double*>(in) + q + Q * p));
          v = make_float4(x.hi, x.lo, 0.f, 0.f);
        } else {
          v = __ldg(static_cast<const float4*>(in) + q + Q * p);
        }
      }
      A[i * CS + p] = v;
    }
    __syncthreads();
    const float4* res = columns_dft<-1>(A, Bf, P, wsh, CS, rad, tw);
    const int wl = Q - q0 < (int64_t)W ? (int)(Q - q0) : W;
    for (int o = threadIdx.x; o < n_out; o += blockDim.x) {
      const int k = kout[o];
      C4 s = zero4();
      for (int i = 0; i < wl; ++i) s = cadd(s, cmul(ld(res[i * CS + k]), ld(__ldg(ostep + (int64_t)o * W + i))));
      const C4 w = tw2<-1>(t0, t1, b, mulmod((uint64_t)q0, (uint64_t)ob[o], Mu, inv));
      acc[o] = st4(cadd(ld(acc[o]), cmul(s, w)));
    }
    __syncthreads();
  }
  for (int o = threadIdx.x; o < n_out; o += blockDim.x) partial[(int64_t)blockIdx.x * n_out + o] = acc[o];
}

// X[o] = sum over blocks of partial[blk][o]: one warp per output, lanes in a
// fixed stride, then a fixed butterfly.
__global__ void k_pr_reduce(const float4* __restrict__ partial, int nb, int n_out, float4* __restrict__ X) {
  const int64_t o = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (o >= n_out) return;   // warp-uniform
  C4 s = zero4();
  for (int blk = lane; blk < nb; blk += 32) s = cadd(s, ld(partial[(int64_t)blk * n_out + o]));
  s.re = df_warp_sum(s.re);
  s.im = df_warp_sum(s.im);
  if (lane == 0) X[o] = st4(s);
}

size_t eval_smem(const PrunedSplit& S) {
  return (size_t)(2 * S.W * (S.P + 1) + S.P + kPrChunk) * sizeof(float4) + (size_t)(S.P + 1) * sizeof(int32_t);
}

size_t fwd_smem(const PrunedSplit& S, int n_out) {
  return (size_t)(2 * S.W * (S.P + 1) + S.P + n_out) * sizeof(float4);
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

bool pruned_split(int64_t M, int64_t n, PrunedSplit* out) {
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
      while (2 * S.W * P <= kPrTile) S.W *= 2;   // W: a power of two, W P <= kPrTile
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
                           int64_t nf_max, const double* scale, void* out, bool out_real, cudaStream_t st) {
  const int64_t M = T.M;
  if (!qf) nf_max = 0;
  const int64_t ne_max = std::max<int64_t>(1, 2 * (na_max + nf_max));
  if (ne_max > (1ll << 30)) SS_FAIL(SS_ERR_INVALID, "pruned evaluation: too many terms");
  PrunedSplit S;
  if (!pruned_split(M, ne_max, &S)) SS_FAIL(SS_ERR_INVALID, "pruned evaluation: M = %lld has no split", (long long)M);
  DevBuf<int64_t> er;
  DevBuf<float4> ev, estep;
  DevBuf<int32_t> boff, kq;
  SS_TRY(er.alloc_tmp(ne_max, st));
  SS_TRY(ev.alloc_tmp(ne_max, st));
  SS_TRY(boff.alloc_tmp(S.P + 1, st));
  SS_TRY(kq.alloc_tmp(ne_max, st));
  SS_TRY(estep.alloc_tmp((size_t)ne_max * S.W, st));
  const int eb = std::min(1024, (S.P + 31) / 32 * 32);
  k_pr_entries<<<1, eb, (S.P + 1) * sizeof(int32_t), st>>>(qa, ca, na_dev, qf, cf, qf ? nf_dev : nullptr, scale, M,
                                                           S.P, kq.get(), er.get(), ev.get(), boff.get());
  SS_LAUNCH_CHECK();
  k_pr_steps<1><<<nblk(ne_max * S.W), 256, 0, st>>>(er.get(), boff.get() + S.P, 0, S.W, M, T.t0.get(), T.t1.get(),
                                                    T.b, estep.get());
  SS_LAUNCH_CHECK();
  const int64_t n_tiles = (S.Q + S.W - 1) / S.W;
  int wsh = 0;
  while ((1 << wsh) < S.W) ++wsh;
  const size_t smem = eval_smem(S);
  int grid = 0;
  ProfScope prof_("k_pr_eval", st);
  if (out_real) {
    SS_TRY(grid_for(k_pr_eval<true>, smem, n_tiles, &grid));
    k_pr_eval<true><<<grid, kPrThreads, smem, st>>>(M, S.P, S.Q, wsh, S.rad, T.t0.get(), T.t1.get(), T.b, er.get(),
                                                    ev.get(), boff.get(), estep.get(), n_tiles, out);
  } else {
    SS_TRY(grid_for(k_pr_eval<false>, smem, n_tiles, &grid));
    k_pr_eval<false><<<grid, kPrThreads, smem, st>>>(M, S.P, S.Q, wsh, S.rad, T.t0.get(), T.t1.get(), T.b, er.get(),
                                                     ev.get(), boff.get(), estep.get(), n_tiles, out);
  }
  SS_LAUNCH_CHECK();
  return SS_OK;
}

ss_status pruned_forward(const TwoLevelTable& T, const void* s, bool in_real, const int64_t* bins, int64_t n_out,
                         float4* X, cudaStream_t st) {
  const int64_t M = T.M;
  if (n_out < 1) return SS_OK;
  PrunedSplit S;
  if (!pruned_split(M, n_out, &S)) SS_FAIL(SS_ERR_INVALID, "pruned transform: M = %lld has no split", (long long)M);
  const int64_t n_tiles = (S.Q + S.W - 1) / S.W;
  int wsh = 0;
  while ((1 << wsh) < S.W) ++wsh;
  for (int64_t o0 = 0; o0 < n_out; o0 += kPrMaxOut) {
    const int nc = (int)std::min<int64_t>(kPrMaxOut, n_out - o0);
    DevBuf<int32_t> kout;
    DevBuf<float4> ostep, partial;
    SS_TRY(kout.alloc_tmp(nc, st));
    SS_TRY(ostep.alloc_tmp((size_t)nc * S.W, st));
    k_pr_kout<<<nblk(nc), 256, 0, st>>>(bins + o0, nc, S.P, kout.get());
    k_pr_steps<-1><<<nblk((int64_t)nc * S.W), 256, 0, st>>>(bins + o0, nullptr, nc, S.W, M, T.t0.get(), T.t1.get(),
                                                             T.b, ostep.get());
    SS_LAUNCH_CHECK();
    const size_t smem = fwd_smem(S, nc);
    int grid = 0;
    if (in_real) {
      SS_TRY(grid_for(k_pr_fwd<true>, smem, n_tiles, &grid));
    } else {
      SS_TRY(grid_for(k_pr_fwd<false>, smem, n_tiles, &grid));
    }
    SS_TRY(partial.alloc_tmp((size_t)grid * nc, st));
    ProfScope prof_("k_pr_fwd", st);
    if (in_real)
      k_pr_fwd<true><<<grid, kPrThreads, smem, st>>>(M, S.P, S.Q, wsh, S.rad, T.t0.get(), T.t1.get(), T.b, s,
                                                     bins + o0, kout.get(), nc, ostep.get(), n_tiles, partial.get());
    else
      k_pr_fwd<false><<<grid, kPrThreads, smem, st>>>(M, S.P, S.Q, wsh, S.rad, T.t0.get(), T.t1.get(), T.b, s,
                                                      bins + o0, kout.get(), nc, ostep.get(), n_tiles, partial.get());
    SS_LAUNCH_CHECK();
    k_pr_reduce<<<nblk((int64_t)nc * 32), 256, 0, st>>>(partial.get(), grid, nc, X + o0);
    SS_LAUNCH_CHECK();
  }
  return SS_OK;
}

}  // namespace ss
