// Monte Carlo form of the proxy error (Lemma ProxyError; Section "Code and
// testing overview"): r(x) = f(x) - f^{s,N}(x) at uniform random points of
// T^d, with f^{s,N} = L[a_hat] u^{s,N} known through its coefficients on
// S^{N+1} (Proposition LExpansion).  The work is a dense trigonometric sum of
// |terms| x |points| exponentials.
//
// Points lie on the grid (2^-32 Z)^d, so the phase k.x mod 1 of every term is
// the exact integer (k.X mod 2^32) / 2^32, formed with wrapping 32-bit
// multiply-adds.  exp(2 pi i ph / 2^32) is the product of three table entries
// (bits 31..21, 20..10 and 9..0 of ph) held in shared memory as double-float
// values, and every product and the running sum are double-float: the whole
// inner loop stays on the FP32 pipe, which issues two orders of magnitude more
// operations per clock than the FP64 pipe on this part.
#include <algorithm>

#include "df.cuh"
#include "ss_internal.cuh"

namespace ss {
namespace {

constexpr int kMcThreads = 256;          // points per block, one per thread
constexpr int kTab0 = 2048;              // exp(2 pi i h / 2^11)
constexpr int kTab1 = 2048;              // exp(2 pi i m / 2^22)
constexpr int kTab2 = 1024;              // exp(2 pi i l / 2^32)
constexpr int kTabAll = kTab0 + kTab1 + kTab2;
constexpr size_t kTabBytes = kTabAll * sizeof(float4);

inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

__global__ void k_mc_tables(float4* tab) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kTabAll) return;
  double num, den;
  if (i < kTab0) {
    num = i; den = 2048.0;
  } else if (i < kTab0 + kTab1) {
    num = i - kTab0; den = 4194304.0;
  } else {
    num = i - kTab0 - kTab1; den = 4294967296.0;
  }
  double s, c;
  sincospi(2.0 * num / den, &s, &c);        // num / den is exact (den a power of two)
  const DF cc = df_split(c), ss_ = df_split(s);
  tab[i] = make_float4(cc.hi, cc.lo, ss_.hi, ss_.lo);
}

// rows of int32 [n][d] -> [n][d4], zero padded (d4 = d rounded up to 4).
__global__ void k_pad_rows(const int32_t* __restrict__ src, int64_t n, int d, int d4, int32_t* __restrict__ dst) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * d4) return;
  const int64_t r = i / d4;
  const int c = (int)(i % d4);
  dst[i] = c < d ? src[r * d + c] : 0;
}

// Term coefficients in double-float, optionally negated.
__global__ void k_coef_df(const double2* __restrict__ c, int64_t n, double sign, float4* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double2 v = c[i];
  const DF re = df_split(sign * v.x), im = df_split(sign * v.y);
  out[i] = make_float4(re.hi, re.lo, im.hi, im.lo);
}

// part[chunk][q] = sum over the chunk's terms t of Re(c_t exp(2 pi i k_t.x_q)).
// Block (x: 256 points, y: one chunk of terms).  Per term the thread forms the
// exact phase, gathers three table entries and does five double-float complex
// half-products: B = c e0, C = B e1, acc += Re(C e2).
__global__ void __launch_bounds__(kMcThreads, 2)
k_mc_terms(const int32_t* __restrict__ K, const float4* __restrict__ coef, int64_t n_terms, int d4,
           const uint32_t* __restrict__ X, int64_t Q, int64_t terms_per_chunk, const float4* __restrict__ tab,
           double* __restrict__ part) {
  extern __shared__ float4 s_tab[];
  for (int i = threadIdx.x; i < kTabAll; i += blockDim.x) s_tab[i] = tab[i];
  __syncthreads();
  const int64_t q = (int64_t)blockIdx.x * kMcThreads + threadIdx.x;
  const bool live = q < Q;
  const int64_t t0 = (int64_t)blockIdx.y * terms_per_chunk;
  const int64_t t1 = (n_terms - t0 < terms_per_chunk) ? n_terms : t0 + terms_per_chunk;
  const int n4 = d4 / 4;
  const uint4* xq = reinterpret_cast<const uint4*>(X + (live ? q : 0) * (int64_t)d4);
  const float4* t_hi = s_tab;
  const float4* t_mid = s_tab + kTab0;
  const float4* t_lo = s_tab + kTab0 + kTab1;
  DF acc{0.f, 0.f};
  for (int64_t t = t0; t < t1; ++t) {
    const int4* kt = reinterpret_cast<const int4*>(K + t * d4);
    uint32_t ph = 0;
    for (int c = 0; c < n4; ++c) {
      const int4 k = __ldg(kt + c);
      const uint4 x = __ldg(xq + c);
      ph += (uint32_t)k.x * x.x + (uint32_t)k.y * x.y + (uint32_t)k.z * x.z + (uint32_t)k.w * x.w;
    }
    const float4 cf = __ldg(coef + t);
    const float4 e0 = t_hi[ph >> 21];
    const float4 e1 = t_mid[(ph >> 10) & 2047u];
    const float4 e2 = t_lo[ph & 1023u];
    DF br{0.f, 0.f}, bi{0.f, 0.f};
    df_fma(br, DF{cf.x, cf.y}, DF{e0.x, e0.y});
    df_fma(br, DF{-cf.z, -cf.w}, DF{e0.z, e0.w});
    df_fma(bi, DF{cf.x, cf.y}, DF{e0.z, e0.w});
    df_fma(bi, DF{cf.z, cf.w}, DF{e0.x, e0.y});
    DF cr{0.f, 0.f}, ci{0.f, 0.f};
    df_fma(cr, br, DF{e1.x, e1.y});
    df_fma(cr, DF{-bi.hi, -bi.lo}, DF{e1.z, e1.w});
    df_fma(ci, br, DF{e1.z, e1.w});
    df_fma(ci, bi, DF{e1.x, e1.y});
    df_fma(acc, cr, DF{e2.x, e2.y});
    df_fma(acc, DF{-ci.hi, -ci.lo}, DF{e2.z, e2.w});
  }
  if (live) part[(int64_t)blockIdx.y * Q + q] = (double)acc.hi + (double)acc.lo;
}

// r[q] = sum_c pf[c][q] + sum_c pg[c][q] (pg holds -f^{s,N}), f[q] = sum_c pf[c][q],
// chunks summed in index order.
__global__ void k_mc_finish(const double* __restrict__ pf, int cf, const double* __restrict__ pg, int cg, int64_t Q,
                            double* __restrict__ r, double* __restrict__ f) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= Q) return;
  double sf = 0.0, sg = 0.0;
  for (int c = 0; c < cf; ++c) sf += pf[(int64_t)c * Q + q];
  for (int c = 0; c < cg; ++c) sg += pg[(int64_t)c * Q + q];
  f[q] = sf;
  r[q] = sf + sg;
}

// Terms split into chunks so that the grid covers the SMs several times over.
int64_t terms_per_chunk(int64_t n_terms, int64_t point_tiles) {
  const int64_t want_blocks = 8LL * 2 * sm_count();
  int64_t chunks = (want_blocks + point_tiles - 1) / point_tiles;
  chunks = std::max<int64_t>(1, std::min<int64_t>(chunks, (n_terms + 63) / 64));
  chunks = std::min<int64_t>(chunks, 65535);
  return (n_terms + chunks - 1) / chunks;
}

ss_status run_terms(const int32_t* K, const float4* coef, int64_t n_terms, int d4, const uint32_t* X, int64_t Q,
                    const float4* tab, DevBuf<double>& part, int* chunks_out, cudaStream_t st) {
  const int64_t tiles = (Q + kMcThreads - 1) / kMcThreads;
  if (n_terms == 0) {
    *chunks_out = 0;
    return SS_OK;
  }
  const int64_t tpc = terms_per_chunk(n_terms, tiles);
  const int chunks = (int)((n_terms + tpc - 1) / tpc);
  SS_TRY(part.alloc((size_t)chunks * Q, st));
  k_mc_terms<<<dim3((unsigned)tiles, (unsigned)chunks), kMcThreads, kTabBytes, st>>>(K, coef, n_terms, d4, X, Q, tpc,
                                                                                   tab, part.get());
  SS_LAUNCH_CHECK();
  *chunks_out = chunks;
  return SS_OK;
}

}  // namespace
}  // namespace ss

using namespace ss;

extern "C" ss_status proxy_mc(ss_stamp s, const double* u_prefix, int64_t n_u, const ss_trig* f, const uint32_t* X,
                              int64_t Q, double* r_out, double* f_out, void* stream) {
  if (!s || !f || (n_u > 0 && !u_prefix) || (Q > 0 && (!X || !r_out || !f_out)))
    SS_FAIL(SS_ERR_INVALID, "proxy_mc: null argument");
  if (f->d != s->d) SS_FAIL(SS_ERR_INVALID, "proxy_mc: dimension %d != %d", f->d, s->d);
  if (n_u < 0 || n_u > s->size) SS_FAIL(SS_ERR_INVALID, "proxy_mc: n_u = %lld outside [0, |S|]", (long long)n_u);
  if (Q < 0 || f->n_terms < 0 || (f->n_terms > 0 && (!f->freq || !f->coef)))
    SS_FAIL(SS_ERR_INVALID, "proxy_mc: bad sizes");
  if (Q == 0) return SS_OK;
  SS_CUDA(cudaFuncSetAttribute(k_mc_terms, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTabBytes));
  cudaStream_t st = as_stream(stream);
  const int d = s->d, d4 = (d + 3) / 4 * 4;
  // rows are read as 16-byte vectors: copy when d is not a multiple of 4 or
  // the caller's array is not 16-byte aligned
  auto needs_copy = [&](const void* p) { return d4 != d || (reinterpret_cast<uintptr_t>(p) & 15u) != 0; };
  DevBuf<float4> tab, cf_f, cf_g;
  DevBuf<int32_t> Kf, Kg, tmp;
  DevBuf<uint32_t> Xp;
  DevBuf<double2> y;
  DevBuf<double> pf, pg;
  SS_TRY(tab.alloc(kTabAll, st));
  k_mc_tables<<<nblk(kTabAll), 256, 0, st>>>(tab.get());
  SS_LAUNCH_CHECK();
  // points, padded
  const uint32_t* Xd = X;
  if (needs_copy(X)) {
    SS_TRY(Xp.alloc((size_t)Q * d4, st));
    k_pad_rows<<<nblk(Q * d4), 256, 0, st>>>(reinterpret_cast<const int32_t*>(X), Q, d, d4,
                                              reinterpret_cast<int32_t*>(Xp.get()));
    SS_LAUNCH_CHECK();
    Xd = Xp.get();
  }
  // f's terms
  const int64_t nf = f->n_terms;
  const int32_t* Kfd = f->freq;
  if (nf > 0) {
    SS_TRY(cf_f.alloc(nf, st));
    k_coef_df<<<nblk(nf), 256, 0, st>>>(reinterpret_cast<const double2*>(f->coef), nf, 1.0, cf_f.get());
    SS_LAUNCH_CHECK();
    if (needs_copy(f->freq)) {
      SS_TRY(Kf.alloc((size_t)nf * d4, st));
      k_pad_rows<<<nblk(nf * d4), 256, 0, st>>>(f->freq, nf, d, d4, Kf.get());
      SS_LAUNCH_CHECK();
      Kfd = Kf.get();
    }
  }
  // f^{s,N} on S: L applied to u (prefix), then S's frequencies, padded
  const int64_t ng = s->size;
  const int32_t* Kgd = nullptr;
  if (ng > 0) {
    SS_TRY(launch_pack64_prefix(s, reinterpret_cast<const double2*>(u_prefix), n_u, st));
    SS_TRY(y.alloc(ng, st));
    SS_TRY(launch_apply64(s, y.get(), st));
    // (L u)_0 = 0 exactly for the diffusion operator (the factor k.l); its
    // stored identity row is for the solve
    if (identity_row(s) >= 0) SS_CUDA(cudaMemsetAsync(y.get() + identity_row(s), 0, sizeof(double2), st));
    SS_TRY(cf_g.alloc(ng, st));
    k_coef_df<<<nblk(ng), 256, 0, st>>>(y.get(), ng, -1.0, cf_g.get());
    SS_LAUNCH_CHECK();
    SS_TRY(tmp.alloc((size_t)ng * d, st));
    SS_TRY((ss_status)stamp_export(s, tmp.get(), nullptr, st));
    if (d4 != d) {
      SS_TRY(Kg.alloc((size_t)ng * d4, st));
      k_pad_rows<<<nblk(ng * d4), 256, 0, st>>>(tmp.get(), ng, d, d4, Kg.get());
      SS_LAUNCH_CHECK();
      Kgd = Kg.get();
    } else {
      Kgd = tmp.get();
    }
  }
  int cfn = 0, cgn = 0;
  SS_TRY(run_terms(Kfd, cf_f.get(), nf, d4, Xd, Q, tab.get(), pf, &cfn, st));
  SS_TRY(run_terms(Kgd, cf_g.get(), ng, d4, Xd, Q, tab.get(), pg, &cgn, st));
  k_mc_finish<<<nblk(Q), 256, 0, st>>>(pf.get(), cfn, pg.get(), cgn, Q, r_out, f_out);
  SS_LAUNCH_CHECK();
  return SS_OK;
}
