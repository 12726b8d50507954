// Stamping set S^N[a_hat](F) (eq. StampSet) built level by level on the GPU,
// and the sliced-ELL neighbour table of the Galerkin operator.
//
// Level n is S^{n-1} + supp(a_hat) minus S^{n-1}.  Candidate c = (parent,
// step j) of level n gets the discovery key c = (parent - start) * s_a + j.
// Every candidate probes the open-addressing table: a slot holding a
// canonical index from an earlier level with the same key drops the
// candidate; an empty slot is claimed with kPending | c; a pending slot with
// the same key takes atomicMin(kPending | c).  After the pass, the winner of
// every new frequency is the candidate with the smallest discovery key, and a
// prefix sum over the winners in discovery order gives the canonical order
// (first discovery over parents in index order and steps in lexicographic
// order).  Keys of pending slots are never stored: they are re-derived from
// the parent key and the step, so a claim is one 64-bit CAS.  Every slot word
// also carries a 31-bit fingerprint of the key hash, so probes compare stored
// keys (up to 12 words at d = 100) only when the fingerprints agree.
#include <atomic>
#include <algorithm>
#include <cmath>
#include <map>

#include "keys.cuh"
#include "scan.cuh"

namespace ss {
namespace {

// a_hat counts as real (a even) when no imaginary part exceeds this fraction
// of max |a_hat|: below the rounding of an FP64 recovery (the FFT leaves
// imaginary parts of order 1e-16 to 1e-14 of the largest coefficient on an
// even a).  The imaginary parts are then dropped at build and every entry
// coefficient is real.
constexpr double kRealTol = 1e-13;

__global__ void k_real_part(double2* av, int n) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) av[j].y = 0.0;
}

struct PrepOut {
  int32_t maxabs_f, maxabs_a;
  int32_t dup_f, dup_a;
  int32_t bad_sym, zero_in_f, bad_herm, j0;
  int32_t f_sym, herm_exact;   // F = -F (F sorted); a_hat_{-p} == conj(a_hat_p) bit for bit
  int32_t a_real;              // every |Im a_hat_p| <= kRealTol max |a_hat| (a even)
  double a0_re, a0_abs, off_l1, amax;
};

__device__ int lexcmp(const int32_t* a, const int32_t* b, int d) {
  for (int c = 0; c < d; ++c) {
    if (a[c] != b[c]) return a[c] < b[c] ? -1 : 1;
  }
  return 0;
}

// Stable lexicographic rank of every row (rank must start at zero); flags
// duplicates.  Thread (i, c) compares row i with rows [chunk c, chunk (c + 1));
// the threads of a warp share c, so the rows of the chunk are broadcast loads.
// Short chunks for small sets (more threads, shorter dependent chains of
// loads), long ones for large sets (fewer atomics).
inline int rank_chunk(int64_t n) { return n <= 8192 ? 16 : 64; }

// Wide rows (d > 16): one block per row i; its warps take the rows j in turn
// and compare 32 coordinates per step (coalesced), the first differing
// coordinate found by a ballot.  rank[i] is written once per block.
constexpr int kLexWarps = 8;

__global__ void __launch_bounds__(32 * kLexWarps) k_lex_rank_wide(const int32_t* __restrict__ f, int64_t n, int d,
                                                                   int32_t* rank, int32_t* dup) {
  __shared__ int32_t s_r[kLexWarps];
  __shared__ int s_du[kLexWarps];
  const int64_t i = blockIdx.x;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int32_t* fi = f + i * d;
  int32_t r = 0;
  bool du = false;
  for (int64_t j = w; j < n; j += kLexWarps) {
    const int32_t* fj = f + j * d;
    int cmp = 0;
    for (int c0 = 0; c0 < d && cmp == 0; c0 += 32) {
      const int c = c0 + lane;
      const int32_t a = c < d ? __ldg(fj + c) : 0, b = c < d ? __ldg(fi + c) : 0;
      const unsigned m = __ballot_sync(0xffffffffu, a != b);
      if (m) {
        const int src = __ffs(m) - 1;
        cmp = __shfl_sync(0xffffffffu, a, src) < __shfl_sync(0xffffffffu, b, src) ? -1 : 1;
      }
    }
    r += (cmp < 0 || (cmp == 0 && j < i)) ? 1 : 0;
    du |= (cmp == 0 && j != i);
  }
  if (lane == 0) {
    s_r[w] = r;
    s_du[w] = du;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int32_t t = 0;
    int any = 0;
    for (int k = 0; k < kLexWarps; ++k) {
      t += s_r[k];
      any |= s_du[k];
    }
    rank[i] = t;
    if (any) atomicExch(dup, 1);
  }
}

__global__ void k_lex_rank(const int32_t* __restrict__ f, int64_t n, int d, int32_t* rank, int32_t* dup, int chunk) {
  const int64_t nc = (n + chunk - 1) / chunk;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * nc) return;
  const int64_t c = t / n, i = t - c * n;
  const int64_t j1 = min(n, (c + 1) * chunk);
  int32_t r = 0;
  bool du = false;
  for (int64_t j = c * chunk; j < j1; ++j) {
    const int cmp = lexcmp(f + j * d, f + i * d, d);
    if (cmp < 0 || (cmp == 0 && j < i)) ++r;
    if (cmp == 0 && j != i) du = true;
  }
  if (r) atomicAdd(rank + i, r);
  if (du) atomicExch(dup, 1);
}

__global__ void k_scatter_rows(const int32_t* __restrict__ f, const double2* __restrict__ v, int64_t n, int d,
                               const int32_t* __restrict__ rank, int32_t* fo, double2* vo) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t r = rank[i];
  for (int c = 0; c < d; ++c) fo[r * d + c] = f[i * d + c];
  if (v) vo[r] = v[i];
}

// One block: ranges, symmetry of supp a_hat (a sorted symmetric set satisfies
// A[j] = -A[s-1-j]), the zero step, Hermitian values, positivity check.
// Input checks and ranges in one block: every thread takes its share of the
// rows, the pairs (p_j, p_{s_a-1-j}) and the |a_hat_j|; thread 0 only adds
// the |a_hat_j| in index order (deterministic) and writes the result.
constexpr int kPrepThreads = 512;

__global__ void __launch_bounds__(kPrepThreads) k_prep(const int32_t* __restrict__ F, int64_t n_f,
                                                       const int32_t* __restrict__ A,
                                                       const double2* __restrict__ av, int s_a, int d, PrepOut* out) {
  __shared__ int32_t s_maxf, s_maxa, s_zf, s_sym, s_herm, s_fasym, s_hinexact, s_aimag;
  __shared__ unsigned long long s_amax;
  __shared__ double s_hyp[4096];
  if (threadIdx.x == 0) {
    s_maxf = 0; s_maxa = 0; s_zf = 0; s_sym = (s_a % 2 == 0); s_herm = 0; s_amax = 0; s_fasym = 0; s_hinexact = 0; s_aimag = 0;
  }
  __syncthreads();
  int32_t mf = 0;
  for (int64_t i = threadIdx.x; i < n_f; i += blockDim.x) {
    bool zero = true;
    for (int c = 0; c < d; ++c) {
      const int32_t x = F[i * d + c];
      mf = max(mf, abs(x));
      zero &= (x == 0);
    }
    if (zero) atomicExch(&s_zf, 1);
    // F sorted lexicographically: F = -F iff row i is minus row n_f - 1 - i
    const int64_t m = n_f - 1 - i;
    for (int c = 0; c < d; ++c)
      if (F[i * d + c] != -F[m * d + c]) atomicExch(&s_fasym, 1);
  }
  atomicMax(&s_maxf, mf);
  int32_t ma = 0;
  for (int64_t i = threadIdx.x; i < (int64_t)s_a * d; i += blockDim.x) ma = max(ma, abs(A[i]));
  atomicMax(&s_maxa, ma);
  const int j0 = (s_a - 1) / 2;
  for (int j = threadIdx.x; j < s_a; j += blockDim.x) {
    const double h = hypot(av[j].x, av[j].y);
    s_hyp[j] = h;
    atomicMax(&s_amax, (unsigned long long)__double_as_longlong(h));   // h >= 0: integer order is value order
    const int m = s_a - 1 - j;
    for (int c = 0; c < d; ++c)
      if (A[j * d + c] != -A[m * d + c]) atomicExch(&s_sym, 1);
  }
  if (threadIdx.x == 0 && s_a % 2 == 1)
    for (int c = 0; c < d; ++c)
      if (A[j0 * d + c] != 0) atomicExch(&s_sym, 1);
  __syncthreads();
  const double amax = __longlong_as_double((long long)s_amax);
  for (int j = threadIdx.x; j < s_a; j += blockDim.x) {
    const int m = s_a - 1 - j;
    if (fabs(av[j].x - av[m].x) > 1e-12 * amax || fabs(av[j].y + av[m].y) > 1e-12 * amax) atomicExch(&s_herm, 1);
    if (!(av[j].x == av[m].x && av[j].y == -av[m].y)) atomicExch(&s_hinexact, 1);
    if (fabs(av[j].y) > kRealTol * amax) atomicExch(&s_aimag, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    out->maxabs_f = s_maxf;
    out->maxabs_a = s_maxa;
    out->zero_in_f = s_zf;
    const int bad_sym = s_sym;
    double off = 0;
    for (int j = 0; j < s_a; ++j)
      if (j != j0) off += s_hyp[j];
    out->bad_sym = bad_sym;
    out->bad_herm = bad_sym ? 0 : s_herm;
    out->j0 = j0;
    out->a0_re = bad_sym ? 0.0 : av[j0].x;
    out->a0_abs = bad_sym ? 0.0 : hypot(av[j0].x, av[j0].y);
    out->off_l1 = off;
    out->amax = amax;
    out->f_sym = !s_fasym;
    out->herm_exact = !bad_sym && !s_hinexact;
    out->a_real = !s_aimag;
  }
}

template <int WT>
__global__ void k_steps(KeyParams P, const int32_t* __restrict__ A, const double2* __restrict__ av, int s_a,
                        uint64_t* stepkey, uint64_t* stepg, int64_t* pnorm, int32_t* pn32, bool wide, double2* ca64,
                        float2* ca32) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= s_a) return;
  uint64_t k[WT];
  pack_key<WT>(A + (int64_t)j * P.d, P, k);
#pragma unroll
  for (int w = 0; w < WT; ++w) stepkey[(int64_t)j * WT + w] = k[w];
  stepg[j] = key_lin<WT>(k) - P.lin_bias;   // key_lin(k + p_j - bias) = key_lin(k) + stepg[j]
  int64_t s = 0;
  for (int c = 0; c < P.d; ++c) s += (int64_t)A[(int64_t)j * P.d + c] * A[(int64_t)j * P.d + c];
  pnorm[j] = s;
  pn32[j] = norm_word(s, wide);
  const double2 a = av[j];
  ca64[j] = make_double2(kTwoPiSq * a.x, kTwoPiSq * a.y);
  ca32[j] = make_float2((float)(kTwoPiSq * a.x), (float)(kTwoPiSq * a.y));
}

// Warp-cooperative packing for wide rows (d > 16): lane l takes coordinates
// c = l, l + 32, ... and ORs its fields into the warp's words in shared memory
// (the fields do not overlap); returns whether every coordinate fits, and the
// row's |k|^2 (both to every lane).  Lanes w < WT then read word w.
constexpr int kPackWarps = 8;

template <int WT>
__device__ __forceinline__ bool warp_pack(const int32_t* __restrict__ k, const KeyParams& P, unsigned long long* words,
                                          int64_t* norm2) {
  const int lane = threadIdx.x & 31;
  if (lane < WT) words[lane] = 0ull;
  __syncwarp();
  bool ok = true;
  int64_t n2 = 0;
  for (int c = lane; c < P.d; c += 32) {
    const int64_t kc = k[c];
    n2 += kc * kc;
    const int64_t v = kc + P.bias_val;
    ok &= (v >= 0) && (v <= (int64_t)P.fieldmask);
    const int wd = c / P.fpw, sh = 64 - P.fb * (c % P.fpw + 1);
    atomicOr(words + wd, (unsigned long long)(((uint64_t)v & P.fieldmask) << sh));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) n2 += __shfl_xor_sync(0xffffffffu, n2, o);
  __syncwarp();
  *norm2 = n2;
  return __all_sync(0xffffffffu, ok);
}

// The linear form of the packed words held by lanes w < WT (sum mod 2^64).
template <int WT>
__device__ __forceinline__ uint64_t warp_lin(uint64_t word) {
  const int lane = threadIdx.x & 31;
  uint64_t lin = lane < WT ? key_lin_coef(lane) * word : 0ull;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) lin += __shfl_xor_sync(0xffffffffu, lin, o);
  return lin;
}

// k_steps with one warp per step (d > 16).
template <int WT>
__global__ void __launch_bounds__(32 * kPackWarps) k_steps_warp(KeyParams P, const int32_t* __restrict__ A,
                                                                const double2* __restrict__ av, int s_a,
                                                                uint64_t* stepkey, uint64_t* stepg, int64_t* pnorm,
                                                                int32_t* pn32, bool wide, double2* ca64,
                                                                float2* ca32) {
  __shared__ unsigned long long s_w[kPackWarps][WT];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int j = blockIdx.x * kPackWarps + w;
  if (j >= s_a) return;   // warp-uniform
  int64_t n2 = 0;
  warp_pack<WT>(A + (int64_t)j * P.d, P, s_w[w], &n2);
  const uint64_t kw = lane < WT ? (uint64_t)s_w[w][lane] : 0ull;
  if (lane < WT) stepkey[(int64_t)j * WT + lane] = kw;
  const uint64_t lin = warp_lin<WT>(kw);
  if (lane != 0) return;
  stepg[j] = lin - P.lin_bias;   // key_lin(k + p_j - bias) = key_lin(k) + stepg[j]
  pnorm[j] = n2;
  pn32[j] = norm_word(n2, wide);
  const double2 a = av[j];
  ca64[j] = make_double2(kTwoPiSq * a.x, kTwoPiSq * a.y);
  ca32[j] = make_float2((float)(kTwoPiSq * a.x), (float)(kTwoPiSq * a.y));
}

// Insert a finalised key (hash hh) with value idx (no duplicates present).
__device__ bool table_insert_final(uint64_t* table, uint64_t capmask, uint64_t hh, uint64_t idx) {
  const uint64_t word = slot_word(slot_fp(hh), idx);
  uint64_t h = hh & capmask;
  for (uint64_t probe = 0; probe <= capmask; ++probe) {
    const uint64_t old = atomicCAS((unsigned long long*)(table + h), (unsigned long long)kEmpty,
                                   (unsigned long long)word);
    if (old == kEmpty) return true;
    h = (h + 1) & capmask;
  }
  return false;
}

template <int WT>
__global__ void k_level0(KeyParams P, const int32_t* __restrict__ F, int64_t n_f, uint64_t* keys, uint64_t* hl,
                         int8_t* level, int64_t* norm, uint64_t* table, uint64_t capmask, int32_t* err,
                         int64_t* zero_idx) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_f) return;
  uint64_t k[WT];
  pack_key<WT>(F + i * P.d, P, k);
#pragma unroll
  for (int w = 0; w < WT; ++w) keys[i * WT + w] = k[w];
  const uint64_t lin = key_lin<WT>(k);
  hl[i] = lin;
  level[i] = 0;
  norm[i] = key_norm<WT>(k, P);
  if (norm[i] == 0) *zero_idx = i;   // only when 0 is in F (allowed for the ADR operator)
  if (!table_insert_final(table, capmask, hash_of_lin(lin), (uint64_t)i)) atomicExch(err, SS_ERR_HASH_FULL);
}

// k_level0 with one warp per row (d > 16).
template <int WT>
__global__ void __launch_bounds__(32 * kPackWarps) k_level0_warp(KeyParams P, const int32_t* __restrict__ F,
                                                                 int64_t n_f, uint64_t* keys, uint64_t* hl,
                                                                 int8_t* level, int64_t* norm, uint64_t* table,
                                                                 uint64_t capmask, int32_t* err, int64_t* zero_idx) {
  __shared__ unsigned long long s_w[kPackWarps][WT];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t i = (int64_t)blockIdx.x * kPackWarps + w;
  if (i >= n_f) return;   // warp-uniform
  int64_t n2 = 0;
  warp_pack<WT>(F + i * P.d, P, s_w[w], &n2);
  const uint64_t kw = lane < WT ? (uint64_t)s_w[w][lane] : 0ull;
  if (lane < WT) keys[i * WT + lane] = kw;
  const uint64_t lin = warp_lin<WT>(kw);
  if (lane != 0) return;
  hl[i] = lin;
  level[i] = 0;
  norm[i] = n2;
  if (n2 == 0) *zero_idx = i;   // only when 0 is in F (allowed for the ADR operator)
  if (!table_insert_final(table, capmask, hash_of_lin(lin), (uint64_t)i)) atomicExch(err, SS_ERR_HASH_FULL);
}

template <int WT>
__global__ void k_pack_rows(KeyParams P, const int32_t* __restrict__ freq, int64_t n, uint64_t* keys, uint64_t* hl) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint64_t k[WT];
  pack_key<WT>(freq + i * P.d, P, k);
#pragma unroll
  for (int w = 0; w < WT; ++w) keys[i * WT + w] = k[w];
  hl[i] = key_lin<WT>(k);
}

__global__ void k_rehash(const uint64_t* __restrict__ hl, int64_t size, uint64_t* table, uint64_t capmask,
                         int32_t* err) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= size) return;
  if (!table_insert_final(table, capmask, hash_of_lin(hl[i]), (uint64_t)i)) atomicExch(err, SS_ERR_HASH_FULL);
}

// (a1 + b1) == (a2 + b2) word by word: two packed frequency + step sums are
// the same frequency (the bias they both carry cancels).
template <int WT>
__device__ __forceinline__ bool sums_equal(const uint64_t* __restrict__ a1, const uint64_t* __restrict__ b1,
                                           const uint64_t* __restrict__ a2, const uint64_t* __restrict__ b2) {
  bool e = true;
  if constexpr (WT % 2 == 0) {
#pragma unroll
    for (int w = 0; w < WT; w += 2) {
      const ulonglong2 x1 = __ldg(reinterpret_cast<const ulonglong2*>(a1 + w));
      const ulonglong2 y1 = __ldg(reinterpret_cast<const ulonglong2*>(b1 + w));
      const ulonglong2 x2 = __ldg(reinterpret_cast<const ulonglong2*>(a2 + w));
      const ulonglong2 y2 = __ldg(reinterpret_cast<const ulonglong2*>(b2 + w));
      e &= (x1.x + y1.x == x2.x + y2.x) & (x1.y + y1.y == x2.y + y2.y);
    }
  } else {
#pragma unroll
    for (int w = 0; w < WT; ++w) e &= __ldg(a1 + w) + __ldg(b1 + w) == __ldg(a2 + w) + __ldg(b2 + w);
  }
  return e;
}

// Candidate pass of one level (see the file comment).  The candidate's hash
// comes from the linear forms (hl[parent] + stepg[j]); words are read only to
// confirm a slot whose fingerprint and linear form agree.
template <int WT>
__global__ void k_insert(KeyParams P, const uint64_t* __restrict__ keys, const uint64_t* __restrict__ hl, int64_t par0,
                         int64_t n_par, int s_a, int j0, const uint64_t* __restrict__ stepkey,
                         const uint64_t* __restrict__ stepg, uint64_t* table, uint64_t capmask, int64_t* slot_of,
                         int32_t* err) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_par * s_a) return;
  const int64_t par = (uint32_t)c / (uint32_t)s_a;   // candidate ids stay below 2^32
  const int j = (int)(c - par * s_a);
  if (j == j0) { slot_of[c] = -1; return; }
  const uint64_t lin = __ldg(hl + par0 + par) + __ldg(stepg + j);
  const uint64_t* pk = keys + (par0 + par) * WT;
  const uint64_t* sk = stepkey + (int64_t)j * WT;
  const uint64_t hh = hash_of_lin(lin), fp = slot_fp(hh);
  const uint64_t mine = kPending | slot_word(fp, (uint64_t)c);
  uint64_t h = hh & capmask;
  for (uint64_t probe = 0; probe <= capmask; ++probe) {
    uint64_t v = __ldcg((const unsigned long long*)(table + h));
    if (v == kEmpty) {
      const uint64_t old = atomicCAS((unsigned long long*)(table + h), (unsigned long long)kEmpty,
                                     (unsigned long long)mine);
      if (old == kEmpty) { slot_of[c] = (int64_t)h; return; }
      v = old;
    }
    if (word_fp(v) == fp) {
      if (v & kPending) {
        const int64_t oc = (int64_t)word_low(v);
        const int64_t opar = (uint32_t)oc / (uint32_t)s_a;
        const int oj = (int)(oc - opar * s_a);
        if (__ldg(hl + par0 + opar) + __ldg(stepg + oj) == lin &&
            sums_equal<WT>(keys + (par0 + opar) * WT, stepkey + (int64_t)oj * WT, pk, sk)) {
          // same key, same fingerprint: the minimum keeps the smallest candidate
          // id (the slot's id only decreases, so a smaller one seen here stays)
          if (oc > c) atomicMin((unsigned long long*)(table + h), (unsigned long long)mine);
          slot_of[c] = (int64_t)h;
          return;
        }
      } else {
        const int64_t o = (int64_t)word_low(v);
        if (__ldg(hl + o) == lin && key_eq_sum<WT>(keys + o * WT, pk, sk, P)) { slot_of[c] = -1; return; }
      }
    }
    h = (h + 1) & capmask;
  }
  atomicExch(err, SS_ERR_HASH_FULL);
  slot_of[c] = -1;
}

// A candidate wins when its slot still holds its own (pending) id: the
// smallest id among the candidates of one new key.
struct WinnerFlag {
  const int64_t* slot_of;
  const uint64_t* table;
  __device__ int32_t operator()(int64_t c) const {
    const int64_t s = slot_of[c];
    if (s < 0) return 0;
    const uint64_t v = __ldg(table + s);
    return ((v & kPending) && word_low(v) == (uint64_t)c) ? 1 : 0;
  }
};

// The winners in canonical order: cand[prefix] = c.
struct WinnerPut {
  int64_t* cand;
  __device__ void operator()(int64_t c, int32_t win, int64_t prefix) const {
    if (win) cand[prefix] = c;
  }
};

// k . p over the fields where the step p is nonzero (k, p packed; a step
// usually touches few coordinates).  The highest set bit of p ^ bias lies in
// the value bits of the first differing field of the word (the guard bit
// above each field is zero in both).
template <int WT>
__device__ __forceinline__ int64_t dot_step(const uint64_t* k, const uint64_t* p, const KeyParams& P) {
  int64_t s = 0;
#pragma unroll
  for (int w = 0; w < WT; ++w) {
    uint64_t x = p[w] ^ P.bias[w];
    while (x) {
      const int f = __clzll(x) / P.fb;
      const int sh = 64 - P.fb * (f + 1);
      const int64_t kv = (int64_t)((k[w] >> sh) & P.fieldmask) - P.bias_val;
      const int64_t pv = (int64_t)((p[w] >> sh) & P.fieldmask) - P.bias_val;
      s += kv * pv;
      x = sh ? (x & ((1ull << sh) - 1)) : 0;
    }
  }
  return s;
}

// One thread per new element t (canonical index base + t), so the key
// arithmetic runs in full warps; the block's new keys are staged in shared
// memory and stored as one contiguous run (coalesced).  |k + p|^2 = |k|^2 +
// |p|^2 + 2 k.p from the parent's norm.
constexpr int kFinThreads = 256;

template <int WT>
__global__ void __launch_bounds__(kFinThreads) k_finalize(KeyParams P, uint64_t* keys, uint64_t* hl, int64_t par0,
                                                          int s_a, const uint64_t* __restrict__ stepkey,
                                                          const uint64_t* __restrict__ stepg,
                                                          const int64_t* __restrict__ pnorm,
                                                          const int64_t* __restrict__ slot_of,
                                                          const int64_t* __restrict__ cand, int64_t added,
                                                          int64_t base, int lvl, int8_t* level, int64_t* norm,
                                                          uint64_t* table, int64_t* zero_idx) {
  __shared__ uint64_t stage[kFinThreads * WT];
  const int64_t t0 = (int64_t)blockIdx.x * kFinThreads;
  const int64_t t = t0 + threadIdx.x;
  if (t < added) {
    const int64_t c = cand[t];
    const int64_t par = (uint32_t)c / (uint32_t)s_a;   // candidate ids stay below 2^32
    const int j = (int)(c - par * s_a);
    uint64_t pk[WT], sk[WT], ck[WT];
    load_key<WT>(keys, par0 + par, pk);
    load_key<WT>(stepkey, j, sk);
    add_keys<WT>(pk, sk, P, ck);
#pragma unroll
    for (int w = 0; w < WT; ++w) stage[threadIdx.x * WT + w] = ck[w];
    const int64_t idx = base + t;
    const uint64_t lin = hl[par0 + par] + __ldg(stepg + j);
    hl[idx] = lin;
    level[idx] = (int8_t)lvl;
    const int64_t nr = norm[par0 + par] + __ldg(pnorm + j) + 2 * dot_step<WT>(pk, sk, P);
    norm[idx] = nr;
    if (nr == 0) *zero_idx = idx;
    table[slot_of[c]] = slot_word(slot_fp(hash_of_lin(lin)), (uint64_t)idx);
  }
  __syncthreads();
  const int64_t rows = added - t0 < kFinThreads ? added - t0 : kFinThreads;
  uint64_t* dst = keys + (base + t0) * WT;
  for (int64_t q = threadIdx.x; q < rows * WT; q += kFinThreads) dst[q] = stage[q];
}

// Neighbour words: for row i and step j, the index of k_i - p_j when it lies
// in S, is not 0, and k_i is not 0; else -1.  Steps j <= j0 are in
// lo[i Ls + j] (L = j0 + 1 of them), steps j > j0 in hi[i Hs + j - L] (H =
// s_a - L); row-major with the row strides Ls, Hs rounded up to multiples of 4
// (16-byte rows, padding -1), so one row moves as a few int4 words.  A row
// is scanned as the virtual slots u < Ls + Hs: lo then hi.
struct NbrView {
  int32_t* lo;
  int32_t* hi;
  int L, H, Ls, Hs;
};

__device__ __forceinline__ const int32_t* nbr_addr(const NbrView& nb, int64_t i, int j) {
  return j < nb.L ? nb.lo + i * nb.Ls + j : nb.hi + i * nb.Hs + (j - nb.L);
}

// Words u .. u + 3 of row i (u a multiple of 4 below Ls + Hs).
__device__ __forceinline__ int4 nbr_chunk(const NbrView& nb, int64_t i, int u) {
  const int32_t* p = u < nb.Ls ? nb.lo + i * nb.Ls + u : nb.hi + i * nb.Hs + (u - nb.Ls);
  return __ldg(reinterpret_cast<const int4*>(p));
}

// Step of virtual slot u, or -1 for padding.
__device__ __forceinline__ int nbr_step(const NbrView& nb, int u) {
  if (u < nb.Ls) return u < nb.L ? u : -1;
  const int h = u - nb.Ls;
  return h < nb.H ? nb.L + h : -1;
}

__device__ __forceinline__ int32_t int4_at(const int4& x, int q) {
  return q == 0 ? x.x : q == 1 ? x.y : q == 2 ? x.z : x.w;
}

// Steps whose lookups (or neighbour words) one thread issues before using
// them: a multiple of 4.
constexpr int kNbrBatch = 8;

// Neighbour lookups.  With keep_zero (the ADR operator) the zero frequency is
// an ordinary row and column.  supp a_hat is sorted and symmetric (p_{s_a-1-j}
// = -p_j, p_j0 = 0), and l = k - p_j lies in S exactly when k = l - p_{s_a-1-j}
// does: for j < j0 the lookup of row i finds l = k_i - p_j and writes
// lo[i][j] = l and hi[l][s_a-1-j] = i, so every pair is probed once (lo is
// written -1 first, hi is filled with -1 beforehand).  One thread per row
// probes kNbrBatch steps at a time (their first table words loaded before any
// is resolved) up to the first slot whose 31-bit fingerprint agrees; the
// warp queues those candidates in shared memory and confirms them with all
// its lanes (the exact word-by-word key comparison), so the comparisons do
// not run divergent once per step.  A candidate that fails (a fingerprint
// collision) resumes its probe sequence.  cnt (zero beforehand) receives
// every row's number of neighbours.
constexpr int kNbrThreads = 256;

template <int WT>
__global__ void __launch_bounds__(kNbrThreads) k_neighbors(KeyParams P, const uint64_t* __restrict__ keys,
                                                           const uint64_t* __restrict__ hl, int64_t size, int s_a,
                                                           int j0, const uint64_t* __restrict__ stepkey,
                                                           const uint64_t* __restrict__ stepg,
                                                           const uint64_t* __restrict__ table, uint64_t capmask,
                                                           const int64_t* __restrict__ zero_dev, bool keep_zero,
                                                           NbrView nb, int32_t* cnt) {
  constexpr int kWarps = kNbrThreads / 32, kQueue = 32 * kNbrBatch;
  __shared__ uint32_t q_tag[kWarps][kQueue];   // lane << 8 | step offset in the batch
  __shared__ uint32_t q_slot[kWarps][kQueue];  // table slot of the candidate
  __shared__ int32_t s_cnt[kNbrThreads];
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const int64_t row0 = (int64_t)blockIdx.x * kNbrThreads + (int64_t)wp * 32;
  const int64_t i = row0 + lane;
  const int64_t zero_idx = keep_zero ? -1 : *zero_dev;
  const bool active = i < size && i != zero_idx;
  s_cnt[threadIdx.x] = active ? 1 : 0;   // the diagonal
  const uint64_t hli = active ? __ldg(hl + i) : 0;
  int4* out = reinterpret_cast<int4*>(nb.lo + i * nb.Ls);
  const unsigned lt = (1u << lane) - 1u;
  for (int jb = 0; jb < nb.Ls; jb += kNbrBatch) {
    uint64_t hh[kNbrBatch], w[kNbrBatch];
#pragma unroll
    for (int q = 0; q < kNbrBatch; ++q) {
      hh[q] = 0;
      w[q] = kEmpty;
      if (active && jb + q < j0) {
        hh[q] = hash_of_lin(hli + __ldg(stepg + (s_a - 1 - (jb + q))));
        w[q] = __ldg(table + (hh[q] & capmask));
      }
    }
    if (i < size) {
#pragma unroll
      for (int q = 0; q < kNbrBatch; q += 4)
        if (jb + q < nb.Ls) {
          int32_t r[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) r[e] = (active && jb + q + e == j0) ? (int32_t)i : -1;
          out[(jb + q) / 4] = make_int4(r[0], r[1], r[2], r[3]);
        }
    }
    int n = 0;
#pragma unroll
    for (int q = 0; q < kNbrBatch; ++q) {
      // first slot with a matching fingerprint, or none
      const uint64_t fp = slot_fp(hh[q]);
      uint64_t h = hh[q] & capmask, v = w[q];
      bool cand = false;
      for (uint64_t probe = 0; probe <= capmask && v != kEmpty; ++probe) {
        if (word_fp(v) == fp) { cand = true; break; }
        h = (h + 1) & capmask;
        v = __ldg(table + h);
      }
      const unsigned m = __ballot_sync(0xffffffffu, cand);
      if (cand) {
        const int pos = n + __popc(m & lt);
        q_tag[wp][pos] = ((uint32_t)lane << 8) | (uint32_t)q;
        q_slot[wp][pos] = (uint32_t)h;
      }
      n += __popc(m);
    }
    __syncwarp();
    for (int e = lane; e < n; e += 32) {
      const int src = (int)(q_tag[wp][e] >> 8), j = jb + (int)(q_tag[wp][e] & 255u);
      const int64_t is = row0 + src;
      const int jr = s_a - 1 - j;   // p_jr = -p_j: k_i - p_j = k_i + p_jr
      const uint64_t* ki = keys + is * WT;
      const uint64_t* sk = stepkey + (int64_t)jr * WT;
      uint64_t h = q_slot[wp][e];
      int64_t o = (int64_t)word_low(__ldg(table + h));
      if (!key_eq_sum<WT>(keys + o * WT, ki, sk, P)) {
        // a fingerprint collision: resume the probe sequence after it
        const uint64_t lin = __ldg(hl + is) + __ldg(stepg + jr);
        const uint64_t hh2 = hash_of_lin(lin), fp = slot_fp(hh2);
        o = -1;
        for (uint64_t probe = 0; probe < capmask; ++probe) {
          h = (h + 1) & capmask;
          const uint64_t v = __ldg(table + h);
          if (v == kEmpty) break;
          if (word_fp(v) == fp && key_eq_sum<WT>(keys + (int64_t)word_low(v) * WT, ki, sk, P)) {
            o = (int64_t)word_low(v);
            break;
          }
        }
      }
      if (o >= 0 && o != zero_idx) {
        nb.lo[is * nb.Ls + j] = (int32_t)o;
        nb.hi[o * nb.Hs + (jr - nb.L)] = (int32_t)is;
        atomicAdd(&s_cnt[wp * 32 + src], 1);
        atomicAdd(cnt + o, 1);
      }
    }
    __syncwarp();
  }
  if (i < size) atomicAdd(cnt + i, s_cnt[threadIdx.x]);
}

// Per-slice widths (max over the slice's 32 rows) and nnz from the row counts.
__global__ void k_slice_widths(const int32_t* __restrict__ cnt, int64_t size, int64_t rows_pad, int32_t* slice_w,
                               unsigned long long* nnz, int32_t* wmax) {
  __shared__ unsigned s_tot[8];   // launched with 256 threads
  __shared__ int32_t s_w[8];
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int32_t c = i < size ? cnt[i] : 0;
  const int32_t w = __reduce_max_sync(0xffffffffu, c);
  const unsigned tot = __reduce_add_sync(0xffffffffu, (unsigned)c);
  if ((threadIdx.x & 31) == 0) {
    if (i < rows_pad) slice_w[i / kSlice] = w;   // rows_pad is a multiple of the warp
    s_tot[threadIdx.x >> 5] = tot;
    s_w[threadIdx.x >> 5] = w;
  }
  __syncthreads();
  if (threadIdx.x == 0) {   // one atomic of each kind per block
    unsigned long long b = 0;
    int32_t m = 0;
    for (int q = 0; q < 8; ++q) {
      b += s_tot[q];
      m = max(m, s_w[q]);
    }
    atomicAdd(nnz, b);
    atomicMax(wmax, m);
  }
}

// Entries of a row in step order, then padding (dummy column rows_pad, zero
// coefficient).  Also stores the FP64 coefficient of every entry,
// (|k|^2 + |l|^2 - |p_j|^2) * 2 pi^2 a_hat_j = 4 pi^2 (k.l) a_hat_j (eq. GF), so
// that the FP64 operator spends four FP64 FMAs per nonzero.
__global__ void k_fill_slices(NbrView nb, int64_t size, int64_t rows_pad, int s_a, int j0,
                              const int32_t* __restrict__ woff, int colbits, const int64_t* __restrict__ norm,
                              const int64_t* __restrict__ pnorm, const double2* __restrict__ ca64, uint32_t* ent,
                              double2* ecoef, bool real) {
  double* ecoef_re = reinterpret_cast<double*>(ecoef);   // real coefficients: one double per entry
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows_pad) return;
  const int64_t s = i / kSlice;
  const int lane = (int)(i % kSlice);
  const int64_t base = (int64_t)woff[s] * kSlice + lane;
  const int w = woff[s + 1] - woff[s];
  int t = 0;
  if (i < size) {
    const int64_t nk = norm[i];
    for (int ub = 0; ub < nb.Ls + nb.Hs; ub += kNbrBatch) {
      int4 x[kNbrBatch / 4];
#pragma unroll
      for (int q = 0; q < kNbrBatch / 4; ++q)
        x[q] = ub + 4 * q < nb.Ls + nb.Hs ? nbr_chunk(nb, i, ub + 4 * q) : make_int4(-1, -1, -1, -1);
      int32_t v[kNbrBatch];
      int64_t nv[kNbrBatch];
#pragma unroll
      for (int q = 0; q < kNbrBatch; ++q) v[q] = int4_at(x[q / 4], q % 4);
#pragma unroll
      for (int q = 0; q < kNbrBatch; ++q) nv[q] = v[q] >= 0 ? __ldg(norm + v[q]) : 0;
#pragma unroll
      for (int q = 0; q < kNbrBatch; ++q) {
        if (v[q] < 0) continue;
        const int j = nbr_step(nb, ub + q);
        const int64_t e = base + (int64_t)t++ * kSlice;
        ent[e] = (uint32_t)v[q] | ((uint32_t)j << colbits);
        const double sc = (double)(nk + nv[q] - pnorm[j]);
        if (real) ecoef_re[e] = sc * ca64[j].x;
        else ecoef[e] = make_double2(sc * ca64[j].x, sc * ca64[j].y);
      }
    }
  }
  const uint32_t pad = (uint32_t)rows_pad | ((uint32_t)j0 << colbits);
  for (; t < w; ++t) {
    ent[base + (int64_t)t * kSlice] = pad;
    if (real) ecoef_re[base + (int64_t)t * kSlice] = 0.0;
    else ecoef[base + (int64_t)t * kSlice] = make_double2(0.0, 0.0);
  }
}

// ADR entries (Remark ADR): for row k and neighbour l = k - p_j,
//   4 pi^2 (k.l) a_hat_j + 2 pi i (l . b_hat_j) + c_hat_j,
// with 4 pi^2 (k.l) a_hat_j = (|k|^2 + |l|^2 - |p_j|^2) * 2 pi^2 a_hat_j formed
// exactly as for the diffusion operator and l . b_hat_j summed over the d
// coordinates of l unpacked from its key.  The entry with l = k (p_j = 0) is
// also the row's Jacobi diagonal.
template <int WT>
__global__ void k_fill_slices_adr(KeyParams P, const uint64_t* __restrict__ keys, NbrView nb,
                                  int64_t size, int64_t rows_pad, int s_a, int j0, const int32_t* __restrict__ woff,
                                  int colbits, const int64_t* __restrict__ norm, const int64_t* __restrict__ pnorm,
                                  const double2* __restrict__ ca64, const double2* __restrict__ bval,
                                  const double2* __restrict__ cval, uint32_t* ent, double2* ecoef, double2* diag) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i > rows_pad) return;
  if (i >= size) {
    diag[i] = make_double2(1.0, 0.0);
    if (i == rows_pad) return;
  }
  const int64_t s = i / kSlice;
  const int lane = (int)(i % kSlice);
  const int64_t base = (int64_t)woff[s] * kSlice + lane;
  const int w = woff[s + 1] - woff[s];
  int t = 0;
  if (i < size) {
    const int64_t nk = norm[i];
    double2 dg = make_double2(1.0, 0.0);
    for (int j = 0; j < s_a; ++j) {
      const int32_t v = *nbr_addr(nb, i, j);
      if (v < 0) continue;
      const int64_t e = base + (int64_t)t++ * kSlice;
      ent[e] = (uint32_t)v | ((uint32_t)j << colbits);
      const double sc = (double)(nk + norm[v] - pnorm[j]);
      double br = 0.0, bi = 0.0;
      const uint64_t* lk = keys + (int64_t)v * WT;
      for (int c = 0; c < P.d; ++c) {
        const double lc = (double)unpack_coord(lk, P, c);
        const double2 b = bval[(int64_t)j * P.d + c];
        br += lc * b.x;
        bi += lc * b.y;
      }
      const double2 cj = cval[j];
      // 2 pi i (br + i bi) = (-2 pi bi) + i (2 pi br)
      const double2 cf = make_double2(sc * ca64[j].x - kTwoPi * bi + cj.x, sc * ca64[j].y + kTwoPi * br + cj.y);
      ecoef[e] = cf;
      if (j == j0) dg = cf;
    }
    if (dg.x == 0.0 && dg.y == 0.0) dg = make_double2(1.0, 0.0);
    diag[i] = dg;
  }
  const uint32_t pad = (uint32_t)rows_pad | ((uint32_t)j0 << colbits);
  for (; t < w; ++t) {
    ent[base + (int64_t)t * kSlice] = pad;
    ecoef[base + (int64_t)t * kSlice] = make_double2(0.0, 0.0);
  }
}

__global__ void k_init_records(const int64_t* __restrict__ norm, int64_t n, bool wide, int32_t* nw32,
                               double2* rec64) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t nr = norm[i];
  nw32[i] = norm_word(nr, wide);
  rec64[i] = make_double2(0.0, 0.0);
}

template <int WT>
__global__ void k_export(KeyParams P, const uint64_t* __restrict__ keys, int64_t size, int32_t* freq) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= size) return;
  for (int c = 0; c < P.d; ++c) freq[i * P.d + c] = unpack_coord(keys + i * WT, P, c);
}

template <int WT>
__global__ void k_lookup(KeyParams P, const uint64_t* __restrict__ keys, const uint64_t* __restrict__ hl,
                         const uint64_t* __restrict__ table, uint64_t capmask, const int32_t* __restrict__ q,
                         int64_t n, int64_t* idx) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint64_t k[WT];
  int64_t r = -1;
  if (pack_key<WT>(q + i * P.d, P, k)) {
    const uint64_t lin = key_lin<WT>(k);
    r = table_find_h(table, capmask, hash_of_lin(lin), hl, lin, [&](int64_t o) {
      bool e = true;
#pragma unroll
      for (int w = 0; w < WT; ++w) e &= __ldg(keys + o * WT + w) == k[w];
      return e;
    });
  }
  idx[i] = r;
}

// The same lookup by one warp per query: the lanes pack the coordinates
// c = lane, lane + 32, ... into the key words (shared-memory OR: the fields do
// not overlap), lane 0 probes, the lanes compare the words of a candidate.
constexpr int kLookupWarps = 8;

template <int WT>
__global__ void __launch_bounds__(32 * kLookupWarps) k_lookup_warp(KeyParams P, const uint64_t* __restrict__ keys,
                                                                   const uint64_t* __restrict__ table, uint64_t capmask,
                                                                   const int32_t* __restrict__ q, int64_t n,
                                                                   int64_t* idx) {
  __shared__ unsigned long long s_key[kLookupWarps][WT];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t i = (int64_t)blockIdx.x * kLookupWarps + w;
  if (i >= n) return;   // warp-uniform
  if (lane < WT) s_key[w][lane] = 0ull;
  __syncwarp();
  bool ok = true;
  for (int c = lane; c < P.d; c += 32) {
    const int64_t v = (int64_t)q[i * P.d + c] + P.bias_val;
    ok &= (v >= 0) && (v <= (int64_t)P.fieldmask);
    const int wd = c / P.fpw, sh = 64 - P.fb * (c % P.fpw + 1);
    atomicOr(&s_key[w][wd], (unsigned long long)(((uint64_t)v & P.fieldmask) << sh));
  }
  __syncwarp();
  int64_t r = -1;
  if (__all_sync(0xffffffffu, ok)) {
    const uint64_t kw = lane < WT ? (uint64_t)s_key[w][lane] : 0ull;
    uint64_t lin = lane < WT ? key_lin_coef(lane) * kw : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lin += __shfl_xor_sync(0xffffffffu, lin, o);
    const uint64_t hh = hash_of_lin(lin), fp = slot_fp(hh);
    uint64_t h = hh & capmask;
    for (uint64_t probe = 0; probe <= capmask; ++probe) {
      const uint64_t v = __ldg(table + h);   // every lane loads the same word
      if (v == kEmpty) break;
      if (word_fp(v) == fp) {
        const int64_t o = (int64_t)word_low(v);
        const bool eq = lane >= WT || __ldg(keys + o * WT + lane) == kw;
        if (__all_sync(0xffffffffu, eq)) {
          r = o;
          break;
        }
      }
      h = (h + 1) & capmask;
    }
  }
  if (lane == 0) idx[i] = r;
}

__global__ void k_scatter_vals(const int64_t* __restrict__ idx, const double2* __restrict__ v, int64_t n,
                               double2* out, unsigned long long* outside) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t r = idx[i];
  if (r >= 0) out[r] = v[i];
  else if (outside) atomicAdd(outside, 1ull);   // counted only when asked for
}

inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

uint64_t next_pow2(uint64_t x) {
  uint64_t p = 1;
  while (p < x) p <<= 1;
  return p;
}

}  // namespace

// ------------------------------------------------------------------ build

// Slot bound of the hash tables built from now on (stamp_set_table_limit; 0: none).
static std::atomic<int64_t> g_table_limit{0};

// Step keys, their linear forms and norms, and the entry scale factors.
static ss_status launch_steps(const KeyParams& P, const int32_t* A, const double2* av, int s_a, uint64_t* stepkey,
                              uint64_t* stepg, int64_t* pnorm, int32_t* pn32, bool wide, double2* ca64, float2* ca32,
                              cudaStream_t st) {
  if (P.d > 16) {
    SS_DISPATCH_WT(P.WT, (k_steps_warp<WT><<<(unsigned)((s_a + kPackWarps - 1) / kPackWarps), 32 * kPackWarps, 0,
                                              st>>>(P, A, av, s_a, stepkey, stepg, pnorm, pn32, wide, ca64, ca32)));
  } else {
    SS_DISPATCH_WT(P.WT, (k_steps<WT><<<nblk(s_a), 256, 0, st>>>(P, A, av, s_a, stepkey, stepg, pnorm, pn32, wide,
                                                                   ca64, ca32)));
  }
  SS_LAUNCH_CHECK();
  return SS_OK;
}

static ss_status grow_table(ss_stamp_s* S, int64_t need, const KeyParams& P, cudaStream_t st, int32_t* d_err) {
  int64_t want = (int64_t)next_pow2((uint64_t)std::max<int64_t>(2 * need, 1024));
  const int64_t lim = g_table_limit.load(std::memory_order_relaxed);
  if (lim > 0) {
    int64_t c = 16;
    while (2 * c <= lim) c *= 2;   // largest power of two <= lim (at least 16)
    want = std::min(want, c);
  }
  if (want <= S->cap) return SS_OK;
  SS_TRY(S->table.alloc(want, st));
  S->cap = want;
  SS_CUDA(cudaMemsetAsync(S->table.get(), 0xff, want * sizeof(uint64_t), st));
  if (S->size > 0) {
    k_rehash<<<nblk(S->size), 256, 0, st>>>(S->hl.get(), S->size, S->table.get(), (uint64_t)want - 1, d_err);
    SS_LAUNCH_CHECK();
  }
  return SS_OK;
}

// The table is sized for the candidates of the last level; when that leaves
// it more than about 8 times larger than S, the lookups that follow probe a
// table of about 4 |S| slots instead (a table that size keeps short probe
// sequences and most of it resident in L2).
static ss_status compact_table(ss_stamp_s* S, cudaStream_t st) {
  int64_t want = (int64_t)next_pow2((uint64_t)std::max<int64_t>(4 * S->size, 1024));
  if (want >= S->cap || S->size == 0) return SS_OK;
  SS_TRY(S->table.alloc(want, st));
  S->cap = want;
  SS_CUDA(cudaMemsetAsync(S->table.get(), 0xff, want * sizeof(uint64_t), st));
  k_rehash<<<nblk(S->size), 256, 0, st>>>(S->hl.get(), S->size, S->table.get(), (uint64_t)want - 1,
                                          S->err_dev.get());
  SS_LAUNCH_CHECK();
  return SS_OK;
}

static ss_status resize_keys(ss_stamp_s* S, int64_t cap, cudaStream_t st);

static ss_status grow_keys(ss_stamp_s* S, int64_t need, cudaStream_t st) {
  const int WT = S->key.WT;
  if ((int64_t)S->keys.n >= need * WT) return SS_OK;
  return resize_keys(S, std::max<int64_t>(need, (int64_t)(S->keys.n / WT) * 2), st);
}

// Keys, levels and norms moved to buffers of cap rows (cap >= size).
static ss_status resize_keys(ss_stamp_s* S, int64_t cap, cudaStream_t st) {
  const int WT = S->key.WT;
  DevBuf<uint64_t> k2, h2;
  DevBuf<int8_t> l2;
  DevBuf<int64_t> n2;
  SS_TRY(k2.alloc(cap * WT, st));
  SS_TRY(h2.alloc(cap, st));
  SS_TRY(l2.alloc(cap, st));
  SS_TRY(n2.alloc(cap + kSlice + 1, st));
  if (S->size > 0) {
    SS_CUDA(cudaMemcpyAsync(k2.get(), S->keys.get(), S->size * WT * sizeof(uint64_t), cudaMemcpyDeviceToDevice, st));
    SS_CUDA(cudaMemcpyAsync(h2.get(), S->hl.get(), S->size * sizeof(uint64_t), cudaMemcpyDeviceToDevice, st));
    SS_CUDA(cudaMemcpyAsync(l2.get(), S->level.get(), S->size, cudaMemcpyDeviceToDevice, st));
    SS_CUDA(cudaMemcpyAsync(n2.get(), S->norm.get(), S->size * sizeof(int64_t), cudaMemcpyDeviceToDevice, st));
  }
  // the old buffers are released on this stream, after the copies
  std::swap(S->keys.p, k2.p); std::swap(S->keys.n, k2.n); std::swap(S->keys.s, k2.s);
  std::swap(S->hl.p, h2.p); std::swap(S->hl.n, h2.n); std::swap(S->hl.s, h2.s);
  std::swap(S->level.p, l2.p); std::swap(S->level.n, l2.n); std::swap(S->level.s, l2.s);
  std::swap(S->norm.p, n2.p); std::swap(S->norm.n, n2.n); std::swap(S->norm.s, n2.s);
  k2.s = st;
  h2.s = st;
  l2.s = st;
  n2.s = st;
  return SS_OK;
}

// |S^N| <= |F| C(s_a - 1 + N, N): an element is some k in F plus a multiset of
// at most N of the s_a - 1 nonzero steps.  Returns min(that, cap).
constexpr int64_t kPresizeCap = 1ll << 22;
static int64_t stamp_size_bound(int64_t n_f, int s_a, int N, int64_t cap) {
  double c = 1.0;   // C(m + i, i), m = s_a - 1, exact while below 2^53
  for (int i = 1; i <= N; ++i) {
    c = c * (double)(s_a - 1 + i) / (double)i;
    if (c * (double)n_f >= (double)cap) return cap;
  }
  return std::min<int64_t>(cap, (int64_t)(c * (double)n_f));
}

// Norm range: |k|^2 <= d maxabs^2 is formed in int64 (and the FP64 entry
// coefficients from |k|^2 + |l|^2 - |p|^2 exactly in FP64 below 2^53).
static bool norms_wide(int d, int64_t maxabs) { return (double)d * (double)maxabs * (double)maxabs >= (double)(1 << 29); }

static ss_status make_layout(int d, int64_t maxabs, KeyLayout* out) {
  if ((double)d * (double)maxabs * (double)maxabs >= 0x1p51)
    SS_FAIL(SS_ERR_KEY_RANGE, "stamp: |k|^2 may reach %g; exact operator coefficients need < 2^51",
            (double)d * maxabs * maxabs);
  int b = 1;
  while (((int64_t)1 << (b - 1)) - 1 < maxabs) ++b;
  KeyLayout L;
  L.d = d;
  L.b = b;
  L.fb = b + 1;
  L.fpw = 64 / L.fb;
  L.W = (d + L.fpw - 1) / L.fpw;
  L.WT = 1;
  while (L.WT < L.W) L.WT <<= 1;
  if (L.W > 8 && L.W <= 12) L.WT = 12;
  if (L.WT > kMaxWords) SS_FAIL(SS_ERR_KEY_RANGE, "stamp: key needs %d words (max %d)", L.W, kMaxWords);
  *out = L;
  return SS_OK;
}

// Candidate buffers of the levels (slot of each candidate, the winners in
// candidate order): sized once by the caller when a bound is known, else
// grown per level.
struct LevelTmp {
  DevBuf<int64_t> slot_of, cand;
};
constexpr int64_t kLevelTmpPresize = 512ll << 20;   // bytes of both, at most

// Levels n_from..n_to of the breadth-first construction (see the file comment).
static ss_status run_levels(ss_stamp_s* S, int n_from, int n_to, cudaStream_t st, LevelTmp& lt) {
  const KeyParams P = make_key_params(S->key);
  const int s_a = S->s_a;
  DevBuf<int64_t> d_total;
  DevBuf<int64_t>& slot_of = lt.slot_of;
  DevBuf<int64_t>& cand = lt.cand;
  SS_TRY(d_total.alloc_tmp(1, st));
  for (int n = n_from; n <= n_to; ++n) {
    const int64_t par0 = S->level_start[n - 1], n_par = S->level_start[n] - par0;
    const int64_t ncand = n_par * s_a;
    if (ncand >= ((int64_t)1 << 32) - 1) SS_FAIL(SS_ERR_KEY_RANGE, "stamp: too many candidates at level %d", n);
    if (ncand == 0) { S->level_start.push_back(S->size); continue; }
    // room for every candidate that may be new, but never more than the
    // multiset bound |S^n| <= |F| C(s_a - 1 + n, n) (the build presized for it)
    int64_t need = S->size + n_par * (s_a - 1);
    const int64_t bnd = stamp_size_bound(S->level_start[1], s_a, n, kPresizeCap);
    if (bnd < kPresizeCap) need = std::min(need, bnd);
    SS_TRY(grow_table(S, need, P, st, S->err_dev.get()));
    SS_TRY(grow_keys(S, need, st));
    SS_TRY(slot_of.ensure_tmp(ncand, st));
    SS_TRY(cand.ensure_tmp(ncand, st));
    {
      ProfScope prof_("k_insert", st);
      SS_DISPATCH_WT(S->key.WT, (k_insert<WT><<<nblk(ncand), 256, 0, st>>>(
                                    P, S->keys.get(), S->hl.get(), par0, n_par, s_a, S->j0, S->stepkey.get(),
                                    S->stepg.get(), S->table.get(), (uint64_t)S->cap - 1, slot_of.get(),
                                    S->err_dev.get())));
    }
    SS_LAUNCH_CHECK();
    {
      // winners (the candidate that holds its slot) in candidate order: one
      // pass computes the flags, their prefix sums and the compaction
      ProfScope prof_("winners", st);
      SS_TRY(scan_lookback(WinnerFlag{slot_of.get(), S->table.get()}, WinnerPut{cand.get()}, ncand, d_total.get(),
                           S->err_dev.get(), st));
    }
    int64_t added = 0;
    int32_t e = 0;
    SS_TRY(read_back(st, {{&added, d_total.get(), sizeof(int64_t)}, {&e, S->err_dev.get(), sizeof(int32_t)}}));
    if (e == SS_ERR_TIMEOUT) SS_FAIL(SS_ERR_TIMEOUT, "stamp: a bounded device wait gave up at level %d", n);
    if (e) SS_FAIL((ss_status)e, "stamp: hash table exhausted at level %d", n);
    SS_TRY(grow_keys(S, S->size + added, st));   // the exact count: the rows k_finalize writes always fit
    if (added > 0) {
      ProfScope prof_("k_finalize", st);
      SS_DISPATCH_WT(S->key.WT, (k_finalize<WT><<<nblk(added, kFinThreads), kFinThreads, 0, st>>>(
                                    P, S->keys.get(), S->hl.get(), par0,
                                                                             s_a, S->stepkey.get(), S->stepg.get(),
                                                                             S->pnorm.get(), slot_of.get(), cand.get(),
                                                                             added,
                                                                             S->size, n, S->level.get(),
                                                                             S->norm.get(), S->table.get(),
                                                                             S->zidx_dev.get())));
    }
    SS_LAUNCH_CHECK();
    S->size += added;
    S->level_start.push_back(S->size);
  }
  return SS_OK;
}

// ---------------------------------------------------- Hermitian half system
//
// For real data (F = -F, a_hat_{-p} = conj(a_hat_p)) S is symmetric and the
// operator maps Hermitian vectors (u_{-k} = conj(u_k)) to Hermitian vectors,
// so for a Hermitian right-hand side the rows k >lex 0 carry the whole
// solution.  The half system keeps those rows ("compact rows", canonical
// order) and reads a neighbour l <lex 0 as conj(u_{-l}).

// mirror[g] = index of -k_g (negation is field-wise 2 bias - v on the packed
// key, no carries since |k_c| < 2^(b-1)); plus[g] = 1 if k_g >lex 0.
template <int WT>
__global__ void k_half_index(KeyParams P, const uint64_t* __restrict__ keys, const uint64_t* __restrict__ hl,
                             int64_t size, const uint64_t* __restrict__ table, uint64_t capmask, int64_t* mirror, int32_t* plus,
                             int32_t* err) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= size) return;
  uint64_t k[WT];
  load_key<WT>(keys, g, k);
  // -k packs as 2 bias - k field by field: its linear form is 2 lin(bias) - lin(k)
  const uint64_t lin = 2 * P.lin_bias - __ldg(hl + g);
  const uint64_t* kg = keys + g * WT;
  const int64_t m = table_find_h(table, capmask, hash_of_lin(lin), nullptr, lin,
                                 [&](int64_t o) { return key_eq_sum<WT>(keys + o * WT, kg, nullptr, P); });
  if (m < 0) atomicExch(err, 1);
  mirror[g] = m;
  // Fields are packed first coordinate first from the top bit down, biased
  // and without carries, so the words compare like the coordinates: k >lex 0
  // iff the word sequence of k exceeds that of the packed zero.
  int p = 0;
#pragma unroll
  for (int w = WT - 1; w >= 0; --w)
    if (k[w] != P.bias[w]) p = k[w] > P.bias[w];
  plus[g] = p;
}

// Indices stay in range even for a set that is not symmetric (a missing -k
// sets the error word and the half system is dropped after the read-back).
__global__ void k_half_rows(const int32_t* __restrict__ plus, const int32_t* __restrict__ ppos,
                            const int64_t* __restrict__ mirror, const int64_t* __restrict__ norm, int64_t size,
                            int64_t zero_idx, int64_t n_plus, int32_t* hpos, int32_t* plus_rows, int64_t* norm_h) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= size) return;
  if (plus[g]) {
    const int32_t i = ppos[g];
    hpos[g] = i;
    if (i < n_plus) {
      plus_rows[i] = (int32_t)g;
      norm_h[i] = norm[g];
    }
  } else if (g == zero_idx || mirror[g] < 0) {
    hpos[g] = -1;
  } else {
    hpos[g] = -2 - ppos[mirror[g]];
  }
}

// Width of every compact row (its stored entries), warp maximum per slice.
__global__ void k_half_widths(const int32_t* __restrict__ plus_rows, int64_t n_plus, int64_t rows_pad_h,
                              const int32_t* __restrict__ woff, const uint32_t* __restrict__ ent, uint32_t colmask,
                              int64_t pad_col, int32_t* slice_w) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows_pad_h) return;
  int32_t cnt = 0;
  if (i < n_plus) {
    const int64_t g = plus_rows[i];
    const int64_t s = g / kSlice;
    const int64_t base = (int64_t)woff[s] * kSlice + (g % kSlice);
    const int w = woff[s + 1] - woff[s];
    for (int t = 0; t < w; ++t)
      if ((int64_t)(ent[base + (int64_t)t * kSlice] & colmask) != pad_col) ++cnt;
  }
  const int32_t m = __reduce_max_sync(0xffffffffu, cnt);
  if ((threadIdx.x & 31) == 0) slice_w[i / kSlice] = m;
}

__global__ void k_half_fill(const int32_t* __restrict__ plus_rows, int64_t n_plus, int64_t rows_pad_h,
                            const int32_t* __restrict__ woff, const uint32_t* __restrict__ ent,
                            const double2* __restrict__ ecoef, uint32_t colmask, int colbits, int64_t pad_col,
                            int colbits_h, int j0, const int32_t* __restrict__ hpos,
                            const int32_t* __restrict__ woff_h, uint32_t* ent_h, double2* ecoef_h, bool real,
                            const int32_t* __restrict__ err) {
  const double* ecoef_re = reinterpret_cast<const double*>(ecoef);
  double* ecoef_h_re = reinterpret_cast<double*>(ecoef_h);
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  // a scan that gave up (err[0]) leaves woff_h and the compact positions
  // incomplete: nothing is written from them
  if (i >= rows_pad_h || __ldg(err) != 0) return;
  const int64_t sh = i / kSlice;
  const int64_t base_h = (int64_t)woff_h[sh] * kSlice + (i % kSlice);
  const int w_h = woff_h[sh + 1] - woff_h[sh];
  int t = 0;
  if (i < n_plus) {
    const int64_t g = plus_rows[i];
    const int64_t s = g / kSlice;
    const int64_t base = (int64_t)woff[s] * kSlice + (g % kSlice);
    const int w = woff[s + 1] - woff[s];
    for (int tf0 = 0; tf0 < w; tf0 += kNbrBatch) {
      // entry words, then the gathered positions, loaded before use
      uint32_t ev[kNbrBatch];
      int32_t hv[kNbrBatch];
#pragma unroll
      for (int q = 0; q < kNbrBatch; ++q)
        ev[q] = tf0 + q < w ? __ldg(ent + base + (int64_t)(tf0 + q) * kSlice) : (uint32_t)pad_col;
#pragma unroll
      for (int q = 0; q < kNbrBatch; ++q) {
        const int64_t c = ev[q] & colmask;
        hv[q] = c == pad_col ? -1 : __ldg(hpos + c);
      }
#pragma unroll
      for (int q = 0; q < kNbrBatch; ++q) {
        const int32_t h = hv[q];
        if (h == -1) continue;   // padding (the zero column is never stored)
        const int64_t e = base + (int64_t)(tf0 + q) * kSlice;
        const uint32_t col = h >= 0 ? (uint32_t)h : (uint32_t)(-2 - h);
        const uint32_t j = ev[q] >> colbits;
        ent_h[base_h + (int64_t)t * kSlice] = col | (j << colbits_h) | (h < 0 ? 0x80000000u : 0u);
        if (real) ecoef_h_re[base_h + (int64_t)t * kSlice] = ecoef_re[e];
        else ecoef_h[base_h + (int64_t)t * kSlice] = ecoef[e];
        ++t;
      }
    }
  }
  for (; t < w_h; ++t) {
    ent_h[base_h + (int64_t)t * kSlice] = (uint32_t)rows_pad_h | ((uint32_t)j0 << colbits_h);
    if (real) ecoef_h_re[base_h + (int64_t)t * kSlice] = 0.0;
    else ecoef_h[base_h + (int64_t)t * kSlice] = make_double2(0.0, 0.0);
  }
}

// Queue the half system of the current set (no synchronisation; the caller's
// read-back returns woff_h and the mirror error flag).
static ss_status build_half(ss_stamp_s* S, cudaStream_t st) {
  S->half_ok = false;
  const int64_t n_plus = (S->size - (S->zero_idx >= 0 ? 1 : 0)) / 2;
  if (!S->half_cand || n_plus < 1 || 2 * n_plus + (S->zero_idx >= 0 ? 1 : 0) != S->size) return SS_OK;
  S->n_plus = n_plus;
  S->rows_pad_h = (n_plus + kSlice - 1) / kSlice * kSlice;
  S->n_slices_h = S->rows_pad_h / kSlice;
  S->colbits_h = 31 - S->jbits;
  if (S->colbits_h < 1 || S->rows_pad_h + 1 > ((int64_t)1 << S->colbits_h)) return SS_OK;   // no room for the conj bit
  const int32_t max_w = S->max_w;
  const KeyParams P = make_key_params(S->key);
  DevBuf<int32_t> plus, ppos, slice_w;
  DevBuf<int64_t> total;
  SS_TRY(plus.alloc_tmp(S->size, st));
  SS_TRY(ppos.alloc_tmp(S->size, st));
  SS_TRY(slice_w.alloc_tmp(S->n_slices_h + 1, st));
  SS_TRY(total.alloc_tmp(1, st));
  SS_TRY(S->mirror.alloc(S->size, st));
  SS_TRY(S->hpos.alloc(S->size, st));
  SS_TRY(S->plus_rows.alloc(S->rows_pad_h, st));
  SS_TRY(S->norm_h.alloc(S->rows_pad_h + 1, st));
  SS_TRY(S->woff_h.alloc(S->n_slices_h + 1, st));
  // Entries of the half table: every compact slice is at most as wide as the
  // widest row it holds; the plus rows of one full slice are consecutive
  // compact rows, so they fall in at most two compact slices and the half
  // table holds at most twice the full table's entries.
  const int64_t cap_h = std::min<int64_t>(S->n_slices_h * (int64_t)max_w * kSlice, 2 * S->n_ent) + 1;
  SS_TRY(S->ent_h.alloc(cap_h, st));
  SS_TRY(S->ecoef_h.alloc(cap_h, st));
  SS_TRY(fill_small(st, {{S->norm_h.get(), (S->rows_pad_h + 1) * sizeof(int64_t), 0},
                         {S->plus_rows.get(), S->rows_pad_h * sizeof(int32_t), 0},
                         {slice_w.get(), (S->n_slices_h + 1) * sizeof(int32_t), 0},
                         {S->err_dev.get() + 3, sizeof(int32_t), 0}}));
  {
    ProfScope prof_("k_half_index", st);
    SS_DISPATCH_WT(S->key.WT, (k_half_index<WT><<<nblk(S->size), 256, 0, st>>>(
                                  P, S->keys.get(), S->hl.get(), S->size, S->table.get(), (uint64_t)S->cap - 1, S->mirror.get(),
                                  plus.get(), S->err_dev.get() + 3)));
  }
  SS_LAUNCH_CHECK();
  SS_TRY(scan_lookback(LbRead{plus.get()}, LbWrite{ppos.get()}, S->size, total.get(), S->err_dev.get(), st));
  {
    ProfScope prof_("k_half_rows", st);
    k_half_rows<<<nblk(S->size), 256, 0, st>>>(plus.get(), ppos.get(), S->mirror.get(), S->norm.get(), S->size,
                                               S->zero_idx, n_plus, S->hpos.get(), S->plus_rows.get(),
                                               S->norm_h.get());
  }
  const uint32_t colmask = colmask_of(S->jbits);
  {
    ProfScope prof_("k_half_widths", st);
    k_half_widths<<<nblk(S->rows_pad_h), 256, 0, st>>>(S->plus_rows.get(), n_plus, S->rows_pad_h, S->slice_off.get(),
                                                       S->ent.get(), colmask, S->rows_pad, slice_w.get());
  }
  SS_LAUNCH_CHECK();
  SS_TRY(scan_lookback(LbRead{slice_w.get()}, LbWrite{S->woff_h.get()}, S->n_slices_h + 1, total.get(),
                       S->err_dev.get(), st));
  {
    ProfScope prof_("k_half_fill", st);
    k_half_fill<<<nblk(S->rows_pad_h), 256, 0, st>>>(S->plus_rows.get(), n_plus, S->rows_pad_h, S->slice_off.get(),
                                                     S->ent.get(), S->ecoef64.get(), colmask, colbits_of(S->jbits),
                                                     S->rows_pad, S->colbits_h, S->j0, S->hpos.get(), S->woff_h.get(),
                                                     S->ent_h.get(), S->ecoef_h.get(), S->a_real, S->err_dev.get());
  }
  SS_LAUNCH_CHECK();
  S->woff_h_host.clear();   // host copy on demand (stamp_host_tables)
  S->half_ok = true;        // confirmed by the caller's read-back of the mirror flag
  return SS_OK;
}

// Error words of a stamp build (err_dev[0]: a device wait that gave up or
// the table exhausted; [3]: some -k of the half system not found).
static ss_status check_words(ss_stamp_s* S, const int32_t* e) {
  S->check_pending = false;
  if (e[0] == SS_ERR_TIMEOUT) SS_FAIL(SS_ERR_TIMEOUT, "stamp: a bounded device wait gave up");
  if (e[0]) SS_FAIL((ss_status)e[0], "stamp: hash table exhausted");
  if (S->half_ok && e[3]) S->half_ok = false;   // some -k not in S: no half system
  return SS_OK;
}

// Neighbour table (sliced ELL), FP64 entry coefficients and apply scratch
// for the current set; settles the stamp's buffers.  The build synchronises
// once for the table's size and once at its end for the error words; with
// `defer` the second synchronisation is left to the caller's next one (the
// one-call pipeline's solve, which copies the words in stream order and
// checks them with its statistics, stamp_check_pending).  Until then the
// half system is only tentative: its consumers are guarded against a failed
// build (no read or write outside the stamp's buffers).
static ss_status build_operator(ss_stamp_s* S, cudaStream_t st, bool defer) {
  const KeyParams P = make_key_params(S->key);
  const int s_a = S->s_a;
  if (S->size >= ((int64_t)1 << 31)) SS_FAIL(SS_ERR_KEY_RANGE, "stamp: |S| = %lld too large", (long long)S->size);
  S->rows_pad = (S->size + kSlice - 1) / kSlice * kSlice;
  S->n_slices = S->rows_pad / kSlice;
  if (S->rows_pad + 1 > ((int64_t)1 << colbits_of(S->jbits)))
    SS_FAIL(SS_ERR_KEY_RANGE, "stamp: |S| = %lld too large for %d-bit columns", (long long)S->size,
            colbits_of(S->jbits));
  SS_TRY(grow_keys(S, S->rows_pad + 1, st));   // norm padded to rows_pad + 1
  {
    ProfScope prof_("compact_table", st);
    SS_TRY(compact_table(S, st));
  }
  if (S->cap > ((int64_t)1 << 32)) SS_FAIL(SS_ERR_KEY_RANGE, "stamp: hash table of %lld slots", (long long)S->cap);
  DevBuf<int32_t> nbr_lo, nbr_hi, cnt, slice_w, d_wmax;
  DevBuf<unsigned long long> d_nnz;
  DevBuf<int64_t> d_total;
  NbrView nb;
  nb.L = S->j0 + 1;
  nb.H = s_a - nb.L;
  nb.Ls = (nb.L + 3) / 4 * 4;
  nb.Hs = (nb.H + 3) / 4 * 4;
  SS_TRY(nbr_lo.alloc_tmp((size_t)S->size * nb.Ls, st));
  SS_TRY(nbr_hi.alloc_tmp((size_t)std::max(S->size * nb.Hs, (int64_t)4), st));
  nb.lo = nbr_lo.get();
  nb.hi = nbr_hi.get();
  SS_TRY(cnt.alloc_tmp(S->size, st));
  SS_TRY(slice_w.alloc_tmp(S->n_slices + 1, st));
  SS_TRY(d_nnz.alloc_tmp(1, st));
  SS_TRY(d_wmax.alloc_tmp(1, st));
  SS_TRY(d_total.alloc_tmp(1, st));
  SS_TRY(fill_small(st, {{S->norm.get() + S->size, (S->rows_pad + 1 - S->size) * sizeof(int64_t), 0},
                         {d_nnz.get(), sizeof(unsigned long long), 0},
                         {d_wmax.get(), sizeof(int32_t), 0},
                         {slice_w.get(), (S->n_slices + 1) * sizeof(int32_t), 0}}));
  {
    ProfScope prof_("k_neighbors", st, true);
    if (nb.Hs > 0) SS_CUDA(cudaMemsetAsync(nb.hi, 0xff, (size_t)S->size * nb.Hs * sizeof(int32_t), st));
    SS_CUDA(cudaMemsetAsync(cnt.get(), 0, (size_t)S->size * sizeof(int32_t), st));
    SS_DISPATCH_WT(S->key.WT, (k_neighbors<WT><<<nblk(S->size, kNbrThreads), kNbrThreads, 0, st>>>(
                                  P, S->keys.get(), S->hl.get(), S->size, s_a, S->j0, S->stepkey.get(), S->stepg.get(),
                                  S->table.get(),
                                  (uint64_t)S->cap - 1, S->zidx_dev.get(), S->adr, nb, cnt.get())));
  }
  {
    ProfScope prof_("k_slice_widths", st);
    k_slice_widths<<<nblk(S->rows_pad), 256, 0, st>>>(cnt.get(), S->size, S->rows_pad, slice_w.get(), d_nnz.get(),
                                                      d_wmax.get());
  }
  SS_LAUNCH_CHECK();
  SS_TRY(S->slice_off.alloc(S->n_slices + 1, st));
  SS_TRY(scan_lookback(LbRead{slice_w.get()}, LbWrite{S->slice_off.get()}, S->n_slices + 1, d_total.get(),
                       S->err_dev.get(), st));
  int64_t total_w = 0;
  unsigned long long hnnz = 0;
  int32_t e0 = 0;
  S->woff_host.clear();   // host copy on demand (stamp_host_tables)
  SS_TRY(read_back(st, {{&total_w, d_total.get(), sizeof(int64_t)},
                        {&hnnz, d_nnz.get(), sizeof(hnnz)},
                        {&S->zero_idx, S->zidx_dev.get(), sizeof(int64_t)},
                        {&S->max_w, d_wmax.get(), sizeof(int32_t)},
                        {&e0, S->err_dev.get(), sizeof(int32_t)}}));
  // the slice offsets size and place every entry below: a scan that gave up
  // is reported before they are used
  if (e0 == SS_ERR_TIMEOUT) SS_FAIL(SS_ERR_TIMEOUT, "stamp: a bounded device wait gave up");
  S->nnz = (int64_t)hnnz;
  S->n_ent = total_w * kSlice;
  SS_TRY(S->ent.alloc(S->n_ent + 1, st));
  SS_TRY(S->ecoef64.alloc(S->n_ent + 1, st));
  S->ecoefdf.release();   // rebuilt from ecoef64 by the next DF64 solve
  S->ecoefdf_h.release();
  if (S->adr) {
    SS_TRY(S->diag64.alloc(S->rows_pad + 1, st));
    SS_DISPATCH_WT(S->key.WT, (k_fill_slices_adr<WT><<<nblk(S->rows_pad + 1), 256, 0, st>>>(
                                  P, S->keys.get(), nb, S->size, S->rows_pad, s_a, S->j0, S->slice_off.get(),
                                  colbits_of(S->jbits), S->norm.get(), S->pnorm.get(), S->ca64.get(), S->bval.get(),
                                  S->cval.get(), S->ent.get(), S->ecoef64.get(), S->diag64.get())));
  } else {
    {
      ProfScope prof_("k_fill_slices", st);
      k_fill_slices<<<nblk(S->rows_pad), 256, 0, st>>>(nb, S->size, S->rows_pad, s_a, S->j0,
                                                       S->slice_off.get(), colbits_of(S->jbits), S->norm.get(),
                                                       S->pnorm.get(), S->ca64.get(), S->ent.get(), S->ecoef64.get(),
                                                       S->a_real);
    }
  }
  SS_LAUNCH_CHECK();
  SS_TRY(S->nw32.alloc(S->rows_pad + 1, st));
  SS_TRY(S->rec64.alloc(S->rows_pad + 1, st));
  k_init_records<<<nblk(S->rows_pad + 1), 256, 0, st>>>(S->norm.get(), S->rows_pad + 1, S->wide, S->nw32.get(),
                                                        S->rec64.get());
  SS_LAUNCH_CHECK();
  SS_TRY(build_half(S, st));
  if (defer) {
    S->check_pending = true;
  } else {
    int32_t e[4] = {0, 0, 0, 0};
    SS_TRY(read_back(st, {{e, S->err_dev.get(), sizeof(e)}}));
    SS_TRY(check_words(S, e));
  }
  // the stamp's buffers outlive this call's stream (synchronised above, or
  // by the caller's next synchronisation before the stamp is handed out)
  S->keys.settle(); S->hl.settle(); S->level.settle(); S->norm.settle(); S->table.settle();
  S->afreq.settle(); S->stepkey.settle(); S->stepg.settle(); S->pnorm.settle(); S->pn32.settle(); S->aval.settle();
  S->ca64.settle(); S->ca32.settle(); S->slice_off.settle(); S->ent.settle(); S->ecoef64.settle();
  S->nw32.settle(); S->rec64.settle(); S->err_dev.settle(); S->zidx_dev.settle(); S->small_arena.settle();
  S->mirror.settle(); S->hpos.settle(); S->plus_rows.settle(); S->woff_h.settle(); S->ent_h.settle();
  S->ecoef_h.settle(); S->norm_h.settle();
  S->bval.settle(); S->cval.settle(); S->diag64.settle();
  return SS_OK;
}

// Re-pack every key (and step) into a wider layout and rebuild the table.
static ss_status relayout(ss_stamp_s* S, const KeyLayout& L2, cudaStream_t st) {
  const KeyParams P1 = make_key_params(S->key), P2 = make_key_params(L2);
  const int d = S->d;
  DevBuf<int32_t> freq;
  SS_TRY(freq.alloc((size_t)std::max<int64_t>(S->size, 1) * d, st));
  SS_DISPATCH_WT(S->key.WT, (k_export<WT><<<nblk(S->size), 256, 0, st>>>(P1, S->keys.get(), S->size, freq.get())));
  SS_LAUNCH_CHECK();
  const int64_t cap_rows = (int64_t)(S->keys.n / S->key.WT);
  DevBuf<uint64_t> k2;
  SS_TRY(k2.alloc((size_t)cap_rows * L2.WT, st));
  SS_DISPATCH_WT(L2.WT, (k_pack_rows<WT><<<nblk(S->size), 256, 0, st>>>(P2, freq.get(), S->size, k2.get(),
                                                                       S->hl.get())));
  SS_LAUNCH_CHECK();
  std::swap(S->keys.p, k2.p); std::swap(S->keys.n, k2.n); std::swap(S->keys.s, k2.s);
  k2.s = st;   // the old keys are freed on this stream, after the export
  S->key = L2;
  SS_TRY(S->stepkey.alloc((size_t)S->s_a * L2.WT, st));
  SS_TRY(S->stepg.alloc(S->s_a, st));
  SS_TRY(launch_steps(P2, S->afreq.get(), S->aval.get(), S->s_a, S->stepkey.get(), S->stepg.get(), S->pnorm.get(),
                      S->pn32.get(), S->wide, S->ca64.get(), S->ca32.get(), st));
  SS_LAUNCH_CHECK();
  const int64_t cap = S->cap;
  S->cap = 0;
  return grow_table(S, std::max<int64_t>(cap / 2, S->size), P2, st, S->err_dev.get());
}

static ss_status build_impl(ss_stamp_s* S, const ss_sparse* a_hat, const int32_t* f_freq, int64_t n_f, int N,
                            cudaStream_t st, bool defer = false) {
  const int d = a_hat->d;
  const int s_a = (int)a_hat->n;
  S->d = d;
  S->N = N;
  S->s_a = s_a;

  // The error words, the zero index and the step tables (canonical step
  // order) as views of one allocation; stepkey sized for the widest packed
  // key, since the layout is known only after the preparation's read-back.
  {
    size_t off = 0;
    auto at = [&](size_t bytes) {
      const size_t o = off;
      off += (bytes + 255) / 256 * 256;
      return o;
    };
    const size_t o_err = at(4 * sizeof(int32_t)), o_z = at(sizeof(int64_t)),
                 o_af = at((size_t)s_a * d * sizeof(int32_t)), o_av = at(s_a * sizeof(double2)),
                 o_sk = at((size_t)s_a * kMaxWords * sizeof(uint64_t)), o_sg = at(s_a * sizeof(uint64_t)),
                 o_pn = at(s_a * sizeof(int64_t)), o_p32 = at(s_a * sizeof(int32_t)),
                 o_c64 = at(s_a * sizeof(double2)), o_c32 = at(s_a * sizeof(float2));
    SS_TRY(S->small_arena.alloc(off, st));
    unsigned char* b = S->small_arena.get();
    S->err_dev.view(reinterpret_cast<int32_t*>(b + o_err), 4);
    S->zidx_dev.view(reinterpret_cast<int64_t*>(b + o_z), 1);
    S->afreq.view(reinterpret_cast<int32_t*>(b + o_af), (size_t)s_a * d);
    S->aval.view(reinterpret_cast<double2*>(b + o_av), s_a);
    S->stepkey.view(reinterpret_cast<uint64_t*>(b + o_sk), (size_t)s_a * kMaxWords);
    S->stepg.view(reinterpret_cast<uint64_t*>(b + o_sg), s_a);
    S->pnorm.view(reinterpret_cast<int64_t*>(b + o_pn), s_a);
    S->pn32.view(reinterpret_cast<int32_t*>(b + o_p32), s_a);
    S->ca64.view(reinterpret_cast<double2*>(b + o_c64), s_a);
    S->ca32.view(reinterpret_cast<float2*>(b + o_c32), s_a);
  }
  DevBuf<int32_t> Fs, rank, rank_a;
  DevBuf<PrepOut> prep;
  SS_TRY(Fs.alloc_tmp(n_f * d, st));
  SS_TRY(rank.alloc_tmp(n_f, st));
  SS_TRY(rank_a.alloc_tmp(s_a, st));
  SS_TRY(prep.alloc_tmp(1, st));
  int32_t* err = S->err_dev.get();
  SS_TRY(fill_small(st, {{err, 4 * sizeof(int32_t), 0}, {S->zidx_dev.get(), sizeof(int64_t), 0xff},
                         {rank.get(), n_f * sizeof(int32_t), 0}, {rank_a.get(), s_a * sizeof(int32_t), 0}}));

  // signed lexicographic order of F and supp a_hat
  const int chf = rank_chunk(n_f), cha = rank_chunk(s_a);
  const int64_t ncf = (n_f + chf - 1) / chf, nca = (s_a + cha - 1) / cha;
  // ranks (rank and rank_a start at zero): per-thread chunks for short rows,
  // one block per row for wide ones
  auto lex_rank = [&](const int32_t* fr, int64_t n, int ch, int64_t nc, int32_t* rk, int32_t* du) {
    if (d > 16) k_lex_rank_wide<<<(unsigned)n, 32 * kLexWarps, 0, st>>>(fr, n, d, rk, du);
    else k_lex_rank<<<nblk(n * nc), 256, 0, st>>>(fr, n, d, rk, du, ch);
  };
  {
    ProfScope prof_("k_lex_rank", st);
    lex_rank(f_freq, n_f, chf, ncf, rank.get(), err + 1);
  }
  k_scatter_rows<<<nblk(n_f), 256, 0, st>>>(f_freq, nullptr, n_f, d, rank.get(), Fs.get(), nullptr);
  {
    ProfScope prof_("k_lex_rank", st);
    lex_rank(a_hat->freq, s_a, cha, nca, rank_a.get(), err + 2);
  }
  k_scatter_rows<<<nblk(s_a), 256, 0, st>>>(a_hat->freq, reinterpret_cast<const double2*>(a_hat->val), s_a, d,
                                            rank_a.get(), S->afreq.get(), S->aval.get());
  {
    ProfScope prof_("k_prep", st);
    k_prep<<<1, kPrepThreads, 0, st>>>(Fs.get(), n_f, S->afreq.get(), S->aval.get(), s_a, d, prep.get());
  }
  SS_LAUNCH_CHECK();
  // While the GPU ranks and prepares: the buffers whose sizes follow from
  // |F|, s_a and N alone.  The table, the rows' linear forms, levels and
  // norms, and the candidate buffers of the levels are sized at once for the
  // whole construction when the bound fits, so that the levels neither grow
  // (copy, rehash) nor allocate; the keys wait for the packed layout.
  S->level_start.assign(1, 0);
  const int64_t pre = std::max<int64_t>(n_f, stamp_size_bound(n_f, s_a, N, kPresizeCap));
  // table load at most 1/4 of the bound (d = 100: 2^23 slots for 1.15 M
  // keys); at load 0.27 the level-3 insert and the lookups ran 20 and 8 us
  // longer (longer probe sequences)
  SS_TRY(grow_table(S, 2 * pre, KeyParams{}, st, err));
  SS_TRY(S->hl.alloc(pre, st));
  SS_TRY(S->level.alloc(pre, st));
  SS_TRY(S->norm.alloc(pre + kSlice + 1, st));
  LevelTmp lt;
  if (N >= 1) {
    // parents of the last level: |S^{N-1}| <= the same multiset bound
    const int64_t par = N >= 2 ? stamp_size_bound(n_f, s_a, N - 1, kPresizeCap) : n_f;
    const int64_t ncand = par * s_a;
    if (par < kPresizeCap && ncand * 2 * (int64_t)sizeof(int64_t) <= kLevelTmpPresize) {
      SS_TRY(lt.slot_of.alloc_tmp(ncand, st));
      SS_TRY(lt.cand.alloc_tmp(ncand, st));
    }
  }
  PrepOut h{};
  int32_t herr[4];
  SS_TRY(read_back(st, {{&h, prep.get(), sizeof(h)}, {herr, err, sizeof(herr)}}));
  if (herr[1]) SS_FAIL(SS_ERR_INVALID, "stamp_build: duplicate frequencies in F");
  if (herr[2]) SS_FAIL(SS_ERR_INVALID, "stamp_build: duplicate frequencies in supp a_hat");
  // the ADR operator's reaction term makes u_hat_0 part of the solution, so f_hat_0 may be nonzero there
  if (h.zero_in_f && !S->adr) SS_FAIL(SS_ERR_INVALID, "stamp_build: F contains k = 0 (f_hat_0 must vanish)");
  if (h.bad_sym) SS_FAIL(SS_ERR_INVALID, "stamp_build: supp a_hat must contain 0 and be closed under negation");
  if (h.bad_herm) SS_FAIL(SS_ERR_INVALID, "stamp_build: a_hat is not Hermitian (a must be real)");
  if (!(h.off_l1 < h.a0_abs)) SS_FAIL(SS_ERR_NOT_ELLIPTIC, "stamp_build: ||a_hat - a_hat_0||_1 = %g >= |a_hat_0| = %g",
                                       h.off_l1, h.a0_abs);
  if (!(h.a0_re > 0)) SS_FAIL(SS_ERR_NOT_ELLIPTIC, "stamp_build: Re(a_hat_0) must be positive");
  S->a0 = h.a0_re;
  S->half_cand = !S->adr && h.f_sym && h.herm_exact;
  // real a_hat: every entry coefficient 2 pi^2 (|k|^2 + |l|^2 - |p|^2) a_hat_p
  // is real (the ADR entries carry the advection and reaction terms)
  S->a_real = !S->adr && h.a_real;
  S->j0 = h.j0;
  S->maxabs_f = h.maxabs_f;
  S->maxabs_a = h.maxabs_a;

  // key layout: every frequency of S^{N+1} must fit (neighbour lookups reach one level further)
  KeyLayout L;
  const int64_t maxabs = (int64_t)h.maxabs_f + (int64_t)(N + 1) * h.maxabs_a;
  SS_TRY(make_layout(d, maxabs, &L));
  S->key = L;
  S->wide = norms_wide(d, maxabs);
  const KeyParams P = make_key_params(L);
  int jb = 0;
  while ((1 << jb) < s_a) ++jb;
  S->jbits = std::max(jb, 1);

  if (S->a_real) {
    k_real_part<<<nblk(s_a), 256, 0, st>>>(S->aval.get(), s_a);
    SS_LAUNCH_CHECK();
  }

  // steps and coefficients in canonical order (afreq and aval were written
  // in that order by the scatter above)
  SS_TRY(launch_steps(P, S->afreq.get(), S->aval.get(), s_a, S->stepkey.get(), S->stepg.get(), S->pnorm.get(),
                      S->pn32.get(), S->wide, S->ca64.get(), S->ca32.get(), st));
  SS_LAUNCH_CHECK();

  // level 0
  SS_TRY(S->keys.alloc((size_t)pre * L.WT, st));
  {
    ProfScope prof_("k_level0", st);
    if (d > 16) {
      SS_DISPATCH_WT(L.WT, (k_level0_warp<WT><<<(unsigned)((n_f + kPackWarps - 1) / kPackWarps), 32 * kPackWarps, 0,
                                                 st>>>(P, Fs.get(), n_f, S->keys.get(), S->hl.get(), S->level.get(),
                                                       S->norm.get(), S->table.get(), (uint64_t)S->cap - 1, err,
                                                       S->zidx_dev.get())));
    } else {
      SS_DISPATCH_WT(L.WT, (k_level0<WT><<<nblk(n_f), 256, 0, st>>>(P, Fs.get(), n_f, S->keys.get(), S->hl.get(),
                                                                    S->level.get(), S->norm.get(), S->table.get(),
                                                                    (uint64_t)S->cap - 1, err, S->zidx_dev.get())));
    }
  }
  SS_LAUNCH_CHECK();
  S->size = n_f;
  S->level_start.push_back(n_f);
  {
    ProfScope prof_("stamp_levels", st);
    SS_TRY(run_levels(S, 1, N, st, lt));
  }
  // give back a large over-reservation of the size bound (the keys stay for
  // lookups, extension and export; the norms are read up to rows_pad + 1)
  const int64_t rows = (int64_t)(S->keys.n / L.WT), keep = S->size + kSlice + 1;
  if (rows > 4 * keep && (double)rows * (8.0 * L.WT + 9.0) > 64e6) SS_TRY(resize_keys(S, keep, st));
  ProfScope prof_("stamp_operator", st);
  return build_operator(S, st, defer);
}

// Buffers replaced during an extension are freed on the extension's stream,
// after the work already queued there.
static void rebind(ss_stamp_s* S, cudaStream_t st) {
  S->keys.s = st;
  S->hl.s = st;
  S->stepg.s = st;
  S->level.s = st;
  S->norm.s = st;
  S->table.s = st;
  S->stepkey.s = st;
  S->slice_off.s = st;
  S->ent.s = st;
  S->ecoef64.s = st;
  S->ecoefdf.s = st;
  S->ecoefdf_h.s = st;
  S->nw32.s = st;
  S->rec64.s = st;
  S->diag64.s = st;
  S->mirror.s = st;
  S->hpos.s = st;
  S->plus_rows.s = st;
  S->woff_h.s = st;
  S->ent_h.s = st;
  S->ecoef_h.s = st;
  S->norm_h.s = st;
}

static ss_status extend_impl(ss_stamp_s* S, int levels, cudaStream_t st) {
  rebind(S, st);
  const int N2 = S->N + levels;
  const int64_t need = (int64_t)S->maxabs_f + (int64_t)(N2 + 1) * S->maxabs_a;
  const int64_t have = ((int64_t)1 << (S->key.b - 1)) - 1;
  const bool wide2 = norms_wide(S->d, need);
  if (need > have) {
    KeyLayout L2;
    SS_TRY(make_layout(S->d, need, &L2));
    S->wide = wide2;
    SS_TRY(relayout(S, L2, st));
  } else if (wide2 != S->wide) {
    // the FP32 norm words of the steps change encoding (the records are
    // rewritten by build_operator)
    S->wide = wide2;
    const KeyParams P = make_key_params(S->key);
    SS_TRY(launch_steps(P, S->afreq.get(), S->aval.get(), S->s_a, S->stepkey.get(), S->stepg.get(), S->pnorm.get(),
                        S->pn32.get(), S->wide, S->ca64.get(), S->ca32.get(), st));
    SS_LAUNCH_CHECK();
  }
  LevelTmp lt;
  SS_TRY(run_levels(S, S->N + 1, N2, st, lt));
  S->N = N2;
  return build_operator(S, st, false);
}

static ss_status build_entry(const ss_sparse* a_hat, const int32_t* f_freq, int64_t n_f, int32_t N, ss_stamp* out,
                             cudaStream_t st, bool defer) {
  if (!a_hat || !out || !f_freq || !a_hat->freq || !a_hat->val)
    SS_FAIL(SS_ERR_INVALID, "stamp_build: null argument");
  if (a_hat->d < 1 || a_hat->n < 1 || n_f < 1 || N < 0 || N > 120)
    SS_FAIL(SS_ERR_INVALID, "stamp_build: need d >= 1, |supp a_hat| >= 1, |F| >= 1, 0 <= N <= 120");
  if (a_hat->n > 4096) SS_FAIL(SS_ERR_INVALID, "stamp_build: |supp a_hat| > 4096");
  *out = nullptr;
  ss_stamp_s* S = new ss_stamp_s();
  ss_status s;
  {
    ProfScope prof_("stamp_build", st);
    s = build_impl(S, a_hat, f_freq, n_f, N, st, defer);
  }
  if (s != SS_OK) {
    cudaStreamSynchronize(st);
    delete S;
    return s;
  }
  *out = S;
  return SS_OK;
}

ss_status stamp_build_pending(const ss_sparse* a_hat, const int32_t* f_freq, int64_t n_f, int32_t N, ss_stamp* out,
                              cudaStream_t st) {
  return build_entry(a_hat, f_freq, n_f, N, out, st, true);
}

ss_status stamp_check_pending(ss_stamp_s* S, const int32_t* e) {
  return S->check_pending ? check_words(S, e) : SS_OK;
}

ss_status stamp_host_tables(ss_stamp_s* S, cudaStream_t st) {
  const bool need_full = (int64_t)S->woff_host.size() != S->n_slices + 1;
  const bool need_half = S->half_ok && (int64_t)S->woff_h_host.size() != S->n_slices_h + 1;
  if (!need_full && !need_half && !S->check_pending) return SS_OK;
  int32_t e[4] = {0, 0, 0, 0};
  if (need_full) S->woff_host.resize(S->n_slices + 1);
  if (need_half) S->woff_h_host.resize(S->n_slices_h + 1);
  SS_TRY(read_back(st, {{e, S->err_dev.get(), sizeof(e)},
                        {need_full ? S->woff_host.data() : nullptr, S->slice_off.get(),
                         need_full ? (S->n_slices + 1) * sizeof(int32_t) : 0},
                        {need_half ? S->woff_h_host.data() : nullptr, S->woff_h.get(),
                         need_half ? (S->n_slices_h + 1) * sizeof(int32_t) : 0}}));
  SS_TRY(stamp_check_pending(S, e));
  if (!S->half_ok) S->woff_h_host.clear();
  return SS_OK;
}
}  // namespace ss

using namespace ss;

extern "C" ss_status stamp_build(const ss_sparse* a_hat, const int32_t* f_freq, int64_t n_f, int32_t N, ss_stamp* out,
                                 void* stream) {
  return build_entry(a_hat, f_freq, n_f, N, out, as_stream(stream), false);
}

namespace {

// Host copy of a device sparse list (small: supports of the data).
ss_status host_sparse(const ss_sparse* g, int d, std::vector<int32_t>* f, std::vector<double2>* v,
                      cudaStream_t st, const char* what) {
  if (!g || g->d != d || g->n < 0 || (g->n > 0 && (!g->freq || !g->val)))
    SS_FAIL(SS_ERR_INVALID, "stamp_build_adr: bad %s", what);
  if (g->n > 4096) SS_FAIL(SS_ERR_INVALID, "stamp_build_adr: |supp %s| > 4096", what);
  f->resize((size_t)g->n * d);
  v->resize((size_t)g->n);
  if (g->n > 0) {
    SS_CUDA(cudaMemcpyAsync(f->data(), g->freq, f->size() * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    SS_CUDA(cudaMemcpyAsync(v->data(), g->val, v->size() * sizeof(double2), cudaMemcpyDeviceToHost, st));
  }
  return SS_OK;
}

// Hermitian: -k present with the conjugate value (a real function).
bool hermitian(const std::map<std::vector<int32_t>, double2>& m) {
  for (const auto& [k, v] : m) {
    std::vector<int32_t> nk(k.size());
    for (size_t c = 0; c < k.size(); ++c) nk[c] = -k[c];
    auto it = m.find(nk);
    if (it == m.end()) return false;
    const double sc = 1e-12 * std::max(1.0, std::hypot(v.x, v.y));
    if (std::fabs(it->second.x - v.x) > sc || std::fabs(it->second.y + v.y) > sc) return false;
  }
  return true;
}

}  // namespace

extern "C" ss_status stamp_build_adr(const ss_sparse* a_hat, const ss_sparse* b_hat, const ss_sparse* c_hat,
                                     const int32_t* f_freq, int64_t n_f, int32_t N, ss_stamp* out, void* stream) {
  if (!a_hat || !b_hat || !c_hat || !out || !f_freq) SS_FAIL(SS_ERR_INVALID, "stamp_build_adr: null argument");
  const int d = a_hat->d;
  if (d < 1 || d > 64 || n_f < 1 || N < 0 || N > 120)
    SS_FAIL(SS_ERR_INVALID, "stamp_build_adr: need 1 <= d <= 64, |F| >= 1, 0 <= N <= 120");
  *out = nullptr;
  cudaStream_t st = as_stream(stream);
  // gather a_hat, the d components of b_hat and c_hat on the host
  std::vector<int32_t> fa, fc;
  std::vector<double2> va, vc;
  std::vector<std::vector<int32_t>> fb(d);
  std::vector<std::vector<double2>> vb(d);
  SS_TRY(host_sparse(a_hat, d, &fa, &va, st, "a_hat"));
  for (int j = 0; j < d; ++j) SS_TRY(host_sparse(b_hat + j, d, &fb[j], &vb[j], st, "b_hat"));
  SS_TRY(host_sparse(c_hat, d, &fc, &vc, st, "c_hat"));
  SS_CUDA(cudaStreamSynchronize(st));
  // union U of the supports in signed lexicographic order (std::map orders
  // int vectors lexicographically), with every coefficient on U
  struct Coef {
    double2 a{0.0, 0.0}, c{0.0, 0.0};
    std::vector<double2> b;
  };
  std::map<std::vector<int32_t>, Coef> U;
  std::map<std::vector<int32_t>, double2> ma, mc;
  std::vector<std::map<std::vector<int32_t>, double2>> mb(d);
  auto add = [&](const std::vector<int32_t>& f, const std::vector<double2>& v, std::map<std::vector<int32_t>, double2>* m,
                 int which) -> bool {
    for (size_t t = 0; t < v.size(); ++t) {
      std::vector<int32_t> k(f.begin() + t * d, f.begin() + (t + 1) * d);
      if (m->count(k)) return false;
      (*m)[k] = v[t];
      Coef& e = U[k];
      if (e.b.empty()) e.b.assign(d, double2{0.0, 0.0});
      if (which < 0) e.a = v[t];
      else if (which == d) e.c = v[t];
      else e.b[which] = v[t];
    }
    return true;
  };
  if (!add(fa, va, &ma, -1)) SS_FAIL(SS_ERR_INVALID, "stamp_build_adr: duplicate frequencies in a_hat");
  for (int j = 0; j < d; ++j)
    if (!add(fb[j], vb[j], &mb[j], j)) SS_FAIL(SS_ERR_INVALID, "stamp_build_adr: duplicate frequencies in b_hat");
  if (!add(fc, vc, &mc, d)) SS_FAIL(SS_ERR_INVALID, "stamp_build_adr: duplicate frequencies in c_hat");
  bool herm = hermitian(ma) && hermitian(mc);
  for (int j = 0; j < d; ++j) herm = herm && hermitian(mb[j]);
  if (!herm) SS_FAIL(SS_ERR_INVALID, "stamp_build_adr: a_hat, b_hat and c_hat must be Hermitian (real data)");
  if ((int64_t)U.size() > 4096) SS_FAIL(SS_ERR_INVALID, "stamp_build_adr: union of the supports > 4096");
  const int64_t s_u = (int64_t)U.size();
  std::vector<int32_t> uf((size_t)s_u * d);
  std::vector<double2> ua(s_u), uc(s_u), ub((size_t)s_u * d);
  int64_t t = 0;
  for (const auto& [k, e] : U) {
    std::copy(k.begin(), k.end(), uf.begin() + t * d);
    ua[t] = e.a;
    uc[t] = e.c;
    std::copy(e.b.begin(), e.b.end(), ub.begin() + t * d);
    ++t;
  }
  ss_stamp_s* S = new ss_stamp_s();
  S->adr = true;
  DevBuf<int32_t> dU;
  DevBuf<double2> dA;
  ss_status r = SS_OK;
  auto up = [&]() -> ss_status {
    SS_TRY(dU.alloc(uf.size(), st));
    SS_TRY(dA.alloc(ua.size(), st));
    SS_TRY(S->bval.alloc(ub.size(), st));
    SS_TRY(S->cval.alloc(uc.size(), st));
    SS_CUDA(cudaMemcpyAsync(dU.get(), uf.data(), uf.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    SS_CUDA(cudaMemcpyAsync(dA.get(), ua.data(), ua.size() * sizeof(double2), cudaMemcpyHostToDevice, st));
    SS_CUDA(cudaMemcpyAsync(S->bval.get(), ub.data(), ub.size() * sizeof(double2), cudaMemcpyHostToDevice, st));
    SS_CUDA(cudaMemcpyAsync(S->cval.get(), uc.data(), uc.size() * sizeof(double2), cudaMemcpyHostToDevice, st));
    const ss_sparse au{d, s_u, dU.get(), reinterpret_cast<const double*>(dA.get())};
    // U is already in canonical step order, so the build keeps bval / cval aligned
    return build_impl(S, &au, f_freq, n_f, N, st);
  };
  r = up();
  if (r != SS_OK) {
    cudaStreamSynchronize(st);
    delete S;
    return r;
  }
  *out = S;
  return SS_OK;
}

extern "C" ss_status stamp_extend(ss_stamp s, int32_t levels, void* stream) {
  if (!s || levels < 0 || s->N + levels > 120) SS_FAIL(SS_ERR_INVALID, "stamp_extend: bad argument");
  if (levels == 0) return SS_OK;
  cudaStream_t st = as_stream(stream);
  drop_solve_ctx(s);   // the solver's work split belongs to the old set
  const ss_status r = extend_impl(s, levels, st);
  if (r != SS_OK) cudaStreamSynchronize(st);
  return r;
}

extern "C" ss_status stamp_set_table_limit(int64_t max_slots) {
  if (max_slots < 0) SS_FAIL(SS_ERR_INVALID, "stamp_set_table_limit: negative bound");
  g_table_limit.store(max_slots, std::memory_order_relaxed);
  return SS_OK;
}

extern "C" void stamp_destroy(ss_stamp s) {
  if (!s) return;
  cudaDeviceSynchronize();
  drop_solve_ctx(s);
  delete s;
}

extern "C" ss_status stamp_real_coefficients(ss_stamp s, int32_t* real) {
  if (!s || !real) SS_FAIL(SS_ERR_INVALID, "stamp_real_coefficients: null argument");
  *real = s->a_real ? 1 : 0;
  return SS_OK;
}

extern "C" ss_status stamp_info(ss_stamp s, int64_t* size, int64_t* nnz, int64_t* zero_index, int32_t* n_levels) {
  if (!s) SS_FAIL(SS_ERR_INVALID, "stamp_info: null stamp");
  if (size) *size = s->size;
  if (nnz) *nnz = s->nnz;
  if (zero_index) *zero_index = s->zero_idx;
  if (n_levels) *n_levels = s->N + 1;
  return SS_OK;
}

extern "C" ss_status stamp_export(ss_stamp s, int32_t* freq_out, int8_t* level_out, void* stream) {
  if (!s) SS_FAIL(SS_ERR_INVALID, "stamp_export: null stamp");
  cudaStream_t st = as_stream(stream);
  if (freq_out) {
    const KeyParams P = make_key_params(s->key);
    SS_DISPATCH_WT(s->key.WT, (k_export<WT><<<nblk(s->size), 256, 0, st>>>(P, s->keys.get(), s->size, freq_out)));
    SS_LAUNCH_CHECK();
  }
  if (level_out) SS_CUDA(cudaMemcpyAsync(level_out, s->level.get(), s->size, cudaMemcpyDeviceToDevice, st));
  return SS_OK;
}

extern "C" ss_status stamp_lookup(ss_stamp s, const int32_t* freq, int64_t n, int64_t* idx_out, void* stream) {
  if (!s || (n > 0 && (!freq || !idx_out))) SS_FAIL(SS_ERR_INVALID, "stamp_lookup: null argument");
  if (n == 0) return SS_OK;
  const KeyParams P = make_key_params(s->key);
  cudaStream_t st = as_stream(stream);
  if (P.d > 16) {   // wide keys: one warp per query
    SS_DISPATCH_WT(s->key.WT, (k_lookup_warp<WT><<<(unsigned)((n + kLookupWarps - 1) / kLookupWarps),
                                                   32 * kLookupWarps, 0, st>>>(P, s->keys.get(), s->table.get(),
                                                                               (uint64_t)s->cap - 1, freq, n,
                                                                               idx_out)));
  } else {
    SS_DISPATCH_WT(s->key.WT, (k_lookup<WT><<<nblk(n), 256, 0, st>>>(P, s->keys.get(), s->hl.get(), s->table.get(),
                                                                    (uint64_t)s->cap - 1, freq, n, idx_out)));
  }
  SS_LAUNCH_CHECK();
  return SS_OK;
}

extern "C" ss_status stamp_scatter(ss_stamp s, const ss_sparse* g, double* out, int64_t* n_outside, void* stream) {
  if (!s || !g || !out) SS_FAIL(SS_ERR_INVALID, "stamp_scatter: null argument");
  if (g->d != s->d) SS_FAIL(SS_ERR_INVALID, "stamp_scatter: dimension %d != %d", g->d, s->d);
  cudaStream_t st = as_stream(stream);
  SS_CUDA(cudaMemsetAsync(out, 0, s->size * sizeof(double2), st));
  if (g->n == 0) {
    if (n_outside) *n_outside = 0;
    return SS_OK;
  }
  DevBuf<int64_t> idx;
  DevBuf<unsigned long long> outside;
  SS_TRY(idx.alloc_tmp(g->n, st));
  if (n_outside) {
    SS_TRY(outside.alloc_tmp(1, st));
    SS_CUDA(cudaMemsetAsync(outside.get(), 0, sizeof(unsigned long long), st));
  }
  SS_TRY(stamp_lookup(s, g->freq, g->n, idx.get(), stream));
  k_scatter_vals<<<nblk(g->n), 256, 0, st>>>(idx.get(), reinterpret_cast<const double2*>(g->val), g->n,
                                             reinterpret_cast<double2*>(out), outside.get());
  SS_LAUNCH_CHECK();
  if (!n_outside) return SS_OK;   // no count asked for: stays asynchronous
  unsigned long long h = 0;
  SS_TRY(read_back(st, {{&h, outside.get(), sizeof(h)}}));
  *n_outside = (int64_t)h;
  return SS_OK;
}
