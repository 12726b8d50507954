// Rank-1 lattices: residues k.z mod M, the reconstructing check, the random
// lattice of Lemma RandomRank1Lattice and a component-by-component search.
#include <algorithm>
#include <cmath>

#include "lattice.cuh"

namespace ss {

// -------------------------------------------------------------- host math

static bool is_prime_host(int64_t n) {
  if (n < 2) return false;
  if (n % 2 == 0) return n == 2;
  for (int64_t i = 3; i * i <= n; i += 2)
    if (n % i == 0) return false;
  return true;
}

int64_t next_prime_host(int64_t n) {
  if (n < 2) n = 2;
  while (!is_prime_host(n)) ++n;
  return n;
}

// Smallest integer >= n whose prime factors are 2, 3, 5, 7 (FFT-friendly).
int64_t next_smooth_host(int64_t n) {
  if (n < 1) n = 1;
  for (;; ++n) {
    int64_t m = n;
    for (int64_t p : {2, 3, 5, 7})
      while (m % p == 0) m /= p;
    if (m == 1) return n;
  }
}

// ---------------------------------------------------------------- kernels

// One warp per row.
__global__ void k_residues(const int32_t* __restrict__ f, int64_t n, int d, LatticeDev L, int64_t* res) {
  const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (i >= n) return;   // warp-uniform
  const int64_t r = residue_warp(f + i * d, d, L);
  if ((threadIdx.x & 31) == 0) res[i] = r;
}

namespace {

__device__ bool rows_equal(const int32_t* a, const int32_t* b, int d) {
  for (int c = 0; c < d; ++c)
    if (a[c] != b[c]) return false;
  return true;
}

__device__ __forceinline__ uint64_t rhash(uint64_t r) {
  r ^= r >> 33;
  r *= 0xff51afd7ed558ccdull;
  r ^= r >> 33;
  return r;
}

// Residue table: slot = index + 1 of the row owning a residue (0 = empty).
__global__ void k_check_insert(const int32_t* __restrict__ f, const int64_t* __restrict__ res, int64_t n, int d,
                               unsigned long long* table, uint64_t capmask, int32_t* flags) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint64_t r = (uint64_t)res[i];
  uint64_t h = rhash(r) & capmask;
  for (uint64_t probe = 0; probe <= capmask; ++probe) {
    const unsigned long long old = atomicCAS(table + h, 0ull, (unsigned long long)(i + 1));
    if (old == 0ull) return;
    const int64_t o = (int64_t)old - 1;
    if ((uint64_t)res[o] == r) {
      if (rows_equal(f + o * d, f + i * d, d)) atomicOr(flags + 0, 1);   // duplicate row
      else atomicOr(flags + 1, 1);                                       // collision
      return;
    }
    h = (h + 1) & capmask;
  }
  atomicOr(flags + 2, 1);
}

// For every row k, is -k present?  (residue of -k is (M - r) mod M)
// One warp per row: the row owning residue M - res[i] is found by probing
// (lane 0's loads, broadcast), then compared with -f_i 32 coordinates at a time.
__global__ void k_check_symmetric(const int32_t* __restrict__ f, const int64_t* __restrict__ res, int64_t n, int d,
                                  int64_t M, const unsigned long long* __restrict__ table, uint64_t capmask,
                                  int32_t* flags) {
  const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= n) return;   // warp-uniform
  const uint64_t r = (uint64_t)((M - res[i]) % M);
  uint64_t h = rhash(r) & capmask;
  int64_t o = -1;
  for (uint64_t probe = 0; probe <= capmask; ++probe) {
    const unsigned long long v = table[h];
    if (v == 0ull) break;
    const int64_t oc = (int64_t)v - 1;
    if ((uint64_t)res[oc] == r) {
      o = oc;
      break;
    }
    h = (h + 1) & capmask;
  }
  bool neg = o >= 0;
  if (neg) {
    const int32_t* a = f + o * d;
    const int32_t* b = f + i * d;
    bool bad = false;
    for (int c = lane; c < d; c += 32) bad |= a[c] != -b[c];
    neg = !__any_sync(0xffffffffu, bad);
  }
  if (!neg && lane == 0) atomicOr(flags + 3, 1);
}

__global__ void k_minmax(const int32_t* __restrict__ f, int64_t n, int d, int32_t* mn, int32_t* mx) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * d) return;
  const int c = (int)(t % d);
  atomicMin(mn + c, f[t]);
  atomicMax(mx + c, f[t]);
}

// CBC: partial residues of coordinates [0, j) are in rho; block b tries
// candidate cand[b] for coordinate j: rho'_i = rho_i + k_ij cand (mod M), and
// fails if two rows with distinct projections onto [0, j] share rho'.
__global__ void k_cbc_try(const int32_t* __restrict__ f, int64_t n, int d, int j, int64_t M,
                          const int64_t* __restrict__ rho, const int64_t* __restrict__ cand, int64_t* scratch,
                          int32_t* fail) {
  const int b = blockIdx.x;
  const uint64_t z = (uint64_t)cand[b];
  int64_t* rp = scratch + (int64_t)b * n;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    int64_t k = f[i * d + j] % M;
    if (k < 0) k += M;
    rp[i] = (int64_t)(((uint64_t)rho[i] + ((uint64_t)k * z) % (uint64_t)M) % (uint64_t)M);
  }
  __syncthreads();
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int64_t i = threadIdx.x; i < n && !bad; i += blockDim.x) {
    const int64_t ri = rp[i];
    for (int64_t q = i + 1; q < n; ++q) {
      if (rp[q] != ri) continue;
      bool same = true;
      for (int c = 0; c <= j; ++c) same &= (f[i * d + c] == f[q * d + c]);
      if (!same) { bad = 1; break; }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) fail[b] = bad;
}

// Same test with the residues and an open-addressing residue -> row table in
// shared memory: a row meeting an earlier row with its residue compares their
// projections (O(n) per candidate instead of all pairs).
__global__ void k_cbc_try_hash(const int32_t* __restrict__ f, int64_t n, int d, int j, int64_t M,
                               const int64_t* __restrict__ rho, const int64_t* __restrict__ cand, int cap,
                               int32_t* fail) {
  extern __shared__ __align__(16) unsigned char smem[];
  int64_t* rp = reinterpret_cast<int64_t*>(smem);
  int32_t* tab = reinterpret_cast<int32_t*>(rp + n);
  __shared__ int bad;
  const uint64_t z = (uint64_t)cand[blockIdx.x];
  if (threadIdx.x == 0) bad = 0;
  for (int i = threadIdx.x; i < cap; i += blockDim.x) tab[i] = -1;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    int64_t k = f[i * d + j] % M;
    if (k < 0) k += M;
    rp[i] = (int64_t)(((uint64_t)rho[i] + ((uint64_t)k * z) % (uint64_t)M) % (uint64_t)M);
  }
  __syncthreads();
  const uint32_t mask = (uint32_t)cap - 1;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const int64_t r = rp[i];
    uint32_t h = (uint32_t)(rhash((uint64_t)r) & mask);
    for (int probe = 0; probe < cap; ++probe) {
      const int32_t old = atomicCAS(tab + h, -1, (int32_t)i);
      if (old == -1) break;
      if (rp[old] == r) {
        bool same = true;
        for (int c = 0; c <= j; ++c) same &= (f[i * d + c] == f[(int64_t)old * d + c]);
        if (!same) atomicExch(&bad, 1);
        break;
      }
      h = (h + 1) & mask;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) fail[blockIdx.x] = bad;
}

__global__ void k_cbc_accept(const int32_t* __restrict__ f, int64_t n, int d, int j, int64_t M,
                             const int64_t* __restrict__ zdev, int64_t* rho) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint64_t z = (uint64_t)zdev[j];
  int64_t k = f[i * d + j] % M;
  if (k < 0) k += M;
  rho[i] = (int64_t)(((uint64_t)rho[i] + ((uint64_t)k * z) % (uint64_t)M) % (uint64_t)M);
}

// First candidate of coordinate j that passed (in stream order); on failure
// records the coordinate and keeps z_j = 1 so the remaining steps stay defined.
__global__ void k_cbc_pick(const int32_t* __restrict__ fail, const int64_t* __restrict__ cand, int n_cand, int j,
                           int64_t* zdev, int32_t* err) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int64_t z = 1;
  int pick = -1;
  for (int c = 0; c < n_cand; ++c)
    if (!fail[c]) { pick = c; break; }
  if (pick >= 0) z = cand[pick];
  else if (*err == 0) *err = j + 1;
  zdev[j] = z;
}

// The whole component-by-component search in one cooperative launch: block c
// tests candidate c of every coordinate in turn.  Each block keeps the partial
// residues rho_i = sum_{c' < j} k_{ic'} z_{c'} mod M of all frequencies in
// shared memory, publishes pass/fail of its candidate for coordinate j, waits
// for the other blocks (bounded wait: on timeout it records SS_ERR_TIMEOUT in
// err[1] and returns), then takes the first candidate that passed - the same
// pick in every block - and adds its column to rho.  Same result as the
// per-coordinate launches below.
__device__ __forceinline__ uint64_t modm(uint64_t x, uint64_t M, uint64_t inv) {
  uint64_t r = x - __umul64hi(x, inv) * M;   // x < 2^62, M < 2^31: quotient estimate short by at most 2
  r = r >= M ? r - M : r;
  return r >= M ? r - M : r;
}

// k mod M in [0, M) by a 32-bit remainder (M < 2^31).
__device__ __forceinline__ uint64_t coord_mod(int32_t k, int64_t M) {
  const int32_t r = k % (int32_t)M;
  return (uint64_t)(r < 0 ? r + (int32_t)M : r);
}

// (a + b) mod M for a, b in [0, M).
__device__ __forceinline__ uint64_t addm(uint64_t a, uint64_t b, uint64_t M) {
  const uint64_t s = a + b;
  return s >= M ? s - M : s;
}

__device__ __forceinline__ long long cbc_timer() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

constexpr int kCbcThreads = 1024;

__global__ void __launch_bounds__(kCbcThreads) k_cbc_all(const int32_t* __restrict__ f, int64_t n, int d, int64_t M,
                                                 const int64_t* __restrict__ cand, int n_cand, int cap,
                                                 int32_t* fail, unsigned* arrive, int64_t* zdev, int32_t* err) {
  extern __shared__ __align__(16) unsigned char smem[];
  int64_t* rho = reinterpret_cast<int64_t*>(smem);
  int64_t* rp = rho + n;
  int32_t* tab = reinterpret_cast<int32_t*>(rp + n);
  __shared__ int bad, pick_s, ok_s;
  const uint64_t inv = ~0ull / (uint64_t)M;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) rho[i] = (int64_t)coord_mod(f[i * d], M);   // z_1 = 1
  if (blockIdx.x == 0 && threadIdx.x == 0) zdev[0] = 1;
  const uint32_t mask = (uint32_t)cap - 1;
  for (int j = 1; j < d; ++j) {
    const uint64_t z = (uint64_t)cand[(int64_t)j * n_cand + blockIdx.x];
    if (threadIdx.x == 0) bad = 0;
    for (int i = threadIdx.x; i < cap; i += blockDim.x) tab[i] = -1;
    __syncthreads();
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x)
      rp[i] = (int64_t)addm((uint64_t)rho[i], modm(coord_mod(f[i * d + j], M) * z, M, inv), M);
    __syncthreads();
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
      const int64_t r = rp[i];
      uint32_t h = (uint32_t)(rhash((uint64_t)r) & mask);
      for (int probe = 0; probe < cap; ++probe) {
        const int32_t old = atomicCAS(tab + h, -1, (int32_t)i);
        if (old == -1) break;
        if (rp[old] == r) {
          bool same = true;
          for (int c = 0; c <= j; ++c) same &= (f[i * d + c] == f[(int64_t)old * d + c]);
          if (!same) atomicExch(&bad, 1);
          break;
        }
        h = (h + 1) & mask;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      fail[(int64_t)j * n_cand + blockIdx.x] = bad;
      unsigned* a = arrive + j;
      asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(a) : "memory");
      const long long t0 = cbc_timer();
      int ok = 1;
      for (;;) {
        unsigned v;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(a) : "memory");
        if (v >= (unsigned)gridDim.x) break;
        if (cbc_timer() - t0 > 2000000000ll) {
          atomicCAS(err + 1, 0, (int)SS_ERR_TIMEOUT);
          ok = 0;
          break;
        }
      }
      int pick = -1;
      if (ok)
        for (int c = 0; c < n_cand; ++c)
          if (!__ldcg(fail + (int64_t)j * n_cand + c)) { pick = c; break; }
      ok_s = ok;
      pick_s = pick;
    }
    __syncthreads();
    if (!ok_s) return;
    const int pick = pick_s;
    const uint64_t zj = pick >= 0 ? (uint64_t)cand[(int64_t)j * n_cand + pick] : 1ull;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      zdev[j] = (int64_t)zj;
      if (pick < 0 && err[0] == 0) err[0] = j + 1;
    }
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x)
      rho[i] = (int64_t)addm((uint64_t)rho[i], modm(coord_mod(f[i * d + j], M) * zj, M, inv), M);
    __syncthreads();
  }
}

inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

}  // namespace

ss_status make_lattice_dev(const ss_lattice* lat, LatticeDev* L) {
  if (!lat || !lat->z) SS_FAIL(SS_ERR_INVALID, "lattice: null argument");
  if (lat->d < 1 || lat->d > kMaxLatticeDim) SS_FAIL(SS_ERR_INVALID, "lattice: d = %d outside 1..%d", lat->d, kMaxLatticeDim);
  if (lat->M < 2 || lat->M >= (1ll << 31)) SS_FAIL(SS_ERR_INVALID, "lattice: M = %lld outside [2, 2^31)", (long long)lat->M);
  L->d = lat->d;
  L->M = lat->M;
  for (int c = 0; c < lat->d; ++c) {
    if (lat->z[c] < 1 || lat->z[c] >= lat->M) SS_FAIL(SS_ERR_INVALID, "lattice: z[%d] = %lld outside [1, M)", c, (long long)lat->z[c]);
    L->z[c] = lat->z[c];
  }
  return SS_OK;
}

ss_status residues(const int32_t* freq, int64_t n, const LatticeDev& L, int64_t* res, cudaStream_t st) {
  ProfScope prof_("k_residues", st);
  if (n == 0) return SS_OK;
  k_residues<<<nblk(n * 32), 256, 0, st>>>(freq, n, L.d, L, res);
  SS_LAUNCH_CHECK();
  return SS_OK;
}

ss_status check_reconstructing_async(const int32_t* freq, int64_t n, const LatticeDev& L, const int64_t* res,
                                     bool need_symmetric, unsigned long long* table, uint64_t cap, int32_t* flags,
                                     cudaStream_t st) {
  ProfScope prof_("lattice_check", st);
  SS_TRY(fill_small(st, {{table, cap * sizeof(unsigned long long), 0}, {flags, 4 * sizeof(int32_t), 0}}));
  if (n == 0) return SS_OK;
  k_check_insert<<<nblk(n), 256, 0, st>>>(freq, res, n, L.d, table, cap - 1, flags);
  if (need_symmetric) k_check_symmetric<<<nblk(n * 32), 256, 0, st>>>(freq, res, n, L.d, L.M, table, cap - 1, flags);
  SS_LAUNCH_CHECK();
  return SS_OK;
}

ss_status reconstructing_status(const int32_t* h, int64_t M) {
  if (h[0]) SS_FAIL(SS_ERR_INVALID, "lattice: duplicate frequencies in the candidate set");
  if (h[2]) SS_FAIL(SS_ERR_HASH_FULL, "lattice: residue table exhausted");
  if (h[1]) SS_FAIL(SS_ERR_NOT_RECONSTRUCTING, "lattice (M = %lld) is not reconstructing for the candidate set",
                    (long long)M);
  if (h[3]) SS_FAIL(SS_ERR_INVALID, "candidate set is not closed under negation");
  return SS_OK;
}

ss_status check_reconstructing(const int32_t* freq, int64_t n, const LatticeDev& L, const int64_t* res,
                               bool need_symmetric, cudaStream_t st) {
  if (n == 0) return SS_OK;
  uint64_t cap = 1;
  while (cap < (uint64_t)(2 * n)) cap <<= 1;
  DevBuf<unsigned long long> table;
  DevBuf<int32_t> flags;
  SS_TRY(table.alloc_tmp(cap, st));
  SS_TRY(flags.alloc_tmp(4, st));
  SS_TRY(fill_small(st, {{table.get(), cap * sizeof(unsigned long long), 0}, {flags.get(), 4 * sizeof(int32_t), 0}}));
  k_check_insert<<<nblk(n), 256, 0, st>>>(freq, res, n, L.d, table.get(), cap - 1, flags.get());
  if (need_symmetric)
    k_check_symmetric<<<nblk(n * 32), 256, 0, st>>>(freq, res, n, L.d, L.M, table.get(), cap - 1, flags.get());
  SS_LAUNCH_CHECK();
  int32_t h[4];
  SS_TRY(read_back(st, {{h, flags.get(), sizeof(h)}}));
  if (h[0]) SS_FAIL(SS_ERR_INVALID, "lattice: duplicate frequencies in the candidate set");
  if (h[2]) SS_FAIL(SS_ERR_HASH_FULL, "lattice: residue table exhausted");
  if (h[1]) SS_FAIL(SS_ERR_NOT_RECONSTRUCTING, "lattice (M = %lld) is not reconstructing for the candidate set",
                    (long long)L.M);
  if (h[3]) SS_FAIL(SS_ERR_INVALID, "candidate set is not closed under negation");
  return SS_OK;
}

static ss_status expansion_of(const int32_t* freq, int64_t n, int d, int64_t* K, cudaStream_t st) {
  DevBuf<int32_t> mm;
  SS_TRY(mm.alloc_tmp(2 * d, st));
  std::vector<int32_t> init(2 * d);
  for (int c = 0; c < d; ++c) { init[c] = INT32_MAX; init[d + c] = INT32_MIN; }
  SS_TRY(upload(st, {{mm.get(), init.data(), 2 * d * sizeof(int32_t)}}));
  if (n > 0) k_minmax<<<nblk(n * d), 256, 0, st>>>(freq, n, d, mm.get(), mm.get() + d);
  SS_LAUNCH_CHECK();
  SS_TRY(read_back(st, {{init.data(), mm.get(), 2 * d * sizeof(int32_t)}}));
  int64_t k = 0;
  for (int c = 0; c < d && n > 0; ++c) k = std::max<int64_t>(k, (int64_t)init[d + c] - init[c]);
  *K = k;
  return SS_OK;
}

}  // namespace ss

using namespace ss;

extern "C" ss_status lattice_size(int64_t K, int64_t n_I, double sigma, int64_t M_min, int64_t* M_out) {
  if (!M_out || !(sigma > 0.0) || sigma > 1.0 || K < 0 || n_I < 0)
    SS_FAIL(SS_ERR_INVALID, "lattice_size: need K >= 0, n_I >= 0, 0 < sigma <= 1");
  const double bound = std::max((double)K, (double)n_I * (double)n_I / sigma);
  if (bound >= 2147483000.0 || M_min >= 2147483000ll) SS_FAIL(SS_ERR_INVALID, "lattice_size: M would exceed 2^31");
  const int64_t lo = (int64_t)std::floor(bound) + 1;
  *M_out = next_prime_host(std::max<int64_t>(lo, M_min));
  return SS_OK;
}

extern "C" ss_status lattice_check(const ss_lattice* lat, const int32_t* freq, int64_t n, void* stream) {
  LatticeDev L;
  SS_TRY(make_lattice_dev(lat, &L));
  if (n > 0 && !freq) SS_FAIL(SS_ERR_INVALID, "lattice_check: null frequencies");
  cudaStream_t st = as_stream(stream);
  DevBuf<int64_t> res;
  SS_TRY(res.alloc_tmp(n, st));
  SS_TRY(residues(freq, n, L, res.get(), st));
  return check_reconstructing(freq, n, L, res.get(), false, st);
}

namespace ss {
namespace {

// The first of `attempts` draws z_c = 1 + raw[a][c] mod (M - 1) that is
// reconstructing for freq (exact check).
ss_status random_draws(const int32_t* freq, int64_t n, int32_t d, int64_t M, const int64_t* raw, int32_t attempts,
                       int64_t* z_out, int32_t* attempt_out, cudaStream_t st) {
  DevBuf<int64_t> res;
  SS_TRY(res.alloc_tmp(n, st));
  std::vector<int64_t> z(d);
  for (int a = 0; a < attempts; ++a) {
    for (int c = 0; c < d; ++c) {
      const int64_t r = raw[(int64_t)a * d + c];
      if (r < 0) SS_FAIL(SS_ERR_INVALID, "lattice_random: raw draws must be non-negative");
      z[c] = 1 + r % (M - 1);
    }
    ss_lattice lat{d, M, z.data()};
    LatticeDev L;
    SS_TRY(make_lattice_dev(&lat, &L));
    SS_TRY(residues(freq, n, L, res.get(), st));
    ss_status s = check_reconstructing(freq, n, L, res.get(), false, st);
    if (s == SS_OK) {
      for (int c = 0; c < d; ++c) z_out[c] = z[c];
      if (attempt_out) *attempt_out = a;
      return SS_OK;
    }
    if (s != SS_ERR_NOT_RECONSTRUCTING) return s;
  }
  SS_FAIL(SS_ERR_NOT_RECONSTRUCTING, "lattice_random: no reconstructing draw among %d attempts (M = %lld)", attempts,
          (long long)M);
}

}  // namespace
}  // namespace ss

extern "C" ss_status lattice_random(const int32_t* freq, int64_t n, int32_t d, double sigma, int64_t M_min,
                                    const int64_t* raw, int32_t attempts, int64_t* z_out, int64_t* M_out,
                                    int32_t* attempt_out, void* stream) {
  if (!freq || !raw || !z_out || !M_out || d < 1 || d > kMaxLatticeDim || attempts < 1)
    SS_FAIL(SS_ERR_INVALID, "lattice_random: bad argument");
  cudaStream_t st = as_stream(stream);
  int64_t K = 0, M = 0;
  SS_TRY(expansion_of(freq, n, d, &K, st));
  SS_TRY(lattice_size(K, n, sigma, M_min, &M));
  SS_TRY(random_draws(freq, n, d, M, raw, attempts, z_out, attempt_out, st));
  *M_out = M;
  return SS_OK;
}

extern "C" ss_status lattice_random_smooth(const int32_t* freq, int64_t n, int32_t d, double sigma, int64_t M_min,
                                           const int64_t* raw, int32_t attempts, int64_t* z_out, int64_t* M_out,
                                           int32_t* attempt_out, void* stream) {
  if (!freq || !raw || !z_out || !M_out || d < 1 || d > kMaxLatticeDim || attempts < 1 || !(sigma > 0.0) ||
      sigma >= 1.0)
    SS_FAIL(SS_ERR_INVALID, "lattice_random_smooth: bad argument");
  cudaStream_t st = as_stream(stream);
  int64_t K = 0;
  SS_TRY(expansion_of(freq, n, d, &K, st));
  const double bound = std::max({(double)K + 1.0, std::ceil((double)n * (double)n / sigma), (double)M_min, 2.0});
  if (bound >= 2147483647.0) SS_FAIL(SS_ERR_INVALID, "lattice_random_smooth: M would exceed 2^31");
  const int64_t M = next_smooth_host((int64_t)bound);
  SS_TRY(random_draws(freq, n, d, M, raw, attempts, z_out, attempt_out, st));
  *M_out = M;
  return SS_OK;
}

extern "C" ss_status lattice_cbc(const int32_t* freq, int64_t n, int32_t d, int64_t M_min, const int64_t* raw,
                                 int32_t n_cand, int64_t* z_out, int64_t* M_out, void* stream) {
  if (!freq || !raw || !z_out || !M_out || d < 1 || d > kMaxLatticeDim || n_cand < 1 || n < 1)
    SS_FAIL(SS_ERR_INVALID, "lattice_cbc: bad argument");
  cudaStream_t st = as_stream(stream);
  int64_t K = 0;
  SS_TRY(expansion_of(freq, n, d, &K, st));
  if (std::max<int64_t>(M_min, K + 1) >= 2147483000ll) SS_FAIL(SS_ERR_INVALID, "lattice_cbc: M would exceed 2^31");
  // the CBC check is exact and needs no prime: take an FFT-friendly length
  const int64_t M = next_smooth_host(std::max<int64_t>(M_min, K + 1));
  // the candidate set must be free of duplicates (checked on the full vectors)
  {
    std::vector<int64_t> one(d, 1);
    ss_lattice lat{d, M, one.data()};
    LatticeDev L;
    SS_TRY(make_lattice_dev(&lat, &L));
  }
  DevBuf<int64_t> rho, cand, scratch, zdev;
  DevBuf<int32_t> fail, err;
  SS_TRY(rho.alloc_tmp(n, st));
  SS_TRY(cand.alloc_tmp((size_t)d * n_cand, st));
  SS_TRY(fail.alloc_tmp(n_cand, st));
  SS_TRY(zdev.alloc_tmp(d, st));
  SS_TRY(err.alloc_tmp(1, st));
  int hash_cap = 1;
  while (hash_cap < 2 * n) hash_cap <<= 1;
  const size_t hash_smem = (size_t)n * sizeof(int64_t) + (size_t)hash_cap * sizeof(int32_t);
  if (hash_smem <= 200 * 1024) {
    if (hash_smem > 48 * 1024)
      SS_CUDA(cudaFuncSetAttribute(k_cbc_try_hash, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hash_smem));
    SS_TRY(scratch.alloc_tmp(1, st));
  } else {
    SS_TRY(scratch.alloc_tmp((size_t)n_cand * n, st));
  }
  // all candidates up front; each coordinate's pick stays on the device
  std::vector<int64_t> hc((size_t)d * n_cand, 1), z(d, 1);
  for (int j = 1; j < d; ++j)
    for (int c = 0; c < n_cand; ++c) {
      const int64_t r = raw[(int64_t)j * n_cand + c];
      if (r < 0) SS_FAIL(SS_ERR_INVALID, "lattice_cbc: raw draws must be non-negative");
      hc[(size_t)j * n_cand + c] = 1 + r % (M - 1);
    }
  SS_TRY(upload(st, {{cand.get(), hc.data(), hc.size() * sizeof(int64_t)}}));
  SS_TRY(fill_small(st, {{rho.get(), n * sizeof(int64_t), 0}, {err.get(), sizeof(int32_t), 0}}));
  // one cooperative launch for all coordinates when the per-block tables fit
  // in shared memory and every candidate's block can be resident at once
  const size_t all_smem = 2 * (size_t)n * sizeof(int64_t) + (size_t)hash_cap * sizeof(int32_t);
  int per_sm = 0;
  bool fused = all_smem <= 200 * 1024 && d > 1;
  if (fused) {
    SS_CUDA(cudaFuncSetAttribute(k_cbc_all, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)all_smem));
    SS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cbc_all, kCbcThreads, all_smem));
    fused = (int64_t)per_sm * sm_count() >= n_cand;
  }
  if (fused) {
    DevBuf<int32_t> fails;
    DevBuf<unsigned> arrive;
    DevBuf<int32_t> err2;
    SS_TRY(fails.alloc_tmp((size_t)d * n_cand, st));
    SS_TRY(arrive.alloc_tmp(d, st));
    SS_TRY(err2.alloc_tmp(2, st));
    SS_TRY(fill_small(st, {{arrive.get(), d * sizeof(unsigned), 0}, {err2.get(), 2 * sizeof(int32_t), 0}}));
    const int32_t* fa = freq;
    int64_t na = n;
    int da = d;
    int64_t Ma = M;
    const int64_t* ca = cand.get();
    int nc = n_cand, hc = hash_cap;
    int32_t* fp = fails.get();
    unsigned* ap = arrive.get();
    int64_t* zp = zdev.get();
    int32_t* ep = err2.get();
    void* args[] = {&fa, &na, &da, &Ma, &ca, &nc, &hc, &fp, &ap, &zp, &ep};
    SS_CUDA(cudaLaunchCooperativeKernel((void*)k_cbc_all, dim3(n_cand), dim3(kCbcThreads), args, all_smem, st));
    SS_LAUNCH_CHECK();
    int32_t herr2[2] = {0, 0};
    SS_TRY(read_back(st, {{z.data(), zdev.get(), d * sizeof(int64_t)}, {herr2, err2.get(), sizeof(herr2)}}));
    if (herr2[1]) SS_FAIL((ss_status)herr2[1], "lattice_cbc: a block of the search timed out waiting for the others");
    if (herr2[0]) SS_FAIL(SS_ERR_NOT_RECONSTRUCTING, "lattice_cbc: no candidate for coordinate %d", herr2[0]);
    for (int c = 0; c < d; ++c) z_out[c] = z[c];
    *M_out = M;
    return SS_OK;
  }
  // coordinate 0: z_1 = 1 (distinct first coordinates have distinct residues since M > K)
  SS_CUDA(cudaMemcpyAsync(zdev.get(), z.data(), sizeof(int64_t), cudaMemcpyHostToDevice, st));
  k_cbc_accept<<<nblk(n), 256, 0, st>>>(freq, n, d, 0, M, zdev.get(), rho.get());
  SS_LAUNCH_CHECK();
  for (int j = 1; j < d; ++j) {
    const int64_t* cj = cand.get() + (size_t)j * n_cand;
    if (hash_smem <= 200 * 1024) {
      k_cbc_try_hash<<<n_cand, 256, hash_smem, st>>>(freq, n, d, j, M, rho.get(), cj, hash_cap, fail.get());
    } else {
      k_cbc_try<<<n_cand, 256, 0, st>>>(freq, n, d, j, M, rho.get(), cj, scratch.get(), fail.get());
    }
    k_cbc_pick<<<1, 32, 0, st>>>(fail.get(), cj, n_cand, j, zdev.get(), err.get());
    k_cbc_accept<<<nblk(n), 256, 0, st>>>(freq, n, d, j, M, zdev.get(), rho.get());
    SS_LAUNCH_CHECK();
  }
  int32_t herr = 0;
  SS_TRY(read_back(st, {{z.data(), zdev.get(), d * sizeof(int64_t)}, {&herr, err.get(), sizeof(int32_t)}}));
  if (herr) SS_FAIL(SS_ERR_NOT_RECONSTRUCTING, "lattice_cbc: no candidate for coordinate %d", herr);
  for (int c = 0; c < d; ++c) z_out[c] = z[c];
  *M_out = M;
  return SS_OK;
}
