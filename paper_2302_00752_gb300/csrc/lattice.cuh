// Rank-1 lattice parameters on the device and exact residues k.z mod M.
#pragma once

#include "ss_internal.cuh"

namespace ss {

constexpr int kMaxLatticeDim = 1024;

struct LatticeDev {
  int d;
  int64_t M;
  int64_t z[kMaxLatticeDim];
};

// (k.z) mod M in [0, M), exact: each product (k_c mod M) z_c < 2^62 is
// reduced by mulmod (Barrett), and the d reduced terms (each < M < 2^31) are
// summed without reduction (below 2^41 for d <= 1024) and reduced once.
__device__ __forceinline__ int64_t residue_of(const int32_t* k, int d, const LatticeDev& L) {
  const uint64_t M = (uint64_t)L.M, inv = ~0ull / M;
  uint64_t acc = 0;
  for (int c = 0; c < d; ++c) {
    int64_t kc = k[c];
    if (kc < 0 || kc >= L.M) {
      kc %= L.M;
      if (kc < 0) kc += L.M;
    }
    acc += mulmod((uint64_t)kc, (uint64_t)L.z[c], M, inv);
  }
  return (int64_t)(acc % M);
}

// The same residue by one warp (every lane gets it): lane l takes the
// coordinates c = l, l + 32, ... (coalesced reads of k and z), the partial
// sums are reduced mod M as they grow and combined in a fixed butterfly.
// Call with the whole warp.
__device__ __forceinline__ int64_t residue_warp(const int32_t* k, int d, const LatticeDev& L) {
  const uint64_t M = (uint64_t)L.M, inv = ~0ull / M;
  uint64_t acc = 0;
  for (int c = (int)(threadIdx.x & 31); c < d; c += 32) {
    int64_t kc = k[c];
    if (kc < 0 || kc >= L.M) {
      kc %= L.M;
      if (kc < 0) kc += L.M;
    }
    acc += mulmod((uint64_t)kc, (uint64_t)L.z[c], M, inv);
    if (acc >= M) acc -= M;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (acc >= M) acc -= M;
  }
  return (int64_t)acc;
}

ss_status make_lattice_dev(const ss_lattice* lat, LatticeDev* L);
ss_status residues(const int32_t* freq, int64_t n, const LatticeDev& L, int64_t* res, cudaStream_t st);
ss_status check_reconstructing(const int32_t* freq, int64_t n, const LatticeDev& L, const int64_t* res,
                               bool need_symmetric, cudaStream_t st);
// Same check left on the device: flags[0] duplicate, [1] collision, [2] table
// full, [3] not closed under negation; reconstructing_status decodes them.
ss_status check_reconstructing_async(const int32_t* freq, int64_t n, const LatticeDev& L, const int64_t* res,
                                     bool need_symmetric, unsigned long long* table, uint64_t cap, int32_t* flags,
                                     cudaStream_t st);
ss_status reconstructing_status(const int32_t* h, int64_t M);
int64_t next_prime_host(int64_t n);

}  // namespace ss
