// Single-pass prefix sums with decoupled look-back.  Every block scans one
// tile of kLbTile values, publishes the tile's sum, then adds the sums of the
// tiles before it (read newest first, until one that already carries its
// inclusive prefix) and publishes its own inclusive prefix.  Blocks take tiles
// in the order they start (an atomic ticket), so every tile a block waits for
// belongs to a block that has started and publishes its sum before it waits
// itself: the waits end.  Each wait is still bounded by wait_ns of the global
// timer; past it the block records SS_ERR_TIMEOUT in *err (when given) and
// goes on with a zero prefix.
//
// The values come from a functor in(c) (non-negative int32 for c < n), the
// results go to out(c, value, exclusive prefix), so a producer and a consumer
// (flags computed on the fly, a compaction) fuse into the one pass.
#pragma once

#include "ss_internal.cuh"

namespace ss {

constexpr int kLbThreads = 256;
constexpr int kLbItems = 8;
constexpr int kLbTile = kLbThreads * kLbItems;

// Status word of a tile: [63:62] 0 nothing yet, 1 tile sum, 2 inclusive
// prefix; [61:0] the value.
constexpr uint64_t kLbSum = 1ull << 62;
constexpr uint64_t kLbIncl = 2ull << 62;
constexpr uint64_t kLbValue = (1ull << 62) - 1;
constexpr long long kLbWaitNs = 2000000000ll;

struct LbScratch {
  uint32_t* ticket;   // zero before the launch
  uint64_t* status;   // [tiles], zero before the launch
  int32_t* err;       // nullable
  long long wait_ns;
};

__device__ __forceinline__ uint64_t lb_load(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void lb_store(uint64_t* p, uint64_t v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ long long lb_timer() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

template <class In, class Out>
__global__ void __launch_bounds__(kLbThreads) k_scan_lookback(In in, Out out, int64_t n, int64_t tiles,
                                                              LbScratch sc, int64_t* d_total) {
  __shared__ uint32_t s_tile;
  __shared__ int64_t s_prefix;
  __shared__ int64_t s_warp[kLbThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_tile = atomicAdd(sc.ticket, 1u);
  __syncthreads();
  const int64_t t = s_tile;
  const int64_t base = t * kLbTile + (int64_t)threadIdx.x * kLbItems;
  int32_t v[kLbItems];
  int64_t s = 0;
#pragma unroll
  for (int q = 0; q < kLbItems; ++q) {
    v[q] = base + q < n ? in(base + q) : 0;
    s += v[q];
  }
  // block-wide inclusive scan of the per-thread sums
  int64_t x = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[warp] = x;
  __syncthreads();
  int64_t before = 0, agg = 0;
#pragma unroll
  for (int w = 0; w < kLbThreads / 32; ++w) {
    if (w < warp) before += s_warp[w];
    agg += s_warp[w];
  }
  if (warp == 0) {
    if (t == 0) {
      if (lane == 0) {
        lb_store(sc.status, kLbIncl | (uint64_t)agg);
        s_prefix = 0;
      }
    } else {
      if (lane == 0) lb_store(sc.status + t, kLbSum | (uint64_t)agg);
      int64_t excl = 0;
      for (int64_t top = t - 1;; top -= 32) {
        const int64_t q = top - lane;
        uint64_t w = q >= 0 ? lb_load(sc.status + q) : kLbIncl;   // before tile 0: prefix 0
        if ((w >> 62) == 0) {
          const long long t0 = lb_timer();
          for (unsigned it = 1; (w >> 62) == 0; ++it) {
            if ((it & 63u) == 0 && lb_timer() - t0 > sc.wait_ns) {
              if (sc.err) atomicCAS(sc.err, 0, (int)SS_ERR_TIMEOUT);
              w = kLbIncl;
              break;
            }
            w = lb_load(sc.status + q);
          }
        }
        const unsigned incl = __ballot_sync(0xffffffffu, (w >> 62) == 2);
        const int stop = incl ? __ffs(incl) - 1 : 31;
        int64_t part = lane <= stop ? (int64_t)(w & kLbValue) : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        excl += part;
        if (incl) break;
      }
      if (lane == 0) {
        lb_store(sc.status + t, kLbIncl | (uint64_t)(excl + agg));
        s_prefix = excl;
      }
    }
  }
  __syncthreads();
  int64_t run = s_prefix + before + x - s;
#pragma unroll
  for (int q = 0; q < kLbItems; ++q) {
    if (base + q < n) out(base + q, v[q], run);
    run += v[q];
  }
  if (t == tiles - 1 && threadIdx.x == 0 && d_total) *d_total = s_prefix + agg;
}

// One pass over n values (asynchronous on st); the total into *d_total
// (device, nullable), a wait that gave up into *err (device, nullable).
template <class In, class Out>
ss_status scan_lookback(In in, Out out, int64_t n, int64_t* d_total, int32_t* err, cudaStream_t st) {
  if (n <= 0) {
    if (d_total) SS_CUDA(cudaMemsetAsync(d_total, 0, sizeof(int64_t), st));
    return SS_OK;
  }
  const int64_t tiles = (n + kLbTile - 1) / kLbTile;
  if (tiles >= ((int64_t)1 << 31)) SS_FAIL(SS_ERR_INVALID, "scan: %lld values are too many", (long long)n);
  DevBuf<uint64_t> buf;   // [0]: ticket, [1 ..]: tile status
  SS_TRY(buf.alloc_tmp(tiles + 1, st));
  SS_CUDA(cudaMemsetAsync(buf.get(), 0, (tiles + 1) * sizeof(uint64_t), st));
  const LbScratch sc{reinterpret_cast<uint32_t*>(buf.get()), buf.get() + 1, err, kLbWaitNs};
  k_scan_lookback<<<(unsigned)tiles, kLbThreads, 0, st>>>(in, out, n, tiles, sc, d_total);
  SS_LAUNCH_CHECK();
  return SS_OK;
}

// Plain exclusive prefix sum of int32 values (out may alias in).
struct LbRead {
  const int32_t* p;
  __device__ int32_t operator()(int64_t c) const { return p[c]; }
};
struct LbWrite {
  int32_t* p;
  __device__ void operator()(int64_t c, int32_t, int64_t excl) const { p[c] = (int32_t)excl; }
};

}  // namespace ss
