// Device-wide exclusive prefix sum of int32 values (used to compact the new
// frontier of each stamping level and to lay out neighbour-table slices).
#include "ss_internal.cuh"

namespace ss {
namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kTile = kScanThreads * kScanItems;

__device__ __forceinline__ int32_t block_exclusive_scan(int32_t v, int32_t* total) {
  __shared__ int32_t warp_sum[kScanThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sum[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int32_t w = (lane < kScanThreads / 32) ? warp_sum[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < kScanThreads / 32) warp_sum[lane] = w;   // inclusive over warps
  }
  __syncthreads();
  int32_t before = (warp > 0) ? warp_sum[warp - 1] : 0;
  *total = warp_sum[kScanThreads / 32 - 1];
  __syncthreads();
  return before + x - v;
}

// Scans one tile per block; writes the tile's total to tile_sum[block] (or to
// *d_total when there is a single tile).
__global__ void k_scan_tiles(const int32_t* __restrict__ in, int32_t* out, int64_t n, int32_t* tile_sum,
                             int64_t* d_total) {
  const int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kScanItems;
  int32_t v[kScanItems];
  int32_t s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    v[i] = (base + i < n) ? in[base + i] : 0;
    s += v[i];
  }
  int32_t tot;
  int32_t run = block_exclusive_scan(s, &tot);
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    if (base + i < n) out[base + i] = run;
    run += v[i];
  }
  if (threadIdx.x == 0) {
    if (tile_sum) tile_sum[blockIdx.x] = tot;
    if (d_total) *d_total = tot;
  }
}

__global__ void k_add_tile_offsets(int32_t* out, int64_t n, const int32_t* __restrict__ tile_off) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] += tile_off[i / kTile];
}

// One block per tile t: adds the sum of the totals of tiles 0..t-1 (summed by
// the block itself, O(t) reads) to the tile's outputs; the last tile also
// writes the grand total.  Replaces a scan of the tile totals plus an offset
// pass when the tiles are few.
constexpr int64_t kPrefixTiles = 16384;
__global__ void __launch_bounds__(kScanThreads) k_add_tile_prefix(int32_t* out, int64_t n,
                                                                  const int32_t* __restrict__ tile_sum,
                                                                  int64_t tiles, int64_t* d_total) {
  __shared__ int32_t warp_sum[kScanThreads / 32];
  const int64_t t = blockIdx.x;
  int32_t acc = 0;
  for (int64_t j = threadIdx.x; j < t; j += kScanThreads) acc += tile_sum[j];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) warp_sum[threadIdx.x >> 5] = acc;
  __syncthreads();
  int32_t off = 0;
#pragma unroll
  for (int w = 0; w < kScanThreads / 32; ++w) off += warp_sum[w];
  const int64_t base = t * kTile;
  for (int i = threadIdx.x; i < kTile && base + i < n; i += kScanThreads) out[base + i] += off;
  if (t == tiles - 1 && threadIdx.x == 0 && d_total) *d_total = (int64_t)off + tile_sum[t];
}

}  // namespace

ss_status exclusive_scan_i32(const int32_t* in, int32_t* out, int64_t n, int64_t* d_total, cudaStream_t st) {
  ProfScope prof_("scan", st);
  if (n <= 0) {
    if (d_total) SS_CUDA(cudaMemsetAsync(d_total, 0, sizeof(int64_t), st));
    return SS_OK;
  }
  const int64_t tiles = (n + kTile - 1) / kTile;
  if (tiles == 1) {
    k_scan_tiles<<<1, kScanThreads, 0, st>>>(in, out, n, nullptr, d_total);
    SS_LAUNCH_CHECK();
    return SS_OK;
  }
  if (tiles <= kPrefixTiles) {
    DevBuf<int32_t> tsum;
    SS_TRY(tsum.alloc_tmp(tiles, st));
    k_scan_tiles<<<(unsigned)tiles, kScanThreads, 0, st>>>(in, out, n, tsum.get(), nullptr);
    k_add_tile_prefix<<<(unsigned)tiles, kScanThreads, 0, st>>>(out, n, tsum.get(), tiles, d_total);
    SS_LAUNCH_CHECK();
    return SS_OK;
  }
  int32_t* sums = nullptr;
  note_alloc();
  SS_CUDA(cudaMallocAsync(&sums, tiles * sizeof(int32_t), st));
  k_scan_tiles<<<(unsigned)tiles, kScanThreads, 0, st>>>(in, out, n, sums, nullptr);
  ss_status s = SS_OK;
  if (cudaGetLastError() != cudaSuccess) s = SS_ERR_CUDA;
  if (s == SS_OK) s = exclusive_scan_i32(sums, sums, tiles, d_total, st);
  if (s == SS_OK) {
    k_add_tile_offsets<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(out, n, sums);
    if (cudaGetLastError() != cudaSuccess) s = SS_ERR_CUDA;
  }
  cudaFreeAsync(sums, st);
  if (s == SS_ERR_CUDA) set_error("scan kernel launch failed");
  return s;
}

}  // namespace ss
