// Microbenchmarks of the rates that bound this library's kernels on the GPU
// they run on (the roofline denominators the copy and GEMM peaks do not
// cover): FP64 and FP32 fused multiply-add throughput, and random gathers of
// 4- to 32-byte records from an L2-resident working set and from HBM.
// Built as a separate library (libss_peaks.so) used by the benchmark only.
//
// Each entry point runs one warm-up launch and then `reps` timed launches
// between CUDA events on the default stream, and returns the best rate.
#include <cuda_runtime.h>

#include <cstdint>

namespace {

constexpr int kChains = 8;   // independent FMA chains per thread

template <typename T>
__global__ void __launch_bounds__(1024) k_fma(T* out, int iters, T a, T b) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-6;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == (T)-1.2345) out[blockIdx.x] = s;   // never true; keeps the chains live
}

// Random gathers of R-byte records (R = 4, 8, 16 or 32) over n_rec records
// (a power of two): per thread a 32-bit LCG picks the record of each step;
// loads bypass L1 (ld.global.cg) so that every request goes to L2.  Eight
// gathers are issued before their values are used (iters: a multiple of 8).
template <int R>
__device__ __forceinline__ uint32_t gather1(const uint4* __restrict__ data, uint32_t idx) {
  if constexpr (R == 4) {
    return __ldcg(reinterpret_cast<const uint32_t*>(data) + idx);
  } else if constexpr (R == 8) {
    const uint2 v = __ldcg(reinterpret_cast<const uint2*>(data) + idx);
    return v.x ^ v.y;
  } else if constexpr (R == 16) {
    const uint4 v = __ldcg(data + idx);
    return v.x ^ v.y ^ v.z ^ v.w;
  } else {
    const uint4 v0 = __ldcg(data + 2 * (size_t)idx), v1 = __ldcg(data + 2 * (size_t)idx + 1);
    return v0.x ^ v0.y ^ v0.z ^ v0.w ^ v1.x ^ v1.y ^ v1.z ^ v1.w;
  }
}

template <int R>
__global__ void __launch_bounds__(256) k_gather(const uint4* __restrict__ data, uint32_t shift, int iters,
                                                 uint32_t* out) {
  uint32_t h = 0x9e3779b9u * (blockIdx.x * blockDim.x + threadIdx.x + 1);
  uint32_t acc = 0;
  for (int i = 0; i < iters; i += 8) {
    uint32_t v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      h = h * 1664525u + 1013904223u;
      v[u] = gather1<R>(data, h >> shift);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) acc ^= v[u];
  }
  if (acc == 0x12345679u) out[0] = acc;
}

int sms() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n;
}

template <typename F>
double best_ms(F launch, int reps) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  launch();   // warm-up
  double best = 1e30;
  for (int r = 0; r < reps; ++r) {
    cudaEventRecord(e0);
    launch();
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return best;
}

template <typename T>
int fma_rate(int reps, double* tflops) {
  T* out = nullptr;
  const int blocks = 4 * sms(), threads = 1024, iters = sizeof(T) == 8 ? 2048 : 65536;
  if (cudaMalloc(&out, blocks * sizeof(T)) != cudaSuccess) return 1;
  const double ms = best_ms([&] { k_fma<T><<<blocks, threads>>>(out, iters, (T)0.999999, (T)1e-7); }, reps);
  const cudaError_t e = cudaGetLastError();
  cudaFree(out);
  if (e != cudaSuccess) return 2;
  *tflops = 2.0 * kChains * (double)iters * blocks * threads / (ms * 1e-3) / 1e12;
  return 0;
}

}  // namespace

// FP64 and FP32 FMA throughput in TFLOP/s (2 flops per FMA).  0 on success.
extern "C" int peak_fma(int reps, double* fp64_tflops, double* fp32_tflops) {
  int r = fma_rate<double>(reps, fp64_tflops);
  if (r) return r;
  return fma_rate<float>(reps, fp32_tflops);
}

// Random gathers of rec_bytes-byte records (4, 8, 16 or 32) from a working set
// of ws_bytes (rounded down to a power-of-two record count).  Writes the useful
// bytes moved per second (GB/s) and the records per second (G/s).  0 on success.
extern "C" int peak_gather(int rec_bytes, int64_t ws_bytes, int reps, double* gbs, double* grecs) {
  if (rec_bytes != 4 && rec_bytes != 8 && rec_bytes != 16 && rec_bytes != 32) return 1;
  int bits = 0;
  while (((int64_t)rec_bytes << (bits + 1)) <= ws_bytes && bits < 31) ++bits;
  if (bits < 1) return 1;
  const int64_t n_rec = (int64_t)1 << bits;
  void* data = nullptr;
  uint32_t* out = nullptr;
  if (cudaMalloc(&data, n_rec * rec_bytes) != cudaSuccess) return 2;
  if (cudaMalloc(&out, sizeof(uint32_t)) != cudaSuccess) {
    cudaFree(data);
    return 2;
  }
  cudaMemset(data, 0x5a, n_rec * rec_bytes);
  const int blocks = 16 * sms(), threads = 256, iters = 256;
  const uint32_t shift = 32u - (uint32_t)bits;
  const uint4* d4 = static_cast<const uint4*>(data);
  auto launch = [&] {
    switch (rec_bytes) {
      case 4: k_gather<4><<<blocks, threads>>>(d4, shift, iters, out); break;
      case 8: k_gather<8><<<blocks, threads>>>(d4, shift, iters, out); break;
      case 16: k_gather<16><<<blocks, threads>>>(d4, shift, iters, out); break;
      default: k_gather<32><<<blocks, threads>>>(d4, shift, iters, out); break;
    }
  };
  const double ms = best_ms(launch, reps);
  const cudaError_t e = cudaGetLastError();
  cudaFree(data);
  cudaFree(out);
  if (e != cudaSuccess) return 3;
  const double recs = (double)blocks * threads * iters;
  *grecs = recs / (ms * 1e-3) / 1e9;
  *gbs = recs * rec_bytes / (ms * 1e-3) / 1e9;
  return 0;
}
