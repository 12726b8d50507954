// Library-wide helpers behind the C ABI: per-thread error text, version,
// device properties.
#include <algorithm>
#include <cstdarg>

#include "ss_internal.cuh"

namespace ss {

static thread_local char g_err[1024] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

void retain_pool() {
  static thread_local int done_dev = -1;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev == done_dev) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t thr = ~0ull;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  done_dev = dev;
}

namespace {

struct PinnedBlock {
  void* p = nullptr;
  size_t n = 0;
  ~PinnedBlock() {
    if (p) cudaFreeHost(p);
  }
};

thread_local PinnedBlock g_pinned;

struct UploadBlock {
  void* p = nullptr;
  size_t n = 0;
  cudaEvent_t done = nullptr;   // recorded after the last copy out of the block
  ~UploadBlock() {
    if (done) cudaEventDestroy(done);
    if (p) cudaFreeHost(p);
  }
};

thread_local UploadBlock g_up;

}  // namespace

ss_status upload(cudaStream_t st, std::initializer_list<HostWrite> parts) {
  size_t total = 0;
  for (const HostWrite& w : parts) total += (w.bytes + 15) / 16 * 16;
  if (!g_up.done) SS_CUDA(cudaEventCreateWithFlags(&g_up.done, cudaEventDisableTiming));
  // the copies queued from the block last time must have run before it is refilled
  SS_CUDA(cudaEventSynchronize(g_up.done));
  if (total > g_up.n) {
    if (g_up.p) {
      cudaFreeHost(g_up.p);
      g_up.p = nullptr;
      g_up.n = 0;
    }
    const size_t n = std::max<size_t>(total, 64 * 1024);
    SS_CUDA(cudaMallocHost(&g_up.p, n));
    g_up.n = n;
  }
  char* base = static_cast<char*>(g_up.p);
  size_t off = 0;
  for (const HostWrite& w : parts) {
    if (w.bytes) {
      std::memcpy(base + off, w.src, w.bytes);
      SS_CUDA(cudaMemcpyAsync(w.dst, base + off, w.bytes, cudaMemcpyHostToDevice, st));
    }
    off += (w.bytes + 15) / 16 * 16;
  }
  SS_CUDA(cudaEventRecord(g_up.done, st));
  return SS_OK;
}

ss_status read_back(cudaStream_t st, std::initializer_list<HostRead> parts) {
  size_t total = 0;
  for (const HostRead& r : parts) total += (r.bytes + 15) / 16 * 16;
  if (total > g_pinned.n) {
    if (g_pinned.p) {
      cudaFreeHost(g_pinned.p);
      g_pinned.p = nullptr;
      g_pinned.n = 0;
    }
    const size_t n = std::max<size_t>(total, 64 * 1024);
    SS_CUDA(cudaMallocHost(&g_pinned.p, n));
    g_pinned.n = n;
  }
  char* base = static_cast<char*>(g_pinned.p);
  size_t off = 0;
  for (const HostRead& r : parts) {
    if (r.bytes) SS_CUDA(cudaMemcpyAsync(base + off, r.src, r.bytes, cudaMemcpyDeviceToHost, st));
    off += (r.bytes + 15) / 16 * 16;
  }
  SS_CUDA(cudaStreamSynchronize(st));
  off = 0;
  for (const HostRead& r : parts) {
    if (r.bytes) std::memcpy(r.dst, base + off, r.bytes);
    off += (r.bytes + 15) / 16 * 16;
  }
  return SS_OK;
}

int sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
  return n > 0 ? n : 1;
}

}  // namespace ss

extern "C" const char* ss_last_error(void) { return ss::g_err; }

extern "C" const char* ss_version(void) { return "sparse-spectral-gb300 0.1 (sm_103a)"; }
