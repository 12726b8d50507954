// Library-wide helpers behind the C ABI: per-thread error text, version,
// device properties.
#include <vector>
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

struct ScratchBlock {
  size_t off, bytes;
  bool live;
};

struct Scratch {
  unsigned char* base = nullptr;
  size_t cap = 0, top = 0, want = 0;
  int64_t spill = 0;
  int dev = -1;
  cudaStream_t st = nullptr;
  cudaEvent_t ev = nullptr;
  std::vector<ScratchBlock> blocks;
};

Scratch& scratch() {
  thread_local Scratch S;
  return S;
}

}  // namespace

void scratch_spill(int64_t bytes) { scratch().spill += bytes; }

void* scratch_take(size_t bytes, cudaStream_t st) {
  Scratch& A = scratch();
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  bytes = (bytes + 255) & ~(size_t)255;
  const size_t need = A.top + bytes + (size_t)(A.spill > 0 ? A.spill : 0);
  if (need > A.want) A.want = need < kScratchMaxCap ? need : kScratchMaxCap;
  if (A.blocks.empty()) {
    if (A.base && (A.dev != dev || A.want > A.cap)) {
      cudaFreeAsync(A.base, A.st);   // after the work queued on the stream that used it
      A.base = nullptr;
      A.cap = 0;
    }
    if (!A.base && A.want > 0) {
      retain_pool();
      const size_t cap = std::min(A.want + A.want / 4, kScratchMaxCap);
      if (cudaMallocAsync(reinterpret_cast<void**>(&A.base), cap, st) != cudaSuccess) {
        cudaGetLastError();
        A.base = nullptr;
        return nullptr;
      }
      A.cap = cap;
      A.dev = dev;
      A.st = st;
    }
    if (A.base && st != A.st) {
      // the new stream waits for the old stream's use of the block
      if (!A.ev && cudaEventCreateWithFlags(&A.ev, cudaEventDisableTiming) != cudaSuccess) return nullptr;
      if (cudaEventRecord(A.ev, A.st) != cudaSuccess || cudaStreamWaitEvent(st, A.ev, 0) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
      }
      A.st = st;
    }
  }
  if (!A.base || A.dev != dev || st != A.st || A.top + bytes > A.cap) return nullptr;
  A.blocks.push_back(ScratchBlock{A.top, bytes, true});
  A.top += bytes;
  return A.base + A.blocks.back().off;
}

void scratch_give(void* p) {
  Scratch& A = scratch();
  const size_t off = static_cast<unsigned char*>(p) - A.base;
  for (auto it = A.blocks.rbegin(); it != A.blocks.rend(); ++it)
    if (it->off == off && it->live) {
      it->live = false;
      break;
    }
  while (!A.blocks.empty() && !A.blocks.back().live) {
    A.top = A.blocks.back().off;
    A.blocks.pop_back();
  }
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
