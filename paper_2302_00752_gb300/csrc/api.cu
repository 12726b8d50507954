// Library-wide helpers behind the C ABI: per-thread error text, version,
// device properties.
#include <atomic>
#include <map>
#include <mutex>
#include <string>
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
      note_alloc();
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
  void* dev = nullptr;   // the block's device-side address (mapped)
  ~PinnedBlock() {
    if (p) cudaFreeHost(p);
  }
};

thread_local PinnedBlock g_pinned;

constexpr int kGatherParts = 8;
constexpr size_t kGatherBytes = 4096;

struct GatherArgs {
  const unsigned char* src[kGatherParts];
  uint32_t bytes[kGatherParts];
  uint32_t off[kGatherParts];
  int n;
};

struct FillArgs {
  unsigned char* dst[kGatherParts];
  size_t bytes[kGatherParts];
  unsigned char value[kGatherParts];
  int n;
};

// Each region: 16-byte words over its 16-byte aligned body, bytes at the ends.
__global__ void k_fill_small(FillArgs a) {
  const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x, nth = (size_t)gridDim.x * blockDim.x;
  for (int k = 0; k < a.n; ++k) {
    unsigned char* p = a.dst[k];
    const size_t nb = a.bytes[k];
    const unsigned char v = a.value[k];
    const size_t mis = (size_t)((16 - ((uintptr_t)p & 15)) & 15);
    const size_t head = mis < nb ? mis : nb;
    const size_t words = (nb - head) / 16;
    const size_t tail0 = head + words * 16;
    const uint32_t w = 0x01010101u * v;
    const uint4 q = make_uint4(w, w, w, w);
    for (size_t i = tid; i < head; i += nth) p[i] = v;
    for (size_t i = tid; i < words; i += nth) reinterpret_cast<uint4*>(p + head)[i] = q;
    for (size_t i = tail0 + tid; i < nb; i += nth) p[i] = v;
  }
}

// Small read-backs: the items copied byte by byte into the mapped pinned block.
__global__ void k_gather_small(GatherArgs a, unsigned char* dst) {
  for (int k = 0; k < a.n; ++k)
    for (uint32_t i = threadIdx.x; i < a.bytes[k]; i += blockDim.x) dst[a.off[k] + i] = a.src[k][i];
}

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
    note_alloc();
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
      g_pinned.dev = nullptr;
    }
    const size_t n = std::max<size_t>(total, 64 * 1024);
    note_alloc();
    SS_CUDA(cudaHostAlloc(&g_pinned.p, n, cudaHostAllocMapped));
    g_pinned.n = n;
    if (cudaHostGetDevicePointer(&g_pinned.dev, g_pinned.p, 0) != cudaSuccess) {
      cudaGetLastError();
      g_pinned.dev = nullptr;
    }
  }
  char* base = static_cast<char*>(g_pinned.p);
  size_t off = 0;
  if (parts.size() >= 2 && parts.size() <= (size_t)kGatherParts && total <= kGatherBytes && g_pinned.dev) {
    // several small items: one kernel writes them into the mapped block
    // instead of one copy call each
    GatherArgs a{};
    for (const HostRead& r : parts) {
      a.src[a.n] = static_cast<const unsigned char*>(r.src);
      a.bytes[a.n] = (uint32_t)r.bytes;
      a.off[a.n] = (uint32_t)off;
      ++a.n;
      off += (r.bytes + 15) / 16 * 16;
    }
    k_gather_small<<<1, 256, 0, st>>>(a, static_cast<unsigned char*>(g_pinned.dev));
    SS_LAUNCH_CHECK();
  } else {
    for (const HostRead& r : parts) {
      if (r.bytes) SS_CUDA(cudaMemcpyAsync(base + off, r.src, r.bytes, cudaMemcpyDeviceToHost, st));
      off += (r.bytes + 15) / 16 * 16;
    }
  }
  SS_CUDA(cudaStreamSynchronize(st));
  off = 0;
  for (const HostRead& r : parts) {
    if (r.bytes) std::memcpy(r.dst, base + off, r.bytes);
    off += (r.bytes + 15) / 16 * 16;
  }
  return SS_OK;
}

ss_status fill_small(cudaStream_t st, std::initializer_list<FillPart> parts) {
  if (parts.size() > (size_t)kGatherParts) SS_FAIL(SS_ERR_INVALID, "fill_small: more than %d regions", kGatherParts);
  FillArgs a{};
  size_t total = 0;
  for (const FillPart& f : parts) {
    if (!f.bytes) continue;
    a.dst[a.n] = static_cast<unsigned char*>(f.dst);
    a.bytes[a.n] = f.bytes;
    a.value[a.n] = f.value;
    ++a.n;
    total += f.bytes;
  }
  if (!a.n) return SS_OK;
  const size_t blocks = std::min<size_t>((total / 16 + 255) / 256 + 1, 4 * (size_t)sm_count());
  k_fill_small<<<(unsigned)blocks, 256, 0, st>>>(a);
  SS_LAUNCH_CHECK();
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

namespace ss {
namespace {
std::atomic<int64_t> g_alloc_count{0};
}  // namespace
void note_alloc() { g_alloc_count.fetch_add(1, std::memory_order_relaxed); }
}  // namespace ss

extern "C" int64_t ss_alloc_count(void) { return ss::g_alloc_count.load(std::memory_order_relaxed); }

extern "C" const char* ss_version(void) { return "sparse-spectral-gb300 0.1 (sm_103a)"; }

// ------------------------------------------------------------ kernel timing

namespace ss {
namespace {

struct ProfPending {
  std::string name;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaStream_t st = nullptr;
  bool ended = false;
};

struct ProfTotals {
  int64_t launches = 0;
  double ms = 0.0;
};

std::atomic<int> g_prof_level{0};
std::mutex g_prof_mu;
std::map<int64_t, ProfPending> g_prof_pending;   // by token
int64_t g_prof_next = 0;
std::vector<cudaEvent_t> g_prof_free;
std::map<std::string, ProfTotals> g_prof_totals;

// Trace: every bracket's start and end relative to the first bracket of the
// session (its start event), at most kProfTraceMax entries.
struct ProfTraceEntry {
  std::string name;
  double t0, t1;
};
constexpr size_t kProfTraceMax = 1 << 16;
cudaEvent_t g_prof_origin = nullptr;
std::vector<ProfTraceEntry> g_prof_trace;

cudaEvent_t prof_event() {
  if (!g_prof_free.empty()) {
    cudaEvent_t e = g_prof_free.back();
    g_prof_free.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

// Resolve every ended pair (waits for its end event); caller holds the lock.
void prof_drain() {
  for (auto it = g_prof_pending.begin(); it != g_prof_pending.end();) {
    ProfPending& p = it->second;
    if (!p.ended) {
      ++it;
      continue;
    }
    float ms = 0.f;
    if (cudaEventSynchronize(p.e1) == cudaSuccess && cudaEventElapsedTime(&ms, p.e0, p.e1) == cudaSuccess) {
      ProfTotals& t = g_prof_totals[p.name];
      t.launches += 1;
      t.ms += ms;
      float a = 0.f, b = 0.f;
      if (g_prof_origin && g_prof_trace.size() < kProfTraceMax &&
          cudaEventElapsedTime(&a, g_prof_origin, p.e0) == cudaSuccess &&
          cudaEventElapsedTime(&b, g_prof_origin, p.e1) == cudaSuccess)
        g_prof_trace.push_back(ProfTraceEntry{p.name, (double)a, (double)b});
      cudaGetLastError();
    } else {
      cudaGetLastError();
    }
    g_prof_free.push_back(p.e0);
    g_prof_free.push_back(p.e1);
    it = g_prof_pending.erase(it);
  }
}

}  // namespace

int prof_level() { return g_prof_level.load(std::memory_order_relaxed); }

int64_t prof_begin(const char* name, cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return -1;
  }
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (g_prof_pending.size() > 4096) prof_drain();   // bound the events held
  if (!g_prof_origin) {   // the session's time origin, just before its first bracket
    if (cudaEventCreate(&g_prof_origin) != cudaSuccess || cudaEventRecord(g_prof_origin, st) != cudaSuccess) {
      cudaGetLastError();
      g_prof_origin = nullptr;
    }
  }
  ProfPending p;
  p.name = name;
  p.st = st;
  p.e0 = prof_event();
  p.e1 = prof_event();
  if (!p.e0 || !p.e1 || cudaEventRecord(p.e0, st) != cudaSuccess) {
    cudaGetLastError();
    if (p.e0) g_prof_free.push_back(p.e0);
    if (p.e1) g_prof_free.push_back(p.e1);
    return -1;
  }
  const int64_t tok = g_prof_next++;
  g_prof_pending.emplace(tok, p);
  return tok;
}

void prof_end(int64_t token) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  auto it = g_prof_pending.find(token);
  if (it == g_prof_pending.end()) return;
  ProfPending& p = it->second;
  if (cudaEventRecord(p.e1, p.st) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  p.ended = true;
}

}  // namespace ss

extern "C" ss_status ss_profile(int32_t on) {
  std::lock_guard<std::mutex> lk(ss::g_prof_mu);
  ss::prof_drain();
  ss::g_prof_totals.clear();
  ss::g_prof_trace.clear();
  if (ss::g_prof_origin) {
    cudaEventDestroy(ss::g_prof_origin);
    ss::g_prof_origin = nullptr;
  }
  ss::g_prof_level.store(on < 0 ? 0 : (on > 2 ? 2 : on), std::memory_order_relaxed);
  return SS_OK;
}

extern "C" ss_status ss_profile_entry(int32_t i, char* name, int32_t name_cap, int64_t* launches, double* total_ms,
                                      int32_t* n_out) {
  std::lock_guard<std::mutex> lk(ss::g_prof_mu);
  ss::prof_drain();
  const int32_t n = (int32_t)ss::g_prof_totals.size();
  if (n_out) *n_out = n;
  if (i < 0 || i >= n) SS_FAIL(SS_ERR_INVALID, "ss_profile_entry: index %d of %d entries", (int)i, (int)n);
  auto it = ss::g_prof_totals.begin();
  std::advance(it, i);
  if (name && name_cap > 0) {
    std::strncpy(name, it->first.c_str(), (size_t)name_cap - 1);
    name[name_cap - 1] = '\0';
  }
  if (launches) *launches = it->second.launches;
  if (total_ms) *total_ms = it->second.ms;
  return SS_OK;
}

extern "C" ss_status ss_profile_trace(int32_t i, char* name, int32_t name_cap, double* t0_ms, double* t1_ms,
                                      int32_t* n_out) {
  std::lock_guard<std::mutex> lk(ss::g_prof_mu);
  ss::prof_drain();
  const int32_t n = (int32_t)ss::g_prof_trace.size();
  if (n_out) *n_out = n;
  if (i < 0 || i >= n) SS_FAIL(SS_ERR_INVALID, "ss_profile_trace: index %d of %d entries", (int)i, (int)n);
  const ss::ProfTraceEntry& e = ss::g_prof_trace[(size_t)i];
  if (name && name_cap > 0) {
    std::strncpy(name, e.name.c_str(), (size_t)name_cap - 1);
    name[name_cap - 1] = '\0';
  }
  if (t0_ms) *t0_ms = e.t0;
  if (t1_ms) *t1_ms = e.t1;
  return SS_OK;
}
