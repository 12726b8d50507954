// Internal declarations shared by the translation units of the library.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <initializer_list>
#include <string>
#include <vector>

#include "../../include/sparse_spectral.h"

namespace ss {

// ----------------------------------------------------------------- errors

void set_error(const char* fmt, ...);

#define SS_CUDA(call)                                                                    \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) {                                                             \
      ss::set_error("%s:%d: %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(e_)); \
      return e_ == cudaErrorMemoryAllocation ? SS_ERR_OOM : SS_ERR_CUDA;                 \
    }                                                                                    \
  } while (0)

#define SS_TRY(call)                  \
  do {                                \
    ss_status s_ = (call);            \
    if (s_ != SS_OK) return s_;       \
  } while (0)

#define SS_FAIL(code, ...)            \
  do {                                \
    ss::set_error(__VA_ARGS__);       \
    return code;                      \
  } while (0)

#define SS_LAUNCH_CHECK() SS_CUDA(cudaGetLastError())

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// Small device-to-host reads.  The pieces are copied into a pinned staging
// block of the calling thread (a copy into pageable memory is a staged,
// blocking transfer of its own), the stream is synchronised once, and the
// bytes are then moved to their destinations.
struct HostRead {
  void* dst;
  const void* src;
  size_t bytes;
};
ss_status read_back(cudaStream_t st, std::initializer_list<HostRead> parts);

// Small host-to-device writes, queued on `st` from a pinned block of the
// calling thread (a pageable source makes the runtime stage each copy while
// the host waits).  The block is reused once the previous upload has run.
struct HostWrite {
  void* dst;
  const void* src;
  size_t bytes;
};
ss_status upload(cudaStream_t st, std::initializer_list<HostWrite> parts);

// Several device regions set to a byte value each by one kernel on `st`
// (at most 8 regions; in place of one memset call per region).
struct FillPart {
  void* dst;
  size_t bytes;
  unsigned char value;
};
ss_status fill_small(cudaStream_t st, std::initializer_list<FillPart> parts);

// ----------------------------------------------------------- device memory

// Keeps freed device memory in the default stream-ordered pool (set once per
// device) so that repeated builds do not go back to the driver.
void retain_pool();

// Counts one device or pinned-host allocation call made by the library
// (reported by ss_alloc_count).
void note_alloc();

// Kernel timing (ss_profile): while it is on, a ProfScope brackets the
// launches made inside its lifetime with a CUDA event pair on their stream
// (not while the stream is being captured into a graph); the device time is
// added to the named entry when the totals are read.  Level 1 brackets the
// main kernels only (a few per pipeline step, so the host spends little on
// event records), level 2 every bracket.
int prof_level();
inline bool prof_on() { return prof_level() > 0; }
int64_t prof_begin(const char* name, cudaStream_t st);
void prof_end(int64_t token);
struct ProfScope {
  int64_t tok = -1;
  ProfScope(const char* name, cudaStream_t st, bool main = false) {
    if (prof_level() >= (main ? 1 : 2)) tok = prof_begin(name, st);
  }
  ~ProfScope() {
    if (tok >= 0) prof_end(tok);
  }
  ProfScope(const ProfScope&) = delete;
  ProfScope& operator=(const ProfScope&) = delete;
};

// Scratch for call-local temporaries: one device block per host thread and
// device, handed out in 256-byte units from the bottom up and given back in
// any order (the top comes down once the blocks above are free).  A block is
// reused in stream order: the scratch follows one stream at a time, and a
// temporary on another stream waits (one event) for what the previous stream
// queued, taken only while nothing is live.  A request that does not fit comes
// from the pool and raises the size the block is regrown to when next idle.
// Requests above kScratchMaxTake go to the pool directly (the scratch saves
// calls, which matters for many small temporaries, not for a few large ones)
// and the block stays below kScratchMaxCap.
// Not for memory that a captured graph or a persistent object keeps.  The
// block stays with its thread (at most kScratchMaxCap) until the thread exits.
constexpr size_t kScratchMaxTake = 16u << 20;
constexpr size_t kScratchMaxCap = 96u << 20;
void* scratch_take(size_t bytes, cudaStream_t st);   // nullptr: use the pool
void scratch_give(void* p);
void scratch_spill(int64_t bytes);                  // pool fallbacks alive (+/-)

// Owning device buffer from the stream-ordered pool: allocated on a stream
// and freed on the same stream (work queued there before the free still sees
// the memory).  settle() moves the free to the legacy stream for buffers that
// outlive the call that made them (the caller synchronised that call's stream).
// alloc_tmp / ensure_tmp take call-local temporaries from the thread's scratch.
template <typename T>
struct DevBuf {
  T* p = nullptr;
  size_t n = 0;
  cudaStream_t s = nullptr;
  int tmp = 0;   // 1: scratch block, 2: pool fallback of alloc_tmp, 3: view of another buffer (not owned)
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { release(); }
  void release() {
    if (p && tmp != 3) {
      if (tmp == 1) {
        scratch_give(p);
      } else {
        cudaFreeAsync(p, s);
        if (tmp == 2) scratch_spill(-(int64_t)(n * sizeof(T)));
      }
    }
    p = nullptr;
    n = 0;
    tmp = 0;
  }
  ss_status alloc_tmp(size_t count, cudaStream_t stream) {
    release();
    if (count == 0) count = 1;
    if (count * sizeof(T) > kScratchMaxTake) return alloc(count, stream);
    if (void* q = scratch_take(count * sizeof(T), stream)) {
      p = static_cast<T*>(q);
      n = count;
      s = stream;
      tmp = 1;
      return SS_OK;
    }
    const ss_status r = alloc(count, stream);
    if (r == SS_OK) {
      tmp = 2;
      scratch_spill((int64_t)(count * sizeof(T)));
    }
    return r;
  }
  ss_status ensure_tmp(size_t count, cudaStream_t stream) { return count <= n ? SS_OK : alloc_tmp(count, stream); }
  // count elements at q inside a buffer that another DevBuf owns (an arena);
  // released without a free, reallocated on its own by alloc()
  void view(T* q, size_t count) {
    release();
    p = q;
    n = count;
    s = nullptr;
    tmp = 3;
  }
  void settle() { s = nullptr; }
  ss_status alloc(size_t count, cudaStream_t stream = nullptr) {
    release();
    retain_pool();
    if (count == 0) count = 1;
    note_alloc();
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&p), count * sizeof(T), stream);
    if (e != cudaSuccess) {
      p = nullptr;
      set_error("device allocation of %zu bytes failed: %s", count * sizeof(T), cudaGetErrorString(e));
      return SS_ERR_OOM;
    }
    n = count;
    s = stream;
    return SS_OK;
  }
  ss_status ensure(size_t count, cudaStream_t stream = nullptr) { return count <= n ? SS_OK : alloc(count, stream); }
  T* get() const { return p; }
};

// ------------------------------------------------------------ constants

constexpr double kTwoPiSq = 19.739208802178716;   // 2 pi^2 (half of the 4 pi^2 in eq. GF)
constexpr double kTwoPi = 6.283185307179586;       // 2 pi (the advection factor 2 pi i of Remark ADR)
constexpr uint64_t kEmpty = ~0ull;                // unused hash slot
constexpr uint64_t kPending = 1ull << 63;         // slot claimed during the current level
constexpr int kMaxWords = 16;                     // packed key words supported
constexpr int kSlice = 32;                        // rows per neighbour-table slice (one warp)

// Packed frequency keys.  Coordinate c sits in word c / fpw at bit offset
// 64 - fb*(c % fpw + 1) (first coordinate most significant) as k_c + 2^(b-1)
// in b bits below one zero guard bit (fb = b + 1).  Unsigned comparison of the
// words in order is signed lexicographic order of the frequencies, and adding
// two packed keys and subtracting the packed bias adds the frequencies field
// by field without carries as long as every result lies in range.
struct KeyLayout {
  int d = 0, W = 0, WT = 1, b = 0, fb = 0, fpw = 0;
};

// ---------------------------------------------------------- stamp handle

}  // namespace ss

struct ss_stamp_s {
  // layout
  int d = 0, N = 0, s_a = 0, j0 = 0, jbits = 0;
  ss::KeyLayout key;
  int64_t size = 0, rows_pad = 0, nnz = 0, zero_idx = -1, n_slices = 0, n_ent = 0;
  std::vector<int64_t> level_start;   // N + 2 entries
  double a0 = 0.0;                    // Re(a_hat_0)
  bool wide = false;                  // |k|^2 may reach 2^29: FP32 norm words hold FP32 values
  // set
  ss::DevBuf<uint64_t> keys;          // [size][WT]
  ss::DevBuf<uint64_t> hl;            // [size] linear form of each key (key_lin; its hash is hash_of_lin)
  ss::DevBuf<int8_t> level;           // [size]
  ss::DevBuf<int64_t> norm;           // [rows_pad + 1] |k|^2 (0 on padding and the dummy row)
  ss::DevBuf<uint64_t> table;         // open-addressing slots
  int64_t cap = 0;
  // coefficient data in canonical step order (supp a_hat sorted lexicographically)
  ss::DevBuf<int32_t> afreq;          // [s_a][d]
  ss::DevBuf<uint64_t> stepkey;       // [s_a][WT] packed p_j
  ss::DevBuf<uint64_t> stepg;         // [s_a] key_lin(stepkey_j) - key_lin(bias)
  ss::DevBuf<int64_t> pnorm;          // [s_a] |p_j|^2
  ss::DevBuf<int32_t> pn32;           // [s_a] FP32 norm words of |p_j|^2 (see norm_word)
  ss::DevBuf<double2> aval;           // [s_a] a_hat_j
  ss::DevBuf<double2> ca64;           // [s_a] 2 pi^2 a_hat_j
  ss::DevBuf<float2> ca32;            // [s_a] same in FP32
  // neighbour table, sliced ELL with 32-row slices, column-major in a slice
  ss::DevBuf<int32_t> slice_off;      // [n_slices + 1], in units of 32 entries (one per row of a slice)
  std::vector<int32_t> woff_host;     // host copy of slice_off, filled on demand (stamp_host_tables)
  int32_t max_w = 0;                  // widest slice (entries per row)
  ss::DevBuf<uint32_t> ent;           // [n_ent] col | (j << colbits)
  ss::DevBuf<double2> ecoef64;        // [n_ent] 2 pi^2 (|k|^2 + |l|^2 - |p_j|^2) a_hat_j per entry (FP64 operator)
  ss::DevBuf<float4> ecoefdf;         // [n_ent + 1] the same as double-float, built on first DF64 solve
  ss::DevBuf<int32_t> nw32;           // [rows_pad + 1] FP32 norm words of |k|^2 (norm_word; 0 on padding)
  // scratch for galerkin_apply (FP64)
  ss::DevBuf<double2> rec64;          // [rows_pad + 1] FP64 values gathered by the FP64 operator
  // build state kept for stamp_extend
  int maxabs_f = 0, maxabs_a = 0;     // largest |coordinate| of F and of supp a_hat
  // operator of Remark ADR (advection b.grad u and reaction c u added; not
  // Hermitian; the zero frequency is an ordinary row and column)
  bool adr = false;
  ss::DevBuf<double2> bval;           // [s_a][d] b_hat_p per step (ADR)
  ss::DevBuf<double2> cval;           // [s_a] c_hat_p per step (ADR)
  ss::DevBuf<double2> diag64;         // [rows_pad + 1] diagonal of the operator (ADR; 1 on padding)
  // Hermitian half system (real data): compact rows k >lex 0 in canonical
  // order; a neighbour l < 0 is read as conj(u_{-l}) (entry bit 31).
  bool half_cand = false;             // F = -F and a_hat exactly Hermitian (set by the build)
  bool a_real = false;                // every a_hat_p real: the entry coefficients are real
  bool half_ok = false;               // half system built for the current set
  int64_t n_plus = 0, rows_pad_h = 0, n_slices_h = 0;
  int colbits_h = 0;                  // half entries: col | j << colbits_h | conj << 31
  ss::DevBuf<int64_t> mirror;         // [size] canonical index of -k
  ss::DevBuf<int32_t> hpos;           // [size] i (k > 0), -2 - i (k < 0, i the row of -k), -1 (k = 0)
  ss::DevBuf<int32_t> plus_rows;      // [rows_pad_h] canonical index of compact row i
  ss::DevBuf<int32_t> woff_h;         // [n_slices_h + 1]
  ss::DevBuf<uint32_t> ent_h;         // col | conj << 31 (dummy column rows_pad_h)
  ss::DevBuf<double2> ecoef_h;        // FP64 entry coefficients of the half table
  ss::DevBuf<int64_t> norm_h;         // [rows_pad_h + 1] |k|^2 of the compact rows (0 on padding)
  ss::DevBuf<float4> ecoefdf_h;       // the half table's coefficients as double-float (first DF64 solve)
  std::vector<int32_t> woff_h_host;   // host copy of woff_h, filled on demand (stamp_host_tables)
  // error words of the build not yet read (stamp_build_pending); the half
  // system is tentative until they are (stamp_check_pending)
  bool check_pending = false;
  // right-hand side and solution kept by sparse_spectral_solve (sol_size rows)
  ss::DevBuf<double2> rhs, sol;
  int64_t sol_size = 0;
  ss::DevBuf<unsigned char> small_arena;   // one allocation for err_dev, zidx_dev and the step tables
  ss::DevBuf<int32_t> err_dev;        // [4] device-side error words
  ss::DevBuf<int64_t> zidx_dev;       // canonical index of k = 0, or -1
};

namespace ss {

// ------------------------------------------------------------- shared API

// Exclusive prefix sum of n int32 values into out (may alias in), total into
// *d_total (device); scratch is library-managed per call.
ss_status exclusive_scan_i32(const int32_t* in, int32_t* out, int64_t n, int64_t* d_total,
                             cudaStream_t st);

// Neighbour-entry encoding.
__host__ __device__ inline uint32_t colmask_of(int jbits) { return (jbits >= 32) ? 0u : (0xffffffffu >> jbits); }
__host__ __device__ inline int colbits_of(int jbits) { return 32 - jbits; }

// Apply launchers used by galerkin_apply and the solver (apply.cu).
ss_status launch_pack64(const ss_stamp_s* s, const double2* u, cudaStream_t st);
ss_status launch_apply64(const ss_stamp_s* s, double2* y, cudaStream_t st);
// u on the first n_u rows of S (a vector on S^N is the prefix of one on
// S^{N+L}), zero on the rest, into the FP64 record array.
ss_status launch_pack64_prefix(const ss_stamp_s* s, const double2* u, int64_t n_u, cudaStream_t st);
// FP32 operator straight from the caller's u (no packing step).
ss_status launch_apply32(const ss_stamp_s* s, const float2* u, float2* y, cudaStream_t st);
// Double-float copy of the FP64 entry coefficients (built once per operator).
ss_status ensure_ecoefdf(ss_stamp_s* s, cudaStream_t st);
ss_status ensure_ecoefdf_half(ss_stamp_s* s, cudaStream_t st);

int sm_count();

// Row replaced by the identity in the operator (the pinned zero frequency of
// the diffusion problem), or -1 (none; the ADR operator keeps row 0).
inline int64_t identity_row(const ss_stamp_s* s) { return s->adr ? -1 : s->zero_idx; }

// sft_recover of a and of f on one lattice and one candidate set (sft.cu):
// the residues and the reconstructing check once, the plan's buffers shared
// in stream order, one read-back for both kept counts.  No s_max limit.
ss_status sft_recover_both(const ss_lattice* lat, const ss_trig* a, const ss_trig* f, ss_precision prec,
                           const int32_t* cand, int64_t n_cand, double tau, int32_t* a_freq, double* a_val,
                           int64_t* n_a, int32_t* f_freq, double* f_val, int64_t* n_f, cudaStream_t st);

// Releases the solver workspace cached for a stamp (solve.cu).
void drop_solve_ctx(const ss_stamp_s* s);

// stamp_build without its final synchronisation (stamp.cu): the build's error
// words are left to the caller's next synchronisation.  The caller copies
// err_dev (4 words) to the host in stream order and passes them to
// stamp_check_pending after that synchronisation, before the stamp is used
// from the host or handed out.
ss_status stamp_build_pending(const ss_sparse* a_hat, const int32_t* f_freq, int64_t n_f, int32_t N, ss_stamp* out,
                              cudaStream_t st);
ss_status stamp_check_pending(ss_stamp_s* S, const int32_t* e);
// Host copies of the slice offsets (woff_host, woff_h_host) for host-side
// planning (batches); one synchronisation when they are missing, which also
// settles a pending check.
ss_status stamp_host_tables(ss_stamp_s* S, cudaStream_t st);

}  // namespace ss

// -------------------------------------------------------- device helpers

namespace ss {

// FP32 operator norm words: |k|^2 as int32 when every norm of the set is below
// 2^29 (then |k|^2 + |l|^2 - |p|^2 = 2 k.l is exact in int32 and rounded to
// FP32 once), otherwise the FP32 value of |k|^2 (2 k.l formed in FP32: k.l is
// close to |k|^2 there, so the sum carries no cancellation beyond FP32
// rounding of the operands; the FP64 operator stays exact).
__host__ __device__ __forceinline__ int32_t norm_word(int64_t n, bool wide) {
#ifdef __CUDA_ARCH__
  return wide ? __float_as_int((float)n) : (int32_t)n;
#else
  if (!wide) return (int32_t)n;
  const float f = (float)n;
  int32_t w;
  std::memcpy(&w, &f, sizeof(w));
  return w;
#endif
}

// (a b) mod M for a, b < M < 2^31 without a 64-bit division in the inner
// loops: Barrett reduction with inv = floor((2^64 - 1) / M); the quotient
// estimate __umul64hi(a b, inv) is at most two below floor(a b / M).
__device__ __forceinline__ uint32_t mulmod(uint64_t a, uint64_t b, uint64_t M, uint64_t inv) {
  const uint64_t x = a * b;
  uint64_t r = x - __umul64hi(x, inv) * M;
  r = r >= M ? r - M : r;
  r = r >= M ? r - M : r;
  return (uint32_t)r;
}

__device__ __forceinline__ uint64_t mix64(uint64_t x) {
  // finaliser of MurmurHash3 (public domain)
  x ^= x >> 33;
  x *= 0xff51afd7ed558ccdull;
  x ^= x >> 33;
  x *= 0xc4ceb9fe1a85ec53ull;
  x ^= x >> 33;
  return x;
}

// Key hash: a linear form of the packed words modulo 2^64 (odd coefficient
// per word) followed by a bijective finaliser.  Linearity lets the hash of a
// neighbour k + p - bias (the packed sum of a frequency and a step) be formed
// from the linear forms of k and of the step by one addition, without
// touching k's words.
__host__ __device__ constexpr uint64_t key_lin_coef(int w) {
  return (0x9e3779b97f4a7c15ull ^ (0xbf58476d1ce4e5b9ull * (uint64_t)(w + 1))) | 1ull;
}

template <int WT>
__device__ __forceinline__ uint64_t key_lin(const uint64_t* k) {
  uint64_t h = 0;
#pragma unroll
  for (int w = 0; w < WT; ++w) h += key_lin_coef(w) * k[w];
  return h;
}

__device__ __forceinline__ uint64_t hash_of_lin(uint64_t lin) { return mix64(lin + 0x632be59bd9b4e019ull); }

template <int WT>
__device__ __forceinline__ uint64_t hash_key(const uint64_t* k) {
  return hash_of_lin(key_lin<WT>(k));
}

template <int WT>
__device__ __forceinline__ bool key_eq(const uint64_t* a, const uint64_t* b) {
  bool eq = true;
#pragma unroll
  for (int w = 0; w < WT; ++w) eq &= (a[w] == b[w]);
  return eq;
}

}  // namespace ss
