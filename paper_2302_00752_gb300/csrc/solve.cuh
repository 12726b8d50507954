// Persistent CG / iterative-refinement solver shared by solve and batch_solve.
#pragma once

#include "apply.cuh"

namespace ss {

constexpr int kNQ = 4;        // partial-sum quantities per slot
constexpr int kMaxInstPerChunk = 32;
constexpr int kMaxWarps = 32;

struct SolveInst {
  int64_t row0, rows, rows_pad, zero_row;
  int32_t coef_off, c_first, c_last, part_base;
  int32_t wide, pad_;       // FP32 norm words of this instance hold FP32 values (norm_word)
  double dscale;            // 4 pi^2 Re(a_hat_0)
  const double2* f;         // caller input, rows entries
  double2* u;               // caller output, rows entries
};

struct Chunk {
  int64_t s0, s1;           // global slice range [s0, s1)
  int32_t inst0, inst1;     // instances touched, inclusive
};

struct InstState {
  double rho[2];            // gamma = <r, u> by iteration parity
  double alpha[2];          // CG step by iteration parity
  double bb;                // ||f||^2
  double rr;                // last residual^2 (FP64 at exit)
  int32_t act[2];           // by iteration parity: CG (FP64) / refinement (FP32) running
  int32_t inn[2];           // by inner-iteration parity: inner CG running (FP32 mode)
  int32_t iters, inner_iters, outer_iters, applies, status, pad_;
  double2 zrho[2], zalpha[2], zomega[2];   // BiCGStab scalars by iteration parity (ADR)
};

struct SolveParams {
  int n_inst, n_chunks;
  const SolveInst* inst;
  const Chunk* chunk;
  InstState* state;
  OpView op;
  const int32_t* slice_inst;   // null for a single instance
  const int64_t* norm;         // |k|^2 per row
  const double2* ca64;
  const float2* ca32;
  const int32_t* pn;           // FP32 norm words of |p_j|^2
  double2* xrec;               // FP64 values of x: gathered for f - L x
  double2* urec64;             // FP64 values of u = D^-1 r: gathered by the FP64 operator
  float4* urec32;              // FP32 records of u: gathered by the FP32 operator
  double2* r;
  double2* w64;                // L u (FP64 mode)
  float2* w32;                 // L u (FP32 operator)
  double2* pd;                 // search direction p
  double2* sd;                 // s = L p
  double2* rhat;               // f - L x (refinement)
  double2* dlt;                // refinement correction (unused by the FP32 inner solve)
  float2* r32;                 // inner CG (FP32): residual, direction, L p, correction
  float2* p32;
  float2* s32;
  float2* d32;
  double* rdiag;               // 1 / D (FP64 mode)
  const double2* cdiag;        // complex diagonal of the ADR operator (BiCGStab), else null
  double2* zrec;               // BiCGStab: records of z = D^-1 s
  double2* tv;                 // BiCGStab: t = L z
  float4* xdf;                 // DF64 CG: x and u = D^-1 r as double-float records
  float4* udf;
  double* part;                // [slots][kNQ]
  unsigned* bar;               // barrier count, generation
  int* counters;               // done, inner started, inner finished
  int* err;
  double tol, inner_tol;
  int max_iter, max_inner, max_outer;
  long long spin_limit;
  int64_t rows_slices;   // > 0: row-wise phases split slices [0, rows_slices) evenly over the blocks
};

// Host-side plan of the static work split.
struct SolvePlan {
  std::vector<SolveInst> inst;
  std::vector<Chunk> chunk;
  int64_t n_parts = 0;
  int grid = 0, block = 256;
  bool row_split = false;   // single instance: the row-wise CG phases split the slices evenly over the blocks
  long long spin_limit = 2000000000ll;   // bound on each grid-barrier wait (ns); below 0: give up at the first poll
  // single instance: the chunk cuts are computed on the device from the
  // device slice table (chunk holds K placeholders); cuts_pending until the
  // cuts have been written into the workspace's chunk table
  bool dev_cuts = false, cuts_pending = false;
  const int32_t* cut_woff = nullptr;
  int64_t cut_n = 0, cut_ov4 = 0;
  const int32_t* cut_err = nullptr;   // the stamp's error words: an error empties every chunk
};

// Device workspace of one solve context (single stamp or batch).
struct SolveWork {
  int64_t rows_total = 0;   // padded rows, plus one dummy record (0: records not set up for this stamp)
  int64_t cap_rows = 0;     // rows the vector and record buffers hold
  int64_t df_rows = -1, bi_rows = -1;   // rows_total the DF64 / BiCGStab dummy records were cleared for
  cudaEvent_t ev[2] = {nullptr, nullptr};
  ~SolveWork() {
    if (ev[0]) cudaEventDestroy(ev[0]);
    if (ev[1]) cudaEventDestroy(ev[1]);
  }
  // the per-row vectors and the barrier / counter / error words: views of
  // one arena (one allocation per workspace)
  template <typename T>
  struct View {
    T* p = nullptr;
    T* get() const { return p; }
    void settle() {}
  };
  DevBuf<unsigned char> arena;
  View<double2> xrec, urec64, r, w64, pd, sd, rhat, dlt;
  DevBuf<double2> zrec, tv;                // BiCGStab only (allocated on first use)
  DevBuf<float4> xdf, udf;                 // DF64 CG only (allocated on first use)
  View<float4> urec32;
  View<float2> w32, r32, p32, s32, d32;
  View<double> rdiag;
  DevBuf<double> part;
  View<unsigned> bar;
  View<int> counters, err;
  DevBuf<InstState> state;
  DevBuf<SolveInst> inst;
  DevBuf<Chunk> chunk;
  int64_t cap_parts = 0;
  int cap_inst = 0, cap_chunk = 0;
};

// The records' norm words are encoded per row: wide_rows (device, one byte per
// row) or, when null, `wide` for every row.
ss_status work_alloc(SolveWork& W, int64_t rows_total, const int64_t* norm, const int8_t* wide_rows, bool wide,
                     cudaStream_t st);
ss_status work_upload(SolveWork& W, SolvePlan& plan, cudaStream_t st);
ss_status max_grid(int mode, int block, int* grid);
// mode: 0 FP64 CG, 1 FP32-refined CG, 2 FP64 BiCGStab (ADR operator; cdiag
// = its complex diagonal, workspace from work_alloc_bicgstab), 3 double-float
// CG (op.ecoefdf set, workspace from work_alloc_df64).
ss_status launch_solve(SolveWork& W, const SolvePlan& plan, const OpView& op, const int32_t* slice_inst,
                       const int64_t* norm, const double2* ca64, const float2* ca32, const int32_t* pn,
                       double tol, int max_iter, int mode, cudaStream_t st,
                       cudaEvent_t ev_begin = nullptr, cudaEvent_t ev_end = nullptr, const double2* cdiag = nullptr,
                       bool zeroed = false);   // zeroed: a single-instance prologue reset the words
ss_status work_alloc_bicgstab(SolveWork& W, cudaStream_t st);
ss_status work_alloc_df64(SolveWork& W, cudaStream_t st);
ss_status read_stats(SolveWork& W, int n_inst, ss_solve_stats* stats, ss_status* worst, cudaStream_t st,
                     cudaEvent_t ev_begin = nullptr, cudaEvent_t ev_end = nullptr);

ss_status plan_chunks(SolvePlan& plan, const std::vector<int32_t>& woff_host, const std::vector<int32_t>& slice_inst_host,
                      int target_chunks, double slice_overhead = 6.0);

}  // namespace ss
