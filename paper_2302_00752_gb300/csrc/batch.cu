// Batched solve: many stamping sets of uneven size in one persistent launch.
//
// batch_create concatenates the instances into one row space (each padded to
// whole 32-row slices, one shared all-zero dummy record at the end), re-encodes
// their neighbour entries with global column indices, and stacks their
// coefficient tables.  The persistent solver (solve.cu) then runs every CG phase
// over all rows at once with per-instance scalars; converged instances drop
// out.  The launch sequence (state resets + the cooperative kernel) can be
// captured in a CUDA graph and replayed.  batch_autotune times the solve over a
// few tile shapes (threads per block, resident blocks per SM, chunks per
// block) and keeps the fastest.
#include <algorithm>
#include <cmath>

#include "solve.cuh"

struct ss_batch_s {
  int n_inst = 0;
  int64_t rows_total = 0, n_slices = 0, n_ent = 0;
  int jbits = 1;
  ss::DevBuf<int64_t> norm;
  ss::DevBuf<int32_t> woff, slice_inst, pn;
  ss::DevBuf<uint32_t> ent;
  ss::DevBuf<double2> ca64, ecoef64;
  ss::DevBuf<float2> ca32;
  std::vector<int32_t> woff_h, slice_inst_h;
  ss::SolvePlan plan;
  ss::SolveWork work;
  // tile shape
  int block = 1024, blocks_per_sm = 1, chunks_per_block = 1;
  bool planned = false;
  int planned_mode = -1;
  // graph
  cudaGraphExec_t graph = nullptr;
  cudaStream_t cap_stream = nullptr;   // capture needs a stream other than the legacy default
  int graph_mode = -1, graph_max_iter = -1;
  double graph_tol = -1;
  ~ss_batch_s() {
    if (graph) cudaGraphExecDestroy(graph);
    if (cap_stream) cudaStreamDestroy(cap_stream);
  }
};

namespace ss {
namespace {

__global__ void k_woff(const int32_t* __restrict__ src, int64_t n, int32_t add, int32_t* dst) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i <= n) dst[i] = src[i] + add;
}

__global__ void k_remap(const uint32_t* __restrict__ src, int64_t n, int src_colbits, uint32_t src_mask,
                        uint32_t local_dummy, uint32_t row0, uint32_t global_dummy, int dst_colbits, uint32_t* dst) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t e = src[i];
  const uint32_t col = e & src_mask, j = e >> src_colbits;
  const uint32_t c2 = (col == local_dummy) ? global_dummy : col + row0;
  dst[i] = c2 | (j << dst_colbits);
}

__global__ void k_fill_i32(int32_t* p, int64_t n, int32_t v) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

ss_status replan(ss_batch_s* b, int mode, cudaStream_t st) {
  int grid_max = 0;
  SS_TRY(max_grid(mode, b->block, &grid_max));
  int grid = grid_max;
  if (b->blocks_per_sm > 0) grid = std::min(grid_max, b->blocks_per_sm * sm_count());
  const int64_t by_size = std::max<int64_t>(1, b->n_slices / 8);
  const int target = (int)std::min<int64_t>((int64_t)grid * b->chunks_per_block, by_size);
  SS_TRY(plan_chunks(b->plan, b->woff_h, b->slice_inst_h, target));
  b->plan.block = b->block;
  b->plan.grid = std::min<int>(grid, (int)b->plan.chunk.size());
  SS_TRY(work_upload(b->work, b->plan, st));
  b->planned = true;
  b->planned_mode = mode;
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  return SS_OK;
}

OpView batch_op(const ss_batch_s* b) {
  OpView op;
  op.woff = b->woff.get();
  op.ent = b->ent.get();
  op.ecoef = b->ecoef64.get();
  op.ecoefdf = nullptr;
  op.colbits = colbits_of(b->jbits);
  op.colmask = colmask_of(b->jbits);
  return op;
}

ss_status run_once(ss_batch_s* b, double tol, int max_iter, ss_precision prec, bool use_graph, cudaStream_t st) {
  const int mode = prec == SS_FP64 ? 0 : 1;
  if (!b->planned || b->planned_mode != mode) SS_TRY(replan(b, mode, st));
  SS_TRY(work_upload(b->work, b->plan, st));   // f/u pointers may have changed
  if (!b->work.ev[0]) {
    SS_CUDA(cudaEventCreate(&b->work.ev[0]));
    SS_CUDA(cudaEventCreate(&b->work.ev[1]));
  }
  if (!use_graph)
    return launch_solve(b->work, b->plan, batch_op(b), b->slice_inst.get(), b->norm.get(), b->ca64.get(),
                        b->ca32.get(), b->pn.get(), tol, max_iter, prec, st, b->work.ev[0], b->work.ev[1]);
  if (!b->graph || b->graph_mode != mode || b->graph_tol != tol || b->graph_max_iter != max_iter) {
    if (b->graph) {
      cudaGraphExecDestroy(b->graph);
      b->graph = nullptr;
    }
    cudaGraph_t g = nullptr;
    if (!b->cap_stream) SS_CUDA(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
    // the upload above must land before the graph runs: the graph is launched on st after it
    SS_CUDA(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
    ss_status s = launch_solve(b->work, b->plan, batch_op(b), b->slice_inst.get(), b->norm.get(), b->ca64.get(),
                               b->ca32.get(), b->pn.get(), tol, max_iter, prec, b->cap_stream);
    cudaError_t e = cudaStreamEndCapture(b->cap_stream, &g);
    if (s != SS_OK) {
      if (g) cudaGraphDestroy(g);
      return s;
    }
    if (e != cudaSuccess) SS_FAIL(SS_ERR_CUDA, "batch_solve: graph capture failed: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      b->graph = nullptr;
      SS_FAIL(SS_ERR_CUDA, "batch_solve: graph instantiation failed: %s", cudaGetErrorString(e));
    }
    b->graph_mode = mode;
    b->graph_tol = tol;
    b->graph_max_iter = max_iter;
  }
  SS_CUDA(cudaEventRecord(b->work.ev[0], st));
  SS_CUDA(cudaGraphLaunch(b->graph, st));
  SS_CUDA(cudaEventRecord(b->work.ev[1], st));
  return SS_OK;
}

ss_status set_pointers(ss_batch_s* b, const double* const* f, double* const* u) {
  for (int i = 0; i < b->n_inst; ++i) {
    if (!f[i] || !u[i]) SS_FAIL(SS_ERR_INVALID, "batch_solve: null vector for instance %d", i);
    b->plan.inst[i].f = reinterpret_cast<const double2*>(f[i]);
    b->plan.inst[i].u = reinterpret_cast<double2*>(u[i]);
  }
  return SS_OK;
}

}  // namespace
}  // namespace ss

using namespace ss;

static ss_status batch_create_impl(ss_batch_s* b, int32_t n, const ss_stamp* stamps, cudaStream_t st) {
  b->n_inst = n;
  int64_t rows = 0, slices = 0, ent = 0, coefs = 0;
  int jb = 1;
  for (int i = 0; i < n; ++i) {
    const ss_stamp_s* s = stamps[i];
    if (!s) SS_FAIL(SS_ERR_INVALID, "batch_create: null stamp %d", i);
    rows += s->rows_pad;
    slices += s->n_slices;
    ent += s->n_ent;
    coefs += s->s_a;
    jb = std::max(jb, s->jbits);
  }
  b->rows_total = rows + 1;   // + dummy record
  b->n_slices = slices;
  b->n_ent = ent;
  b->jbits = jb;
  if (b->rows_total > ((int64_t)1 << colbits_of(jb)) || ent / kSlice >= INT32_MAX)
    SS_FAIL(SS_ERR_KEY_RANGE, "batch_create: %lld rows do not fit %d-bit columns", (long long)b->rows_total,
            colbits_of(jb));
  SS_TRY(b->norm.alloc(b->rows_total, st));
  SS_TRY(b->woff.alloc(slices + 1, st));
  SS_TRY(b->slice_inst.alloc(slices, st));
  SS_TRY(b->ent.alloc(ent + 1, st));
  SS_TRY(b->ecoef64.alloc(ent + 1, st));
  SS_TRY(b->ca64.alloc(coefs, st));
  SS_TRY(b->ca32.alloc(coefs, st));
  SS_TRY(b->pn.alloc(coefs, st));
  DevBuf<int8_t> wide_rows;
  SS_TRY(wide_rows.alloc(b->rows_total, st));
  SS_CUDA(cudaMemsetAsync(wide_rows.get(), 0, b->rows_total, st));
  b->woff_h.assign(slices + 1, 0);
  b->slice_inst_h.assign(slices, 0);
  b->plan.inst.assign(n, SolveInst{});
  int64_t row0 = 0, s0 = 0, e0 = 0, c0 = 0;
  const uint32_t global_dummy = (uint32_t)(b->rows_total - 1);
  for (int i = 0; i < n; ++i) {
    const ss_stamp_s* s = stamps[i];
    SS_CUDA(cudaMemcpyAsync(b->norm.get() + row0, s->norm.get(), s->rows_pad * sizeof(int64_t),
                            cudaMemcpyDeviceToDevice, st));
    if (s->wide) SS_CUDA(cudaMemsetAsync(wide_rows.get() + row0, 1, s->rows_pad, st));
    k_woff<<<nblk(s->n_slices + 1), 256, 0, st>>>(s->slice_off.get(), s->n_slices, (int32_t)(e0 / kSlice),
                                                  b->woff.get() + s0);
    k_remap<<<nblk(s->n_ent), 256, 0, st>>>(s->ent.get(), s->n_ent, colbits_of(s->jbits), colmask_of(s->jbits),
                                            (uint32_t)s->rows_pad, (uint32_t)row0, global_dummy, colbits_of(jb),
                                            b->ent.get() + e0);
    k_fill_i32<<<nblk(s->n_slices), 256, 0, st>>>(b->slice_inst.get() + s0, s->n_slices, i);
    SS_CUDA(cudaMemcpyAsync(b->ecoef64.get() + e0, s->ecoef64.get(), s->n_ent * sizeof(double2),
                            cudaMemcpyDeviceToDevice, st));
    SS_LAUNCH_CHECK();
    SS_CUDA(cudaMemcpyAsync(b->ca64.get() + c0, s->ca64.get(), s->s_a * sizeof(double2), cudaMemcpyDeviceToDevice, st));
    SS_CUDA(cudaMemcpyAsync(b->ca32.get() + c0, s->ca32.get(), s->s_a * sizeof(float2), cudaMemcpyDeviceToDevice, st));
    SS_CUDA(cudaMemcpyAsync(b->pn.get() + c0, s->pn32.get(), s->s_a * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
    const std::vector<int32_t>& w = s->woff_host;
    if ((int64_t)w.size() != s->n_slices + 1) SS_FAIL(SS_ERR_INVALID, "batch_create: stamp %d has no slice table", i);
    for (int64_t q = 0; q <= s->n_slices; ++q) b->woff_h[s0 + q] = w[q] + (int32_t)(e0 / kSlice);
    for (int64_t q = 0; q < s->n_slices; ++q) b->slice_inst_h[s0 + q] = i;
    SolveInst& in = b->plan.inst[i];
    in.row0 = row0;
    in.rows = s->size;
    in.rows_pad = s->rows_pad;
    in.zero_row = s->zero_idx >= 0 ? row0 + s->zero_idx : -1;
    in.coef_off = (int32_t)c0;
    in.dscale = 2.0 * kTwoPiSq * s->a0;
    in.wide = s->wide ? 1 : 0;
    row0 += s->rows_pad;
    s0 += s->n_slices;
    e0 += s->n_ent;
    c0 += s->s_a;
  }
  SS_CUDA(cudaMemsetAsync(b->norm.get() + (b->rows_total - 1), 0, sizeof(int64_t), st));
  SS_TRY(work_alloc(b->work, b->rows_total, b->norm.get(), wide_rows.get(), false, st));
  SS_CUDA(cudaStreamSynchronize(st));
  b->norm.settle(); b->woff.settle(); b->slice_inst.settle(); b->ent.settle();
  b->ca64.settle(); b->ca32.settle(); b->pn.settle(); b->ecoef64.settle();
  return SS_OK;
}

extern "C" ss_status batch_create(int32_t n_inst, const ss_stamp* stamps, ss_batch* out, void* stream) {
  if (!out || !stamps || n_inst < 1) SS_FAIL(SS_ERR_INVALID, "batch_create: bad argument");
  for (int i = 0; i < n_inst; ++i)
    if (stamps[i] && stamps[i]->adr) SS_FAIL(SS_ERR_INVALID, "batch_create: ADR stamps are solved one at a time");
  *out = nullptr;
  ss_batch_s* b = new ss_batch_s();
  ss_status s = batch_create_impl(b, n_inst, stamps, as_stream(stream));
  if (s != SS_OK) {
    cudaStreamSynchronize(as_stream(stream));
    delete b;
    return s;
  }
  *out = b;
  return SS_OK;
}

extern "C" void batch_destroy(ss_batch b) {
  if (!b) return;
  cudaDeviceSynchronize();
  delete b;
}

extern "C" ss_status batch_solve(ss_batch b, const double* const* f, double* const* u, double tol, int32_t max_iter,
                                 ss_precision prec, int32_t use_graph, ss_solve_stats* stats, void* stream) {
  if (!b || !f || !u) SS_FAIL(SS_ERR_INVALID, "batch_solve: null argument");
  if (!(tol > 0.0) || max_iter < 1) SS_FAIL(SS_ERR_INVALID, "batch_solve: need tol > 0 and max_iter >= 1");
  if (prec != SS_FP64 && prec != SS_FP32) SS_FAIL(SS_ERR_INVALID, "batch_solve: bad precision");
  cudaStream_t st = as_stream(stream);
  SS_TRY(set_pointers(b, f, u));
  SS_TRY(run_once(b, tol, max_iter, prec, use_graph != 0, st));
  ss_status worst;
  SS_TRY(read_stats(b->work, b->n_inst, stats, &worst, st, b->work.ev[0], b->work.ev[1]));
  return worst;
}

extern "C" ss_status batch_autotune(ss_batch b, const double* const* f, double* const* u, double tol,
                                    int32_t max_iter, ss_precision prec, double* best_ms, void* stream) {
  if (!b || !f || !u) SS_FAIL(SS_ERR_INVALID, "batch_autotune: null argument");
  cudaStream_t st = as_stream(stream);
  SS_TRY(set_pointers(b, f, u));
  struct Cfg { int block, bps, cpb; };
  const Cfg cands[] = {{1024, 1, 1}, {1024, 1, 2}, {512, 2, 1}, {512, 1, 1}, {256, 0, 1}, {256, 4, 2}, {128, 0, 2}};
  cudaEvent_t e0, e1;
  SS_CUDA(cudaEventCreate(&e0));
  SS_CUDA(cudaEventCreate(&e1));
  double best = 1e300;
  Cfg pick = cands[0];
  const int mode = prec == SS_FP64 ? 0 : 1;
  ss_status result = SS_OK;
  for (const Cfg& c : cands) {
    b->block = c.block;
    b->blocks_per_sm = c.bps;
    b->chunks_per_block = c.cpb;
    result = replan(b, mode, st);
    if (result != SS_OK) break;
    result = run_once(b, tol, max_iter, prec, false, st);   // warm-up
    if (result != SS_OK) break;
    cudaEventRecord(e0, st);
    result = run_once(b, tol, max_iter, prec, false, st);
    if (result != SS_OK) break;
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess) { result = SS_ERR_CUDA; break; }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    ss_status worst;
    result = read_stats(b->work, b->n_inst, nullptr, &worst, st);
    if (result != SS_OK) break;
    if (worst == SS_OK && ms < best) {
      best = ms;
      pick = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (result != SS_OK) return result;
  b->block = pick.block;
  b->blocks_per_sm = pick.bps;
  b->chunks_per_block = pick.cpb;
  SS_TRY(replan(b, mode, st));
  if (best_ms) *best_ms = best;
  return SS_OK;
}

extern "C" ss_status batch_config(ss_batch b, int32_t* block, int32_t* blocks_per_sm, int32_t* chunks_per_block,
                                  int32_t* grid, int32_t* n_chunks) {
  if (!b) SS_FAIL(SS_ERR_INVALID, "batch_config: null batch");
  if (block) *block = b->block;
  if (blocks_per_sm) *blocks_per_sm = b->blocks_per_sm;
  if (chunks_per_block) *chunks_per_block = b->chunks_per_block;
  if (grid) *grid = b->plan.grid;
  if (n_chunks) *n_chunks = (int32_t)b->plan.chunk.size();
  return SS_OK;
}

extern "C" ss_status batch_set_config(ss_batch b, int32_t block, int32_t blocks_per_sm, int32_t chunks_per_block) {
  if (!b || (block != 128 && block != 256 && block != 512 && block != 1024) || blocks_per_sm < 0 ||
      chunks_per_block < 1)
    SS_FAIL(SS_ERR_INVALID, "batch_set_config: block in {128,256,512,1024}, blocks_per_sm >= 0, chunks >= 1");
  b->block = block;
  b->blocks_per_sm = blocks_per_sm;
  b->chunks_per_block = chunks_per_block;
  b->planned = false;
  return SS_OK;
}
