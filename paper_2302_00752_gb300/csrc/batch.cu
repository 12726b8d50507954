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
  bool conj = false;                  // built from the instances' Hermitian half systems
  bool realc = false;                 // every instance's a_hat real: real entry coefficients
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
  // half systems of all instances (real data), solved in place of the full
  // batch when every right-hand side is Hermitian: compact vectors, the full
  // index of every compact row and of its mirror, and per full row its
  // instance, its index and its compact position (hpos convention)
  ss_batch_s* half_b = nullptr;
  bool use_half = true;
  std::vector<int64_t> row0_h;
  ss::DevBuf<double2> fc, uc;
  ss::DevBuf<int32_t> gsrc, gmir, srow_inst, slocal, shpos, hflag;
  ss::DevBuf<uint64_t> fptr, uptr;
  int64_t n_full_rows = 0;
  int32_t* hflag_host = nullptr;
  ~ss_batch_s() {
    if (graph) cudaGraphExecDestroy(graph);
    if (cap_stream) cudaStreamDestroy(cap_stream);
    if (hflag_host) cudaFreeHost(hflag_host);
    delete half_b;
  }
};

namespace ss {
namespace {

__global__ void k_woff(const int32_t* __restrict__ src, int64_t n, int32_t add, int32_t* dst) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i <= n) dst[i] = src[i] + add;
}

// Local entry -> batch entry: column shifted by the instance's first row (the
// local dummy becomes the batch's dummy), step index kept, conjugation bit
// (half systems, bit 31) kept.
__global__ void k_remap(const uint32_t* __restrict__ src, int64_t n, int src_colbits, uint32_t src_mask,
                        uint32_t src_jmask, uint32_t local_dummy, uint32_t row0, uint32_t global_dummy,
                        int dst_colbits, uint32_t* dst) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t e = src[i];
  const uint32_t col = e & src_mask, j = (e >> src_colbits) & src_jmask;
  const uint32_t c2 = (col == local_dummy) ? global_dummy : col + row0;
  dst[i] = c2 | (j << dst_colbits) | (e & 0x80000000u & ~(src_jmask << src_colbits));
}

// Compact right-hand side of the half batch from the callers' vectors, with
// the check that every f is Hermitian (f_{-k} == conj(f_k) bit for bit).
__global__ void k_bgather(const uint64_t* __restrict__ fptr, const int32_t* __restrict__ slice_inst,
                          const int32_t* __restrict__ gsrc, const int32_t* __restrict__ gmir, int64_t rows,
                          double2* fc, int32_t* flag) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rows) return;
  const int32_t g = gsrc[r];
  if (g < 0) return;   // padding row
  const double2* f = reinterpret_cast<const double2*>(fptr[slice_inst[r / ss::kSlice]]);
  const double2 a = f[g], b = f[gmir[r]];
  if (!(a.x == b.x && a.y == -b.y)) atomicExch(flag, 1);
  fc[r] = a;
}

// u of every instance from the compact solution (hpos convention: >= 0 the
// compact row, -1 the zero frequency, -2 - i the conjugate of compact row i).
__global__ void k_bscatter(const uint64_t* __restrict__ uptr, const int32_t* __restrict__ srow_inst,
                           const int32_t* __restrict__ slocal, const int32_t* __restrict__ shpos, int64_t n,
                           const double2* __restrict__ uc) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  double2* u = reinterpret_cast<double2*>(uptr[srow_inst[q]]);
  const int32_t h = shpos[q];
  double2 v = make_double2(0.0, 0.0);
  if (h >= 0) v = uc[h];
  else if (h <= -2) { v = uc[-2 - h]; v.y = -v.y; }
  u[slocal[q]] = v;
}

__global__ void k_half_maps(const int32_t* __restrict__ plus_rows, const int64_t* __restrict__ mirror,
                            const int32_t* __restrict__ hpos, int64_t n_plus, int64_t rows_pad_h, int64_t size,
                            int64_t row0_h, int32_t inst, int32_t* gsrc, int32_t* gmir, int32_t* srow_inst,
                            int32_t* slocal, int32_t* shpos) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < rows_pad_h) {
    const int32_t g = t < n_plus ? plus_rows[t] : -1;
    gsrc[t] = g;
    gmir[t] = g >= 0 ? (int32_t)mirror[g] : -1;
  }
  if (t < size) {
    srow_inst[t] = inst;
    slocal[t] = (int32_t)t;
    const int32_t h = hpos[t];
    shpos[t] = h >= 0 ? (int32_t)(row0_h + h) : (h == -1 ? -1 : (int32_t)(-2 - (row0_h + (-2 - h))));
  }
}

__global__ void k_widen_real(const double* __restrict__ in, int64_t n, double2* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = make_double2(in[i], 0.0);
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
  op.colbits = b->conj ? 31 - b->jbits : colbits_of(b->jbits);
  op.colmask = (uint32_t)((1ull << op.colbits) - 1);
  op.jmask = (1u << b->jbits) - 1u;
  op.conj = b->conj;
  op.realc = b->realc;
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

namespace {

// One instance's system as the batch builder sees it: the full operator of a
// stamp, or its Hermitian half system.
struct SysIn {
  int64_t rows, rows_pad, n_slices, n_ent, zero_row;
  const int64_t* norm;
  const int32_t* woff;
  const std::vector<int32_t>* woff_host;
  const uint32_t* ent;
  const double2* ecoef;
  int colbits, jbits;
  uint32_t colmask;
};

SysIn full_in(const ss_stamp_s* s) {
  return SysIn{s->size, s->rows_pad, s->n_slices, s->n_ent, s->zero_idx, s->norm.get(), s->slice_off.get(),
               &s->woff_host, s->ent.get(), s->ecoef64.get(), colbits_of(s->jbits), s->jbits,
               colmask_of(s->jbits)};
}

SysIn half_in(const ss_stamp_s* s) {
  const int64_t n_ent_h = s->woff_h_host.empty() ? 0 : (int64_t)s->woff_h_host.back() * kSlice;
  return SysIn{s->n_plus, s->rows_pad_h, s->n_slices_h, n_ent_h, -1, s->norm_h.get(), s->woff_h.get(),
               &s->woff_h_host, s->ent_h.get(), s->ecoef_h.get(), s->colbits_h, s->jbits,
               (uint32_t)((1u << s->colbits_h) - 1u)};
}

}  // namespace

static ss_status batch_create_impl(ss_batch_s* b, int32_t n, const ss_stamp* stamps, bool half, cudaStream_t st) {
  b->n_inst = n;
  b->conj = half;
  std::vector<SysIn> in(n);
  int64_t rows = 0, slices = 0, ent = 0, coefs = 0;
  int jb = 1;
  b->realc = true;
  for (int i = 0; i < n; ++i) {
    const ss_stamp_s* s = stamps[i];
    if (!s) SS_FAIL(SS_ERR_INVALID, "batch_create: null stamp %d", i);
    b->realc = b->realc && s->a_real;
    in[i] = half ? half_in(s) : full_in(s);
    rows += in[i].rows_pad;
    slices += in[i].n_slices;
    ent += in[i].n_ent;
    coefs += s->s_a;
    jb = std::max(jb, s->jbits);
  }
  b->rows_total = rows + 1;   // + dummy record
  b->n_slices = slices;
  b->n_ent = ent;
  b->jbits = jb;
  const int dst_colbits = half ? 31 - jb : colbits_of(jb);
  if (dst_colbits < 1 || b->rows_total > ((int64_t)1 << dst_colbits) || ent / kSlice >= INT32_MAX)
    SS_FAIL(SS_ERR_KEY_RANGE, "batch_create: %lld rows do not fit %d-bit columns", (long long)b->rows_total,
            dst_colbits);
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
    const SysIn& x = in[i];
    SS_CUDA(cudaMemcpyAsync(b->norm.get() + row0, x.norm, x.rows_pad * sizeof(int64_t), cudaMemcpyDeviceToDevice,
                            st));
    if (s->wide) SS_CUDA(cudaMemsetAsync(wide_rows.get() + row0, 1, x.rows_pad, st));
    k_woff<<<nblk(x.n_slices + 1), 256, 0, st>>>(x.woff, x.n_slices, (int32_t)(e0 / kSlice), b->woff.get() + s0);
    k_remap<<<nblk(x.n_ent), 256, 0, st>>>(x.ent, x.n_ent, x.colbits, x.colmask, (1u << x.jbits) - 1u,
                                           (uint32_t)x.rows_pad, (uint32_t)row0, global_dummy, dst_colbits,
                                           b->ent.get() + e0);
    k_fill_i32<<<nblk(x.n_slices), 256, 0, st>>>(b->slice_inst.get() + s0, x.n_slices, i);
    // entry coefficients: one double per entry when every stamp's are real
    // (the batch keeps that layout), else double2 (a real stamp's widened)
    if (b->realc)
      SS_CUDA(cudaMemcpyAsync(reinterpret_cast<double*>(b->ecoef64.get()) + e0, x.ecoef, x.n_ent * sizeof(double),
                              cudaMemcpyDeviceToDevice, st));
    else if (s->a_real)
      k_widen_real<<<nblk(x.n_ent), 256, 0, st>>>(reinterpret_cast<const double*>(x.ecoef), x.n_ent,
                                                  b->ecoef64.get() + e0);
    else
      SS_CUDA(cudaMemcpyAsync(b->ecoef64.get() + e0, x.ecoef, x.n_ent * sizeof(double2), cudaMemcpyDeviceToDevice, st));
    SS_LAUNCH_CHECK();
    SS_CUDA(cudaMemcpyAsync(b->ca64.get() + c0, s->ca64.get(), s->s_a * sizeof(double2), cudaMemcpyDeviceToDevice, st));
    SS_CUDA(cudaMemcpyAsync(b->ca32.get() + c0, s->ca32.get(), s->s_a * sizeof(float2), cudaMemcpyDeviceToDevice, st));
    SS_CUDA(cudaMemcpyAsync(b->pn.get() + c0, s->pn32.get(), s->s_a * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
    const std::vector<int32_t>& w = *x.woff_host;
    if ((int64_t)w.size() != x.n_slices + 1) SS_FAIL(SS_ERR_INVALID, "batch_create: stamp %d has no slice table", i);
    for (int64_t q = 0; q <= x.n_slices; ++q) b->woff_h[s0 + q] = w[q] + (int32_t)(e0 / kSlice);
    for (int64_t q = 0; q < x.n_slices; ++q) b->slice_inst_h[s0 + q] = i;
    SolveInst& si = b->plan.inst[i];
    si.row0 = row0;
    si.rows = x.rows;
    si.rows_pad = x.rows_pad;
    si.zero_row = x.zero_row >= 0 ? row0 + x.zero_row : -1;
    si.coef_off = (int32_t)c0;
    si.dscale = 2.0 * kTwoPiSq * s->a0;
    si.wide = s->wide ? 1 : 0;
    row0 += x.rows_pad;
    s0 += x.n_slices;
    e0 += x.n_ent;
    c0 += s->s_a;
  }
  SS_CUDA(cudaMemsetAsync(b->norm.get() + (b->rows_total - 1), 0, sizeof(int64_t), st));
  SS_TRY(work_alloc(b->work, b->rows_total, b->norm.get(), wide_rows.get(), false, st));
  SS_CUDA(cudaStreamSynchronize(st));
  b->norm.settle(); b->woff.settle(); b->slice_inst.settle(); b->ent.settle();
  b->ca64.settle(); b->ca32.settle(); b->pn.settle(); b->ecoef64.settle();
  return SS_OK;
}

// The half batch and the maps between the callers' vectors and its rows.
static ss_status batch_create_half(ss_batch_s* b, int32_t n, const ss_stamp* stamps, cudaStream_t st) {
  ss_batch_s* h = new ss_batch_s();
  ss_status r = batch_create_impl(h, n, stamps, true, st);
  if (r != SS_OK) {
    cudaStreamSynchronize(st);
    delete h;
    return r;
  }
  b->half_b = h;
  const int64_t rows_h = h->rows_total;
  int64_t full_rows = 0;
  for (int i = 0; i < n; ++i) full_rows += stamps[i]->size;
  b->n_full_rows = full_rows;
  SS_TRY(b->fc.alloc(rows_h, st));
  SS_TRY(b->uc.alloc(rows_h, st));
  SS_TRY(b->gsrc.alloc(rows_h, st));
  SS_TRY(b->gmir.alloc(rows_h, st));
  SS_TRY(b->srow_inst.alloc(full_rows, st));
  SS_TRY(b->slocal.alloc(full_rows, st));
  SS_TRY(b->shpos.alloc(full_rows, st));
  SS_TRY(b->hflag.alloc(1, st));
  SS_TRY(b->fptr.alloc(n, st));
  SS_TRY(b->uptr.alloc(n, st));
  SS_CUDA(cudaMemsetAsync(b->fc.get(), 0, rows_h * sizeof(double2), st));
  SS_CUDA(cudaMemsetAsync(b->gsrc.get(), 0xff, rows_h * sizeof(int32_t), st));   // -1: the dummy row
  b->row0_h.assign(n, 0);
  int64_t q0 = 0;
  for (int i = 0; i < n; ++i) {
    const ss_stamp_s* s = stamps[i];
    const int64_t row0_h = h->plan.inst[i].row0;
    b->row0_h[i] = row0_h;
    const int64_t m = std::max<int64_t>(s->rows_pad_h, s->size);
    k_half_maps<<<nblk(m), 256, 0, st>>>(s->plus_rows.get(), s->mirror.get(), s->hpos.get(), s->n_plus,
                                         s->rows_pad_h, s->size, row0_h, i, b->gsrc.get() + row0_h,
                                         b->gmir.get() + row0_h, b->srow_inst.get() + q0, b->slocal.get() + q0,
                                         b->shpos.get() + q0);
    SS_LAUNCH_CHECK();
    // the half batch reads and writes the compact vectors, always at the same place
    h->plan.inst[i].f = b->fc.get() + row0_h;
    h->plan.inst[i].u = b->uc.get() + row0_h;
    q0 += s->size;
  }
  if (!b->hflag_host) {
    note_alloc();
    SS_CUDA(cudaMallocHost(&b->hflag_host, sizeof(int32_t)));
  }
  SS_CUDA(cudaStreamSynchronize(st));
  b->fc.settle(); b->uc.settle(); b->gsrc.settle(); b->gmir.settle(); b->srow_inst.settle();
  b->slocal.settle(); b->shpos.settle(); b->hflag.settle(); b->fptr.settle(); b->uptr.settle();
  return SS_OK;
}

extern "C" ss_status batch_create(int32_t n_inst, const ss_stamp* stamps, ss_batch* out, void* stream) {
  if (!out || !stamps || n_inst < 1) SS_FAIL(SS_ERR_INVALID, "batch_create: bad argument");
  cudaStream_t st = as_stream(stream);
  // host copies of the slice offsets: the batch's tables are laid out on the host
  for (int i = 0; i < n_inst; ++i)
    if (stamps[i]) SS_TRY(stamp_host_tables(stamps[i], st));
  bool all_half = true;
  for (int i = 0; i < n_inst; ++i) {
    if (stamps[i] && stamps[i]->adr) SS_FAIL(SS_ERR_INVALID, "batch_create: ADR stamps are solved one at a time");
    all_half = all_half && stamps[i] && stamps[i]->half_ok;
  }
  *out = nullptr;
  ss_batch_s* b = new ss_batch_s();
  ss_status s = batch_create_impl(b, n_inst, stamps, false, st);
  // real data throughout: the half batch as well (one that does not fit its
  // column bits is left out; the full batch serves)
  if (s == SS_OK && all_half && batch_create_half(b, n_inst, stamps, st) != SS_OK) {
    delete b->half_b;
    b->half_b = nullptr;
  }
  if (s != SS_OK) {
    cudaStreamSynchronize(st);
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

namespace {

// Keep the half batch's tile shape equal to the batch's.
void sync_config(ss_batch_s* b) {
  ss_batch_s* h = b->half_b;
  if (!h) return;
  if (h->block != b->block || h->blocks_per_sm != b->blocks_per_sm || h->chunks_per_block != b->chunks_per_block) {
    h->block = b->block;
    h->blocks_per_sm = b->blocks_per_sm;
    h->chunks_per_block = b->chunks_per_block;
    h->planned = false;
  }
}

// Compact right-hand sides of the half batch from the callers' vectors (and
// the Hermitian check, read back with the statistics).
ss_status gather_half(ss_batch_s* b, const double* const* f, double* const* u, cudaStream_t st) {
  ss_batch_s* h = b->half_b;
  const size_t bytes = (size_t)b->n_inst * sizeof(uint64_t);
  SS_TRY(upload(st, {{b->fptr.get(), f, bytes}, {b->uptr.get(), u, bytes}}));
  SS_CUDA(cudaMemsetAsync(b->hflag.get(), 0, sizeof(int32_t), st));
  k_bgather<<<nblk(h->rows_total - 1), 256, 0, st>>>(b->fptr.get(), h->slice_inst.get(), b->gsrc.get(),
                                                      b->gmir.get(), h->rows_total - 1, b->fc.get(), b->hflag.get());
  SS_LAUNCH_CHECK();
  return SS_OK;
}

// The half batch end to end; *used is false when some f was not Hermitian
// (the callers' u are then to be recomputed by the full batch).
ss_status run_half(ss_batch_s* b, const double* const* f, double* const* u, double tol, int max_iter,
                   ss_precision prec, bool use_graph, ss_solve_stats* stats, ss_status* worst, bool* used,
                   cudaStream_t st) {
  ss_batch_s* h = b->half_b;
  sync_config(b);
  SS_TRY(gather_half(b, f, u, st));
  SS_TRY(run_once(h, tol, max_iter, prec, use_graph, st));
  k_bscatter<<<nblk(b->n_full_rows), 256, 0, st>>>(b->uptr.get(), b->srow_inst.get(), b->slocal.get(),
                                                   b->shpos.get(), b->n_full_rows, b->uc.get());
  SS_LAUNCH_CHECK();
  SS_CUDA(cudaMemcpyAsync(b->hflag_host, b->hflag.get(), sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  SS_TRY(read_stats(h->work, b->n_inst, stats, worst, st, h->work.ev[0], h->work.ev[1]));
  *used = *b->hflag_host == 0;
  if (*used && stats)
    for (int i = 0; i < b->n_inst; ++i) {
      stats[i].half_system = 1;
      stats[i].real_coefficients = h->realc;
    }
  return SS_OK;
}

}  // namespace

extern "C" ss_status batch_solve(ss_batch b, const double* const* f, double* const* u, double tol, int32_t max_iter,
                                 ss_precision prec, int32_t use_graph, ss_solve_stats* stats, void* stream) {
  if (!b || !f || !u) SS_FAIL(SS_ERR_INVALID, "batch_solve: null argument");
  if (!(tol > 0.0) || max_iter < 1) SS_FAIL(SS_ERR_INVALID, "batch_solve: need tol > 0 and max_iter >= 1");
  if (prec != SS_FP64 && prec != SS_FP32) SS_FAIL(SS_ERR_INVALID, "batch_solve: bad precision");
  for (int i = 0; i < b->n_inst; ++i)
    if (!f[i] || !u[i]) SS_FAIL(SS_ERR_INVALID, "batch_solve: null vector for instance %d", i);
  cudaStream_t st = as_stream(stream);
  ss_status worst;
  if (b->half_b && b->use_half) {
    bool used = false;
    SS_TRY(run_half(b, f, u, tol, max_iter, prec, use_graph != 0, stats, &worst, &used, st));
    if (used) return worst;
  }
  SS_TRY(set_pointers(b, f, u));
  SS_TRY(run_once(b, tol, max_iter, prec, use_graph != 0, st));
  SS_TRY(read_stats(b->work, b->n_inst, stats, &worst, st, b->work.ev[0], b->work.ev[1]));
  if (stats)
    for (int i = 0; i < b->n_inst; ++i) stats[i].real_coefficients = b->realc;
  return worst;
}

extern "C" ss_status batch_set_symmetry(ss_batch b, int32_t use_half) {
  if (!b) SS_FAIL(SS_ERR_INVALID, "batch_set_symmetry: null batch");
  b->use_half = use_half != 0;
  return SS_OK;
}

extern "C" ss_status batch_autotune(ss_batch b, const double* const* f, double* const* u, double tol,
                                    int32_t max_iter, ss_precision prec, double* best_ms, void* stream) {
  if (!b || !f || !u) SS_FAIL(SS_ERR_INVALID, "batch_autotune: null argument");
  cudaStream_t st = as_stream(stream);
  // the system batch_solve runs: the half batch when there is one
  ss_batch_s* t = (b->half_b && b->use_half) ? b->half_b : b;
  if (t == b) SS_TRY(set_pointers(b, f, u));
  else SS_TRY(gather_half(b, f, u, st));
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
    t->block = c.block;
    t->blocks_per_sm = c.bps;
    t->chunks_per_block = c.cpb;
    result = replan(t, mode, st);
    if (result != SS_OK) break;
    result = run_once(t, tol, max_iter, prec, false, st);   // warm-up
    if (result != SS_OK) break;
    cudaEventRecord(e0, st);
    result = run_once(t, tol, max_iter, prec, false, st);
    if (result != SS_OK) break;
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess) { result = SS_ERR_CUDA; break; }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    ss_status worst;
    result = read_stats(t->work, t->n_inst, nullptr, &worst, st);
    if (result != SS_OK) break;
    if (worst == SS_OK && ms < best) {
      best = ms;
      pick = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (result != SS_OK) return result;
  for (ss_batch_s* x : {b, b->half_b}) {
    if (!x) continue;
    x->block = pick.block;
    x->blocks_per_sm = pick.bps;
    x->chunks_per_block = pick.cpb;
    x->planned = false;
  }
  SS_TRY(replan(t, mode, st));
  if (best_ms) *best_ms = best;
  return SS_OK;
}

extern "C" ss_status batch_config(ss_batch b, int32_t* block, int32_t* blocks_per_sm, int32_t* chunks_per_block,
                                  int32_t* grid, int32_t* n_chunks) {
  if (!b) SS_FAIL(SS_ERR_INVALID, "batch_config: null batch");
  const ss_batch_s* t = (b->half_b && b->use_half) ? b->half_b : b;
  if (block) *block = b->block;
  if (blocks_per_sm) *blocks_per_sm = b->blocks_per_sm;
  if (chunks_per_block) *chunks_per_block = b->chunks_per_block;
  if (grid) *grid = t->plan.grid;
  if (n_chunks) *n_chunks = (int32_t)t->plan.chunk.size();
  return SS_OK;
}

extern "C" ss_status batch_set_config(ss_batch b, int32_t block, int32_t blocks_per_sm, int32_t chunks_per_block) {
  if (!b || (block != 128 && block != 256 && block != 512 && block != 1024) || blocks_per_sm < 0 ||
      chunks_per_block < 1)
    SS_FAIL(SS_ERR_INVALID, "batch_set_config: block in {128,256,512,1024}, blocks_per_sm >= 0, chunks >= 1");
  for (ss_batch_s* x : {b, b->half_b}) {
    if (!x) continue;
    x->block = block;
    x->blocks_per_sm = blocks_per_sm;
    x->chunks_per_block = chunks_per_block;
    x->planned = false;
  }
  return SS_OK;
}
