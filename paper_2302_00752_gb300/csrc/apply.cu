// galerkin_apply: y = L_{N,s} u on the stamping set (eq. FiniteGalerkinOperator).
// One thread per row, one warp per 32-row slice of the sliced-ELL table: the
// index stream is read coalesced (column-major inside a slice).  FP64: the
// values of u are first packed into a record array and gathered from there
// beside the stored entry coefficients.  FP32: u_l is gathered straight from
// the caller's array and |l|^2 from the stamp's norm words.
#include <algorithm>

#include "apply.cuh"

namespace ss {
namespace {

__global__ void k_pack64(const double2* __restrict__ u, int64_t size, double2* rec) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < size) rec[i] = u[i];
}

__global__ void __launch_bounds__(256) k_apply64(OpView op, int64_t size, int64_t rows_pad,
                                                 const double2* __restrict__ rec, int64_t zero_idx,
                                                 double2* __restrict__ y) {
  const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= rows_pad) return;
  const int64_t s = row / kSlice;
  const int lane = (int)(row % kSlice);
  double2 acc = row_apply64(op, s, lane, rec);
  if (row == zero_idx) acc = rec[row];
  if (row < size) y[row] = acc;
}

// One row per thread; 40 registers (six 256-thread blocks per SM) keep four
// index words and eight gathers in flight per thread.
template <bool WIDE>
__global__ void __launch_bounds__(256, 6) k_apply32(OpView op, int64_t size, int64_t rows_pad,
                                                    const int32_t* __restrict__ nw, const float2* __restrict__ u,
                                                    const float2* __restrict__ ca, const int32_t* __restrict__ pn,
                                                    int64_t zero_idx, float2* __restrict__ y) {
  const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= rows_pad) return;
  const int64_t s = row / kSlice;
  const int lane = (int)(row % kSlice);
  float2 acc = row_apply32_direct<WIDE, 4>(op, s, lane, __ldg(nw + row), size, u, nw, ca, pn);
  if (row < size) y[row] = row == zero_idx ? u[row] : acc;
}

inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// u on the first n_u rows (a solution on S^N is the prefix of S^{N+L}), zero after.
__global__ void k_pack64_prefix(const double2* __restrict__ u, int64_t n_u, int64_t size, double2* rec) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < size) rec[i] = i < n_u ? u[i] : make_double2(0.0, 0.0);
}

constexpr int kNormThreads = 256;

// Per block: sum |f - y|^2 and |f|^2 over a fixed row range, fixed tree.
__global__ void k_resid_partials(const double2* __restrict__ f, const double2* __restrict__ y, int64_t n,
                                 int64_t rows_per_block, double2* part) {
  __shared__ double2 sh[kNormThreads];
  const int64_t r0 = (int64_t)blockIdx.x * rows_per_block;
  const int64_t r1 = min(n, r0 + rows_per_block);
  double num = 0.0, den = 0.0;
  for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
    const double2 a = f[i], b = y[i];
    const double ex = a.x - b.x, ey = a.y - b.y;
    num += ex * ex + ey * ey;
    den += a.x * a.x + a.y * a.y;
  }
  sh[threadIdx.x] = make_double2(num, den);
  __syncthreads();
  for (int o = kNormThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      sh[threadIdx.x].x += sh[threadIdx.x + o].x;
      sh[threadIdx.x].y += sh[threadIdx.x + o].y;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void k_sum_partials(const double2* __restrict__ part, int n, double2* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double2 s = make_double2(0.0, 0.0);
  for (int i = 0; i < n; ++i) {
    s.x += part[i].x;
    s.y += part[i].y;
  }
  *out = s;
}

__global__ void k_ecoef_df(const double2* __restrict__ in, int64_t n, bool real, float4* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double2 c = real ? make_double2(reinterpret_cast<const double*>(in)[i], 0.0) : in[i];
  out[i] = cdf(df_split(c.x), df_split(c.y));
}

}  // namespace

ss_status ensure_ecoefdf(ss_stamp_s* s, cudaStream_t st) {
  if (s->ecoefdf.get()) return SS_OK;
  const int64_t n = s->n_ent + 1;
  SS_TRY(s->ecoefdf.alloc(n, st));
  k_ecoef_df<<<nblk(n), 256, 0, st>>>(s->ecoef64.get(), n, s->a_real, s->ecoefdf.get());
  SS_LAUNCH_CHECK();
  SS_CUDA(cudaStreamSynchronize(st));
  s->ecoefdf.settle();
  return SS_OK;
}

ss_status ensure_ecoefdf_half(ss_stamp_s* s, cudaStream_t st) {
  if (s->ecoefdf_h.get()) return SS_OK;
  const int64_t n = s->ecoef_h.n;
  SS_TRY(s->ecoefdf_h.alloc(n, st));
  k_ecoef_df<<<nblk(n), 256, 0, st>>>(s->ecoef_h.get(), n, s->a_real, s->ecoefdf_h.get());
  SS_LAUNCH_CHECK();
  SS_CUDA(cudaStreamSynchronize(st));
  s->ecoefdf_h.settle();
  return SS_OK;
}

OpView op_view(const ss_stamp_s* s) {
  OpView op;
  op.woff = s->slice_off.get();
  op.ent = s->ent.get();
  op.ecoef = s->ecoef64.get();
  op.ecoefdf = s->ecoefdf.get();
  op.colbits = colbits_of(s->jbits);
  op.colmask = colmask_of(s->jbits);
  op.realc = s->a_real;
  return op;
}

ss_status launch_pack64(const ss_stamp_s* s, const double2* u, cudaStream_t st) {
  k_pack64<<<nblk(s->size), 256, 0, st>>>(u, s->size, s->rec64.get());
  SS_LAUNCH_CHECK();
  return SS_OK;
}

ss_status launch_pack64_prefix(const ss_stamp_s* s, const double2* u, int64_t n_u, cudaStream_t st) {
  k_pack64_prefix<<<nblk(s->size), 256, 0, st>>>(u, n_u, s->size, s->rec64.get());
  SS_LAUNCH_CHECK();
  return SS_OK;
}

ss_status launch_apply64(const ss_stamp_s* s, double2* y, cudaStream_t st) {
  {
    ProfScope prof_("k_apply64", st, true);
    k_apply64<<<nblk(s->rows_pad), 256, 0, st>>>(op_view(s), s->size, s->rows_pad, s->rec64.get(), identity_row(s), y);
  }
  SS_LAUNCH_CHECK();
  return SS_OK;
}

ss_status launch_apply32(const ss_stamp_s* s, const float2* u, float2* y, cudaStream_t st) {
  if (s->adr) SS_FAIL(SS_ERR_INVALID, "the FP32 operator is not available for ADR stamps (use SS_FP64)");
  if (s->wide)
    {
      ProfScope prof_("k_apply32", st, true);
      k_apply32<true><<<nblk(s->rows_pad), 256, 0, st>>>(op_view(s), s->size, s->rows_pad, s->nw32.get(), u,
                                                         s->ca32.get(), s->pn32.get(), s->zero_idx, y);
    }
  else
    {
      ProfScope prof_("k_apply32", st, true);
      k_apply32<false><<<nblk(s->rows_pad), 256, 0, st>>>(op_view(s), s->size, s->rows_pad, s->nw32.get(), u,
                                                          s->ca32.get(), s->pn32.get(), s->zero_idx, y);
    }
  SS_LAUNCH_CHECK();
  return SS_OK;
}

}  // namespace ss

using namespace ss;

extern "C" ss_status galerkin_apply(ss_stamp s, const void* u, void* y, ss_precision prec, void* stream) {
  if (!s || !u || !y) SS_FAIL(SS_ERR_INVALID, "galerkin_apply: null argument");
  cudaStream_t st = as_stream(stream);
  if (s->size == 0) return SS_OK;
  if (prec == SS_FP64) {
    SS_TRY(launch_pack64(s, reinterpret_cast<const double2*>(u), st));
    return launch_apply64(s, reinterpret_cast<double2*>(y), st);
  }
  if (prec == SS_FP32)
    return launch_apply32(s, reinterpret_cast<const float2*>(u), reinterpret_cast<float2*>(y), st);
  SS_FAIL(SS_ERR_INVALID, "galerkin_apply: unknown precision %d", (int)prec);
}

extern "C" ss_status proxy_residual(ss_stamp s, const double* u_prefix, int64_t n_u, const double* f_on_S,
                                    double* out2, void* stream) {
  if (!s || !f_on_S || !out2 || (n_u > 0 && !u_prefix)) SS_FAIL(SS_ERR_INVALID, "proxy_residual: null argument");
  if (n_u < 0 || n_u > s->size) SS_FAIL(SS_ERR_INVALID, "proxy_residual: n_u = %lld outside [0, |S|]", (long long)n_u);
  cudaStream_t st = as_stream(stream);
  SS_TRY(launch_pack64_prefix(s, reinterpret_cast<const double2*>(u_prefix), n_u, st));
  DevBuf<double2> y, part, sum;
  const int64_t rows_per_block = 4096;
  const int nb = (int)std::max<int64_t>(1, (s->size + rows_per_block - 1) / rows_per_block);
  SS_TRY(y.alloc(s->size, st));
  SS_TRY(part.alloc(nb, st));
  SS_TRY(sum.alloc(1, st));
  SS_TRY(launch_apply64(s, y.get(), st));
  k_resid_partials<<<nb, kNormThreads, 0, st>>>(reinterpret_cast<const double2*>(f_on_S), y.get(), s->size,
                                                rows_per_block, part.get());
  k_sum_partials<<<1, 32, 0, st>>>(part.get(), nb, sum.get());
  SS_LAUNCH_CHECK();
  double2 h;
  SS_CUDA(cudaMemcpyAsync(&h, sum.get(), sizeof(h), cudaMemcpyDeviceToHost, st));
  SS_CUDA(cudaStreamSynchronize(st));
  out2[0] = h.x;
  out2[1] = h.y;
  return SS_OK;
}
