// Persistent Jacobi-preconditioned CG for L_{N,s} u = f (eq.
// SparseSpectralSFTEquation), one cooperative launch per solve.
//
// The rows of one or many instances form one row space cut into 32-row slices
// (one warp each).  The slices are split once into contiguous chunks (static
// work units); every CG phase walks the block's chunks, and a grid-wide barrier
// separates phases.  Inner products are reduced deterministically: per chunk
// and instance, each lane adds its rows in slice order, each warp folds its
// lanes with a fixed butterfly, the block adds its warps in order into one
// partial slot, and every block that needs a scalar sums that
// instance's slots with the same fixed warp reduction.  Per-instance state that
// crosses phases (rho, active flags) is double-buffered by iteration parity and
// written only by the instance's owner block (the one holding its first
// chunk), so no phase reads a value that is written in the same phase.
//
// Modes
//   FP64  plain CG on the FP64 operator.
//   FP32  iterative refinement: r = f - L x with the FP64 operator, then CG on
//         the FP32 operator with FP32 vectors (inner products reduced in FP64,
//         FP64 scalars) to a relative reduction inner_tol, then x += delta in
//         FP64.
//   ADR   BiCGStab on the FP64 operator of Remark ADR (not Hermitian), right
//         Jacobi preconditioning with its complex diagonal.
// The CG preconditioner is D_k = 4 pi^2 Re(a_hat_0) |k|^2 (the diagonal of L),
// 1 on the zero row and on padding rows.
#include <algorithm>
#include <mutex>
#include <cmath>
#include <type_traits>

#include "solve.cuh"

namespace ss {
namespace {

struct Smem {
  double acc[kMaxWarps][kMaxInstPerChunk][kNQ];
  double ca[kMaxInstPerChunk];
  double cb[kMaxInstPerChunk];
  double cc[kMaxInstPerChunk];
  double cd[kMaxInstPerChunk];
  float dfs[kMaxInstPerChunk][4];   // DF64 CG: alpha and beta as double-float
  int32_t flag[kMaxInstPerChunk];
};

__device__ __forceinline__ long long gtimer() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned arrive_acq_rel(unsigned* p) {
  unsigned v;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid-wide barrier (all blocks are co-resident: cooperative launch).  The
// arrival is a release-acquire add on the count; the last block resets the
// count and publishes the next generation with a release add, which the others
// poll with acquire loads (no sleep between polls: the waits are short).  A
// wait longer than spin_limit ns sets SS_ERR_TIMEOUT and returns false; so
// does any error already posted by another block.
__device__ bool grid_sync(const SolveParams& P) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned* gen = P.bar + 1;
    const unsigned g = ld_acquire(gen);
    const unsigned arrived = arrive_acq_rel(P.bar) + 1u;
    int ok = 1;
    if (arrived == gridDim.x) {
      asm volatile("st.relaxed.gpu.global.u32 [%0], 0;" ::"l"(P.bar) : "memory");
      asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(gen) : "memory");
    } else {
      const long long t0 = gtimer();
      for (unsigned it = 1; ld_acquire(gen) == g; ++it) {
        if (it == 1 || (it & 255u) == 0) {
          if (*(volatile int*)P.err) { ok = 0; break; }
          if (gtimer() - t0 > P.spin_limit) {
            atomicCAS(P.err, 0, (int)SS_ERR_TIMEOUT);
            ok = 0;
            break;
          }
        }
      }
    }
    s_ok = ok;   // an error posted elsewhere stops the waiters in their poll loop
  }
  __syncthreads();
  return s_ok != 0;
}

// Counter read by one thread and broadcast to the block (uniform control flow).
__device__ int block_counter(const SolveParams& P, int idx) {
  __shared__ int s_cnt;
  __syncthreads();
  if (threadIdx.x == 0) s_cnt = atomicAdd(P.counters + idx, 0);
  __syncthreads();
  return s_cnt;
}

// Sums of the kNQ quantities over the partial slots of instance i, by one warp
// in a fixed order (lane-strided, then a fixed butterfly; lane 0's result is
// broadcast), so every block that needs them gets the same bits.  Loads of four
// slots per lane are issued before they are added.
__device__ void inst_sums(const SolveParams& P, int i, double out[kNQ]) {
  const int lane = threadIdx.x & 31;
  const SolveInst& in = P.inst[i];
  const int len = in.c_last - in.c_first + 1;
  const double2* base = reinterpret_cast<const double2*>(P.part + (int64_t)in.part_base * kNQ);
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  int c = lane;
  for (; c + 96 < len; c += 128) {
    double2 x[8];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      x[2 * u] = __ldcg(base + 2 * (c + 32 * u));
      x[2 * u + 1] = __ldcg(base + 2 * (c + 32 * u) + 1);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      a0 += x[2 * u].x;
      a1 += x[2 * u].y;
      a2 += x[2 * u + 1].x;
      a3 += x[2 * u + 1].y;
    }
  }
  for (; c < len; c += 32) {
    const double2 x0 = __ldcg(base + 2 * c), x1 = __ldcg(base + 2 * c + 1);
    a0 += x0.x;
    a1 += x0.y;
    a2 += x1.x;
    a3 += x1.y;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a0 += __shfl_xor_sync(0xffffffffu, a0, o);
    a1 += __shfl_xor_sync(0xffffffffu, a1, o);
    a2 += __shfl_xor_sync(0xffffffffu, a2, o);
    a3 += __shfl_xor_sync(0xffffffffu, a3, o);
  }
  out[0] = __shfl_sync(0xffffffffu, a0, 0);
  out[1] = __shfl_sync(0xffffffffu, a1, 0);
  out[2] = __shfl_sync(0xffffffffu, a2, 0);
  out[3] = __shfl_sync(0xffffffffu, a3, 0);
}

__device__ __forceinline__ double warp_reduce(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Lane accumulators of run_phase: FP64; double-float for the DF64 CG and FP32
// for the FP32 inner solve (kept on the FP32 pipe, converted to FP64 once per
// warp fold).
__device__ __forceinline__ void acc_add(double& a, double b) { a += b; }
__device__ __forceinline__ void acc_add(float& a, float b) { a += b; }
__device__ __forceinline__ double acc_fold(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return (double)v;
}
__device__ __forceinline__ void acc_add(DF& a, DF b) { a = df_add(a, b); }
__device__ __forceinline__ double acc_fold(double v) { return warp_reduce(v); }
__device__ __forceinline__ double acc_fold(DF v) { return df_to_double(df_warp_sum(v)); }

// Run one phase over the block's chunks.  Partial sums: every lane adds its
// rows' values in slice order, the warp folds its lanes once per run of slices
// of one instance (fixed butterfly), the block adds its warps in order.
//   scal(c, ch, k, i, owner): per instance of the chunk (one warp each), fills
//                             sm.ca/cb/flag[k] and does the owner's bookkeeping;
//   row(g, s, lane, i, k, vals): per row, sets vals[q] for q in qmask; with
//                             INTO the row adds to the lane's running sums
//                             itself (vals is then the running sums: the FP64
//                             CG accumulates its inner products by FMA, two
//                             FP64 operations per complex product instead of
//                             three).
template <class Acc = double, bool INTO = false, class Scal, class Row>
__device__ void run_phase(const SolveParams& P, Smem& sm, unsigned qmask, Scal scal, Row row) {
  const int nw = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int c = blockIdx.x; c < P.n_chunks; c += gridDim.x) {
    const Chunk ch = P.chunk[c];
    const int ni = ch.inst1 - ch.inst0 + 1;
    if (qmask)
      for (int t = threadIdx.x; t < nw * kMaxInstPerChunk * kNQ; t += blockDim.x)
        (&sm.acc[0][0][0])[t] = 0.0;
    for (int k = warp; k < ni; k += nw) {
      const int i = ch.inst0 + k;
      scal(c, ch, k, i, c == P.inst[i].c_first, lane);
    }
    __syncthreads();
    int cur_k = -1;
    Acc run[kNQ] = {};
    for (int64_t s = ch.s0 + warp; s < ch.s1; s += nw) {
      const int i = P.slice_inst ? __ldg(P.slice_inst + s) : 0;
      const int k = i - ch.inst0;
      const int64_t g = s * kSlice + lane;
      if constexpr (INTO) {
        if (qmask && k != cur_k) {
          if (cur_k >= 0) {
#pragma unroll
            for (int q = 0; q < kNQ; ++q) {
              const double t = (qmask & (1u << q)) ? acc_fold(run[q]) : 0.0;
              if (lane == 0) sm.acc[warp][cur_k][q] += t;
            }
          }
          for (int q = 0; q < kNQ; ++q) run[q] = Acc{};
          cur_k = k;
        }
        row(g, s, lane, i, k, run);
        continue;
      }
      Acc vals[kNQ] = {};
      row(g, s, lane, i, k, vals);
      if (qmask) {
        // lanes keep their own running sums; the butterfly runs once per
        // instance run of the warp (warp-uniform branch), not once per slice
        if (k != cur_k) {
          if (cur_k >= 0) {
#pragma unroll
            for (int q = 0; q < kNQ; ++q) {
              const double t = (qmask & (1u << q)) ? acc_fold(run[q]) : 0.0;
              if (lane == 0) sm.acc[warp][cur_k][q] += t;
            }
          }
          for (int q = 0; q < kNQ; ++q) run[q] = Acc{};
          cur_k = k;
        }
#pragma unroll
        for (int q = 0; q < kNQ; ++q)
          if (qmask & (1u << q)) acc_add(run[q], vals[q]);
      }
    }
    if (qmask && cur_k >= 0) {
#pragma unroll
      for (int q = 0; q < kNQ; ++q) {
        const double t = (qmask & (1u << q)) ? acc_fold(run[q]) : 0.0;
        if (lane == 0) sm.acc[warp][cur_k][q] += t;
      }
    }
    __syncthreads();
    if (qmask) {
      for (int t = threadIdx.x; t < ni * kNQ; t += blockDim.x) {
        const int k = t / kNQ, q = t % kNQ;
        if (!(qmask & (1u << q))) continue;
        double v = 0.0;
        for (int w = 0; w < nw; ++w) v += sm.acc[w][k][q];
        const SolveInst& in = P.inst[ch.inst0 + k];
        P.part[(int64_t)(in.part_base + (c - in.c_first)) * kNQ + q] = v;
      }
    }
    __syncthreads();
  }
}

// Row-wise phase of one instance (no neighbour reads, no partial sums): with
// P.rows_slices > 0 the slices are split evenly over the blocks, so that the
// work follows the rows rather than the entries the apply chunks are balanced
// by; block 0 does the owner's bookkeeping.  Otherwise the chunks of run_phase.
template <class Scal, class Row>
__device__ void run_rows(const SolveParams& P, Smem& sm, Scal scal, Row row) {
  if (P.rows_slices <= 0) {
    run_phase(P, sm, 0u, scal, row);
    return;
  }
  const int nw = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t s0 = P.rows_slices * blockIdx.x / gridDim.x, s1 = P.rows_slices * (blockIdx.x + 1) / gridDim.x;
  const Chunk ch{s0, s1, 0, 0};
  if (warp == 0) scal(0, ch, 0, 0, blockIdx.x == 0, lane);
  __syncthreads();
  for (int64_t s = s0 + warp; s < s1; s += nw) {
    double vals[kNQ] = {};
    row(s * kSlice + lane, s, lane, 0, 0, vals);
  }
  __syncthreads();
}

// Power-of-two scale of an inner (FP32) solve: the residual handed to it has
// RMS entry near 1, so that the FP32 inner products r.D^-1 r and p.Lp stay far
// from FP32 underflow however small the outer residual and however large the
// Jacobi diagonal 4 pi^2 a_0 |k|^2 get.  Exact in FP64; 1 when rr = 0.
__device__ __forceinline__ double inner_scale(double rr, int64_t rows) {
  if (!(rr > 0.0)) return 1.0;
  return ldexp(1.0, -ilogb(sqrt(rr / (double)(rows > 0 ? rows : 1))));
}

__device__ __forceinline__ double jacobi(const SolveParams& P, const SolveInst& in, int64_t g) {
  const int64_t nk = __ldg(P.norm + g);
  return nk > 0 ? in.dscale * (double)nk : 1.0;
}

__device__ __forceinline__ float jacobi32(const SolveParams& P, const SolveInst& in, int64_t g) {
  const int64_t nk = __ldg(P.norm + g);
  return nk > 0 ? (float)in.dscale * (float)nk : 1.0f;
}

__device__ __forceinline__ double2 f_at(const SolveInst& in, int64_t g) {
  const int64_t l = g - in.row0;
  return l < in.rows ? in.f[l] : make_double2(0.0, 0.0);
}

__device__ __forceinline__ double2 apply64_row(const SolveParams& P, const SolveInst& in, int64_t s, int lane,
                                               int64_t g, const double2* rec) {
  if (g == in.zero_row) return __ldcg(rec + g);
  return row_apply64<true>(P.op, s, lane, rec);
}

__device__ __forceinline__ float2 apply32_row(const SolveParams& P, const SolveInst& in, int64_t s, int lane,
                                              int64_t g) {
  if (g == in.zero_row) {
    const float4 v = __ldcg(P.urec32 + g);
    return make_float2(v.x, v.y);
  }
  return row_apply32<true>(P.op, s, lane, __ldg(P.norm + g), in.wide != 0, P.urec32, P.ca32 + in.coef_off,
                           P.pn + in.coef_off);
}

__device__ __forceinline__ void owner_done(const SolveParams& P, InstState& st, int status) {
  st.status = status;
  atomicAdd(P.counters + 0, 1);
}

// ------------------------------------------------------------ CG recurrences
//
// Both modes use the Chronopoulos-Gear form of preconditioned CG, which needs
// one reduction per iteration (two grid barriers instead of three):
//   p_i = u_i + beta_i p_{i-1},  s_i = w_i + beta_i s_{i-1}   (s_i = L p_i)
//   x_{i+1} = x_i + alpha_i p_i, r_{i+1} = r_i - alpha_i s_i, u_{i+1} = D^-1 r_{i+1}
//   w_{i+1} = L u_{i+1};  gamma = <r,u>, delta = <w,u>
//   beta_{i+1} = gamma_{i+1}/gamma_i,
//   alpha_{i+1} = gamma_{i+1} / (delta_{i+1} - beta_{i+1} gamma_{i+1} / alpha_i),
// with beta_0 = 0, alpha_0 = gamma_0 / delta_0.  Phase X does the scalars and
// the vector updates, phase Y the operator and the three inner products
// (gamma, delta, |r|^2).  Partial slot q3 holds |f|^2.

struct Coeffs {
  double alpha, beta;
};

__device__ __forceinline__ Coeffs cg_coeffs(int it, double gam, double del, double gam_prev, double alpha_prev) {
  Coeffs c;
  if (it == 0) {
    c.beta = 0.0;
    c.alpha = gam / del;
  } else {
    c.beta = gam / gam_prev;
    c.alpha = gam / (del - c.beta * gam / alpha_prev);
  }
  return c;
}

// --------------------------------------------------------------- FP64 CG

__device__ void solve_fp64(const SolveParams& P, Smem& sm) {
  const double tol2 = P.tol * P.tol;
  auto noscal = [](int, const Chunk&, int, int, bool, int) {};
  // The residual is kept as r = D u (D the Jacobi diagonal, u = D^-1 r the
  // preconditioned residual and the gathered record): the vector phase
  // updates u = u - alpha D^-1 s directly, and the apply phase forms
  // <r, u> = sum D |u|^2 and <r, r> = sum D^2 |u|^2.  No r vector is read or
  // written (152 instead of 184 bytes per row and iteration in the vector
  // phase); P.r holds D (one double per row).
  double* dg = reinterpret_cast<double*>(P.r);
  // x = 0, u = D^-1 f, p = s = 0; |f|^2
  run_phase(P, sm, 0b1000u, noscal, [&](int64_t g, int64_t, int, int i, int, double* v) {
    const SolveInst& in = P.inst[i];
    const double2 f = f_at(in, g);
    const double dk = jacobi(P, in, g), rD = 1.0 / dk;
    P.rdiag[g] = rD;
    dg[g] = dk;
    P.xrec[g] = make_double2(0.0, 0.0);
    P.urec64[g] = make_double2(f.x * rD, f.y * rD);
    P.pd[g] = make_double2(0.0, 0.0);
    P.sd[g] = make_double2(0.0, 0.0);
    v[3] = f.x * f.x + f.y * f.y;
  });
  if (!grid_sync(P)) return;
  auto phase_y = [&](unsigned par) {
    run_phase<double, true>(P, sm, 0b0111u, [&](int, const Chunk&, int k, int i, bool, int lane) {
      if (lane == 0) sm.flag[k] = par > 1 ? 1 : __ldcg(&P.state[i].act[par]);
    }, [&](int64_t g, int64_t s, int lane, int i, int k, double* v) {
      if (!sm.flag[k]) return;
      const SolveInst& in = P.inst[i];
      const double2 w = apply64_row(P, in, s, lane, g, P.urec64);
      const double2 u = P.urec64[g];
      const double dk = dg[g];
      P.w64[g] = w;
      const double du = dk * fma(u.y, u.y, u.x * u.x);   // D |u|^2 = <r, u> of this row
      v[0] += du;
      v[1] = fma(w.y, u.y, fma(w.x, u.x, v[1]));
      v[2] = fma(dk, du, v[2]);                           // |r|^2 = D^2 |u|^2
    });
  };
  phase_y(2);   // every instance
  if (!grid_sync(P)) return;
  for (int it = 0;; ++it) {
    const int cur = it & 1, nxt = cur ^ 1;
    run_rows(P, sm, [&](int, const Chunk&, int k, int i, bool owner, int lane) {
      double t[kNQ];
      inst_sums(P, i, t);
      if (lane == 0) {
        InstState& st = P.state[i];
        const int act = it == 0 ? 1 : __ldcg(&st.act[cur]);
        const double bb = it == 0 ? t[3] : __ldcg(&st.bb);
        const bool conv = t[2] <= tol2 * bb;
        const bool cap = it >= P.max_iter;
        const Coeffs cf = cg_coeffs(it, t[0], t[1], it ? __ldcg(&st.rho[cur]) : 0.0,
                                    it ? __ldcg(&st.alpha[cur]) : 0.0);
        const bool go = act && !conv && !cap;
        sm.flag[k] = go;
        sm.ca[k] = cf.alpha;
        sm.cb[k] = cf.beta;
        if (owner) {
          if (it == 0) {
            st.bb = bb;
            st.applies = 1;
            st.outer_iters = 1;
          }
          st.act[nxt] = go;
          st.rho[nxt] = t[0];
          st.alpha[nxt] = cf.alpha;
          if (act) {
            st.rr = t[2];
            st.iters = it;
            if (conv) owner_done(P, st, SS_OK);
            else if (cap) owner_done(P, st, SS_ERR_NOT_CONVERGED);
            else st.applies += 1;
          }
        }
      }
    }, [&](int64_t g, int64_t, int, int i, int k, double*) {
      if (!sm.flag[k]) return;
      const double a = sm.ca[k], b = sm.cb[k];
      double2 u = P.urec64[g];
      const double2 w = P.w64[g];
      double2 p = P.pd[g], sv = P.sd[g], x = P.xrec[g];
      p.x = u.x + b * p.x; p.y = u.y + b * p.y;
      sv.x = w.x + b * sv.x; sv.y = w.y + b * sv.y;
      x.x += a * p.x; x.y += a * p.y;
      const double t = a * P.rdiag[g];   // u - alpha D^-1 s = D^-1 (r - alpha s)
      u.x = fma(-t, sv.x, u.x);
      u.y = fma(-t, sv.y, u.y);
      P.pd[g] = p;
      P.sd[g] = sv;
      P.xrec[g] = x;
      P.urec64[g] = u;
    });
    if (!grid_sync(P)) return;
    if (block_counter(P, 0) >= P.n_inst) break;
    phase_y(nxt);
    if (!grid_sync(P)) return;
  }
  // true residual f - L x in FP64, and the output
  run_phase(P, sm, 0b0100u, noscal, [&](int64_t g, int64_t s, int lane, int i, int, double* v) {
    const SolveInst& in = P.inst[i];
    const double2 y = apply64_row(P, in, s, lane, g, P.xrec);
    const double2 f = f_at(in, g);
    const double2 r = make_double2(f.x - y.x, f.y - y.y);
    v[2] = r.x * r.x + r.y * r.y;
    const int64_t l = g - in.row0;
    if (l < in.rows) in.u[l] = P.xrec[g];
  });
  if (!grid_sync(P)) return;
  run_phase(P, sm, 0u, [&](int, const Chunk&, int, int i, bool owner, int lane) {
    double t[kNQ];
    inst_sums(P, i, t);
    if (owner && lane == 0) {
      P.state[i].rr = t[2];
      P.state[i].applies += 1;
    }
  }, [](int64_t, int64_t, int, int, int, double*) {});
}

// ------------------------------------------------------------ DF64 CG
//
// The FP64 CG above in double-float arithmetic: vectors, records, entry
// coefficients and the Jacobi factors are unevaluated float pairs, every
// product and sum is an error-free-transformation double-float operation on
// the FP32 pipe (about 2^-48 relative each), partial sums stay double-float
// until the warp fold; the CG scalars, the stopping test and the final
// residual f - L x are FP64.  Same recurrences, same phases.

__device__ void solve_df64(const SolveParams& P, Smem& sm) {
  const double tol2 = P.tol * P.tol;
  auto noscal = [](int, const Chunk&, int, int, bool, int) {};
  float4* r4 = reinterpret_cast<float4*>(P.r);
  float4* w4 = reinterpret_cast<float4*>(P.w64);
  float4* p4 = reinterpret_cast<float4*>(P.pd);
  float4* s4 = reinterpret_cast<float4*>(P.sd);
  // r = f, x = 0, u = D^-1 r, p = s = 0; |f|^2 (FP64)
  run_phase(P, sm, 0b1000u, noscal, [&](int64_t g, int64_t, int, int i, int, double* v) {
    const SolveInst& in = P.inst[i];
    const double2 f = f_at(in, g);
    const DF rD = df_split(1.0 / jacobi(P, in, g));
    P.d32[g] = make_float2(rD.hi, rD.lo);
    const DF fr = df_split(f.x), fi = df_split(f.y);
    r4[g] = cdf(fr, fi);
    P.xdf[g] = make_float4(0.f, 0.f, 0.f, 0.f);
    P.udf[g] = cdf(df_mul(rD, fr), df_mul(rD, fi));
    p4[g] = make_float4(0.f, 0.f, 0.f, 0.f);
    s4[g] = make_float4(0.f, 0.f, 0.f, 0.f);
    v[3] = f.x * f.x + f.y * f.y;
  });
  if (!grid_sync(P)) return;
  auto phase_y = [&](unsigned par) {
    run_phase<DF>(P, sm, 0b0111u, [&](int, const Chunk&, int k, int i, bool, int lane) {
      if (lane == 0) sm.flag[k] = par > 1 ? 1 : __ldcg(&P.state[i].act[par]);
    }, [&](int64_t g, int64_t s, int lane, int i, int k, DF* v) {
      if (!sm.flag[k]) return;
      const SolveInst& in = P.inst[i];
      const float4 w = (g == in.zero_row) ? __ldcg(P.udf + g) : row_applydf<true>(P.op, s, lane, P.udf);
      const float4 u = P.udf[g], r = r4[g];
      w4[g] = w;
      DF a{0.f, 0.f}, b{0.f, 0.f}, c{0.f, 0.f};
      df_fma(a, re_of(r), re_of(u));
      df_fma(a, im_of(r), im_of(u));
      df_fma(b, re_of(w), re_of(u));
      df_fma(b, im_of(w), im_of(u));
      df_fma(c, re_of(r), re_of(r));
      df_fma(c, im_of(r), im_of(r));
      v[0] = a;
      v[1] = b;
      v[2] = c;
    });
  };
  phase_y(2);   // every instance
  if (!grid_sync(P)) return;
  for (int it = 0;; ++it) {
    const int cur = it & 1, nxt = cur ^ 1;
    run_rows(P, sm, [&](int, const Chunk&, int k, int i, bool owner, int lane) {
      double t[kNQ];
      inst_sums(P, i, t);
      if (lane == 0) {
        InstState& st = P.state[i];
        const int act = it == 0 ? 1 : __ldcg(&st.act[cur]);
        const double bb = it == 0 ? t[3] : __ldcg(&st.bb);
        const bool conv = t[2] <= tol2 * bb;
        const bool cap = it >= P.max_iter;
        const Coeffs cf = cg_coeffs(it, t[0], t[1], it ? __ldcg(&st.rho[cur]) : 0.0,
                                    it ? __ldcg(&st.alpha[cur]) : 0.0);
        const bool go = act && !conv && !cap;
        sm.flag[k] = go;
        const DF a = df_split(cf.alpha), b = df_split(cf.beta);
        sm.dfs[k][0] = a.hi;
        sm.dfs[k][1] = a.lo;
        sm.dfs[k][2] = b.hi;
        sm.dfs[k][3] = b.lo;
        if (owner) {
          if (it == 0) {
            st.bb = bb;
            st.applies = 1;
            st.outer_iters = 1;
          }
          st.act[nxt] = go;
          st.rho[nxt] = t[0];
          st.alpha[nxt] = cf.alpha;
          if (act) {
            st.rr = t[2];
            st.iters = it;
            if (conv) owner_done(P, st, SS_OK);
            else if (cap) owner_done(P, st, SS_ERR_NOT_CONVERGED);
            else st.applies += 1;
          }
        }
      }
    }, [&](int64_t g, int64_t, int, int, int k, double*) {
      if (!sm.flag[k]) return;
      const DF a{sm.dfs[k][0], sm.dfs[k][1]}, b{sm.dfs[k][2], sm.dfs[k][3]};
      const float4 u = P.udf[g], w = w4[g], po = p4[g], so = s4[g], xo = P.xdf[g], ro = r4[g];
      // p = u + beta p, s = w + beta s
      DF pr = re_of(u), pi = im_of(u), sr = re_of(w), si = im_of(w);
      df_fma(pr, b, re_of(po));
      df_fma(pi, b, im_of(po));
      df_fma(sr, b, re_of(so));
      df_fma(si, b, im_of(so));
      // x += alpha p, r -= alpha s
      DF xr = re_of(xo), xi = im_of(xo), rr = re_of(ro), ri = im_of(ro);
      df_fma(xr, a, pr);
      df_fma(xi, a, pi);
      const DF na = df_neg(a);
      df_fma(rr, na, sr);
      df_fma(ri, na, si);
      const float2 d = P.d32[g];
      const DF rD{d.x, d.y};
      p4[g] = cdf(pr, pi);
      s4[g] = cdf(sr, si);
      P.xdf[g] = cdf(xr, xi);
      r4[g] = cdf(rr, ri);
      P.udf[g] = cdf(df_mul(rD, rr), df_mul(rD, ri));
    });
    if (!grid_sync(P)) return;
    if (block_counter(P, 0) >= P.n_inst) break;
    phase_y(nxt);
    if (!grid_sync(P)) return;
  }
  // true residual f - L x (double-float operator, FP64 difference), and the output
  run_phase(P, sm, 0b0100u, noscal, [&](int64_t g, int64_t s, int lane, int i, int, double* v) {
    const SolveInst& in = P.inst[i];
    const float4 y4 = (g == in.zero_row) ? __ldcg(P.xdf + g) : row_applydf<true>(P.op, s, lane, P.xdf);
    const double2 f = f_at(in, g);
    const double2 r = make_double2(f.x - df_to_double(re_of(y4)), f.y - df_to_double(im_of(y4)));
    v[2] = r.x * r.x + r.y * r.y;
    const int64_t l = g - in.row0;
    const float4 x = P.xdf[g];
    if (l < in.rows) in.u[l] = make_double2(df_to_double(re_of(x)), df_to_double(im_of(x)));
  });
  if (!grid_sync(P)) return;
  run_phase(P, sm, 0u, [&](int, const Chunk&, int, int i, bool owner, int lane) {
    double t[kNQ];
    inst_sums(P, i, t);
    if (owner && lane == 0) {
      P.state[i].rr = t[2];
      P.state[i].applies += 1;
    }
  }, [](int64_t, int64_t, int, int, int, double*) {});
}

// ------------------------------------------------- FP32 CG in FP64 refinement

__device__ void solve_refined(const SolveParams& P, Smem& sm) {
  const double tol2 = P.tol * P.tol, itol2 = P.inner_tol * P.inner_tol;
  auto noscal = [](int, const Chunk&, int, int, bool, int) {};
  // x = 0; |f|^2
  run_phase(P, sm, 0b1000u, noscal, [&](int64_t g, int64_t, int, int i, int, double* v) {
    const double2 f = f_at(P.inst[i], g);
    P.xrec[g] = make_double2(0.0, 0.0);
    v[3] = f.x * f.x + f.y * f.y;
  });
  if (!grid_sync(P)) return;
  run_phase(P, sm, 0u, [&](int, const Chunk&, int, int i, bool owner, int lane) {
    double t[kNQ];
    inst_sums(P, i, t);
    if (owner && lane == 0) {
      InstState& st = P.state[i];
      st.bb = t[3];
      st.rr = t[3];
      st.act[0] = t[3] > 0.0;
      if (!(t[3] > 0.0)) owner_done(P, st, SS_OK);
    }
  }, [](int64_t, int64_t, int, int, int, double*) {});
  if (!grid_sync(P)) return;
  for (int ot = 0;; ++ot) {
    const int ocur = ot & 1, onxt = ocur ^ 1;
    // rhat = f - L64 x, |rhat|^2
    run_phase(P, sm, 0b0100u, [&](int, const Chunk&, int k, int i, bool owner, int lane) {
      if (lane == 0) {
        sm.flag[k] = __ldcg(&P.state[i].act[ocur]);
        if (owner && sm.flag[k]) P.state[i].applies += 1;
      }
    }, [&](int64_t g, int64_t s, int lane, int i, int k, double* v) {
      if (!sm.flag[k]) return;
      const SolveInst& in = P.inst[i];
      const double2 y = apply64_row(P, in, s, lane, g, P.xrec);
      const double2 f = f_at(in, g);
      const double2 r = make_double2(f.x - y.x, f.y - y.y);
      P.rhat[g] = r;
      v[2] = r.x * r.x + r.y * r.y;
    });
    if (!grid_sync(P)) return;
    // outer test; inner start (all FP32): r = rhat * scale, delta = 0, u = D^-1 r, p = s = 0
    run_phase(P, sm, 0u, [&](int, const Chunk&, int k, int i, bool owner, int lane) {
      double t[kNQ];
      inst_sums(P, i, t);
      if (lane == 0) {
        InstState& st = P.state[i];
        const int act = __ldcg(&st.act[ocur]);
        const bool conv = t[2] <= tol2 * __ldcg(&st.bb);
        const bool cap = ot >= P.max_outer;
        const bool go = act && !conv && !cap;
        sm.flag[k] = go;
        sm.ca[k] = inner_scale(t[2], P.inst[i].rows);
        if (owner) {
          st.act[onxt] = go;
          st.inn[0] = go;
          if (act) {
            st.rr = t[2];
            if (conv) owner_done(P, st, SS_OK);
            else if (cap) owner_done(P, st, SS_ERR_NOT_CONVERGED);
            else {
              st.outer_iters = ot + 1;
              st.applies += 1;
              atomicAdd(P.counters + 1, 1);
            }
          }
        }
      }
    }, [&](int64_t g, int64_t, int, int i, int k, double*) {
      if (!sm.flag[k]) return;
      const SolveInst& in = P.inst[i];
      const double2 rh = P.rhat[g];
      const double sc = sm.ca[k];
      const float2 r = make_float2((float)(rh.x * sc), (float)(rh.y * sc));
      const float rD = 1.0f / jacobi32(P, in, g);
      P.r32[g] = r;
      P.d32[g] = make_float2(0.f, 0.f);
      P.p32[g] = make_float2(0.f, 0.f);
      P.s32[g] = make_float2(0.f, 0.f);
      reinterpret_cast<float2*>(P.urec32 + g)[0] = make_float2(r.x * rD, r.y * rD);
    });
    if (!grid_sync(P)) return;
    if (block_counter(P, 0) >= P.n_inst) break;
    // inner CG on the FP32 operator with FP32 vectors; inner products are
    // formed per row in FP32 and reduced in FP64, scalars stay FP64
    // the inner products of the FP32 inner solve (relative tolerance 1e-5)
    // are summed in FP32 per lane and in FP64 from the warp fold on
    auto phase_y = [&](int par) {
      run_phase<float>(P, sm, 0b0111u, [&](int, const Chunk&, int k, int i, bool, int lane) {
        if (lane == 0) sm.flag[k] = __ldcg(&P.state[i].inn[par]);
      }, [&](int64_t g, int64_t s, int lane, int i, int k, float* v) {
        if (!sm.flag[k]) return;
        const SolveInst& in = P.inst[i];
        const float2 w = apply32_row(P, in, s, lane, g);
        const float4 u = P.urec32[g];
        const float2 r = P.r32[g];
        P.w32[g] = w;
        v[0] = r.x * u.x + r.y * u.y;
        v[1] = w.x * u.x + w.y * u.y;
        v[2] = r.x * r.x + r.y * r.y;
      });
    };
    phase_y(0);
    if (!grid_sync(P)) return;
    for (int it = 0;; ++it) {
      const int cur = it & 1, nxt = cur ^ 1;
      run_phase(P, sm, 0u, [&](int, const Chunk&, int k, int i, bool owner, int lane) {
        double t[kNQ];
        inst_sums(P, i, t);
        if (lane == 0) {
          InstState& st = P.state[i];
          const int act = __ldcg(&st.inn[cur]);
          const double rr = __ldcg(&st.rr), sc = inner_scale(rr, P.inst[i].rows);
          const bool conv = t[2] <= itol2 * rr * sc * sc;     // r32 carries the scale
          const bool cap = it >= P.max_inner;
          const Coeffs cf = cg_coeffs(it, t[0], t[1], it ? __ldcg(&st.rho[cur]) : 0.0,
                                      it ? __ldcg(&st.alpha[cur]) : 0.0);
          const bool go = act && !conv && !cap;
          sm.flag[k] = go;
          sm.ca[k] = cf.alpha;
          sm.cb[k] = cf.beta;
          if (owner) {
            st.inn[nxt] = go;
            st.rho[nxt] = t[0];
            st.alpha[nxt] = cf.alpha;
            if (act) {
              if (go) {
                st.inner_iters += 1;
                st.applies += 1;
              } else {
                atomicAdd(P.counters + 2, 1);
              }
            }
          }
        }
      }, [&](int64_t g, int64_t, int, int i, int k, double*) {
        if (!sm.flag[k]) return;
        const SolveInst& in = P.inst[i];
        const float a = (float)sm.ca[k], b = (float)sm.cb[k];
        const float4 u = P.urec32[g];
        const float2 w = P.w32[g];
        float2 p = P.p32[g], sv = P.s32[g], dl = P.d32[g], r = P.r32[g];
        p.x = fmaf(b, p.x, u.x); p.y = fmaf(b, p.y, u.y);
        sv.x = fmaf(b, sv.x, w.x); sv.y = fmaf(b, sv.y, w.y);
        dl.x = fmaf(a, p.x, dl.x); dl.y = fmaf(a, p.y, dl.y);
        r.x = fmaf(-a, sv.x, r.x); r.y = fmaf(-a, sv.y, r.y);
        const float rD = 1.0f / jacobi32(P, in, g);
        P.p32[g] = p;
        P.s32[g] = sv;
        P.d32[g] = dl;
        P.r32[g] = r;
        reinterpret_cast<float2*>(P.urec32 + g)[0] = make_float2(r.x * rD, r.y * rD);
      });
      if (!grid_sync(P)) return;
      if (block_counter(P, 2) >= block_counter(P, 1)) break;
      phase_y(nxt);
      if (!grid_sync(P)) return;
    }
    // x += delta
    run_phase(P, sm, 0u, [&](int, const Chunk&, int k, int i, bool, int lane) {
      if (lane == 0) {
        sm.flag[k] = __ldcg(&P.state[i].act[onxt]);
        sm.ca[k] = 1.0 / inner_scale(__ldcg(&P.state[i].rr), P.inst[i].rows);
      }
    }, [&](int64_t g, int64_t, int, int, int k, double*) {
      if (!sm.flag[k]) return;
      double2 x = P.xrec[g];
      const float2 dl = P.d32[g];
      const double us = sm.ca[k];
      x.x += (double)dl.x * us;
      x.y += (double)dl.y * us;
      P.xrec[g] = x;
    });
    if (!grid_sync(P)) return;
  }
  run_phase(P, sm, 0u, noscal, [&](int64_t g, int64_t, int, int i, int, double*) {
    const SolveInst& in = P.inst[i];
    const int64_t l = g - in.row0;
    if (l < in.rows) in.u[l] = P.xrec[g];
  });
}

// ------------------------------------------------- BiCGStab (ADR operator)
//
// The operator of Remark ADR is not Hermitian.  BiCGStab (van der Vorst, 1992)
// with right Jacobi preconditioning y = D^-1 p, D = diag L (complex), and the
// shadow residual r^ = r_0 = f:
//   rho = <r^, r>, beta = (rho / rho_prev) (alpha / omega)
//   p = r + beta (p - omega v),  v = L D^-1 p
//   alpha = rho / <r^, v>,  s = r - alpha v,  x += alpha D^-1 p
//   t = L D^-1 s,  omega = <t, s> / <t, t>,  x += omega D^-1 s,  r = s - omega t
// with <a, b> = sum conj(a) b.  Five phases per iteration, each closed by a
// grid barrier; every block recomputes the scalars from the deterministic
// partial sums, and the owner keeps rho, alpha and omega by iteration parity.
// The half step stops the iteration when |s| already meets the tolerance
// (x = x + alpha y is then the answer).  A vanishing or non-finite scalar
// restarts the direction (beta = 0) or skips the step (alpha or omega = 0);
// the iteration cap then reports non-convergence.

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  const double n = b.x * b.x + b.y * b.y;
  if (n == 0.0) return make_double2(0.0, 0.0);
  return make_double2((a.x * b.x + a.y * b.y) / n, (a.y * b.x - a.x * b.y) / n);
}
__device__ __forceinline__ double2 finite_or_zero(double2 a) {
  return (isfinite(a.x) && isfinite(a.y)) ? a : make_double2(0.0, 0.0);
}
// conj(a) b
__device__ __forceinline__ double2 cdot(double2 a, double2 b) {
  return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}

__device__ void solve_bicgstab(const SolveParams& P, Smem& sm) {
  const double tol2 = P.tol * P.tol;
  auto noscal = [](int, const Chunk&, int, int, bool, int) {};
  // x = 0, r = r^ = f, p = v = 0, dlt = D^-1;  <r^, r> = |f|^2 + 0 i (q0, q1), |r|^2 (q2), |f|^2 (q3).
  // q1 is written (as zero) too: the first iteration reads rho = (q0, q1),
  // and a slot left out would hold whatever an earlier phase or solve left there.
  run_phase(P, sm, 0b1111u, noscal, [&](int64_t g, int64_t, int, int i, int, double* v) {
    const double2 f = f_at(P.inst[i], g);
    P.xrec[g] = make_double2(0.0, 0.0);
    P.r[g] = f;
    P.rhat[g] = f;
    P.pd[g] = make_double2(0.0, 0.0);
    P.w64[g] = make_double2(0.0, 0.0);
    P.dlt[g] = cdiv(make_double2(1.0, 0.0), __ldg(P.cdiag + g));
    const double ff = f.x * f.x + f.y * f.y;
    v[0] = ff;
    v[2] = ff;
    v[3] = ff;
  });
  if (!grid_sync(P)) return;
  for (int it = 0;; ++it) {
    const int cur = it & 1, nxt = cur ^ 1;
    // A: test, beta; p = r + beta (p - omega v); y = D^-1 p (records of urec64)
    run_phase(P, sm, 0u, [&](int, const Chunk&, int k, int i, bool owner, int lane) {
      double t[kNQ];
      inst_sums(P, i, t);
      if (lane == 0) {
        InstState& st = P.state[i];
        // inn[par]: the instance finished at the half step of that iteration
        const int act = it == 0 ? 1 : (__ldcg(&st.act[cur]) && !__ldcg(&st.inn[cur]));
        const double bb = it == 0 ? t[3] : __ldcg(&st.bb);
        const bool conv = t[2] <= tol2 * bb;
        const bool cap = it >= P.max_iter;
        const bool go = act && !conv && !cap;
        const double2 rho = make_double2(t[0], t[1]);
        double2 beta = make_double2(0.0, 0.0), om = make_double2(0.0, 0.0);
        if (it > 0) {
          om = __ldcg(&st.zomega[cur]);
          beta = finite_or_zero(cmul(cdiv(rho, __ldcg(&st.zrho[cur])), cdiv(__ldcg(&st.zalpha[cur]), om)));
        }
        sm.flag[k] = go;
        sm.ca[k] = beta.x;
        sm.cb[k] = beta.y;
        sm.cc[k] = om.x;
        sm.cd[k] = om.y;
        if (owner) {
          if (it == 0) {
            st.bb = bb;
            st.outer_iters = 1;
          }
          st.act[nxt] = go;
          st.zrho[nxt] = rho;
          if (act) {
            st.rr = t[2];
            st.iters = it;
            if (conv) owner_done(P, st, SS_OK);
            else if (cap) owner_done(P, st, SS_ERR_NOT_CONVERGED);
          }
        }
      }
    }, [&](int64_t g, int64_t, int, int, int k, double*) {
      if (!sm.flag[k]) return;
      const double2 beta = make_double2(sm.ca[k], sm.cb[k]), om = make_double2(sm.cc[k], sm.cd[k]);
      const double2 r = P.r[g], v = P.w64[g];
      double2 p = P.pd[g];
      const double2 q = make_double2(p.x - (om.x * v.x - om.y * v.y), p.y - (om.x * v.y + om.y * v.x));
      p = make_double2(r.x + (beta.x * q.x - beta.y * q.y), r.y + (beta.x * q.y + beta.y * q.x));
      P.pd[g] = p;
      P.urec64[g] = cmul(P.dlt[g], p);
    });
    if (!grid_sync(P)) return;
    if (block_counter(P, 0) >= P.n_inst) break;
    // B: v = L y;  <r^, v>
    run_phase(P, sm, 0b0011u, [&](int, const Chunk&, int k, int i, bool owner, int lane) {
      if (lane == 0) {
        sm.flag[k] = __ldcg(&P.state[i].act[nxt]);
        if (owner && sm.flag[k]) P.state[i].applies += 1;
      }
    }, [&](int64_t g, int64_t s, int lane, int i, int k, double* v) {
      if (!sm.flag[k]) return;
      const double2 w = apply64_row(P, P.inst[i], s, lane, g, P.urec64);
      P.w64[g] = w;
      const double2 q = cdot(P.rhat[g], w);
      v[0] = q.x;
      v[1] = q.y;
    });
    if (!grid_sync(P)) return;
    // C: alpha = rho / <r^, v>; s = r - alpha v; x += alpha y; z = D^-1 s;  |s|^2
    run_phase(P, sm, 0b0100u, [&](int, const Chunk&, int k, int i, bool owner, int lane) {
      double t[kNQ];
      inst_sums(P, i, t);
      if (lane == 0) {
        InstState& st = P.state[i];
        const double2 alpha = finite_or_zero(cdiv(__ldcg(&st.zrho[nxt]), make_double2(t[0], t[1])));
        sm.flag[k] = __ldcg(&st.act[nxt]);
        sm.ca[k] = alpha.x;
        sm.cb[k] = alpha.y;
        if (owner) st.zalpha[nxt] = alpha;
      }
    }, [&](int64_t g, int64_t, int, int, int k, double* vq) {
      if (!sm.flag[k]) return;
      const double2 alpha = make_double2(sm.ca[k], sm.cb[k]);
      const double2 r = P.r[g], v = P.w64[g], y = P.urec64[g];
      const double2 av = cmul(alpha, v), ay = cmul(alpha, y);
      const double2 s = make_double2(r.x - av.x, r.y - av.y);
      double2 x = P.xrec[g];
      x.x += ay.x;
      x.y += ay.y;
      P.xrec[g] = x;
      P.sd[g] = s;
      P.zrec[g] = cmul(P.dlt[g], s);
      vq[2] = s.x * s.x + s.y * s.y;
    });
    if (!grid_sync(P)) return;
    // D: half-step test on |s|; t = L z;  <t, s>, <t, t>
    run_phase(P, sm, 0b0111u, [&](int, const Chunk&, int k, int i, bool owner, int lane) {
      double t[kNQ];
      inst_sums(P, i, t);
      if (lane == 0) {
        InstState& st = P.state[i];
        const int act = __ldcg(&st.act[nxt]);
        const bool half = act && t[2] <= tol2 * __ldcg(&st.bb);
        sm.flag[k] = act && !half;
        if (owner) {
          st.inn[nxt] = half;
          if (half) {
            st.rr = t[2];
            st.iters = it + 1;
            owner_done(P, st, SS_OK);
          } else if (act) {
            st.applies += 1;
          }
        }
      }
    }, [&](int64_t g, int64_t s, int lane, int i, int k, double* v) {
      if (!sm.flag[k]) return;
      const double2 t = apply64_row(P, P.inst[i], s, lane, g, P.zrec);
      P.tv[g] = t;
      const double2 q = cdot(t, P.sd[g]);
      v[0] = q.x;
      v[1] = q.y;
      v[2] = t.x * t.x + t.y * t.y;
    });
    if (!grid_sync(P)) return;
    // E: omega = <t, s> / <t, t>; x += omega z; r = s - omega t;  <r^, r>, |r|^2
    run_phase(P, sm, 0b0111u, [&](int, const Chunk&, int k, int i, bool owner, int lane) {
      double t[kNQ];
      inst_sums(P, i, t);
      if (lane == 0) {
        InstState& st = P.state[i];
        const double2 om =
            finite_or_zero(t[2] > 0.0 ? make_double2(t[0] / t[2], t[1] / t[2]) : make_double2(0.0, 0.0));
        sm.flag[k] = __ldcg(&st.act[nxt]) && !__ldcg(&st.inn[nxt]);
        sm.ca[k] = om.x;
        sm.cb[k] = om.y;
        if (owner) st.zomega[nxt] = om;
      }
    }, [&](int64_t g, int64_t, int, int, int k, double* v) {
      if (!sm.flag[k]) return;
      const double2 om = make_double2(sm.ca[k], sm.cb[k]);
      const double2 s = P.sd[g], t = P.tv[g], z = P.zrec[g];
      const double2 oz = cmul(om, z), ot = cmul(om, t);
      double2 x = P.xrec[g];
      x.x += oz.x;
      x.y += oz.y;
      P.xrec[g] = x;
      const double2 r = make_double2(s.x - ot.x, s.y - ot.y);
      P.r[g] = r;
      const double2 q = cdot(P.rhat[g], r);
      v[0] = q.x;
      v[1] = q.y;
      v[2] = r.x * r.x + r.y * r.y;
    });
    if (!grid_sync(P)) return;
  }
  // true residual f - L x in FP64, and the output
  run_phase(P, sm, 0b0100u, noscal, [&](int64_t g, int64_t s, int lane, int i, int, double* v) {
    const SolveInst& in = P.inst[i];
    const double2 y = apply64_row(P, in, s, lane, g, P.xrec);
    const double2 f = f_at(in, g);
    const double2 r = make_double2(f.x - y.x, f.y - y.y);
    v[2] = r.x * r.x + r.y * r.y;
    const int64_t l = g - in.row0;
    if (l < in.rows) in.u[l] = P.xrec[g];
  });
  if (!grid_sync(P)) return;
  run_phase(P, sm, 0u, [&](int, const Chunk&, int, int i, bool owner, int lane) {
    double t[kNQ];
    inst_sums(P, i, t);
    if (owner && lane == 0) {
      P.state[i].rr = t[2];
      P.state[i].applies += 1;
    }
  }, [](int64_t, int64_t, int, int, int, double*) {});
}

template <int MODE>
__global__ void __launch_bounds__(1024) k_solve(SolveParams P) {
  __shared__ Smem sm;
  if constexpr (MODE == 0) solve_fp64(P, sm);
  else if constexpr (MODE == 1) solve_refined(P, sm);
  else if constexpr (MODE == 2) solve_bicgstab(P, sm);
  else solve_df64(P, sm);
}

__global__ void k_init_solve_records(const int64_t* __restrict__ norm, int64_t n, const int8_t* __restrict__ wide_rows,
                                     bool wide, double2* xrec, double2* prec64, float4* prec32) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n) return;
  const int64_t nr = norm[g];
  const bool wd = wide_rows ? wide_rows[g] != 0 : wide;
  xrec[g] = make_double2(0.0, 0.0);
  prec64[g] = make_double2(0.0, 0.0);
  prec32[g] = make_float4(0.f, 0.f, __int_as_float(norm_word(nr, wd)), 0.f);
}

inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// Chunk cuts of one instance, computed where the slice table lives (one
// block of kPlanThreads threads; no host copy of the widths and no host
// synchronisation).  Slice s weighs 4 (woff[s+1] - woff[s]) + ov4 (quarter
// units, exact in int64); pw(s) = 4 woff[s] + ov4 s is the weight of slices
// [0, s).  Stamping operators order their rows by level: interior rows
// (every step of supp a_hat) first, then the last level's rows with a few
// entries each.  When the first slice t narrower than half the widest one has
// no wider slice after it, [0, t) and [t, n) get their own chunks, shared by
// weight (a chunk holding the transition gives its first warps an interior
// slice plus boundary slices in the later rounds of the warp loop).  Within a
// range of K' chunks, cut c sits at the slice boundary whose prefix weight is
// nearest c/K' of the range's weight, so every block gets one chunk within
// half a slice of the mean.  A sequential pass then makes the cuts strictly
// increasing (K <= n).  If the stamp's build reported an error (err[0]; its
// check may still be pending) every chunk is empty and the solve reads no
// entry.  The slice table is staged in shared memory when it fits.
constexpr int kPlanThreads = 1024;
constexpr int kPlanMaxK = 8192;            // chunks of one instance
constexpr int kPlanSmemWoff = 40960;       // slice offsets staged in shared memory up to this count

__device__ void plan_cuts_block(const int32_t* __restrict__ woff_g, int64_t n, int K, int64_t ov4,
                                const int32_t* __restrict__ stamp_err, Chunk* out) {
  extern __shared__ int32_t sm_plan[];
  __shared__ int32_t s_wmax;
  __shared__ unsigned long long s_t;
  __shared__ int s_bad, s_fix;
  const int tid = threadIdx.x;
  const bool staged = n + 1 <= kPlanSmemWoff;
  int32_t* cut = sm_plan + (staged ? kPlanSmemWoff : 0);   // [K + 1]
  if (tid == 0) {
    s_wmax = 0;
    s_t = (unsigned long long)n;
    s_bad = 0;
    s_fix = 0;
  }
  if (staged) {
    // kStage loads in flight per thread before the first store (the table
    // holds at most kPlanSmemWoff words: ceil(40960 / 1024) = 40 per thread)
    constexpr int kStage = 8;
    for (int64_t s0 = tid; s0 <= n; s0 += (int64_t)kStage * blockDim.x) {
      int32_t v[kStage];
#pragma unroll
      for (int q = 0; q < kStage; ++q) {
        const int64_t s = s0 + (int64_t)q * blockDim.x;
        v[q] = s <= n ? __ldg(woff_g + s) : 0;
      }
#pragma unroll
      for (int q = 0; q < kStage; ++q) {
        const int64_t s = s0 + (int64_t)q * blockDim.x;
        if (s <= n) sm_plan[s] = v[q];
      }
    }
  }
  __syncthreads();
  const int32_t* woff = staged ? sm_plan : woff_g;
  if (stamp_err && __ldg(stamp_err) != 0) {
    for (int c = tid; c < K; c += blockDim.x) out[c] = Chunk{0, 0, 0, 0};
    return;
  }
  int32_t wm = 0;
  for (int64_t s = tid; s < n; s += blockDim.x) wm = max(wm, woff[s + 1] - woff[s]);
  wm = __reduce_max_sync(0xffffffffu, wm);
  if ((tid & 31) == 0) atomicMax(&s_wmax, wm);
  __syncthreads();
  const int32_t wmax = s_wmax;
  for (int64_t s = tid; s < n; s += blockDim.x)
    if (2 * (woff[s + 1] - woff[s]) < wmax) {
      atomicMin(&s_t, (unsigned long long)s);
      break;   // a thread's slices ascend: its first hit is its smallest
    }
  __syncthreads();
  const int64_t t = (int64_t)s_t;
  for (int64_t s = t + tid; s < n; s += blockDim.x)
    if (2 * (woff[s + 1] - woff[s]) >= wmax) s_bad = 1;
  __syncthreads();
  auto pw = [&](int64_t s) { return 4 * (int64_t)woff[s] + ov4 * s; };
  const bool split = t > 0 && t < n && !s_bad && K >= 2;
  const int64_t pn = pw(n);
  int k1 = K;
  if (split) {
    const int64_t r = (2 * pw(t) * K + pn) / (2 * pn);   // K pw(t) / pw(n), rounded
    k1 = (int)(r < 1 ? 1 : (r > K - 1 ? K - 1 : r));
  }
  for (int c = tid + 1; c < K; c += blockDim.x) {
    int64_t a = 0, b = n, kr = K, cr = c;
    if (split) {
      if (c < k1) {
        b = t;
        kr = k1;
      } else {
        a = t;
        kr = K - k1;
        cr = c - k1;
      }
    }
    int64_t cs;
    if (cr == 0) {
      cs = a;   // the region boundary
    } else {
      // smallest s in (a, b] with kr (pw(s) - pw(a)) >= cr (pw(b) - pw(a)), or s - 1 if nearer
      // (pw < 2^39 and kr <= 2^13: the products fit in int64)
      const int64_t base = pw(a), tgt = (pw(b) - base) * cr;
      int64_t lo = a + 1, hi = b;
      while (lo < hi) {
        const int64_t mid = lo + (hi - lo) / 2;
        if ((pw(mid) - base) * kr >= tgt) hi = mid;
        else lo = mid + 1;
      }
      if (lo - 1 > a && tgt - (pw(lo - 1) - base) * kr < (pw(lo) - base) * kr - tgt) --lo;
      cs = lo;
    }
    cut[c] = (int32_t)cs;
  }
  if (tid == 0) {
    cut[0] = 0;
    cut[K] = (int32_t)n;
  }
  __syncthreads();
  for (int c = tid; c < K; c += blockDim.x)
    if (cut[c] >= cut[c + 1]) s_fix = 1;
  __syncthreads();
  if (s_fix && tid == 0) {   // only when a slice outweighs a chunk: one sequential pass
    for (int c = 1; c < K; ++c) cut[c] = max(cut[c], cut[c - 1] + 1);
    for (int c = K - 1; c >= 1; --c) cut[c] = min(cut[c], cut[c + 1] - 1);
  }
  __syncthreads();
  for (int c = tid; c < K; c += blockDim.x) out[c] = Chunk{cut[c], cut[c + 1], 0, 0};
}

// Everything a single-instance solve writes before its kernel starts, in one
// launch of one block: the barrier, counter and error words, the instance
// state, one caller word (the half system's Hermitian flag), the instance
// descriptor, and the chunk cuts when the plan is new (plan_cuts_block).
struct Prologue {
  unsigned* bar;
  int* counters;
  int* err;
  InstState* state;
  int32_t* extra;
  SolveInst* inst_dst;
  SolveInst inst;
  int cuts;
  const int32_t* woff;
  int64_t n, ov4;
  int K;
  const int32_t* stamp_err;
  Chunk* chunk;
};

__global__ void __launch_bounds__(kPlanThreads) k_solve_prologue(Prologue p) {
  const int tid = threadIdx.x;
  if (tid < 2) p.bar[tid] = 0u;
  if (tid < 4) p.counters[tid] = 0;
  if (tid == 0) {
    *p.err = 0;
    if (p.extra) *p.extra = 0;
    *p.inst_dst = p.inst;
  }
  static_assert(sizeof(InstState) % sizeof(int32_t) == 0, "InstState is zeroed in 32-bit words");
  for (int i = tid; i < (int)(sizeof(InstState) / sizeof(int32_t)); i += blockDim.x)
    reinterpret_cast<int32_t*>(p.state)[i] = 0;
  if (p.cuts) plan_cuts_block(p.woff, p.n, p.K, p.ov4, p.stamp_err, p.chunk);
}

}  // namespace

// ---------------------------------------------------------------- host side

// The single-instance plan: K chunks (c_first 0, c_last K - 1, one partial
// slot each) whose cuts the prologue computes on the device.
static void plan_single(SolvePlan& plan, int64_t n_slices, int target, const int32_t* woff_dev, double overhead,
                        const int32_t* stamp_err) {
  const int K = (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)target, n_slices, (int64_t)kPlanMaxK}));
  plan.chunk.assign(K, Chunk{0, 0, 0, 0});
  plan.n_parts = K;
  SolveInst& in = plan.inst[0];
  in.c_first = 0;
  in.c_last = K - 1;
  in.part_base = 0;
  plan.dev_cuts = true;
  plan.cuts_pending = true;
  plan.cut_woff = woff_dev;
  plan.cut_n = n_slices;
  plan.cut_ov4 = std::llround(4.0 * overhead);
  plan.cut_err = stamp_err;
}

// The prologue of a single-instance (dev_cuts) plan into the given words and
// tables; the chunk cuts only when the plan's are not in `chunk` yet.
static ss_status launch_prologue(SolvePlan& plan, unsigned* bar, int* counters, int* err, InstState* state,
                                 int32_t* extra, SolveInst* inst_dst, Chunk* chunk, cudaStream_t st) {
  Prologue p{};
  p.bar = bar;
  p.counters = counters;
  p.err = err;
  p.state = state;
  p.extra = extra;
  p.inst_dst = inst_dst;
  p.inst = plan.inst[0];
  p.cuts = plan.cuts_pending ? 1 : 0;
  p.woff = plan.cut_woff;
  p.n = plan.cut_n;
  p.ov4 = plan.cut_ov4;
  p.K = (int)plan.chunk.size();
  p.stamp_err = plan.cut_err;
  p.chunk = chunk;
  const size_t smem =
      p.cuts ? ((plan.cut_n + 1 <= kPlanSmemWoff ? (size_t)kPlanSmemWoff : 0) + (size_t)p.K + 1) * sizeof(int32_t) : 0;
  // the attribute belongs to the current device: set with every planning launch
  if (smem > 48 * 1024)
    SS_CUDA(cudaFuncSetAttribute(k_solve_prologue, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_solve_prologue<<<1, kPlanThreads, smem, st>>>(p);
  SS_LAUNCH_CHECK();
  plan.cuts_pending = false;
  return SS_OK;
}

ss_status plan_chunks(SolvePlan& plan, const std::vector<int32_t>& woff, const std::vector<int32_t>& slice_inst,
                      int target_chunks, double slice_overhead) {
  const int64_t n_slices = (int64_t)woff.size() - 1;
  const int n_inst = (int)plan.inst.size();
  plan.chunk.clear();
  if (n_slices <= 0) SS_FAIL(SS_ERR_INVALID, "solve: empty operator");
  // weight of a slice: its entries (gathers) plus the vector work of 32 rows
  // (small when the row-wise phases split the rows on their own)
  auto weight = [&](int64_t s) { return (double)(woff[s + 1] - woff[s]) + slice_overhead; };
  auto inst_of = [&](int64_t s) { return slice_inst.empty() ? 0 : slice_inst[s]; };
  // running cuts over the instances' slices (batches; a single instance is
  // cut on the device by the solve prologue)
  {
    double total = 0;
    for (int64_t s = 0; s < n_slices; ++s) total += weight(s);
    const double target = total / std::max(1, target_chunks);
    int64_t s0 = 0;
    double acc = 0;
    for (int64_t s = 0; s < n_slices; ++s) {
      acc += weight(s);
      const bool last = s + 1 == n_slices;
      bool cut = last || acc >= target;
      if (!last && inst_of(s + 1) - inst_of(s0) + 1 > kMaxInstPerChunk) cut = true;
      if (cut) {
        plan.chunk.push_back(Chunk{s0, s + 1, inst_of(s0), inst_of(s)});
        s0 = s + 1;
        acc = 0;
      }
    }
  }
  for (auto& in : plan.inst) { in.c_first = INT32_MAX; in.c_last = -1; }
  for (int c = 0; c < (int)plan.chunk.size(); ++c)
    for (int i = plan.chunk[c].inst0; i <= plan.chunk[c].inst1; ++i) {
      plan.inst[i].c_first = std::min(plan.inst[i].c_first, c);
      plan.inst[i].c_last = std::max(plan.inst[i].c_last, c);
    }
  int32_t base = 0;
  for (int i = 0; i < n_inst; ++i) {
    if (plan.inst[i].c_last < 0) SS_FAIL(SS_ERR_INVALID, "solve: instance %d has no rows", i);
    plan.inst[i].part_base = base;
    base += plan.inst[i].c_last - plan.inst[i].c_first + 1;
  }
  plan.n_parts = base;
  return SS_OK;
}

ss_status work_alloc(SolveWork& W, int64_t rows_total, const int64_t* norm, const int8_t* wide_rows, bool wide,
                     cudaStream_t st) {
  if (W.rows_total == rows_total) return SS_OK;
  if (W.cap_rows >= rows_total) {
    // a workspace kept from an earlier stamp: new records, same buffers
    W.rows_total = rows_total;
    k_init_solve_records<<<nblk(rows_total), 256, 0, st>>>(norm, rows_total, wide_rows, wide, W.xrec.get(),
                                                           W.urec64.get(), W.urec32.get());
    SS_LAUNCH_CHECK();
    return SS_OK;
  }
  W.rows_total = rows_total;
  W.cap_rows = rows_total;
  W.df_rows = W.bi_rows = -1;
  {
    // one allocation, carved in 256-byte aligned pieces
    size_t off = 0;
    auto take = [&](auto& view, size_t count) {
      using T = typename std::remove_pointer<decltype(view.p)>::type;
      view.p = reinterpret_cast<T*>(off);   // offset for now, rebased below
      off += (count * sizeof(T) + 255) / 256 * 256;
    };
    const size_t n = (size_t)rows_total;
    take(W.xrec, n); take(W.urec64, n); take(W.urec32, n); take(W.r, n); take(W.w64, n); take(W.w32, n);
    take(W.pd, n); take(W.sd, n); take(W.rhat, n); take(W.dlt, n); take(W.r32, n); take(W.p32, n);
    take(W.s32, n); take(W.d32, n); take(W.rdiag, n); take(W.bar, 2); take(W.counters, 4); take(W.err, 1);
    SS_TRY(W.arena.alloc(off, st));
    const uintptr_t b = reinterpret_cast<uintptr_t>(W.arena.get());
    auto rebase = [&](auto& view) {
      using T = typename std::remove_pointer<decltype(view.p)>::type;
      view.p = reinterpret_cast<T*>(b + reinterpret_cast<uintptr_t>(view.p));
    };
    rebase(W.xrec); rebase(W.urec64); rebase(W.urec32); rebase(W.r); rebase(W.w64); rebase(W.w32);
    rebase(W.pd); rebase(W.sd); rebase(W.rhat); rebase(W.dlt); rebase(W.r32); rebase(W.p32);
    rebase(W.s32); rebase(W.d32); rebase(W.rdiag); rebase(W.bar); rebase(W.counters); rebase(W.err);
  }
  k_init_solve_records<<<nblk(rows_total), 256, 0, st>>>(norm, rows_total, wide_rows, wide, W.xrec.get(),
                                                         W.urec64.get(), W.urec32.get());
  SS_LAUNCH_CHECK();
  // The workspace is reused by later calls, possibly on other streams: both
  // callers synchronise `st` before they return (solve when it reads the
  // statistics, batch_create right after this), which orders those calls
  // after these allocations.
  W.arena.settle();
  return SS_OK;
}

ss_status work_alloc_bicgstab(SolveWork& W, cudaStream_t st) {
  if (W.zrec.n >= (size_t)W.rows_total && W.tv.n >= (size_t)W.rows_total) {
    if (W.bi_rows != W.rows_total) {   // the dummy row of this row count must read as zero
      SS_CUDA(cudaMemsetAsync(W.zrec.get() + (W.rows_total - 1), 0, sizeof(double2), st));
      W.bi_rows = W.rows_total;
    }
    return SS_OK;
  }
  W.bi_rows = W.rows_total;
  SS_TRY(W.zrec.alloc(W.rows_total, st));
  SS_TRY(W.tv.alloc(W.rows_total, st));
  SS_CUDA(cudaMemsetAsync(W.zrec.get(), 0, W.rows_total * sizeof(double2), st));
  SS_CUDA(cudaStreamSynchronize(st));
  W.zrec.settle();
  W.tv.settle();
  return SS_OK;
}

ss_status work_alloc_df64(SolveWork& W, cudaStream_t st) {
  if (W.xdf.n >= (size_t)W.rows_total && W.udf.n >= (size_t)W.rows_total) {
    if (W.df_rows != W.rows_total) {   // the dummy record of this row count must read as zero
      SS_CUDA(cudaMemsetAsync(W.xdf.get() + (W.rows_total - 1), 0, sizeof(float4), st));
      SS_CUDA(cudaMemsetAsync(W.udf.get() + (W.rows_total - 1), 0, sizeof(float4), st));
      W.df_rows = W.rows_total;
    }
    return SS_OK;
  }
  W.df_rows = W.rows_total;
  SS_TRY(W.xdf.alloc(W.rows_total, st));
  SS_TRY(W.udf.alloc(W.rows_total, st));
  // the dummy record (last row) must read as zero
  SS_CUDA(cudaMemsetAsync(W.xdf.get(), 0, W.rows_total * sizeof(float4), st));
  SS_CUDA(cudaMemsetAsync(W.udf.get(), 0, W.rows_total * sizeof(float4), st));
  SS_CUDA(cudaStreamSynchronize(st));
  W.xdf.settle();
  W.udf.settle();
  return SS_OK;
}

ss_status work_upload(SolveWork& W, SolvePlan& plan, cudaStream_t st) {
  const int n_inst = (int)plan.inst.size(), n_chunk = (int)plan.chunk.size();
  if (n_inst > W.cap_inst) { SS_TRY(W.inst.alloc(n_inst, st)); SS_TRY(W.state.alloc(n_inst, st)); W.cap_inst = n_inst; }
  if (n_chunk > W.cap_chunk) {
    SS_TRY(W.chunk.alloc(n_chunk, st));
    W.cap_chunk = n_chunk;
    plan.cuts_pending = plan.dev_cuts;   // a new chunk table: its cuts are written again
  }
  if (plan.n_parts > W.cap_parts) { SS_TRY(W.part.alloc(plan.n_parts * kNQ, st)); W.cap_parts = plan.n_parts; }
  W.inst.settle(); W.state.settle(); W.chunk.settle(); W.part.settle();   // reused across calls (see read_stats)
  if (plan.dev_cuts) return SS_OK;   // descriptor, cuts and zeroed words: work_prologue
  return upload(st, {{W.inst.get(), plan.inst.data(), n_inst * sizeof(SolveInst)},
                     {W.chunk.get(), plan.chunk.data(), n_chunk * sizeof(Chunk)}});
}

// The prologue of a single-instance plan into its workspace (after
// work_upload); `extra` is one more word to zero (or null).  The solve is then
// launched with zeroed = true.
static ss_status work_prologue(SolveWork& W, SolvePlan& plan, int32_t* extra, cudaStream_t st) {
  return launch_prologue(plan, W.bar.get(), W.counters.get(), W.err.get(), W.state.get(), extra, W.inst.get(),
                         W.chunk.get(), st);
}

ss_status max_grid(int mode, int block, int* grid) {
  // resident blocks per SM, looked up once per device, mode and block size
  static std::mutex mu;
  static int cache[64][4][4] = {};
  int dev = 0;
  SS_CUDA(cudaGetDevice(&dev));
  const int bi = block == 128 ? 0 : block == 256 ? 1 : block == 512 ? 2 : 3;
  if (dev >= 0 && dev < 64 && mode >= 0 && mode < 4) {
    std::lock_guard<std::mutex> lk(mu);
    if (cache[dev][mode][bi] > 0) {
      *grid = cache[dev][mode][bi] * sm_count();
      return SS_OK;
    }
  }
  int nb = 0;
  if (mode == 0) SS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_solve<0>, block, 0));
  else if (mode == 1) SS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_solve<1>, block, 0));
  else if (mode == 2) SS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_solve<2>, block, 0));
  else SS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_solve<3>, block, 0));
  if (nb < 1) SS_FAIL(SS_ERR_CUDA, "solve: kernel does not fit on an SM with %d threads", block);
  if (dev >= 0 && dev < 64 && mode >= 0 && mode < 4) {
    std::lock_guard<std::mutex> lk(mu);
    cache[dev][mode][bi] = nb;
  }
  *grid = nb * sm_count();
  return SS_OK;
}

// Fill params and launch (capturable: no host synchronisation).
ss_status launch_solve(SolveWork& W, const SolvePlan& plan, const OpView& op, const int32_t* slice_inst,
                       const int64_t* norm, const double2* ca64, const float2* ca32, const int32_t* pn,
                       double tol, int max_iter, int mode, cudaStream_t st, cudaEvent_t ev_begin,
                       cudaEvent_t ev_end, const double2* cdiag, bool zeroed) {
  if (mode == 2 && (!cdiag || !W.zrec.get() || !W.tv.get()))
    SS_FAIL(SS_ERR_INVALID, "solve: BiCGStab needs the operator diagonal and its workspace");
  if (mode == 3 && (!op.ecoefdf || !W.xdf.get() || !W.udf.get()))
    SS_FAIL(SS_ERR_INVALID, "solve: DF64 CG needs double-float coefficients and its workspace");
  SolveParams P{};
  P.n_inst = (int)plan.inst.size();
  P.n_chunks = (int)plan.chunk.size();
  P.inst = W.inst.get();
  P.chunk = W.chunk.get();
  P.state = W.state.get();
  P.op = op;
  P.slice_inst = slice_inst;
  P.norm = norm;
  P.ca64 = ca64;
  P.ca32 = ca32;
  P.pn = pn;
  P.xrec = W.xrec.get();
  P.urec64 = W.urec64.get();
  P.urec32 = W.urec32.get();
  P.r = W.r.get();
  P.w64 = W.w64.get();
  P.w32 = W.w32.get();
  P.pd = W.pd.get();
  P.sd = W.sd.get();
  P.rhat = W.rhat.get();
  P.dlt = W.dlt.get();
  P.r32 = W.r32.get();
  P.p32 = W.p32.get();
  P.s32 = W.s32.get();
  P.d32 = W.d32.get();
  P.rdiag = W.rdiag.get();
  P.cdiag = cdiag;
  P.zrec = W.zrec.get();
  P.tv = W.tv.get();
  P.xdf = W.xdf.get();
  P.udf = W.udf.get();
  P.part = W.part.get();
  P.bar = W.bar.get();
  P.counters = W.counters.get();
  P.err = W.err.get();
  P.tol = tol;
  P.inner_tol = 1e-5;
  P.max_iter = max_iter;
  P.max_inner = std::max(1, std::min(max_iter, 200));
  P.max_outer = std::max(1, max_iter);
  P.spin_limit = plan.spin_limit;   // 2 s unless solve_set_wait_limit changed it
  const int64_t n_sl = plan.dev_cuts ? plan.cut_n : plan.chunk.back().s1;
  P.rows_slices = plan.row_split && P.n_inst == 1 && !slice_inst ? n_sl : 0;
  if (!zeroed) {
    SS_TRY(fill_small(st, {{W.bar.get(), 2 * sizeof(unsigned), 0}, {W.counters.get(), 4 * sizeof(int), 0}}));
    SS_CUDA(cudaMemsetAsync(W.err.get(), 0, sizeof(int), st));
    SS_CUDA(cudaMemsetAsync(W.state.get(), 0, plan.inst.size() * sizeof(InstState), st));
  }
  // cooperative launch: all blocks co-resident (required by the grid barrier);
  // expressed as a launch attribute so that it can be captured in a graph
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(plan.grid);
  cfg.blockDim = dim3(plan.block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (ev_begin) SS_CUDA(cudaEventRecord(ev_begin, st));
  {
    static const char* const names[4] = {"k_solve<0>", "k_solve<1>", "k_solve<2>", "k_solve<3>"};
    ProfScope prof_(names[mode & 3], st, true);
    if (mode == 0) SS_CUDA(cudaLaunchKernelEx(&cfg, k_solve<0>, P));
    else if (mode == 1) SS_CUDA(cudaLaunchKernelEx(&cfg, k_solve<1>, P));
    else if (mode == 2) SS_CUDA(cudaLaunchKernelEx(&cfg, k_solve<2>, P));
    else SS_CUDA(cudaLaunchKernelEx(&cfg, k_solve<3>, P));
  }
  if (ev_end) SS_CUDA(cudaEventRecord(ev_end, st));
  return SS_OK;
}

ss_status read_stats(SolveWork& W, int n_inst, ss_solve_stats* stats, ss_status* worst, cudaStream_t st,
                     cudaEvent_t ev_begin, cudaEvent_t ev_end) {
  std::vector<InstState> hs(n_inst);
  int herr = 0;
  SS_TRY(read_back(st, {{hs.data(), W.state.get(), n_inst * sizeof(InstState)}, {&herr, W.err.get(), sizeof(int)}}));
  float kms = 0.f;
  if (ev_begin && ev_end) cudaEventElapsedTime(&kms, ev_begin, ev_end);
  *worst = SS_OK;
  if (herr) {
    *worst = (ss_status)herr;
    set_error("solve: a device-side wait gave up (status %d)", herr);
  }
  for (int i = 0; i < n_inst; ++i) {
    const InstState& s = hs[i];
    if (stats) {
      stats[i].status = herr ? herr : s.status;
      stats[i].outer_iters = s.outer_iters;
      stats[i].inner_iters = s.inner_iters ? s.inner_iters : s.iters;
      stats[i].applies = s.applies;
      stats[i].rel_residual = s.bb > 0 ? std::sqrt(s.rr / s.bb) : 0.0;
      stats[i].kernel_ms = kms;
      stats[i].half_system = 0;
      stats[i].real_coefficients = 0;
    }
    if (*worst == SS_OK && s.status != SS_OK) {
      *worst = (ss_status)s.status;
      set_error("solve: instance %d did not converge (relative residual %.3e)", i,
                s.bb > 0 ? std::sqrt(s.rr / s.bb) : 0.0);
    }
  }
  return SS_OK;
}

}  // namespace ss

// ------------------------------------------------------- per-stamp solve state

struct ss_solve_ctx {
  ss::SolveWork work;
  ss::SolvePlan plan;
  int planned_mode = -1;
  int block = 1024, blocks_per_sm = 1, chunks_per_block = 1;   // tile shape (solve_set_config)
  long long wait_ns = 2000000000ll;   // grid-barrier wait bound (solve_set_wait_limit)
  double2* f0_host = nullptr;   // pinned copy of f_hat_0, checked after the solve's own synchronisation
  // Hermitian half system (FP64 CG): its own plan and workspace, the compact
  // right-hand side and solution, and the "f is not Hermitian" flag
  bool use_half = true;
  ss_solve_ctx* half = nullptr;
  ss::DevBuf<double2> fh, uh;
  ss::DevBuf<int32_t> hflag;
  int32_t* hflag_host = nullptr;
  int32_t* chk_host = nullptr;   // pinned copy of a pending stamp's error words (stamp_build_pending)
  ~ss_solve_ctx() {
    if (f0_host) cudaFreeHost(f0_host);
    if (hflag_host) cudaFreeHost(hflag_host);
    if (chk_host) cudaFreeHost(chk_host);
    delete half;
  }
};

namespace ss {

// Weight of a slice in the chunk cuts beyond its entries, in entry rows (one
// unit = one entry per row of the slice).  Fitted to per-block clock counts
// of the apply phases on the d = 100 operator (interior slices of width 41,
// boundary slices of width 4): an interior slice took 5.8 times a boundary
// slice in the FP64 CG, (41 + 3.75) / (4 + 3.75), whose boundary rows carry
// three FP64 inner products and the record loads and stores besides their
// entries; 7.6 times in the double-float CG, whose row work runs on the FP32
// pipes.  The FP32-refined and BiCGStab solves do their vector updates in the
// chunks too (no even row split of those phases).
static double slice_overhead(int mode) {
  switch (mode) {
    case 0: return 3.75;   // FP64 CG
    case 3: return 1.5;    // DF64 CG
    case 1: return 2.0;    // FP32-refined
    default: return 6.0;   // BiCGStab
  }
}

static ss_status stamp_plan(ss_stamp_s* s, ss_solve_ctx& C, int mode, cudaStream_t st) {
  if (C.planned_mode == mode) return SS_OK;
  if (!s->slice_off.get() || s->n_slices < 1) SS_FAIL(SS_ERR_INVALID, "solve: stamp has no slice table");
  C.plan.inst.assign(1, SolveInst{});
  SolveInst& in = C.plan.inst[0];
  in.row0 = 0;
  in.rows = s->size;
  in.rows_pad = s->rows_pad;
  in.zero_row = identity_row(s);
  in.coef_off = 0;
  in.dscale = 2.0 * kTwoPiSq * s->a0;   // 4 pi^2 Re(a_hat_0)
  in.wide = s->wide ? 1 : 0;
  int grid = 0;
  C.plan.block = C.block;
  SS_TRY(max_grid(mode, C.plan.block, &grid));
  if (C.blocks_per_sm > 0) grid = std::min(grid, C.blocks_per_sm * sm_count());
  const int by_size = (int)std::max<int64_t>(1, s->n_slices / 8);   // at least 8 slices per chunk
  const int target = std::min<int64_t>((int64_t)grid * C.chunks_per_block, by_size);
  // FP64 and DF64 CG: the vector updates run over an even split of the rows,
  // the apply phases over chunks balanced by entries
  C.plan.row_split = mode == 0 || mode == 3;
  plan_single(C.plan, s->n_slices, target, s->slice_off.get(), slice_overhead(mode), s->err_dev.get());
  C.plan.grid = std::min<int>(grid, (int)C.plan.chunk.size());
  SS_TRY(work_alloc(C.work, s->rows_pad + 1, s->norm.get(), nullptr, s->wide, st));
  if (mode == 2) SS_TRY(work_alloc_bicgstab(C.work, st));
  if (mode == 3) {
    SS_TRY(ensure_ecoefdf(s, st));
    SS_TRY(work_alloc_df64(C.work, st));
  }
  C.planned_mode = mode;   // the plan goes to the device with the call's f and u (solve)
  return SS_OK;
}

// Plan and workspace of the Hermitian half system (FP64, FP32-refined and DF64 modes).
static ss_status stamp_plan_half(ss_stamp_s* s, ss_solve_ctx& H, int mode, cudaStream_t st) {
  if (H.planned_mode == mode) return SS_OK;
  if (!s->woff_h.get() || s->n_slices_h < 1) SS_FAIL(SS_ERR_INVALID, "solve: no half-system table");
  H.plan.inst.assign(1, SolveInst{});
  SolveInst& in = H.plan.inst[0];
  in.row0 = 0;
  in.rows = s->n_plus;
  in.rows_pad = s->rows_pad_h;
  in.zero_row = -1;                      // k = 0 is not a row of the half system
  in.coef_off = 0;
  in.dscale = 2.0 * kTwoPiSq * s->a0;
  in.wide = s->wide ? 1 : 0;
  int grid = 0;
  H.plan.block = H.block;
  SS_TRY(max_grid(mode, H.plan.block, &grid));
  if (H.blocks_per_sm > 0) grid = std::min(grid, H.blocks_per_sm * sm_count());
  const int by_size = (int)std::max<int64_t>(1, s->n_slices_h / 8);
  const int target = std::min<int64_t>((int64_t)grid * H.chunks_per_block, by_size);
  H.plan.row_split = mode == 0 || mode == 3;
  plan_single(H.plan, s->n_slices_h, target, s->woff_h.get(), slice_overhead(mode), s->err_dev.get());
  H.plan.grid = std::min<int>(grid, (int)H.plan.chunk.size());
  SS_TRY(work_alloc(H.work, s->rows_pad_h + 1, s->norm_h.get(), nullptr, s->wide, st));
  if (mode == 3) {
    SS_TRY(ensure_ecoefdf_half(s, st));
    SS_TRY(work_alloc_df64(H.work, st));
  }
  H.planned_mode = mode;
  return SS_OK;
}

namespace {

// Compact right-hand side f_h[i] = f[k_i] (k_i > 0); flags an f that is not
// Hermitian (f_{-k} != conj(f_k) bit for bit) so the full system is solved instead.
__global__ void k_half_gather(const double2* __restrict__ f, const int32_t* __restrict__ plus_rows,
                              const int64_t* __restrict__ mirror, int64_t n_plus, double2* f_h, int32_t* flag) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_plus) return;
  const int64_t g = plus_rows[i];
  const int64_t m = mirror[g];   // -1: -k not found (the stamp's check fails): solved as the full system
  const double2 a = f[g];
  if (m < 0) {
    atomicExch(flag, 1);
  } else {
    const double2 b = f[m];
    if (!(a.x == b.x && a.y == -b.y)) atomicExch(flag, 1);
  }
  f_h[i] = a;
}

// u on S from the compact solution: u_k (k > 0), conj(u_{-k}) (k < 0), 0 (k = 0).
__global__ void k_half_scatter(const double2* __restrict__ u_h, const int32_t* __restrict__ hpos, int64_t size,
                               int64_t n_plus, double2* u) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= size) return;
  const int32_t h = hpos[g];
  // positions outside the compact rows only come from a half system whose
  // build failed (reported by the stamp's check); nothing is read there
  if (h == -1 || h >= n_plus || (h < -1 && -2 - (int64_t)h >= n_plus)) {
    u[g] = make_double2(0.0, 0.0);
  } else if (h >= 0) {
    u[g] = u_h[h];
  } else {
    const double2 v = u_h[-2 - h];
    u[g] = make_double2(v.x, -v.y);
  }
}

}  // namespace

}  // namespace ss

using namespace ss;

// The per-stamp context lives in a side table keyed by the stamp pointer so
// that the stamp layout stays independent of the solver.
#include <mutex>
#include <unordered_map>
static std::mutex g_ctx_mu;
static std::unordered_map<const ss_stamp_s*, ss_solve_ctx*> g_ctx;

namespace ss {
// Contexts of destroyed stamps are kept (a few) with their device buffers and
// given to the next stamps: a new stamp then needs no allocation for its
// solves, only new records (work_alloc re-initialises them for its rows).
static std::vector<ss_solve_ctx*> g_spare_ctx;
constexpr size_t kMaxSpareCtx = 4;

static void reset_ctx(ss_solve_ctx* C) {
  C->planned_mode = -1;
  C->work.rows_total = 0;
  C->block = 1024;
  C->blocks_per_sm = 1;
  C->chunks_per_block = 1;
  C->use_half = true;
  C->wait_ns = 2000000000ll;
  if (C->half) reset_ctx(C->half);
}

void drop_solve_ctx(const ss_stamp_s* s) {
  std::lock_guard<std::mutex> lk(g_ctx_mu);
  auto it = g_ctx.find(s);
  if (it != g_ctx.end()) {
    ss_solve_ctx* C = it->second;
    g_ctx.erase(it);
    if (g_spare_ctx.size() < kMaxSpareCtx) {
      reset_ctx(C);
      g_spare_ctx.push_back(C);
    } else {
      delete C;
    }
  }
}
}  // namespace ss

static ss_solve_ctx* solve_ctx(const ss_stamp_s* s) {
  std::lock_guard<std::mutex> lk(g_ctx_mu);
  auto& slot = g_ctx[s];
  if (!slot) {
    if (!g_spare_ctx.empty()) {
      slot = g_spare_ctx.back();
      g_spare_ctx.pop_back();
    } else {
      slot = new ss_solve_ctx();
    }
  }
  return slot;
}

extern "C" ss_status solve_set_config(ss_stamp s, int32_t block, int32_t blocks_per_sm, int32_t chunks_per_block) {
  if (!s || (block != 128 && block != 256 && block != 512 && block != 1024) || blocks_per_sm < 0 ||
      chunks_per_block < 1)
    SS_FAIL(SS_ERR_INVALID, "solve_set_config: block in {128,256,512,1024}, blocks_per_sm >= 0, chunks >= 1");
  ss_solve_ctx* C = solve_ctx(s);
  C->block = block;
  C->blocks_per_sm = blocks_per_sm;
  C->chunks_per_block = chunks_per_block;
  C->planned_mode = -1;
  return SS_OK;
}

extern "C" ss_status solve_set_wait_limit(ss_stamp s, int64_t ns) {
  if (!s || ns < 0) SS_FAIL(SS_ERR_INVALID, "solve_set_wait_limit: null stamp or negative limit");
  solve_ctx(s)->wait_ns = ns == 0 ? -1 : (long long)ns;   // 0: give up at the first poll
  return SS_OK;
}

extern "C" ss_status solve_set_symmetry(ss_stamp s, int32_t use_half) {
  if (!s) SS_FAIL(SS_ERR_INVALID, "solve_set_symmetry: null stamp");
  solve_ctx(s)->use_half = use_half != 0;
  return SS_OK;
}

extern "C" ss_status solve(ss_stamp s, const double* f_on_S, double* u_on_S, double tol, int32_t max_iter,
                           ss_precision prec, ss_solve_stats* stats, void* stream) {
  if (!s || !f_on_S || !u_on_S) SS_FAIL(SS_ERR_INVALID, "solve: null argument");
  if (!(tol > 0.0) || max_iter < 1) SS_FAIL(SS_ERR_INVALID, "solve: need tol > 0 and max_iter >= 1");
  if (prec != SS_FP64 && prec != SS_FP32 && prec != SS_DF64) SS_FAIL(SS_ERR_INVALID, "solve: bad precision");
  cudaStream_t st = as_stream(stream);
  if (s->adr && prec != SS_FP64) SS_FAIL(SS_ERR_INVALID, "solve: ADR stamps solve in SS_FP64 (BiCGStab)");
  ss_solve_ctx* C = solve_ctx(s);
  // Host checks read back with the solve's statistics (one synchronisation
  // for all), queued behind the solve kernel so that they do not delay it:
  // f_hat_0 (must vanish) and the error words of a stamp whose build left
  // them to this synchronisation (the one-call pipeline).
  const bool pending = s->check_pending;
  const bool check_f0 = !s->adr && s->zero_idx >= 0;
  bool checks_queued = false;
  auto queue_checks = [&]() -> ss_status {
    if (checks_queued) return SS_OK;
    checks_queued = true;
    if (pending) {
      if (!C->chk_host) {
        note_alloc();
        SS_CUDA(cudaMallocHost(&C->chk_host, 4 * sizeof(int32_t)));
      }
      SS_CUDA(cudaMemcpyAsync(C->chk_host, s->err_dev.get(), 4 * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    }
    if (check_f0) {
      if (!C->f0_host) {
        note_alloc();
        SS_CUDA(cudaMallocHost(&C->f0_host, sizeof(double2)));
      }
      SS_CUDA(cudaMemcpyAsync(C->f0_host, reinterpret_cast<const double2*>(f_on_S) + s->zero_idx, sizeof(double2),
                              cudaMemcpyDeviceToHost, st));
    }
    return SS_OK;
  };
  const int mode = s->adr ? 2 : (prec == SS_FP64 ? 0 : (prec == SS_FP32 ? 1 : 3));
  if (mode != 2 && s->half_ok && C->use_half) {
    // Real data: solve the Hermitian half system (rows k >lex 0, neighbours
    // below read as conjugates), then unfold; if f turns out not to be
    // Hermitian the full system below is solved instead.
    if (!C->half) C->half = new ss_solve_ctx();
    ss_solve_ctx* H = C->half;
    if (H->block != C->block || H->blocks_per_sm != C->blocks_per_sm || H->chunks_per_block != C->chunks_per_block) {
      H->block = C->block;
      H->blocks_per_sm = C->blocks_per_sm;
      H->chunks_per_block = C->chunks_per_block;
      H->planned_mode = -1;
    }
    SS_TRY(stamp_plan_half(s, *H, mode, st));
    SS_TRY(C->fh.ensure(s->rows_pad_h, st));
    SS_TRY(C->uh.ensure(s->rows_pad_h, st));
    SS_TRY(C->hflag.ensure(1, st));
    if (!C->hflag_host) {
      note_alloc();
      SS_CUDA(cudaMallocHost(&C->hflag_host, sizeof(int32_t)));
    }
    H->plan.inst[0].f = C->fh.get();
    H->plan.inst[0].u = C->uh.get();
    SS_TRY(work_upload(H->work, H->plan, st));
    SS_TRY(work_prologue(H->work, H->plan, C->hflag.get(), st));   // also clears the Hermitian flag
    const unsigned gb = (unsigned)((s->n_plus + 255) / 256), sb = (unsigned)((s->size + 255) / 256);
    k_half_gather<<<gb, 256, 0, st>>>(reinterpret_cast<const double2*>(f_on_S), s->plus_rows.get(), s->mirror.get(),
                                      s->n_plus, C->fh.get(), C->hflag.get());
    SS_LAUNCH_CHECK();
    OpView hop;
    hop.woff = s->woff_h.get();
    hop.ent = s->ent_h.get();
    hop.ecoef = s->ecoef_h.get();
    hop.ecoefdf = s->ecoefdf_h.get();
    hop.colbits = s->colbits_h;
    hop.colmask = (1u << s->colbits_h) - 1u;
    hop.jmask = (1u << s->jbits) - 1u;
    hop.conj = true;
    hop.realc = s->a_real;
    if (!H->work.ev[0]) {
      SS_CUDA(cudaEventCreate(&H->work.ev[0]));
      SS_CUDA(cudaEventCreate(&H->work.ev[1]));
    }
    H->plan.spin_limit = C->wait_ns;
    SS_TRY(launch_solve(H->work, H->plan, hop, nullptr, s->norm_h.get(), s->ca64.get(), s->ca32.get(), s->pn32.get(),
                        tol, max_iter, mode, st, H->work.ev[0], H->work.ev[1], nullptr, true));
    k_half_scatter<<<sb, 256, 0, st>>>(C->uh.get(), s->hpos.get(), s->size, s->n_plus,
                                       reinterpret_cast<double2*>(u_on_S));
    SS_LAUNCH_CHECK();
    SS_CUDA(cudaMemcpyAsync(C->hflag_host, C->hflag.get(), sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    SS_TRY(queue_checks());
    ss_status worst;
    ss_solve_stats one{};
    SS_TRY(read_stats(H->work, 1, &one, &worst, st, H->work.ev[0], H->work.ev[1]));
    C->fh.settle();
    C->uh.settle();
    C->hflag.settle();
    if (pending) SS_TRY(stamp_check_pending(s, C->chk_host));   // may withdraw the half system
    if (*C->hflag_host == 0 && s->half_ok) {
      one.half_system = 1;
      one.real_coefficients = s->a_real;
      if (check_f0 && (C->f0_host->x != 0.0 || C->f0_host->y != 0.0)) {
        one.status = SS_ERR_INVALID;
        if (stats) *stats = one;
        SS_FAIL(SS_ERR_INVALID, "solve: f_hat_0 must be 0 (mean-zero forcing)");
      }
      if (stats) *stats = one;
      return worst;
    }
  }
  SS_TRY(stamp_plan(s, *C, mode, st));
  C->plan.inst[0].f = reinterpret_cast<const double2*>(f_on_S);
  C->plan.inst[0].u = reinterpret_cast<double2*>(u_on_S);
  SS_TRY(work_upload(C->work, C->plan, st));
  SS_TRY(work_prologue(C->work, C->plan, nullptr, st));
  OpView op;
  op.woff = s->slice_off.get();
  op.ent = s->ent.get();
  op.ecoef = s->ecoef64.get();
  op.ecoefdf = s->ecoefdf.get();
  op.colbits = colbits_of(s->jbits);
  op.colmask = colmask_of(s->jbits);
  op.realc = s->a_real;
  if (!C->work.ev[0]) {
    SS_CUDA(cudaEventCreate(&C->work.ev[0]));
    SS_CUDA(cudaEventCreate(&C->work.ev[1]));
  }
  C->plan.spin_limit = C->wait_ns;
  SS_TRY(launch_solve(C->work, C->plan, op, nullptr, s->norm.get(), s->ca64.get(), s->ca32.get(), s->pn32.get(), tol,
                      max_iter, mode, st, C->work.ev[0], C->work.ev[1], s->adr ? s->diag64.get() : nullptr, true));
  SS_TRY(queue_checks());
  ss_status worst;
  ss_solve_stats one{};
  SS_TRY(read_stats(C->work, 1, &one, &worst, st, C->work.ev[0], C->work.ev[1]));
  if (pending) SS_TRY(stamp_check_pending(s, C->chk_host));
  one.real_coefficients = s->a_real;
  if (check_f0 && (C->f0_host->x != 0.0 || C->f0_host->y != 0.0)) {
    one.status = SS_ERR_INVALID;
    if (stats) *stats = one;
    SS_FAIL(SS_ERR_INVALID, "solve: f_hat_0 must be 0 (mean-zero forcing)");
  }
  if (stats) *stats = one;
  return worst;
}

// ------------------------------------------------------ allocation-free solve
//
// solve_noalloc runs the same persistent solver as solve() (the full system,
// never the Hermitian half system; the same work split as solve() with its
// default tile shape) but takes all of its workspace from one file-scope
// device array instead of allocating it.
// It serves callers that may not allocate device memory once they run:
// plug-ins inside a host application that owns all device memory, code that
// must not stall on cudaMalloc (allocation synchronises the device), or code
// that runs under a fixed device-memory budget set at start-up.  The array holds a stamping set of at
// most kNoAllocRows padded rows (stamps of up to 32,736 frequencies, a few MB
// of device memory on every GPU that loads the library, kept until exit).

namespace ss {
namespace {

constexpr int64_t kNoAllocRows = 32768;                 // padded rows of S
constexpr int64_t kNoAllocRecs = kNoAllocRows + 1;      // plus the dummy record
constexpr int kNoAllocChunks = 1024;
constexpr int64_t kNoAllocParts = kNoAllocChunks + 1;

constexpr size_t a256(size_t x) { return (x + 255) / 256 * 256; }

// byte offsets of the workspace inside the array
constexpr size_t kOffXrec = 0;
constexpr size_t kOffU64 = kOffXrec + a256(2 * kNoAllocRecs * sizeof(double2));
constexpr size_t kOffU32 = kOffU64 + a256(2 * kNoAllocRecs * sizeof(double2));
constexpr size_t kOffR = kOffU32 + a256(kNoAllocRecs * sizeof(float4));
constexpr size_t kOffW64 = kOffR + a256(kNoAllocRecs * sizeof(double2));
constexpr size_t kOffPd = kOffW64 + a256(kNoAllocRecs * sizeof(double2));
constexpr size_t kOffSd = kOffPd + a256(kNoAllocRecs * sizeof(double2));
constexpr size_t kOffRhat = kOffSd + a256(kNoAllocRecs * sizeof(double2));
constexpr size_t kOffDlt = kOffRhat + a256(kNoAllocRecs * sizeof(double2));
constexpr size_t kOffW32 = kOffDlt + a256(kNoAllocRecs * sizeof(double2));
constexpr size_t kOffR32 = kOffW32 + a256(kNoAllocRecs * sizeof(float2));
constexpr size_t kOffP32 = kOffR32 + a256(kNoAllocRecs * sizeof(float2));
constexpr size_t kOffS32 = kOffP32 + a256(kNoAllocRecs * sizeof(float2));
constexpr size_t kOffD32 = kOffS32 + a256(kNoAllocRecs * sizeof(float2));
constexpr size_t kOffRdiag = kOffD32 + a256(kNoAllocRecs * sizeof(float2));
constexpr size_t kOffPart = kOffRdiag + a256(kNoAllocRecs * sizeof(double));
constexpr size_t kOffBar = kOffPart + a256(kNoAllocParts * kNQ * sizeof(double));
constexpr size_t kOffCnt = kOffBar + 256;
constexpr size_t kOffErr = kOffCnt + 256;
constexpr size_t kOffState = kOffErr + 256;
constexpr size_t kOffInst = kOffState + a256(sizeof(InstState));
constexpr size_t kOffChunk = kOffInst + a256(sizeof(SolveInst));
constexpr size_t kNoAllocBytes = kOffChunk + a256(kNoAllocChunks * sizeof(Chunk));

}  // namespace
}  // namespace ss

// The shared workspace (one per device; every call uses all of it).
static __device__ __align__(256) unsigned char ss_noalloc_scratch[ss::kNoAllocBytes];

namespace ss {
namespace {

std::mutex g_noalloc_mu;
unsigned char* g_noalloc_base[64] = {};

// Device address of the array for the current device, looked up once per
// device (host code cannot use the array's name as a device address).
ss_status noalloc_base(unsigned char** out) {
  int dev = 0;
  SS_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) SS_FAIL(SS_ERR_INVALID, "solve_noalloc: device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_base[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, ss_noalloc_scratch);
    if (e != cudaSuccess || !p)
      SS_FAIL(SS_ERR_CUDA, "solve_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
    g_noalloc_base[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_noalloc_base[dev];
  return SS_OK;
}

}  // namespace
}  // namespace ss

extern "C" ss_status solve_noalloc(ss_stamp s, const double* f_on_S, double* u_on_S, double tol, int32_t max_iter,
                                   ss_precision prec, ss_solve_stats* stats, void* stream) {
  if (!s || !f_on_S || !u_on_S) SS_FAIL(SS_ERR_INVALID, "solve_noalloc: null argument");
  if (!(tol > 0.0) || max_iter < 1) SS_FAIL(SS_ERR_INVALID, "solve_noalloc: need tol > 0 and max_iter >= 1");
  if (prec != SS_FP64 && prec != SS_FP32) SS_FAIL(SS_ERR_INVALID, "solve_noalloc: bad precision");
  if (s->adr) SS_FAIL(SS_ERR_INVALID, "solve_noalloc: ADR stamps are solved by solve (BiCGStab)");
  if (s->rows_pad > kNoAllocRows)
    SS_FAIL(SS_ERR_INVALID,
            "solve_noalloc: |S| = %lld (%lld padded rows) exceeds the allocation-free workspace of %lld rows",
            (long long)s->size, (long long)s->rows_pad, (long long)kNoAllocRows);
  cudaStream_t st = as_stream(stream);
  unsigned char* base = nullptr;
  SS_TRY(noalloc_base(&base));
  if (!s->slice_off.get() || s->n_slices < 1) SS_FAIL(SS_ERR_INVALID, "solve_noalloc: stamp has no slice table");
  // static work split, as solve() with its default tile shape: the cuts are
  // computed on the device into the workspace's chunk table
  const int mode = prec == SS_FP64 ? 0 : 1;
  SolvePlan plan;
  plan.inst.assign(1, SolveInst{});
  SolveInst& in = plan.inst[0];
  in.row0 = 0;
  in.rows = s->size;
  in.rows_pad = s->rows_pad;
  in.zero_row = s->zero_idx;
  in.coef_off = 0;
  in.dscale = 2.0 * kTwoPiSq * s->a0;
  in.wide = s->wide ? 1 : 0;
  in.f = reinterpret_cast<const double2*>(f_on_S);
  in.u = reinterpret_cast<double2*>(u_on_S);
  plan.block = 1024;
  int grid = 0;
  SS_TRY(max_grid(mode, plan.block, &grid));
  grid = std::min(grid, sm_count());
  const int by_size = (int)std::max<int64_t>(1, s->n_slices / 8);
  // FP64 CG: the vector updates over an even split of the rows (as solve())
  plan.row_split = mode == 0;
  plan_single(plan, s->n_slices, std::min(grid, by_size), s->slice_off.get(), slice_overhead(mode), s->err_dev.get());
  plan.grid = std::min<int>(grid, (int)plan.chunk.size());
  if ((int)plan.chunk.size() > kNoAllocChunks || plan.n_parts > kNoAllocParts)
    SS_FAIL(SS_ERR_INVALID, "solve_noalloc: work split exceeds the workspace tables");
  // pointers into the shared workspace
  auto at = [&](size_t off) { return static_cast<void*>(base + off); };
  SolveInst* d_inst = static_cast<SolveInst*>(at(kOffInst));
  Chunk* d_chunk = static_cast<Chunk*>(at(kOffChunk));
  InstState* d_state = static_cast<InstState*>(at(kOffState));
  unsigned* d_bar = static_cast<unsigned*>(at(kOffBar));
  int* d_cnt = static_cast<int*>(at(kOffCnt));
  int* d_err = static_cast<int*>(at(kOffErr));
  // the array keeps the previous call's contents: the prologue writes the
  // descriptor and the cuts and resets what must start at zero (barrier,
  // counters, error word, instance state); the records are set up below
  SS_TRY(launch_prologue(plan, d_bar, d_cnt, d_err, d_state, nullptr, d_inst, d_chunk, st));
  const int64_t recs = s->rows_pad + 1;
  k_init_solve_records<<<nblk(recs), 256, 0, st>>>(s->norm.get(), recs, nullptr, s->wide,
                                                  static_cast<double2*>(at(kOffXrec)),
                                                  static_cast<double2*>(at(kOffU64)), static_cast<float4*>(at(kOffU32)));
  SS_LAUNCH_CHECK();
  SolveParams P{};
  P.n_inst = 1;
  P.n_chunks = (int)plan.chunk.size();
  P.inst = d_inst;
  P.chunk = d_chunk;
  P.state = d_state;
  P.op.woff = s->slice_off.get();
  P.op.ent = s->ent.get();
  P.op.ecoef = s->ecoef64.get();
  P.op.colbits = colbits_of(s->jbits);
  P.op.colmask = colmask_of(s->jbits);
  P.op.realc = s->a_real;
  P.slice_inst = nullptr;
  P.norm = s->norm.get();
  P.ca64 = s->ca64.get();
  P.ca32 = s->ca32.get();
  P.pn = s->pn32.get();
  P.xrec = static_cast<double2*>(at(kOffXrec));
  P.urec64 = static_cast<double2*>(at(kOffU64));
  P.urec32 = static_cast<float4*>(at(kOffU32));
  P.r = static_cast<double2*>(at(kOffR));
  P.w64 = static_cast<double2*>(at(kOffW64));
  P.pd = static_cast<double2*>(at(kOffPd));
  P.sd = static_cast<double2*>(at(kOffSd));
  P.rhat = static_cast<double2*>(at(kOffRhat));
  P.dlt = static_cast<double2*>(at(kOffDlt));
  P.w32 = static_cast<float2*>(at(kOffW32));
  P.r32 = static_cast<float2*>(at(kOffR32));
  P.p32 = static_cast<float2*>(at(kOffP32));
  P.s32 = static_cast<float2*>(at(kOffS32));
  P.d32 = static_cast<float2*>(at(kOffD32));
  P.rdiag = static_cast<double*>(at(kOffRdiag));
  P.part = static_cast<double*>(at(kOffPart));
  P.bar = d_bar;
  P.counters = d_cnt;
  P.err = d_err;
  P.tol = tol;
  P.inner_tol = 1e-5;
  P.max_iter = max_iter;
  P.max_inner = std::max(1, std::min(max_iter, 200));
  P.max_outer = std::max(1, max_iter);
  P.spin_limit = 2000000000ll;
  P.rows_slices = plan.row_split ? plan.cut_n : 0;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(plan.grid);
  cfg.blockDim = dim3(plan.block);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (mode == 0) SS_CUDA(cudaLaunchKernelEx(&cfg, k_solve<0>, P));
  else SS_CUDA(cudaLaunchKernelEx(&cfg, k_solve<1>, P));
  // statistics, error word and f_hat_0 read back with one synchronisation
  InstState hs;
  int herr = 0;
  double2 f0 = make_double2(0.0, 0.0);
  SS_CUDA(cudaMemcpyAsync(&hs, d_state, sizeof(hs), cudaMemcpyDeviceToHost, st));
  SS_CUDA(cudaMemcpyAsync(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  if (s->zero_idx >= 0)
    SS_CUDA(cudaMemcpyAsync(&f0, reinterpret_cast<const double2*>(f_on_S) + s->zero_idx, sizeof(f0),
                            cudaMemcpyDeviceToHost, st));
  SS_CUDA(cudaStreamSynchronize(st));
  const double rel = hs.bb > 0 ? std::sqrt(hs.rr / hs.bb) : 0.0;
  if (stats) {
    stats->status = herr ? herr : hs.status;
    stats->outer_iters = hs.outer_iters;
    stats->inner_iters = hs.inner_iters ? hs.inner_iters : hs.iters;
    stats->applies = hs.applies;
    stats->rel_residual = rel;
    stats->kernel_ms = 0.0;
    stats->half_system = 0;
    stats->real_coefficients = s->a_real;
  }
  if (f0.x != 0.0 || f0.y != 0.0) {
    if (stats) stats->status = SS_ERR_INVALID;
    SS_FAIL(SS_ERR_INVALID, "solve_noalloc: f_hat_0 must be 0 (mean-zero forcing)");
  }
  if (herr) SS_FAIL((ss_status)herr, "solve_noalloc: a device-side wait gave up (status %d)", herr);
  if (hs.status != SS_OK) SS_FAIL((ss_status)hs.status, "solve_noalloc: not converged (relative residual %.3e)", rel);
  return SS_OK;
}
