// Algorithm 1 of the paper in one library call: lattice, SFT of a and of f on
// it, stamping set S^N[a_hat](supp f_hat), right-hand side on S and the solve.
// The stages are the library's own entry points, called back to back on one
// stream; running them from here keeps the host between two stages in native
// code (the stages that must read a size back synchronise, as they do when
// called one by one).
#include <algorithm>
#include <vector>

#include "ss_internal.cuh"

using namespace ss;

namespace {

ss_status choose_lattice(const ss_lattice_spec* ls, const int32_t* cand, int64_t n_cand, int64_t* z, int64_t* M,
                         cudaStream_t st) {
  const int d = ls->d;
  switch (ls->kind) {
    case SS_LATTICE_GIVEN:
      if (!ls->z || ls->M < 2) SS_FAIL(SS_ERR_INVALID, "sparse_spectral_solve: given lattice needs z and M >= 2");
      std::copy(ls->z, ls->z + d, z);
      *M = ls->M;
      return SS_OK;
    case SS_LATTICE_CBC:
      return lattice_cbc(cand, n_cand, d, ls->M_min, ls->raw, ls->n_raw, z, M, st);
    case SS_LATTICE_RANDOM:
    case SS_LATTICE_RANDOM_SMOOTH: {
      int32_t attempt = 0;
      auto fn = ls->kind == SS_LATTICE_RANDOM ? lattice_random : lattice_random_smooth;
      return fn(cand, n_cand, d, ls->sigma, ls->M_min, ls->raw, ls->n_raw, z, M, &attempt, st);
    }
    default:
      SS_FAIL(SS_ERR_INVALID, "sparse_spectral_solve: unknown lattice kind %d", (int)ls->kind);
  }
}

ss_status run(const ss_lattice_spec* ls, const ss_trig* a, const ss_trig* f, const int32_t* cand, int64_t n_cand,
              int32_t N, double tau, ss_precision sft_prec, ss_precision solve_prec, double tol, int32_t max_iter,
              int64_t* z_out, int64_t* M_out, ss_stamp* stamp_out, double* u_out, int64_t u_cap,
              ss_solve_stats* stats, cudaStream_t st) {
  const int d = ls->d;
  std::vector<int64_t> z(d, 1);
  int64_t M = 0;
  SS_TRY(choose_lattice(ls, cand, n_cand, z.data(), &M, st));
  const ss_lattice lat{d, M, z.data()};
  // recovered coefficients: at most one per candidate
  DevBuf<int32_t> af, ff;
  DevBuf<double2> av, fv;
  SS_TRY(af.alloc_tmp((size_t)n_cand * d, st));
  SS_TRY(ff.alloc_tmp((size_t)n_cand * d, st));
  SS_TRY(av.alloc_tmp(n_cand, st));
  SS_TRY(fv.alloc_tmp(n_cand, st));
  int64_t n_a = 0, n_f = 0;
  SS_TRY(sft_recover_both(&lat, a, f, sft_prec, cand, n_cand, tau, af.get(), reinterpret_cast<double*>(av.get()), &n_a,
                          ff.get(), reinterpret_cast<double*>(fv.get()), &n_f, st));
  if (n_a < 1 || n_f < 1)
    SS_FAIL(SS_ERR_INVALID, "sparse_spectral_solve: %s has no coefficient above the threshold", n_a < 1 ? "a" : "f");
  const ss_sparse a_hat{d, n_a, af.get(), reinterpret_cast<const double*>(av.get())};
  ss_stamp s = nullptr;
  // the build's final error words are read with the solve's statistics (one
  // synchronisation fewer between the stamp and the solve)
  SS_TRY(stamp_build_pending(&a_hat, ff.get(), n_f, N, &s, st));
  ss_status r = SS_OK;
  do {
    r = s->sol.alloc(std::max<int64_t>(s->size, 1), st);
    if (r != SS_OK) break;
    r = s->rhs.alloc(std::max<int64_t>(s->size, 1), st);
    if (r != SS_OK) break;
    const ss_sparse f_hat{d, n_f, ff.get(), reinterpret_cast<const double*>(fv.get())};
    r = stamp_scatter(s, &f_hat, reinterpret_cast<double*>(s->rhs.get()), nullptr, st);
    if (r != SS_OK) break;
    r = solve(s, reinterpret_cast<const double*>(s->rhs.get()), reinterpret_cast<double*>(s->sol.get()), tol,
              max_iter, solve_prec, stats, st);
    s->sol_size = s->size;
    if (u_out && s->size <= u_cap) {
      const cudaError_t e = cudaMemcpyAsync(u_out, s->sol.get(), s->size * sizeof(double2),
                                            cudaMemcpyDeviceToDevice, st);
      if (e != cudaSuccess) {
        set_error("sparse_spectral_solve: copy of the solution failed: %s", cudaGetErrorString(e));
        r = SS_ERR_CUDA;
      }
    }
    // both buffers outlive this call (solve synchronised the stream)
    s->sol.settle();
    s->rhs.settle();
  } while (false);
  if (s->check_pending) {   // the solve stopped before it read the build's error words
    const ss_status rc = stamp_host_tables(s, st);
    if (rc != SS_OK) r = rc;
  }
  if (r != SS_OK && r != SS_ERR_NOT_CONVERGED) {
    const std::string msg = ss_last_error();
    stamp_destroy(s);
    SS_FAIL(r, "%s", msg.c_str());
  }
  std::copy(z.begin(), z.end(), z_out);
  *M_out = M;
  *stamp_out = s;
  return r;
}

}  // namespace

extern "C" ss_status sparse_spectral_solve(const ss_lattice_spec* lat, const ss_trig* a, const ss_trig* f,
                                           const int32_t* cand, int64_t n_cand, int32_t N, double tau,
                                           ss_precision sft_prec, ss_precision solve_prec, double tol,
                                           int32_t max_iter, int64_t* z_out, int64_t* M_out, ss_stamp* stamp_out,
                                           double* u_out, int64_t u_cap, ss_solve_stats* stats, void* stream) {
  if (!lat || !a || !f || !cand || n_cand < 1 || !z_out || !M_out || !stamp_out)
    SS_FAIL(SS_ERR_INVALID, "sparse_spectral_solve: null argument");
  *stamp_out = nullptr;
  if (lat->d < 1 || a->d != lat->d || f->d != lat->d)
    SS_FAIL(SS_ERR_INVALID, "sparse_spectral_solve: dimensions of the lattice, a and f differ");
  return run(lat, a, f, cand, n_cand, N, tau, sft_prec, solve_prec, tol, max_iter, z_out, M_out, stamp_out, u_out,
             u_cap, stats, as_stream(stream));
}

extern "C" ss_status stamp_solution(ss_stamp s, double* u_out, void* stream) {
  if (!s || !u_out) SS_FAIL(SS_ERR_INVALID, "stamp_solution: null argument");
  if (s->sol_size <= 0 || !s->sol.get())
    SS_FAIL(SS_ERR_INVALID, "stamp_solution: the stamp holds no solution (made by sparse_spectral_solve)");
  SS_CUDA(cudaMemcpyAsync(u_out, s->sol.get(), s->sol_size * sizeof(double2), cudaMemcpyDeviceToDevice,
                          as_stream(stream)));
  return SS_OK;
}
