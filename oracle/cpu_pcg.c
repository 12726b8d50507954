/* TEST INFRASTRUCTURE ONLY: the multi-core CPU baseline of the oracle's solve.
 * The library never links it.  Jacobi-preconditioned CG (Algorithm 1, last
 * step) on the explicit CSR operator that oracle.galerkin.galerkin_matrix
 * assembles from eq. GF, complex FP64 values interleaved (re, im), with the
 * recurrences of oracle.solve.pcg; the sparse products and the inner products
 * run row-parallel over OpenMP threads. */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static void spmv(int64_t n, const int64_t* ip, const int32_t* ix, const double* v, const double* x, double* y) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double re = 0.0, im = 0.0;
    for (int64_t e = ip[i]; e < ip[i + 1]; ++e) {
      const double ar = v[2 * e], ai = v[2 * e + 1];
      const double xr = x[2 * (int64_t)ix[e]], xi = x[2 * (int64_t)ix[e] + 1];
      re += ar * xr - ai * xi;
      im += ar * xi + ai * xr;
    }
    y[2 * i] = re;
    y[2 * i + 1] = im;
  }
}

/* Re sum conj(a_i) b_i */
static double dot_re(int64_t n, const double* a, const double* b) {
  double s = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : s)
  for (int64_t i = 0; i < 2 * n; ++i) s += a[i] * b[i];
  return s;
}

static void precondition(int64_t n, const double* r, const double* D, double* z) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    z[2 * i] = r[2 * i] / D[i];
    z[2 * i + 1] = r[2 * i + 1] / D[i];
  }
}

/* Solves L x = b from x = 0 until ||r|| <= tol ||b|| (recursive residual) or
 * max_iter iterations; x holds 2n doubles.  Returns the number of iterations,
 * or -1 when a work vector cannot be allocated. */
int pcg_csr(int64_t n, const int64_t* ip, const int32_t* ix, const double* v, const double* b, const double* D,
            double tol, int max_iter, int threads, double* x) {
#ifdef _OPENMP
  if (threads > 0) omp_set_num_threads(threads);
#endif
  double* r = malloc(sizeof(double) * 2 * n);
  double* z = malloc(sizeof(double) * 2 * n);
  double* p = malloc(sizeof(double) * 2 * n);
  double* q = malloc(sizeof(double) * 2 * n);
  if (!r || !z || !p || !q) {
    free(r); free(z); free(p); free(q);
    return -1;
  }
  memset(x, 0, sizeof(double) * 2 * n);
  memcpy(r, b, sizeof(double) * 2 * n);
  const double bnorm = sqrt(dot_re(n, b, b));
  int it = 0;
  if (bnorm > 0.0) {
    precondition(n, r, D, z);
    memcpy(p, z, sizeof(double) * 2 * n);
    double rho = dot_re(n, r, z);
    double rn = 1.0;
    while (rn > tol && it < max_iter) {
      spmv(n, ip, ix, v, p, q);
      const double alpha = rho / dot_re(n, p, q);
#pragma omp parallel for schedule(static)
      for (int64_t i = 0; i < 2 * n; ++i) {
        x[i] += alpha * p[i];
        r[i] -= alpha * q[i];
      }
      ++it;
      rn = sqrt(dot_re(n, r, r)) / bnorm;
      precondition(n, r, D, z);
      const double rho_new = dot_re(n, r, z);
      const double beta = rho_new / rho;
#pragma omp parallel for schedule(static)
      for (int64_t i = 0; i < 2 * n; ++i) p[i] = z[i] + beta * p[i];
      rho = rho_new;
    }
  }
  free(r); free(z); free(p); free(q);
  return it;
}

int pcg_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
