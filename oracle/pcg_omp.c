/*
 * Jacobi-preconditioned conjugate gradients (Section 3.1 of Zhu & Gleich,
 * arXiv:1501.03105) in plain C with OpenMP, FP64 throughout.
 *
 * TEST INFRASTRUCTURE ONLY: this file belongs to the oracle.  It is called
 * by the oracle's Python wrapper (oracle/pcg_omp.py), which only tests/, the
 * smoke check and the CPU-baseline leg of bench.py use; it shares no code
 * with the CUDA library.
 *
 * It is the recurrence of oracle.pirmcut.pcg_jacobi written out in C, the
 * same steps in the same order, with the matrix-vector product, the vector
 * updates and the inner products split over OpenMP threads (the CPU baseline
 * of the design is timed on one thread and on every host core):
 *   r = b - A x;  stop if ||r|| <= tol ||b||
 *   z = D^-1 r;  p = z;  rz = (r, z)
 *   repeat:  q = A p;  alpha = rz / (p, q);  x += alpha p;  r -= alpha q
 *            stop if ||r|| <= tol ||b|| or maxit reached
 *            z = D^-1 r;  rz' = (r, z);  beta = rz' / rz;  p = z + beta p
 * A is a symmetric positive definite CSR matrix (the reduced Laplacian
 * L~ of Eq. reduced-laplacian-system), D its diagonal.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#ifdef _OPENMP
#include <omp.h>
#endif

static void spmv(int64_t n, const int64_t* indptr, const int32_t* indices, const double* data,
                 const double* v, double* out) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int64_t e = indptr[i]; e < indptr[i + 1]; ++e) s += data[e] * v[indices[e]];
    out[i] = s;
  }
}

static double dot(int64_t n, const double* a, const double* b) {
  double s = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : s)
  for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

/*
 * x holds the start vector on entry and the solution on return.
 * Returns 0 on success, 1 when a buffer could not be allocated, 2 when the
 * matrix has a zero on its diagonal.  *iters receives the iterations taken,
 * *rel the final ||r|| / ||b|| of the recurrence (0 when b = 0).
 */
int oracle_pcg_jacobi(int64_t n, const int64_t* indptr, const int32_t* indices,
                      const double* data, const double* b, double* x, double tol, int64_t maxit,
                      int threads, int64_t* iters, double* rel) {
#ifdef _OPENMP
  if (threads > 0) omp_set_num_threads(threads);
#else
  (void)threads;
#endif
  *iters = 0;
  *rel = 0.0;
  double* dinv = (double*)malloc(sizeof(double) * (size_t)(n ? n : 1));
  double* r = (double*)malloc(sizeof(double) * (size_t)(n ? n : 1));
  double* z = (double*)malloc(sizeof(double) * (size_t)(n ? n : 1));
  double* p = (double*)malloc(sizeof(double) * (size_t)(n ? n : 1));
  double* q = (double*)malloc(sizeof(double) * (size_t)(n ? n : 1));
  int status = 0;
  if (!dinv || !r || !z || !p || !q) {
    status = 1;
    goto done;
  }
  /* the diagonal of A */
  for (int64_t i = 0; i < n; ++i) {
    double d = 0.0;
    for (int64_t e = indptr[i]; e < indptr[i + 1]; ++e)
      if (indices[e] == i) d += data[e];
    if (d == 0.0) {
      status = 2;
      goto done;
    }
    dinv[i] = 1.0 / d;
  }
  const double bnorm = sqrt(dot(n, b, b));
  if (bnorm == 0.0) {
    for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
    goto done;
  }
  spmv(n, indptr, indices, data, x, q);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) r[i] = b[i] - q[i];
  double rnorm = sqrt(dot(n, r, r));
  if (rnorm <= tol * bnorm) {
    *rel = rnorm / bnorm;
    goto done;
  }
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    z[i] = dinv[i] * r[i];
    p[i] = z[i];
  }
  double rz = dot(n, r, z);
  int64_t it = 0;
  while (it < maxit) {
    spmv(n, indptr, indices, data, p, q);
    const double alpha = rz / dot(n, p, q);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
      x[i] += alpha * p[i];
      r[i] -= alpha * q[i];
    }
    ++it;
    rnorm = sqrt(dot(n, r, r));
    if (rnorm <= tol * bnorm) break;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) z[i] = dinv[i] * r[i];
    const double rz_new = dot(n, r, z);
    const double beta = rz_new / rz;
    rz = rz_new;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
  }
  *iters = it;
  *rel = rnorm / bnorm;
done:
  free(dinv);
  free(r);
  free(z);
  free(p);
  free(q);
  return status;
}

/* Threads an OpenMP parallel region of this library gets by default. */
int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
