/* CPU block PCG baseline for the transfer matrix T = A^-1 B (test and
 * measurement infrastructure, not part of the GPU library).
 *
 * The paper's forward solve (Sec. 2.3.1) is a conjugate-gradient iteration
 * with a diagonal preconditioner, one right-hand side per electrode
 * (App. A.4: each column of T solves A t = b for one column of B).  This is
 * that iteration in plain FP64 C, every column an independent PCG run, the
 * columns stored side by side (node-major n x L) so that one pass over the
 * sparse matrix serves all of them.  Rows are split over OpenMP threads; dot
 * products are summed per thread and then in thread order.
 *
 *   precond 0: Jacobi, d_i = a_ii;  1: lumped diagonal, d_i = sum_j |a_ij|.
 *   A column stops once its recurrence residual satisfies |r|_2 <= tol |b|_2.
 *   Returns the largest iteration count, or -1 on bad arguments / memory.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static int nthreads_of(int req) {
#ifdef _OPENMP
  return req > 0 ? req : omp_get_max_threads();
#else
  (void)req;
  return 1;
#endif
}

int zi_cpu_block_pcg(int64_t n, const int32_t* rowptr, const int32_t* colind, const double* vals, int L,
                     const double* B, double tol, int maxit, int precond, double* T, int32_t* iters,
                     int nthreads) {
  if (n <= 0 || L <= 0 || !rowptr || !colind || !vals || !B || !T) return -1;
  const int nt = nthreads_of(nthreads);
  const size_t nl = (size_t)n * (size_t)L;
  double* dinv = malloc(sizeof(double) * (size_t)n);
  double* R = malloc(sizeof(double) * nl);
  double* P = malloc(sizeof(double) * nl);
  double* Q = malloc(sizeof(double) * nl);
  double* part = calloc((size_t)nt * 3 * (size_t)L, sizeof(double));
  double* rho = malloc(sizeof(double) * (size_t)L);
  double* stop2 = malloc(sizeof(double) * (size_t)L);
  double* alpha = malloc(sizeof(double) * (size_t)L);
  double* beta = malloc(sizeof(double) * (size_t)L);
  int* active = malloc(sizeof(int) * (size_t)L);
  int rc = 0;
  if (!dinv || !R || !P || !Q || !part || !rho || !stop2 || !alpha || !beta || !active) {
    rc = -1;
    goto done;
  }
  /* preconditioner */
  for (int64_t i = 0; i < n; ++i) {
    double d = 0.0;
    for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
      if (precond == 1)
        d += fabs(vals[k]);
      else if (colind[k] == i)
        d = vals[k];
    }
    dinv[i] = d != 0.0 ? 1.0 / d : 0.0;
  }
  /* x = 0, r = b, p = D^-1 r; rho = r.D^-1 r; stop2 = tol^2 |b|^2 */
  memset(T, 0, sizeof(double) * nl);
  memcpy(R, B, sizeof(double) * nl);
  for (int c = 0; c < L; ++c) rho[c] = stop2[c] = 0.0;
  for (int64_t i = 0; i < n; ++i)
    for (int c = 0; c < L; ++c) {
      const double r = R[i * L + c];
      P[i * L + c] = dinv[i] * r;
      rho[c] += r * dinv[i] * r;
      stop2[c] += r * r;
    }
  int nact = 0;
  for (int c = 0; c < L; ++c) {
    stop2[c] *= tol * tol;
    active[c] = stop2[c] > 0.0;
    nact += active[c];
    if (iters) iters[c] = 0;
  }
  int it = 0;
  while (nact > 0 && it < maxit) {
    /* Q = A P and the column dots p.q */
    memset(part, 0, sizeof(double) * (size_t)nt * 3 * (size_t)L);
#pragma omp parallel num_threads(nt)
    {
#ifdef _OPENMP
      const int t = omp_get_thread_num();
#else
      const int t = 0;
#endif
      double* pq = part + (size_t)t * 3 * L;
#pragma omp for schedule(static)
      for (int64_t i = 0; i < n; ++i) {
        double* q = Q + i * L;
        for (int c = 0; c < L; ++c) q[c] = 0.0;
        for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
          const double a = vals[k];
          const double* p = P + (int64_t)colind[k] * L;
          for (int c = 0; c < L; ++c) q[c] += a * p[c];
        }
        const double* p = P + i * L;
        for (int c = 0; c < L; ++c) pq[c] += p[c] * q[c];
      }
    }
    for (int c = 0; c < L; ++c) {
      double s = 0.0;
      for (int t = 0; t < nt; ++t) s += part[(size_t)t * 3 * L + c];
      alpha[c] = (active[c] && s > 0.0) ? rho[c] / s : 0.0;
    }
    /* x += alpha p, r -= alpha q, with r.r and r.D^-1 r */
    memset(part, 0, sizeof(double) * (size_t)nt * 3 * (size_t)L);
#pragma omp parallel num_threads(nt)
    {
#ifdef _OPENMP
      const int t = omp_get_thread_num();
#else
      const int t = 0;
#endif
      double* rr = part + (size_t)t * 3 * L + L;
      double* rz = part + (size_t)t * 3 * L + 2 * L;
#pragma omp for schedule(static)
      for (int64_t i = 0; i < n; ++i)
        for (int c = 0; c < L; ++c) {
          const int64_t e = i * L + c;
          T[e] += alpha[c] * P[e];
          const double r = R[e] - alpha[c] * Q[e];
          R[e] = r;
          rr[c] += r * r;
          rz[c] += r * dinv[i] * r;
        }
    }
    ++it;
    nact = 0;
    for (int c = 0; c < L; ++c) {
      double rr = 0.0, rz = 0.0;
      for (int t = 0; t < nt; ++t) {
        rr += part[(size_t)t * 3 * L + L + c];
        rz += part[(size_t)t * 3 * L + 2 * L + c];
      }
      beta[c] = 0.0;
      if (!active[c]) continue;
      if (iters) iters[c] = it;
      if (rr <= stop2[c] || !(rz > 0.0)) {
        active[c] = 0;
        continue;
      }
      beta[c] = rz / rho[c];
      rho[c] = rz;
      ++nact;
    }
    /* p = D^-1 r + beta p for the columns still running */
#pragma omp parallel for num_threads(nt) schedule(static)
    for (int64_t i = 0; i < n; ++i)
      for (int c = 0; c < L; ++c)
        if (active[c]) P[i * L + c] = dinv[i] * R[i * L + c] + beta[c] * P[i * L + c];
  }
  rc = it;
done:
  free(dinv);
  free(R);
  free(P);
  free(Q);
  free(part);
  free(rho);
  free(stop2);
  free(alpha);
  free(beta);
  free(active);
  return rc;
}
