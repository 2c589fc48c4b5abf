/*
 * CPU oracle for the eigenvalues of a real symmetric tridiagonal matrix
 * T = tridiag(e, d, e) -- TEST INFRASTRUCTURE ONLY.
 *
 * Only tests/, __graft_entry__.smoke() and the cpu_baseline / reference leg of
 * bench.py may load this library.  The CUDA solver never calls it, shares no
 * code with it, and fails loudly if its own extension is missing.
 *
 * What is computed is the plain definition of the result of the paper's
 * eigenvalue-only divide and conquer (Sec. 3.1 problem setting; Theorem
 * "BR computes the same eigenvalues as conventional D&C"): the multiset of
 * eigenvalues of T, in ascending order.  Two independent routes:
 *
 *  1. Sturm-count bisection (oracle_eigvals_bisect / _select).  The number of
 *     eigenvalues of T below x equals the number of negative pivots of the
 *     LDL^T factorisation of T - xI (Sylvester's law of inertia):
 *         q_1 = d_1 - x,   q_i = (d_i - x) - e_{i-1}^2 / q_{i-1}.
 *     A pivot whose magnitude falls below pivmin is replaced by -pivmin so the
 *     recurrence never divides by zero; pivmin = DBL_MIN * max(1, max e_i^2).
 *     Eigenvalue k (0-based) is the infimum of {x : count(x) > k}; it is
 *     bracketed by the Gershgorin interval and bisected until the bracket is
 *     narrower than max(2 eps |x|, eps ||T||_1), eps = DBL_EPSILON.
 *
 *     The same count for many query points (oracle_sturm_counts) certifies a
 *     computed spectrum without bisecting it: lambda_k lies in [x - g, x + g)
 *     exactly when count(x - g) <= k and count(x + g) >= k + 1.
 *
 *  2. Dense cyclic Jacobi (oracle_jacobi_eigh) for n <= 64: a sweep of plane
 *     rotations that annihilate each off-diagonal entry in turn until the
 *     off-diagonal Frobenius mass is below 1e-30 of the total.  Returns
 *     eigenvalues and eigenvectors (columns), unsorted.
 *
 * Both are plain loops in IEEE double precision; the bisection loop runs one
 * eigenvalue index per OpenMP iteration.  Nothing here is blocked, fused or
 * reordered beyond the definitions above.
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ||T||_1 = max_j (|e_{j-1}| + |d_j| + |e_j|), the gate's matrix norm. */
double oracle_tridiag_norm1(int64_t n, const double* d, const double* e) {
  double best = 0.0;
  for (int64_t j = 0; j < n; ++j) {
    double s = fabs(d[j]);
    if (j > 0) s += fabs(e[j - 1]);
    if (j + 1 < n) s += fabs(e[j]);
    if (s > best) best = s;
  }
  return best;
}

static double pivmin_of(int64_t n, const double* e) {
  double m = 1.0;
  for (int64_t i = 0; i + 1 < n; ++i) {
    double t = e[i] * e[i];
    if (t > m) m = t;
  }
  return DBL_MIN * m;
}

/* Number of eigenvalues of T strictly below x (negative LDL^T pivots). */
int64_t oracle_sturm_count(int64_t n, const double* d, const double* e, double x) {
  double pivmin = pivmin_of(n, e);
  int64_t count = 0;
  double q = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    if (i == 0) {
      q = d[0] - x;
    } else {
      q = (d[i] - x) - (e[i - 1] * e[i - 1]) / q;
    }
    if (fabs(q) < pivmin) q = -pivmin;
    if (q < 0.0) ++count;
  }
  return count;
}

/* Same count with a precomputed pivmin and squared off-diagonals. */
static int64_t count_below(int64_t n, const double* d, const double* e2, double pivmin,
                           double x) {
  int64_t count = 0;
  double q = d[0] - x;
  if (fabs(q) < pivmin) q = -pivmin;
  if (q < 0.0) ++count;
  for (int64_t i = 1; i < n; ++i) {
    q = (d[i] - x) - e2[i - 1] / q;
    if (fabs(q) < pivmin) q = -pivmin;
    if (q < 0.0) ++count;
  }
  return count;
}

static void gershgorin(int64_t n, const double* d, const double* e, double* lo, double* hi) {
  double a = INFINITY, b = -INFINITY;
  for (int64_t j = 0; j < n; ++j) {
    double r = 0.0;
    if (j > 0) r += fabs(e[j - 1]);
    if (j + 1 < n) r += fabs(e[j]);
    if (d[j] - r < a) a = d[j] - r;
    if (d[j] + r > b) b = d[j] + r;
  }
  *lo = a;
  *hi = b;
}

/* Eigenvalues with 0-based ascending indices ks[0..nk) -> out[0..nk).
 * Returns the number of OpenMP threads used. */
int oracle_eigvals_bisect_select(int64_t n, const double* d, const double* e, int64_t nk,
                                 const int64_t* ks, double* out) {
  if (n <= 0 || nk <= 0) return 0;
  double* e2 = (double*)malloc(sizeof(double) * (size_t)(n > 1 ? n - 1 : 1));
  for (int64_t i = 0; i + 1 < n; ++i) e2[i] = e[i] * e[i];
  double pivmin = pivmin_of(n, e);
  double tnorm = oracle_tridiag_norm1(n, d, e);
  double glo, ghi;
  gershgorin(n, d, e, &glo, &ghi);
  /* widen so that count(glo) = 0 and count(ghi) = n hold after rounding */
  double pad = 2.0 * DBL_EPSILON * tnorm + 2.0 * pivmin;
  glo -= pad;
  ghi += pad;
  double abstol = DBL_EPSILON * tnorm;
  int used = 1;
#pragma omp parallel
  {
#ifdef _OPENMP
#pragma omp single
    used = omp_get_num_threads();
#endif
#pragma omp for schedule(dynamic, 4)
    for (int64_t t = 0; t < nk; ++t) {
      int64_t k = ks[t];
      double lo = glo, hi = ghi; /* invariant: count(lo) <= k < count(hi) */
      for (int it = 0; it < 200; ++it) {
        double width = hi - lo;
        double scale = fmax(fabs(lo), fabs(hi));
        if (width <= fmax(2.0 * DBL_EPSILON * scale, abstol)) break;
        double mid = lo + 0.5 * width;
        if (mid <= lo || mid >= hi) break;
        if (count_below(n, d, e2, pivmin, mid) > k)
          hi = mid;
        else
          lo = mid;
      }
      out[t] = lo + 0.5 * (hi - lo);
    }
  }
  free(e2);
  return used;
}

/* counts[t] = number of eigenvalues of T strictly below xs[t], t in [0, nx): the
 * count of count_below for many query points (used to certify a computed
 * spectrum: lambda_k >= x  <=>  count(x) <= k, and lambda_k < x  <=>  count(x) >= k+1).
 * Query points are taken eight at a time so that the eight independent pivot
 * recurrences share one pass over d and e; each recurrence performs exactly the
 * operations of count_below, in the same order, so every count equals the
 * single-point count bit for bit.  Returns the number of OpenMP threads used. */
int oracle_sturm_counts(int64_t n, const double* d, const double* e, int64_t nx,
                        const double* xs, int64_t* counts) {
  if (nx <= 0) return 0;
  if (n <= 0) {
    for (int64_t t = 0; t < nx; ++t) counts[t] = 0;
    return 1;
  }
  double* e2 = (double*)malloc(sizeof(double) * (size_t)(n > 1 ? n - 1 : 1));
  for (int64_t i = 0; i + 1 < n; ++i) e2[i] = e[i] * e[i];
  const double pivmin = pivmin_of(n, e);
  int used = 1;
#pragma omp parallel
  {
#ifdef _OPENMP
#pragma omp single
    used = omp_get_num_threads();
#endif
#pragma omp for schedule(dynamic, 1)
    for (int64_t t0 = 0; t0 < nx; t0 += 8) {
      const int64_t nb = (nx - t0 < 8) ? nx - t0 : 8;
      double x[8], q[8];
      int64_t c[8];
      for (int j = 0; j < 8; ++j) {
        x[j] = xs[t0 + (j < nb ? j : nb - 1)];
        q[j] = d[0] - x[j];
        if (fabs(q[j]) < pivmin) q[j] = -pivmin;
        c[j] = (q[j] < 0.0) ? 1 : 0;
      }
      for (int64_t i = 1; i < n; ++i) {
        for (int j = 0; j < 8; ++j) {
          q[j] = (d[i] - x[j]) - e2[i - 1] / q[j];
          if (fabs(q[j]) < pivmin) q[j] = -pivmin;
          c[j] += (q[j] < 0.0) ? 1 : 0;
        }
      }
      for (int64_t j = 0; j < nb; ++j) counts[t0 + j] = c[j];
    }
  }
  free(e2);
  return used;
}

/* All n eigenvalues in ascending order.  Returns the OpenMP thread count. */
int oracle_eigvals_bisect(int64_t n, const double* d, const double* e, double* lam) {
  if (n <= 0) return 0;
  int64_t* ks = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  for (int64_t k = 0; k < n; ++k) ks[k] = k;
  int used = oracle_eigvals_bisect_select(n, d, e, n, ks, lam);
  free(ks);
  return used;
}

/* Dense symmetric eigen-decomposition by cyclic Jacobi, n <= 64.
 * a: n*n row-major symmetric (destroyed); w: eigenvalues; v: n*n row-major,
 * column j is the eigenvector of w[j].  Returns the number of sweeps, or -1 if
 * 100 sweeps did not converge. */
int oracle_jacobi_eigh(int n, double* a, double* w, double* v) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) v[i * n + j] = (i == j) ? 1.0 : 0.0;
  double total = 0.0;
  for (int i = 0; i < n * n; ++i) total += a[i] * a[i];
  int sweep;
  for (sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) off += 2.0 * a[p * n + q] * a[p * n + q];
    if (off <= 1e-30 * total || off == 0.0) break;
    for (int p = 0; p < n; ++p) {
      for (int q = p + 1; q < n; ++q) {
        double apq = a[p * n + q];
        if (apq == 0.0) continue;
        double app = a[p * n + p], aqq = a[q * n + q];
        /* rotation angle that zeroes a_pq: cot(2 phi) = (aqq - app) / (2 apq) */
        double theta = (aqq - app) / (2.0 * apq);
        double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        double c = 1.0 / sqrt(t * t + 1.0);
        double s = t * c;
        /* A <- J^T A J with J the (p,q) plane rotation [c s; -s c] */
        for (int k = 0; k < n; ++k) {
          double akp = a[k * n + p], akq = a[k * n + q];
          a[k * n + p] = c * akp - s * akq;
          a[k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {
          double apk = a[p * n + k], aqk = a[q * n + k];
          a[p * n + k] = c * apk - s * aqk;
          a[q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          double vkp = v[k * n + p], vkq = v[k * n + q];
          v[k * n + p] = c * vkp - s * vkq;
          v[k * n + q] = s * vkp + c * vkq;
        }
      }
    }
  }
  for (int i = 0; i < n; ++i) w[i] = a[i * n + i];
  return sweep < 100 ? sweep : -1;
}
