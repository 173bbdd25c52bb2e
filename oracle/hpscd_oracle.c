/*
 * CPU oracle for the HPSCD column sweep (Algorithm 1 of "Algorithmic Solution
 * for Systems of Linear Equations, in O(mn) time").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or calls
 * this file: only the tests, the smoke check and the benchmark's CPU-baseline
 * leg do.  It shares no code, header or constant with the CUDA library.
 *
 * Arithmetic: IEEE float64 throughout, strictly sequential summation order
 * (i = 0..m-1), true division.  X is read in its stored type (float32,
 * bfloat16 or IEEE binary16 bit patterns, or float64) and promoted exactly to
 * float64, so the system being solved is exactly the stored one.
 *
 * Readings of the paper taken here (each is listed in the design notes):
 *   - the residual is e = y - X·a (Algorithm 1, the initialisation of e, and
 *     Sec. 3), not X·a - y as the prose of Sec. 2 once writes it;
 *   - a column with <X_j,X_j> = 0 is skipped (da = 0): the paper is silent;
 *   - the stopping test ("break if under a certain threshold", Sec. 2) runs
 *     once per sweep, after column n, on r_s = ||e_s||_2 / ||y||_2
 *     (r_s = ||e_s||_2 when y = 0);
 *       REL_RES:    stop after sweep s >= 0 when r_s <= tol
 *       REL_CHANGE: stop after sweep s >= 1 when |r_{s-1} - r_s| < tol * r_{s-1}
 *                   (or when r_{s-1} == 0)
 *       NONE:       run exactly max_sweeps sweeps;
 *   - hist[0] is the residual of the initial guess (before any sweep).
 * Parity status: pinned (closed forms, Gaussian elimination, normal-equation
 * least squares, orthogonality and monotonicity invariants, Gauss-Seidel
 * equivalence), see tests/test_oracle_pins.py.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_F32 0
#define OR_BF16 1
#define OR_F64 2
#define OR_F16 3
#define OR_COL 0
#define OR_ROW 1
#define OR_STOP_REL_RES 0
#define OR_STOP_REL_CHANGE 1
#define OR_STOP_NONE 2
#define OR_OK 0
#define OR_INVALID 1
#define OR_NOT_CONVERGED 2
#define OR_NONFINITE 3
#define OR_NOMEM 4

static double bf16_to_f64(uint16_t b) {
  uint32_t u = (uint32_t)b << 16;
  float f;
  memcpy(&f, &u, sizeof f);
  return (double)f;
}

/* IEEE 754 binary16 bit pattern to float64, from the format's definition:
 * sign, 5 exponent bits (bias 15), 10 fraction bits; exponent 0 holds the
 * subnormals fraction·2^-24, exponent 31 the infinities and NaNs.  Every
 * binary16 value is exact in float64. */
static double f16_to_f64(uint16_t h) {
  const int ex = (h >> 10) & 31, fr = h & 1023;
  double v;
  if (ex == 0) v = ldexp((double)fr, -24);
  else if (ex == 31) v = fr ? NAN : INFINITY;
  else v = ldexp((double)(fr + 1024), ex - 25);
  return (h & 0x8000) ? -v : v;
}

/* Element X(i, j) promoted to float64. */
static double x_elem(const void* X, int dt, int lay, int64_t ld, int64_t i, int64_t j) {
  int64_t idx = (lay == OR_COL) ? j * ld + i : i * ld + j;
  if (dt == OR_F32) return (double)((const float*)X)[idx];
  if (dt == OR_BF16) return bf16_to_f64(((const uint16_t*)X)[idx]);
  if (dt == OR_F16) return f16_to_f64(((const uint16_t*)X)[idx]);
  return ((const double*)X)[idx];
}

/* Column X_j promoted to float64 into col[0..m-1]. */
static void load_column(const void* X, int dt, int lay, int64_t ld, int64_t m, int64_t j,
                        double* col) {
  if (lay == OR_COL) {
    const int64_t base = j * ld;
    if (dt == OR_F32) {
      const float* p = (const float*)X + base;
      for (int64_t i = 0; i < m; ++i) col[i] = (double)p[i];
    } else if (dt == OR_BF16) {
      const uint16_t* p = (const uint16_t*)X + base;
      for (int64_t i = 0; i < m; ++i) col[i] = bf16_to_f64(p[i]);
    } else if (dt == OR_F16) {
      const uint16_t* p = (const uint16_t*)X + base;
      for (int64_t i = 0; i < m; ++i) col[i] = f16_to_f64(p[i]);
    } else {
      memcpy(col, (const double*)X + base, (size_t)m * sizeof(double));
    }
    return;
  }
  for (int64_t i = 0; i < m; ++i) col[i] = x_elem(X, dt, lay, ld, i, j);
}

static double norm2(const double* v, int64_t m) {
  double s = 0.0;
  for (int64_t i = 0; i < m; ++i) s += v[i] * v[i];
  return sqrt(s);
}

static int valid_args(const void* X, int dt, int lay, int64_t m, int64_t n, int64_t ld) {
  if (m < 0 || n < 0) return 0;
  if (dt != OR_F32 && dt != OR_BF16 && dt != OR_F64 && dt != OR_F16) return 0;
  if (lay != OR_COL && lay != OR_ROW) return 0;
  if (lay == OR_COL && ld < (m > 1 ? m : 1)) return 0;
  if (lay == OR_ROW && ld < (n > 1 ? n : 1)) return 0;
  if (!X && m > 0 && n > 0) return 0;
  return 1;
}

/*
 * e = y - X·a in float64 (the residual definition of Algorithm 1 and Sec. 3).
 * Writes e[0..m-1]; returns ||e||_2 through *enorm (may be NULL).
 */
int hpscd_oracle_residual(const void* X, int dt, int lay, int64_t m, int64_t n, int64_t ld,
                          const double* y, const double* a, double* e, double* enorm) {
  if (!valid_args(X, dt, lay, m, n, ld) || (!y && m > 0) || (!a && n > 0) || (!e && m > 0))
    return OR_INVALID;
  for (int64_t i = 0; i < m; ++i) e[i] = y[i];
  if (lay == OR_COL) {
    double* col = (double*)malloc((size_t)(m > 0 ? m : 1) * sizeof(double));
    if (!col) return OR_NOMEM;
    for (int64_t j = 0; j < n; ++j) {
      load_column(X, dt, lay, ld, m, j, col);
      for (int64_t i = 0; i < m; ++i) e[i] -= col[i] * a[j];
    }
    free(col);
  } else {
    for (int64_t i = 0; i < m; ++i) {
      double s = 0.0;
      for (int64_t j = 0; j < n; ++j) s += x_elem(X, dt, lay, ld, i, j) * a[j];
      e[i] -= s;
    }
  }
  if (enorm) *enorm = norm2(e, m);
  return OR_OK;
}

/*
 * Algorithm 1 (HPSCD), literally, in float64.
 *
 *   a <- a0 (0_n when a0 == NULL)                     initial guess
 *   e <- y - X·a                                       initial residual
 *   d_j <- <X_j, X_j>  for every j                     the denominator of the
 *                                                      column step; X is
 *                                                      constant, so it is
 *                                                      formed once
 *   for s = 1..max_sweeps:
 *     for j = 1..n (in order):
 *       da  <- <X_j, e> / d_j       (Eq. da2; skipped when d_j == 0)
 *       e   <- e - X_j·da           (Eq. ek1-ek)
 *       a_j <- a_j + da
 *     hist[s] <- ||e|| / ||y||, then the stopping test
 *
 * Row-major X is first copied to column-major float64 storage so that each
 * column is read contiguously; the arithmetic is unchanged.
 *
 * max_col_steps >= 0 stops after that many single-column steps in total
 * (k = (s-1)·n + j counts them), even mid-sweep, to expose intermediate
 * states for the invariant checks; -1 disables it.
 *
 * Outputs: a_out[n], e_out[m] (may be NULL), hist[max_sweeps+1] (may be NULL),
 * *sweeps_done (number of completed sweeps; may be NULL).
 * Returns OR_OK when the stopping rule was met (or for STOP_NONE / column-step
 * limits), OR_NOT_CONVERGED when max_sweeps ran out first, OR_NONFINITE when a
 * residual norm is not finite, OR_INVALID for bad arguments.
 */
int hpscd_oracle_solve(const void* X, int dt, int lay, int64_t m, int64_t n, int64_t ld,
                       const double* y, const double* a0, double tol, int64_t max_sweeps,
                       int stop_rule, int64_t max_col_steps, double* a_out, double* e_out,
                       double* hist, int64_t* sweeps_done) {
  if (!valid_args(X, dt, lay, m, n, ld) || (!y && m > 0) || (!a_out && n > 0) ||
      max_sweeps < 0 || (stop_rule < 0 || stop_rule > 2) || !(tol >= 0.0))
    return OR_INVALID;

  const void* Xc = X;
  int dtc = dt, layc = lay;
  int64_t ldc = ld;
  double* Xcopy = NULL;
  if (lay == OR_ROW && m > 0 && n > 0) {
    Xcopy = (double*)malloc((size_t)m * (size_t)n * sizeof(double));
    if (!Xcopy) return OR_NOMEM;
    for (int64_t i = 0; i < m; ++i)
      for (int64_t j = 0; j < n; ++j) Xcopy[j * m + i] = x_elem(X, dt, lay, ld, i, j);
    Xc = Xcopy;
    dtc = OR_F64;
    layc = OR_COL;
    ldc = m;
  }

  double* e = (double*)malloc((size_t)(m > 0 ? m : 1) * sizeof(double));
  double* col = (double*)malloc((size_t)(m > 0 ? m : 1) * sizeof(double));
  double* d = (double*)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
  if (!e || !col || !d) {
    free(e); free(col); free(d); free(Xcopy);
    return OR_NOMEM;
  }

  /* a <- a0 (or 0_n); e <- y - X·a. */
  for (int64_t j = 0; j < n; ++j) a_out[j] = a0 ? a0[j] : 0.0;
  for (int64_t i = 0; i < m; ++i) e[i] = y[i];
  for (int64_t j = 0; j < n; ++j) {
    if (a_out[j] == 0.0) continue;
    load_column(Xc, dtc, layc, ldc, m, j, col);
    for (int64_t i = 0; i < m; ++i) e[i] -= col[i] * a_out[j];
  }
  /* d_j = <X_j, X_j>. */
  for (int64_t j = 0; j < n; ++j) {
    load_column(Xc, dtc, layc, ldc, m, j, col);
    double s = 0.0;
    for (int64_t i = 0; i < m; ++i) s += col[i] * col[i];
    d[j] = s;
  }

  const double ynorm = norm2(y, m);
  const double scale = ynorm > 0.0 ? ynorm : 1.0;
  double r_prev = norm2(e, m) / scale;
  if (hist) hist[0] = r_prev;
  int status = OR_NOT_CONVERGED;
  int64_t s_done = 0;
  int64_t steps = 0;
  int stopped_mid = 0;

  if (!isfinite(r_prev)) {
    status = OR_NONFINITE;
  } else if (stop_rule == OR_STOP_REL_RES && r_prev <= tol) {
    status = OR_OK;
  } else if (stop_rule == OR_STOP_NONE && max_sweeps == 0) {
    status = OR_OK;
  } else if (max_col_steps == 0) {
    status = OR_OK;
  } else {
    for (int64_t s = 1; s <= max_sweeps; ++s) {
      for (int64_t j = 0; j < n; ++j) {
        load_column(Xc, dtc, layc, ldc, m, j, col);
        double num = 0.0;
        for (int64_t i = 0; i < m; ++i) num += col[i] * e[i];
        const double da = d[j] > 0.0 ? num / d[j] : 0.0;
        for (int64_t i = 0; i < m; ++i) e[i] -= col[i] * da;
        a_out[j] += da;
        ++steps;
        if (max_col_steps > 0 && steps >= max_col_steps) {
          stopped_mid = 1;
          break;
        }
      }
      if (stopped_mid && steps % (n > 0 ? n : 1) != 0) {
        status = OR_OK;
        break;
      }
      s_done = s;
      const double r = norm2(e, m) / scale;
      if (hist) hist[s] = r;
      if (!isfinite(r)) {
        status = OR_NONFINITE;
        break;
      }
      if (stopped_mid) {
        status = OR_OK;
        break;
      }
      if (stop_rule == OR_STOP_REL_RES && r <= tol) {
        status = OR_OK;
        break;
      }
      if (stop_rule == OR_STOP_REL_CHANGE && (r_prev == 0.0 || fabs(r_prev - r) < tol * r_prev)) {
        status = OR_OK;
        break;
      }
      if (stop_rule == OR_STOP_NONE && s == max_sweeps) {
        status = OR_OK;
        break;
      }
      r_prev = r;
    }
  }
  if (e_out)
    for (int64_t i = 0; i < m; ++i) e_out[i] = e[i];
  if (sweeps_done) *sweeps_done = s_done;
  free(e);
  free(col);
  free(d);
  free(Xcopy);
  return status;
}

/*
 * Algorithm 1 as hpscd_oracle_solve (initial guess a0 or 0_n, REL_RES /
 * REL_CHANGE / NONE once per sweep), with the two row loops of every column
 * step -- the dot <X_j, e> and the correction e <- e - X_j·da -- split over
 * `threads` threads (OpenMP; the CPU baseline).  The column order stays
 * sequential: thread t owns rows [m·t/T, m·(t+1)/T), sums its part of the dot
 * in row order, and every thread adds the T parts in thread order, so all of
 * them take the same da.  With threads = 1 this is hpscd_oracle_solve's
 * arithmetic exactly; with T > 1 only the summation order of the dots and
 * norms differs.  *threads_used receives T (1 when built without OpenMP).
 * Column-major or row-major X (row-major is copied to column-major float64
 * first, as hpscd_oracle_solve does).
 */
#ifdef _OPENMP
#include <omp.h>
#endif

static double dot_rows(const void* X, int dt, int64_t base, const double* e, int64_t i0, int64_t i1) {
  double s = 0.0;
  if (dt == OR_F32) {
    const float* p = (const float*)X + base;
    for (int64_t i = i0; i < i1; ++i) s += (double)p[i] * e[i];
  } else if (dt == OR_BF16) {
    const uint16_t* p = (const uint16_t*)X + base;
    for (int64_t i = i0; i < i1; ++i) s += bf16_to_f64(p[i]) * e[i];
  } else if (dt == OR_F16) {
    const uint16_t* p = (const uint16_t*)X + base;
    for (int64_t i = i0; i < i1; ++i) s += f16_to_f64(p[i]) * e[i];
  } else {
    const double* p = (const double*)X + base;
    for (int64_t i = i0; i < i1; ++i) s += p[i] * e[i];
  }
  return s;
}

static void axpy_rows(const void* X, int dt, int64_t base, double da, double* e, int64_t i0, int64_t i1) {
  if (dt == OR_F32) {
    const float* p = (const float*)X + base;
    for (int64_t i = i0; i < i1; ++i) e[i] -= (double)p[i] * da;
  } else if (dt == OR_BF16) {
    const uint16_t* p = (const uint16_t*)X + base;
    for (int64_t i = i0; i < i1; ++i) e[i] -= bf16_to_f64(p[i]) * da;
  } else if (dt == OR_F16) {
    const uint16_t* p = (const uint16_t*)X + base;
    for (int64_t i = i0; i < i1; ++i) e[i] -= f16_to_f64(p[i]) * da;
  } else {
    const double* p = (const double*)X + base;
    for (int64_t i = i0; i < i1; ++i) e[i] -= p[i] * da;
  }
}

int hpscd_oracle_solve_mt(const void* X, int dt, int lay, int64_t m, int64_t n, int64_t ld,
                          const double* y, const double* a0, double tol, int64_t max_sweeps,
                          int stop_rule, int threads, double* a_out, double* hist,
                          int64_t* sweeps_done, int* threads_used) {
  if (!valid_args(X, dt, lay, m, n, ld) || (!y && m > 0) || (!a_out && n > 0) ||
      max_sweeps < 0 || (stop_rule < 0 || stop_rule > 2) || !(tol >= 0.0) || threads < 1)
    return OR_INVALID;
#ifndef _OPENMP
  threads = 1;
#endif
  if (threads_used) *threads_used = threads;
  const void* Xc = X;
  int dtc = dt;
  int64_t ldc = ld;
  double* Xcopy = NULL;
  if (lay == OR_ROW && m > 0 && n > 0) {
    Xcopy = (double*)malloc((size_t)m * (size_t)n * sizeof(double));
    if (!Xcopy) return OR_NOMEM;
    for (int64_t c = 0; c < n; ++c)
      for (int64_t r = 0; r < m; ++r) Xcopy[c * m + r] = x_elem(X, dt, lay, ld, r, c);
    Xc = Xcopy;
    dtc = OR_F64;
    ldc = m;
  }
  const int T = threads;
  double* e = (double*)malloc((size_t)(m > 0 ? m : 1) * sizeof(double));
  double* d = (double*)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
  double* part = (double*)calloc((size_t)2 * T * 8, sizeof(double));  /* [2][T] at a stride of 8 */
  if (!e || !d || !part) {
    free(e); free(d); free(part); free(Xcopy);
    return OR_NOMEM;
  }
  for (int64_t j = 0; j < n; ++j) a_out[j] = a0 ? a0[j] : 0.0;
  int status = OR_NOT_CONVERGED;
  int64_t s_done = 0;
  int stop = 0;
  double ynorm = 0.0, r_prev = 0.0;

#pragma omp parallel num_threads(T)
  {
#ifdef _OPENMP
    const int t = omp_get_thread_num();
#else
    const int t = 0;
#endif
    const int64_t i0 = m * t / T, i1 = m * (t + 1) / T;
    /* e <- y - X·a, d_j <- <X_j, X_j>, ||y||: each thread its rows, then in thread order */
    for (int64_t i = i0; i < i1; ++i) e[i] = y[i];
    for (int64_t j = 0; j < n; ++j)
      if (a_out[j] != 0.0) axpy_rows(Xc, dtc, j * ldc, a_out[j], e, i0, i1);
    for (int64_t j = 0; j < n; ++j) {
      double sq = 0.0;
      if (dtc == OR_F32) {
        const float* p = (const float*)Xc + j * ldc;
        for (int64_t i = i0; i < i1; ++i) sq += (double)p[i] * (double)p[i];
      } else if (dtc == OR_BF16) {
        const uint16_t* p = (const uint16_t*)Xc + j * ldc;
        for (int64_t i = i0; i < i1; ++i) sq += bf16_to_f64(p[i]) * bf16_to_f64(p[i]);
      } else if (dtc == OR_F16) {
        const uint16_t* p = (const uint16_t*)Xc + j * ldc;
        for (int64_t i = i0; i < i1; ++i) sq += f16_to_f64(p[i]) * f16_to_f64(p[i]);
      } else {
        const double* p = (const double*)Xc + j * ldc;
        for (int64_t i = i0; i < i1; ++i) sq += p[i] * p[i];
      }
      part[((j & 1) * T + t) * 8] = sq;
#pragma omp barrier
      if (t == 0) {
        double tot = 0.0;
        for (int k = 0; k < T; ++k) tot += part[((j & 1) * T + k) * 8];
        d[j] = tot;
      }
    }
    double yy = 0.0, ee = 0.0;
    for (int64_t i = i0; i < i1; ++i) { yy += y[i] * y[i]; ee += e[i] * e[i]; }
#pragma omp barrier
    part[t * 8] = yy;
    part[(T + t) * 8] = ee;
#pragma omp barrier
    if (t == 0) {
      double ys = 0.0, es = 0.0;
      for (int k = 0; k < T; ++k) { ys += part[k * 8]; es += part[(T + k) * 8]; }
      ynorm = sqrt(ys);
      const double scale = ynorm > 0.0 ? ynorm : 1.0;
      r_prev = sqrt(es) / scale;
      if (hist) hist[0] = r_prev;
      if (!isfinite(r_prev)) { status = OR_NONFINITE; stop = 1; }
      else if (stop_rule == OR_STOP_REL_RES && r_prev <= tol) { status = OR_OK; stop = 1; }
      else if (stop_rule == OR_STOP_NONE && max_sweeps == 0) { status = OR_OK; stop = 1; }
    }
#pragma omp barrier
    for (int64_t sw = 1; sw <= max_sweeps && !stop; ++sw) {
      for (int64_t j = 0; j < n; ++j) {
        /* da <- <X_j, e> / d_j (Eq. da2); e <- e - X_j·da (Eq. ek1-ek); a_j += da */
        part[((j & 1) * T + t) * 8] = dot_rows(Xc, dtc, j * ldc, e, i0, i1);
#pragma omp barrier
        double num = 0.0;
        for (int k = 0; k < T; ++k) num += part[((j & 1) * T + k) * 8];
        const double dj = d[j], da = dj > 0.0 ? num / dj : 0.0;
        axpy_rows(Xc, dtc, j * ldc, da, e, i0, i1);
        if (t == 0) a_out[j] = a_out[j] + da;
      }
      double es = 0.0;
      for (int64_t i = i0; i < i1; ++i) es += e[i] * e[i];
#pragma omp barrier
      part[t * 8] = es;
#pragma omp barrier
      if (t == 0) {
        double tot = 0.0;
        for (int k = 0; k < T; ++k) tot += part[k * 8];
        const double r = sqrt(tot) / (ynorm > 0.0 ? ynorm : 1.0);
        s_done = sw;
        if (hist) hist[sw] = r;
        if (!isfinite(r)) { status = OR_NONFINITE; stop = 1; }
        else if (stop_rule == OR_STOP_REL_RES && r <= tol) { status = OR_OK; stop = 1; }
        else if (stop_rule == OR_STOP_REL_CHANGE && (r_prev == 0.0 || fabs(r_prev - r) < tol * r_prev)) {
          status = OR_OK; stop = 1;
        } else if (stop_rule == OR_STOP_NONE && sw == max_sweeps) { status = OR_OK; stop = 1; }
        r_prev = r;
      }
#pragma omp barrier
    }
  }
  if (sweeps_done) *sweeps_done = s_done;
  free(e);
  free(d);
  free(part);
  free(Xcopy);
  return status;
}

/*
 * Algorithm 2 (HPSCDP, Sec. 7), literally, in float64.
 *
 *   a <- a0 (or 0_n); e <- y - X·a
 *   for s = 1..max_sweeps:
 *     aprev <- a
 *     for each block jj = {k, ..., k+thr-1} of thr consecutive columns
 *         (the last block holds the n mod thr remaining columns):
 *       for every k in jj, against the SAME e:  a_k <- a_k + <X_k, e> / <X_k, X_k>
 *       e <- e - X_jj·(a_jj - aprev_jj)
 *     hist[s] <- ||e|| / ||y||, then the stopping test (as in Algorithm 1)
 * thr = 1 is Algorithm 1; thr >= n updates every column from one residual.
 * Zero columns are skipped (da = 0).  Returns like hpscd_oracle_solve.
 */
int hpscd_oracle_solve_blocks(const void* X, int dt, int lay, int64_t m, int64_t n, int64_t ld,
                              const double* y, const double* a0, int64_t thr, double tol,
                              int64_t max_sweeps, int stop_rule, double* a_out, double* e_out,
                              double* hist, int64_t* sweeps_done) {
  if (!valid_args(X, dt, lay, m, n, ld) || (!y && m > 0) || (!a_out && n > 0) ||
      max_sweeps < 0 || (stop_rule < 0 || stop_rule > 2) || !(tol >= 0.0) || thr < 1)
    return OR_INVALID;
  double* e = (double*)malloc((size_t)(m > 0 ? m : 1) * sizeof(double));
  double* col = (double*)malloc((size_t)(m > 0 ? m : 1) * sizeof(double));
  double* d = (double*)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
  double* aprev = (double*)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
  if (!e || !col || !d || !aprev) {
    free(e); free(col); free(d); free(aprev);
    return OR_NOMEM;
  }
  for (int64_t j = 0; j < n; ++j) a_out[j] = a0 ? a0[j] : 0.0;
  for (int64_t i = 0; i < m; ++i) e[i] = y[i];
  for (int64_t c = 0; c < n; ++c) {
    load_column(X, dt, lay, ld, m, c, col);
    double sq = 0.0;
    for (int64_t i = 0; i < m; ++i) {
      e[i] -= col[i] * a_out[c];
      sq += col[i] * col[i];
    }
    d[c] = sq;
  }
  const double ynorm = norm2(y, m);
  const double scale = ynorm > 0.0 ? ynorm : 1.0;
  double r_prev = norm2(e, m) / scale;
  if (hist) hist[0] = r_prev;
  int status = OR_NOT_CONVERGED;
  int64_t s_done = 0;
  if (!isfinite(r_prev)) {
    status = OR_NONFINITE;
  } else if ((stop_rule == OR_STOP_REL_RES && r_prev <= tol) ||
             (stop_rule == OR_STOP_NONE && max_sweeps == 0)) {
    status = OR_OK;
  } else {
    for (int64_t s = 1; s <= max_sweeps; ++s) {
      for (int64_t j = 0; j < n; ++j) aprev[j] = a_out[j];
      for (int64_t k0 = 0; k0 < n; k0 += thr) {
        const int64_t k1 = k0 + thr < n ? k0 + thr : n;
        /* every column of the block against the same e */
        for (int64_t k = k0; k < k1; ++k) {
          load_column(X, dt, lay, ld, m, k, col);
          double dot = 0.0;
          for (int64_t i = 0; i < m; ++i) dot += col[i] * e[i];
          a_out[k] += d[k] > 0.0 ? dot / d[k] : 0.0;
        }
        /* e <- e - X_jj (a_jj - aprev_jj) */
        for (int64_t k = k0; k < k1; ++k) {
          const double delta = a_out[k] - aprev[k];
          if (delta == 0.0) continue;
          load_column(X, dt, lay, ld, m, k, col);
          for (int64_t i = 0; i < m; ++i) e[i] -= col[i] * delta;
        }
      }
      s_done = s;
      const double r = norm2(e, m) / scale;
      if (hist) hist[s] = r;
      if (!isfinite(r)) { status = OR_NONFINITE; break; }
      if (stop_rule == OR_STOP_REL_RES && r <= tol) { status = OR_OK; break; }
      if (stop_rule == OR_STOP_REL_CHANGE && (r_prev == 0.0 || fabs(r_prev - r) < tol * r_prev)) {
        status = OR_OK;
        break;
      }
      if (stop_rule == OR_STOP_NONE && s == max_sweeps) { status = OR_OK; break; }
      r_prev = r;
    }
  }
  if (e_out)
    for (int64_t i = 0; i < m; ++i) e_out[i] = e[i];
  if (sweeps_done) *sweeps_done = s_done;
  free(e); free(col); free(d); free(aprev);
  return status;
}

/*
 * Algorithm 3 (HPSCDF, Sec. 8), literally, in float64, for F steps.
 *
 *   a <- 0_n; e <- y; J <- (); d_j <- <X_j, X_j>  (the diagonal of X^T X)
 *   for f = 1..F:
 *     da   <- (X^T e) ⊘ d                       (elementwise; 0 where d_j = 0)
 *     E_j  <- sum_i (e_i - X_ij·da_j)^2         for every j
 *     jhat <- argmin_j E_j                      (lowest j among equal values)
 *     J    <- (J, jhat)  when jhat is not in J yet
 *     a_jhat <- a_jhat + da_jhat;  e <- e - X_jhat·da_jhat
 *     hist[f] <- ||e|| / ||y||
 * Outputs: sel[f-1] = jhat of step f (F entries), a_out[n], hist[F+1] (may
 * be NULL).  Returns OR_OK or OR_INVALID / OR_NOMEM.
 */
int hpscd_oracle_select(const void* X, int dt, int lay, int64_t m, int64_t n, int64_t ld,
                        const double* y, int64_t F, int64_t* sel, double* a_out, double* hist) {
  if (!valid_args(X, dt, lay, m, n, ld) || (!y && m > 0) || (!a_out && n > 0) || F < 0 ||
      (!sel && F > 0) || n < 1)
    return OR_INVALID;
  double* e = (double*)malloc((size_t)(m > 0 ? m : 1) * sizeof(double));
  double* col = (double*)malloc((size_t)(m > 0 ? m : 1) * sizeof(double));
  double* d = (double*)malloc((size_t)n * sizeof(double));
  double* da = (double*)malloc((size_t)n * sizeof(double));
  if (!e || !col || !d || !da) {
    free(e); free(col); free(d); free(da);
    return OR_NOMEM;
  }
  for (int64_t j = 0; j < n; ++j) a_out[j] = 0.0;
  for (int64_t i = 0; i < m; ++i) e[i] = y[i];
  for (int64_t c = 0; c < n; ++c) {
    load_column(X, dt, lay, ld, m, c, col);
    double sq = 0.0;
    for (int64_t i = 0; i < m; ++i) sq += col[i] * col[i];
    d[c] = sq;
  }
  const double ynorm = norm2(y, m);
  const double scale = ynorm > 0.0 ? ynorm : 1.0;
  if (hist) hist[0] = norm2(e, m) / scale;
  for (int64_t f = 1; f <= F; ++f) {
    for (int64_t c = 0; c < n; ++c) {
      load_column(X, dt, lay, ld, m, c, col);
      double corr = 0.0;
      for (int64_t i = 0; i < m; ++i) corr += col[i] * e[i];
      da[c] = d[c] > 0.0 ? corr / d[c] : 0.0;
    }
    int64_t jhat = 0;
    double best = 0.0;
    for (int64_t j = 0; j < n; ++j) {
      load_column(X, dt, lay, ld, m, j, col);
      double E = 0.0;
      for (int64_t i = 0; i < m; ++i) {
        const double r = e[i] - col[i] * da[j];
        E += r * r;
      }
      if (j == 0 || E < best) { best = E; jhat = j; }
    }
    sel[f - 1] = jhat;
    a_out[jhat] += da[jhat];
    load_column(X, dt, lay, ld, m, jhat, col);
    for (int64_t i = 0; i < m; ++i) e[i] -= col[i] * da[jhat];
    if (hist) hist[f] = norm2(e, m) / scale;
  }
  free(e); free(col); free(d); free(da);
  return OR_OK;
}

/*
 * Algorithm 1 with a given column order per sweep (Sec. 2: instead of taking
 * j = 1..n in turn, each step may take a randomly chosen index j), literally,
 * in float64.  The random indices are an input: step k of sweep s updates
 * column order[(s-1)·n + k], k = 0..n-1; an index may repeat within a sweep
 * (drawn with replacement) and a column may be left out of a sweep.
 *
 *   a <- a0 (or 0_n); e <- y - X·a; d_j <- <X_j, X_j>
 *   for s = 1..max_sweeps:
 *     for k = 0..n-1:
 *       q     <- order[(s-1)·n + k]
 *       step  <- <X_q, e> / d_q        (Eq. da2; 0 when d_q == 0)
 *       e     <- e - X_q·step          (Eq. ek1-ek)
 *       a_q   <- a_q + step
 *     hist[s] <- ||e|| / ||y||, then the stopping test (as in Algorithm 1)
 * order holds max_sweeps·n entries, each in [0, n).  Returns like
 * hpscd_oracle_solve (OR_INVALID for an index outside [0, n)).
 */
int hpscd_oracle_solve_order(const void* X, int dt, int lay, int64_t m, int64_t n, int64_t ld,
                             const double* y, const double* a0, const int64_t* order,
                             double tol, int64_t max_sweeps, int stop_rule, double* a_out,
                             double* e_out, double* hist, int64_t* sweeps_done) {
  if (!valid_args(X, dt, lay, m, n, ld) || (!y && m > 0) || (!a_out && n > 0) ||
      max_sweeps < 0 || (stop_rule < 0 || stop_rule > 2) || !(tol >= 0.0) ||
      (!order && max_sweeps > 0 && n > 0))
    return OR_INVALID;
  for (int64_t k = 0; k < max_sweeps * n; ++k)
    if (order[k] < 0 || order[k] >= n) return OR_INVALID;
  double* e = (double*)malloc((size_t)(m > 0 ? m : 1) * sizeof(double));
  double* xq = (double*)malloc((size_t)(m > 0 ? m : 1) * sizeof(double));
  double* dq = (double*)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
  if (!e || !xq || !dq) {
    free(e); free(xq); free(dq);
    return OR_NOMEM;
  }
  for (int64_t q = 0; q < n; ++q) a_out[q] = a0 ? a0[q] : 0.0;
  for (int64_t i = 0; i < m; ++i) e[i] = y[i];
  for (int64_t q = 0; q < n; ++q) {
    load_column(X, dt, lay, ld, m, q, xq);
    double ss = 0.0;
    for (int64_t i = 0; i < m; ++i) ss += xq[i] * xq[i];
    dq[q] = ss;
    if (a_out[q] != 0.0)
      for (int64_t i = 0; i < m; ++i) e[i] = e[i] - xq[i] * a_out[q];
  }
  const double ynorm = norm2(y, m);
  const double scale = ynorm > 0.0 ? ynorm : 1.0;
  double r_prev = norm2(e, m) / scale;
  if (hist) hist[0] = r_prev;
  int status = OR_NOT_CONVERGED;
  int64_t s_done = 0;
  if (!isfinite(r_prev)) {
    status = OR_NONFINITE;
  } else if ((stop_rule == OR_STOP_REL_RES && r_prev <= tol) ||
             (stop_rule == OR_STOP_NONE && max_sweeps == 0)) {
    status = OR_OK;
  } else {
    for (int64_t s = 1; s <= max_sweeps; ++s) {
      for (int64_t k = 0; k < n; ++k) {
        const int64_t q = order[(s - 1) * n + k];
        load_column(X, dt, lay, ld, m, q, xq);
        double g = 0.0;
        for (int64_t i = 0; i < m; ++i) g += xq[i] * e[i];
        const double step = dq[q] > 0.0 ? g / dq[q] : 0.0;
        for (int64_t i = 0; i < m; ++i) e[i] = e[i] - xq[i] * step;
        a_out[q] = a_out[q] + step;
      }
      s_done = s;
      const double r = norm2(e, m) / scale;
      if (hist) hist[s] = r;
      if (!isfinite(r)) { status = OR_NONFINITE; break; }
      if ((stop_rule == OR_STOP_REL_RES && r <= tol) ||
          (stop_rule == OR_STOP_REL_CHANGE && (r_prev == 0.0 || fabs(r_prev - r) < tol * r_prev)) ||
          (stop_rule == OR_STOP_NONE && s == max_sweeps)) {
        status = OR_OK;
        break;
      }
      r_prev = r;
    }
  }
  if (e_out)
    for (int64_t i = 0; i < m; ++i) e_out[i] = e[i];
  if (sweeps_done) *sweeps_done = s_done;
  free(e); free(xq); free(dq);
  return status;
}

/*
 * Algorithm 3 followed by the feature-removal loop of Sec. 8, literally, in
 * float64.  The loop is one sentence in the paper: a feature is removed when,
 * for the updated errors, a feature not yet selected gives lower errors than an
 * existing one.  Read as an exact swap step over the selected set
 * S = {k : a_k != 0}, repeated at most R times:
 *   for every k in S and j not in S (d_j > 0):
 *     e'    <- e + X_k·a_k                          (k removed)
 *     dj    <- <X_j, e'> / <X_j, X_j>               (j refitted, Eq. da2)
 *     E_kj  <- sum_i (e'_i - X_ij·dj)^2
 *   (k*, j*) <- argmin E_kj (lowest k, then lowest j, on ties)
 *   if E_k*j* < ||e||^2:  a_k* <- 0,  a_j* <- dj*,  e <- e' - X_j*·dj*
 *   else stop.
 * Outputs: sel[F] as hpscd_oracle_select; swaps[2·R] the (k*, j*) of each swap
 * made (-1 after the last); hist[F + 1 + R] (after the F steps, the residual
 * ||e|| / ||y|| after each swap); *nswaps.  Returns OR_OK or OR_INVALID /
 * OR_NOMEM.
 */
int hpscd_oracle_select_swap(const void* X, int dt, int lay, int64_t m, int64_t n, int64_t ld,
                             const double* y, int64_t F, int64_t R, int64_t* sel,
                             int64_t* swaps, double* a_out, double* hist, int64_t* nswaps) {
  if (R < 0 || (!swaps && R > 0) || !nswaps) return OR_INVALID;
  int st = hpscd_oracle_select(X, dt, lay, m, n, ld, y, F, sel, a_out, hist);
  if (st != OR_OK) return st;
  double* e = (double*)malloc((size_t)(m > 0 ? m : 1) * sizeof(double));
  double* ep = (double*)malloc((size_t)(m > 0 ? m : 1) * sizeof(double));
  double* xk = (double*)malloc((size_t)(m > 0 ? m : 1) * sizeof(double));
  double* xj = (double*)malloc((size_t)(m > 0 ? m : 1) * sizeof(double));
  double* dd = (double*)malloc((size_t)n * sizeof(double));
  if (!e || !ep || !xk || !xj || !dd) {
    free(e); free(ep); free(xk); free(xj); free(dd);
    return OR_NOMEM;
  }
  /* the residual of the selection's coefficients, recomputed from a */
  for (int64_t i = 0; i < m; ++i) e[i] = y[i];
  for (int64_t c = 0; c < n; ++c) {
    load_column(X, dt, lay, ld, m, c, xk);
    double q = 0.0;
    for (int64_t i = 0; i < m; ++i) q += xk[i] * xk[i];
    dd[c] = q;
    if (a_out[c] != 0.0)
      for (int64_t i = 0; i < m; ++i) e[i] = e[i] - xk[i] * a_out[c];
  }
  const double ynorm = norm2(y, m);
  const double scale = ynorm > 0.0 ? ynorm : 1.0;
  int64_t done = 0;
  for (int64_t r = 0; r < R; ++r) {
    double ee = 0.0;
    for (int64_t i = 0; i < m; ++i) ee += e[i] * e[i];
    int64_t bk = -1, bj = -1;
    double bestE = 0.0, bestd = 0.0;
    for (int64_t k = 0; k < n; ++k) {
      if (a_out[k] == 0.0) continue;
      load_column(X, dt, lay, ld, m, k, xk);
      for (int64_t i = 0; i < m; ++i) ep[i] = e[i] + xk[i] * a_out[k];
      for (int64_t j = 0; j < n; ++j) {
        if (a_out[j] != 0.0 || !(dd[j] > 0.0)) continue;
        load_column(X, dt, lay, ld, m, j, xj);
        double t = 0.0;
        for (int64_t i = 0; i < m; ++i) t += xj[i] * ep[i];
        const double dj = t / dd[j];
        double E = 0.0;
        for (int64_t i = 0; i < m; ++i) {
          const double u = ep[i] - xj[i] * dj;
          E += u * u;
        }
        if (bk < 0 || E < bestE) { bestE = E; bk = k; bj = j; bestd = dj; }
      }
    }
    if (bk < 0 || !(bestE < ee)) break;
    load_column(X, dt, lay, ld, m, bk, xk);
    load_column(X, dt, lay, ld, m, bj, xj);
    for (int64_t i = 0; i < m; ++i) e[i] = (e[i] + xk[i] * a_out[bk]) - xj[i] * bestd;
    a_out[bk] = 0.0;
    a_out[bj] = bestd;
    swaps[2 * done] = bk;
    swaps[2 * done + 1] = bj;
    ++done;
    if (hist) hist[F + done] = norm2(e, m) / scale;
  }
  for (int64_t r = done; r < R; ++r) { swaps[2 * r] = -1; swaps[2 * r + 1] = -1; }
  *nswaps = done;
  free(e); free(ep); free(xk); free(xj); free(dd);
  return OR_OK;
}
