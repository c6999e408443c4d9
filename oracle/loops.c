/*
 * CPU oracle for the four region bodies -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, obviously correct scalar loops in float64.  Only the tests,
 * the smoke check and the bench's CPU-baseline leg may load this library; the
 * product path never does.  Nothing here is shared with the CUDA sources.
 *
 * The paper's running example is a vector update (Listings 1-5, Section 2 and
 * Section 3.2); its evaluation adapts HPC loops (Table 3: Heat, a finite
 * difference stencil; AMGMk relax, a CSR sweep).  The four bodies below are
 * the synthetic stand-ins named for the adaptive region's variants:
 *   daxpy   y <- a*x + y
 *   jacobi7 u' = (sum of the 6 face neighbours) / 6 on N^3 unknowns, zero
 *           Dirichlet ghosts outside the cube
 *   heat7   u' = u + alpha (sum of the 6 face neighbours - 6 u): one explicit
 *           (forward Euler) step of the heat equation on the same grid, the
 *           finite-difference scheme of Table 3's Heat, alpha = kappa dt / h^2
 *   spmv    y = A x for CSR A, each row summed in column-list order
 *   nbody   a_i = sum_j m_j (r_j - r_i) / (|r_j - r_i|^2 + eps^2)^(3/2)
 * The outer loops carry an OpenMP "parallel for" so the timed CPU baseline
 * can use the host's cores; it changes no arithmetic or summation order.
 *
 * Compiled with -O2 -ffp-contract=off so that a*x+y is a rounded product
 * followed by a rounded sum, as written.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void or_set_threads(int t) {
#ifdef _OPENMP
  if (t > 0) omp_set_num_threads(t);
#else
  (void)t;
#endif
}

/* ---------------------------------------------------------------- daxpy */
/* y[i] <- a*x[i] + y[i], product then sum, each rounded (no contraction). */
void or_daxpy(int64_t n, double a, const double *x, double *y) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) y[i] = a * x[i] + y[i];
}

/* Same update with one fused multiply-add per element (a second legal
 * rounding of the same definition). */
void or_daxpy_fma(int64_t n, double a, const double *x, double *y) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) y[i] = fma(a, x[i], y[i]);
}

/* ---------------------------------------------------------------- Jacobi */
/* Value of unknown (i, j, k) or 0 outside [0, N)^3 (Dirichlet ghost). */
static double at(const double *u, int64_t N, int64_t i, int64_t j, int64_t k) {
  if (i < 0 || j < 0 || k < 0 || i >= N || j >= N || k >= N) return 0.0;
  return u[(k * N + j) * N + i];
}

/* One sweep: out = (W + E + S + N + D + U) / 6, summed in that order. */
void or_jacobi7_sweep(int64_t N, const double *in, double *out) {
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < N; ++k)
    for (int64_t j = 0; j < N; ++j)
      for (int64_t i = 0; i < N; ++i) {
        double s = at(in, N, i - 1, j, k);
        s = s + at(in, N, i + 1, j, k);
        s = s + at(in, N, i, j - 1, k);
        s = s + at(in, N, i, j + 1, k);
        s = s + at(in, N, i, j, k - 1);
        s = s + at(in, N, i, j, k + 1);
        out[(k * N + j) * N + i] = s / 6.0;
      }
}

/* `sweeps` sweeps starting from u0; the result is written to `out`.
 * `work` must hold N^3 doubles.  u0 is not modified. */
void or_jacobi7(int64_t N, int sweeps, const double *u0, double *out, double *work) {
  const int64_t n3 = N * N * N;
  if (sweeps <= 0) {
    memcpy(out, u0, (size_t)n3 * sizeof(double));
    return;
  }
  /* ping-pong so that the last sweep lands in `out` */
  const double *src = u0;
  for (int s = 0; s < sweeps; ++s) {
    double *dst = ((sweeps - 1 - s) % 2 == 0) ? out : work;
    or_jacobi7_sweep(N, src, dst);
    src = dst;
  }
}

/* ---------------------------------------------------------------- Heat */
/* One explicit step: out = u + alpha * (s - 6 u), s = W + E + S + N + D + U
 * summed in that order, each operation rounded as written. */
void or_heat7_step(int64_t N, double alpha, const double *in, double *out) {
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < N; ++k)
    for (int64_t j = 0; j < N; ++j)
      for (int64_t i = 0; i < N; ++i) {
        double s = at(in, N, i - 1, j, k);
        s = s + at(in, N, i + 1, j, k);
        s = s + at(in, N, i, j - 1, k);
        s = s + at(in, N, i, j + 1, k);
        s = s + at(in, N, i, j, k - 1);
        s = s + at(in, N, i, j, k + 1);
        const double u = in[(k * N + j) * N + i];
        out[(k * N + j) * N + i] = u + alpha * (s - 6.0 * u);
      }
}

/* `steps` steps starting from u0, result in `out`; `work` holds N^3
 * doubles; u0 is not modified. */
void or_heat7(int64_t N, int steps, double alpha, const double *u0, double *out, double *work) {
  const int64_t n3 = N * N * N;
  if (steps <= 0) {
    memcpy(out, u0, (size_t)n3 * sizeof(double));
    return;
  }
  const double *src = u0;
  for (int s = 0; s < steps; ++s) {
    double *dst = ((steps - 1 - s) % 2 == 0) ? out : work;
    or_heat7_step(N, alpha, src, dst);
    src = dst;
  }
}

/* ---------------------------------------------------------------- SpMV */
/* y[r] = sum over k in [rowptr[r], rowptr[r+1]) of val[k] * x[col[k]],
 * accumulated left to right; an empty row gives 0. */
void or_spmv(int64_t rows, const int32_t *rowptr, const int32_t *col, const double *val,
             const double *x, double *y) {
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t r = 0; r < rows; ++r) {
    double s = 0.0;
    for (int64_t k = rowptr[r]; k < rowptr[r + 1]; ++k) s = s + val[k] * x[col[k]];
    y[r] = s;
  }
}

/* Same sums for a list of rows only (sampled checks at full size); also
 * returns sum_k |val_k * x_col_k| per row, the scale of the row's rounding. */
void or_spmv_rows(int64_t count, const int64_t *which, const int32_t *rowptr, const int32_t *col,
                  const double *val, const double *x, double *y, double *absum) {
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t t = 0; t < count; ++t) {
    int64_t r = which[t];
    double s = 0.0, a = 0.0;
    for (int64_t k = rowptr[r]; k < rowptr[r + 1]; ++k) {
      double p = val[k] * x[col[k]];
      s = s + p;
      a = a + fabs(p);
    }
    y[t] = s;
    absum[t] = a;
  }
}

/* Row-length statistics used as selector features: rows, nnz, mean, variance
 * (population) and maximum of nnz per row, in float64 from exact integers. */
void or_csr_row_stats(int64_t rows, const int32_t *rowptr, double *out5) {
  int64_t nnz = (int64_t)rowptr[rows] - rowptr[0];
  double mean = rows > 0 ? (double)nnz / (double)rows : 0.0;
  double ss = 0.0;
  int64_t mx = 0;
  for (int64_t r = 0; r < rows; ++r) {
    int64_t len = (int64_t)rowptr[r + 1] - rowptr[r];
    double d = (double)len - mean;
    ss += d * d;
    if (len > mx) mx = len;
  }
  out5[0] = (double)rows;
  out5[1] = (double)nnz;
  out5[2] = mean;
  out5[3] = rows > 0 ? ss / (double)rows : 0.0;
  out5[4] = (double)mx;
}

/* ---------------------------------------------------------------- n-body */
/* Acceleration of body i: sum over all j (j = i contributes exactly 0) of
 * m_j d / (|d|^2 + eps^2)^(3/2), d = r_j - r_i, G = 1.  Inputs are float32
 * (x, y, z, m) records promoted to float64; the sum runs j = 0 .. N-1. */
static void accel_one(int64_t N, const float *p4, int64_t i, double eps2, double *a3) {
  double xi = p4[4 * i], yi = p4[4 * i + 1], zi = p4[4 * i + 2];
  double ax = 0.0, ay = 0.0, az = 0.0;
  for (int64_t j = 0; j < N; ++j) {
    double dx = (double)p4[4 * j] - xi;
    double dy = (double)p4[4 * j + 1] - yi;
    double dz = (double)p4[4 * j + 2] - zi;
    double r2 = dx * dx + dy * dy + dz * dz + eps2;
    double inv = 1.0 / (r2 * sqrt(r2));
    double s = (double)p4[4 * j + 3] * inv;
    ax += s * dx;
    ay += s * dy;
    az += s * dz;
  }
  a3[0] = ax;
  a3[1] = ay;
  a3[2] = az;
}

void or_nbody(int64_t N, const float *p4, double eps, double *acc3) {
  const double eps2 = eps * eps;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t i = 0; i < N; ++i) accel_one(N, p4, i, eps2, acc3 + 3 * i);
}

/* Accelerations of a list of bodies only (sampled checks at full size). */
void or_nbody_rows(int64_t N, const float *p4, double eps, int64_t count, const int64_t *which,
                   double *acc3) {
  const double eps2 = eps * eps;
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t t = 0; t < count; ++t) accel_one(N, p4, which[t], eps2, acc3 + 3 * t);
}

/* Batched form: `count` independent systems, system b holding bodies
 * [offs[b], offs[b+1]) of the concatenated array; bodies interact only
 * within their own system. */
void or_nbody_batched(int64_t count, const int32_t *offs, const float *p4, double eps,
                      double *acc3) {
  for (int64_t b = 0; b < count; ++b) {
    int64_t o = offs[b], n = (int64_t)offs[b + 1] - offs[b];
    or_nbody(n, p4 + 4 * o, eps, acc3 + 3 * o);
  }
}
