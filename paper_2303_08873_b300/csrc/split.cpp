// Loops over HOST-resident data split between the GPU and the host cores.
//
// The paper's co-scheduling use case (Section 3.2, "Co-Scheduling GPU and CPU
// execution", Listing 5): the region's variants are numeric, [0.0:1.0:0.1],
// each the fraction of the iteration space given to the GPU; the GPU part's
// inputs are mapped to the device, its loop runs asynchronously (nowait),
// the host cores run the remaining iterations as a parallel loop, and the
// region waits for both before the GPU part's results are mapped back.  With
// the fractions 0 and 1 only it is the device-selection use case (Section
// 3.2, "Selection of optimal execution device", Listing 3: variants cpu and
// gpu).  Sections 5.2 and 5.4 evaluate both.
//
// Here the GPU part is one of the loop's CUDA variants on caller-owned device
// buffers, with one cudaMemcpyAsync per input slice in and one for the result
// slice out on the caller's stream; the host part is an OpenMP loop in this
// file (the library's own host code), started after the GPU work is enqueued
// so the two overlap.  Each call blocks until both parts are done.
#include <cuda_runtime.h>
#include <omp.h>

#include <cmath>
#include <cstdint>

#include "ar.h"
#include "ar_loops.h"

namespace {

// First index of the host part: round(f * n), the fraction's share of the
// iteration space rounded to the nearest iteration.
int64_t split_point(double f, int64_t n) {
  const double m = std::floor(f * (double)n + 0.5);
  return m <= 0.0 ? 0 : (m >= (double)n ? n : (int64_t)m);
}

bool bad_fraction(double f) { return !(f >= 0.0 && f <= 1.0); }

int status_of(cudaError_t e) { return e == cudaSuccess ? AR_OK : AR_ERR_CUDA; }

}  // namespace

extern "C" int ar_daxpy_split(double gpu_fraction, const ar_daxpy_split_args* a, void* stream) {
  if (!a || bad_fraction(gpu_fraction) || a->n < 0) return AR_ERR_ARG;
  if (a->n == 0) return AR_OK;
  const int64_t n = a->n, m = split_point(gpu_fraction, n);
  if (!a->x || !a->y || (m > 0 && (!a->x_dev || !a->y_dev))) return AR_ERR_ARG;
  if (a->gpu_variant < 0 || a->gpu_variant >= ar_loop_num_variants(AR_LOOP_DAXPY)) return AR_ERR_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int rc = AR_OK;
  if (m > 0) {
    const size_t b = sizeof(double) * (size_t)m;
    rc = status_of(cudaMemcpyAsync(a->x_dev, a->x, b, cudaMemcpyHostToDevice, s));
    if (rc == AR_OK) rc = status_of(cudaMemcpyAsync(a->y_dev, a->y, b, cudaMemcpyHostToDevice, s));
    if (rc == AR_OK) rc = ar_daxpy(a->gpu_variant, m, a->a, a->x_dev, a->y_dev, stream);
    if (rc == AR_OK) rc = status_of(cudaMemcpyAsync(a->y, a->y_dev, b, cudaMemcpyDeviceToHost, s));
    if (rc != AR_OK) {
      cudaStreamSynchronize(s);  // nothing of this call stays in flight
      return rc;
    }
  }
  // host part: the same fused multiply-add per element as the device
  const double alpha = a->a;
  const double* x = a->x;
  double* y = a->y;
#pragma omp parallel for schedule(static)
  for (int64_t i = m; i < n; ++i) y[i] = std::fma(alpha, x[i], y[i]);
  return m > 0 ? status_of(cudaStreamSynchronize(s)) : AR_OK;
}

extern "C" int ar_spmv_split(double gpu_fraction, const ar_spmv_split_args* a, void* stream) {
  if (!a || bad_fraction(gpu_fraction) || a->rows < 0 || a->nnz < 0 || a->nnz > 0x7fffffffLL || a->cols < 0)
    return AR_ERR_ARG;
  if (a->rows == 0) return AR_OK;
  if (!a->rowptr || !a->y || (a->nnz > 0 && (!a->col || !a->val || !a->x))) return AR_ERR_ARG;
  if (a->rowptr[0] != 0 || a->rowptr[a->rows] != a->nnz) return AR_ERR_ARG;
  const int64_t rows = a->rows, m = split_point(gpu_fraction, rows);
  if (m > 0 && (!a->rowptr_dev || !a->y_dev || (a->nnz > 0 && (!a->col_dev || !a->val_dev || !a->x_dev))))
    return AR_ERR_ARG;
  if (a->gpu_variant < 0 || a->gpu_variant >= ar_loop_num_variants(AR_LOOP_SPMV)) return AR_ERR_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int rc = AR_OK;
  if (m > 0) {
    const int64_t nz = a->rowptr[m];  // nonzeros of the GPU's rows
    rc = status_of(cudaMemcpyAsync(a->rowptr_dev, a->rowptr, sizeof(int32_t) * (size_t)(m + 1),
                                   cudaMemcpyHostToDevice, s));
    if (rc == AR_OK && nz > 0)
      rc = status_of(cudaMemcpyAsync(a->col_dev, a->col, sizeof(int32_t) * (size_t)nz, cudaMemcpyHostToDevice, s));
    if (rc == AR_OK && nz > 0)
      rc = status_of(cudaMemcpyAsync(a->val_dev, a->val, sizeof(double) * (size_t)nz, cudaMemcpyHostToDevice, s));
    if (rc == AR_OK && nz > 0 && a->cols > 0)
      rc = status_of(cudaMemcpyAsync(a->x_dev, a->x, sizeof(double) * (size_t)a->cols, cudaMemcpyHostToDevice, s));
    if (rc == AR_OK)
      rc = ar_spmv(a->gpu_variant, m, nz, a->rowptr_dev, a->col_dev, a->val_dev, a->x_dev, a->y_dev, a->workspace,
                   a->workspace_bytes, stream);
    if (rc == AR_OK)
      rc = status_of(cudaMemcpyAsync(a->y, a->y_dev, sizeof(double) * (size_t)m, cudaMemcpyDeviceToHost, s));
    if (rc != AR_OK) {
      cudaStreamSynchronize(s);
      return rc;
    }
  }
  // host part: one row per iteration, products summed by fused multiply-add
  // in nonzero order (the thread-per-row order of the device variants)
  const int32_t* rp = a->rowptr;
  const int32_t* col = a->col;
  const double* val = a->val;
  const double* x = a->x;
  double* y = a->y;
#pragma omp parallel for schedule(dynamic, 1024)
  for (int64_t r = m; r < rows; ++r) {
    double acc = 0.0;
    for (int32_t k = rp[r]; k < rp[r + 1]; ++k) acc = std::fma(val[k], x[col[k]], acc);
    y[r] = acc;
  }
  return m > 0 ? status_of(cudaStreamSynchronize(s)) : AR_OK;
}

namespace ar {

// Region launchers: the variant's numeric value is the GPU fraction.
int daxpy_split_launch(void* args, int, double value, void* stream, void*) {
  return ar_daxpy_split(value, static_cast<const ar_daxpy_split_args*>(args), stream);
}
int spmv_split_launch(void* args, int, double value, void* stream, void*) {
  return ar_spmv_split(value, static_cast<const ar_spmv_split_args*>(args), stream);
}

}  // namespace ar

extern "C" int ar_region_add_split(ar_region* r, int loop, double begin, double end, double step, int* out_count) {
  if (!r || begin < 0.0 || end > 1.0) return AR_ERR_ARG;
  if (loop == AR_LOOP_DAXPY) return ar_variant_register_range(r, begin, end, step, ar::daxpy_split_launch, nullptr, out_count);
  if (loop == AR_LOOP_SPMV) return ar_variant_register_range(r, begin, end, step, ar::spmv_split_launch, nullptr, out_count);
  return AR_ERR_ARG;
}

extern "C" int ar_split_threads(void) { return omp_get_max_threads(); }
