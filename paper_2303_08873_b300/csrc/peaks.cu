// Issue-rate microbenchmarks for the roofline denominators: eight independent
// dependent chains of fused multiply-adds per thread on every SM, timed with
// CUDA events.  B300 issues float64 at a small fraction of its float32 rate,
// so the float64 rate bounds the native float64 loop variants.
#include "common.cuh"

namespace ar {
namespace {

template <typename T>
__global__ void __launch_bounds__(256) fma_chains(T* out, int iters, T a, T b) {
  T acc[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) acc[c] = (T)(threadIdx.x * 1e-3 + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[c] = fma(acc[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < 8; ++c) s += acc[c];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
int rate(int iters, double* out_rate) {
  const int blocks = device_sms() * 8, threads = 256;
  T* buf = nullptr;
  if (cudaMalloc(&buf, sizeof(T) * blocks * threads) != cudaSuccess) return AR_ERR_OOM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  int rc = AR_OK;
  for (int rep = 0; rep < 4 && rc == AR_OK; ++rep) {
    cudaEventRecord(e0);
    fma_chains<T><<<blocks, threads>>>(buf, iters, (T)0.999, (T)1e-7);
    cudaEventRecord(e1);
    if (cudaEventSynchronize(e1) != cudaSuccess) rc = AR_ERR_CUDA;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best) best = ms;  // first run is a warm-up
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(buf);
  if (rc == AR_OK) *out_rate = (double)blocks * threads * iters * 8 / (best * 1e-3);
  return rc;
}

}  // namespace
}  // namespace ar

extern "C" int ar_measure_fma_rates(double* fp64_fma_per_s, double* fp32_fma_per_s) {
  double r64 = 0, r32 = 0;
  int rc = ar::rate<double>(2048, &r64);
  if (rc == AR_OK) rc = ar::rate<float>(16384, &r32);
  if (rc != AR_OK) return rc;
  if (fp64_fma_per_s) *fp64_fma_per_s = r64;
  if (fp32_fma_per_s) *fp32_fma_per_s = r32;
  return AR_OK;
}
