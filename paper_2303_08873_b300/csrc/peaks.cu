// Issue-rate microbenchmarks for the roofline denominators: eight independent
// dependent chains of fused multiply-adds per thread on every SM, timed with
// CUDA events.  B300 issues float64 at a small fraction of its float32 rate,
// so the float64 rate bounds the native float64 loop variants.  The packed
// float32 form (FFMA2, two lanes' FMAs per instruction) is measured apart:
// on B300 it reaches about 91 % of the scalar float32 lane rate.
#define AR_TU 7
#include <type_traits>

#include "common.cuh"

namespace ar {
namespace {

__device__ __forceinline__ double chain_fma(double x, double a, double b) { return fma(x, a, b); }
__device__ __forceinline__ float chain_fma(float x, float a, float b) { return fmaf(x, a, b); }
__device__ __forceinline__ float2 chain_fma(float2 x, float2 a, float2 b) { return __ffma2_rn(x, a, b); }
template <typename T>
__device__ __forceinline__ T chain_init(double v) { return (T)v; }
template <>
__device__ __forceinline__ float2 chain_init<float2>(double v) { return make_float2((float)v, (float)(v + 0.5)); }
__device__ __forceinline__ double chain_add(double x, double y) { return x + y; }
__device__ __forceinline__ float chain_add(float x, float y) { return x + y; }
__device__ __forceinline__ float2 chain_add(float2 x, float2 y) { return make_float2(x.x + y.x, x.y + y.y); }

// T = float2 issues packed FFMA2 instructions (two float32 lanes' FMAs each).
template <typename T>
__global__ void __launch_bounds__(256) fma_chains(T* out, int iters, T a, T b) {
  T acc[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) acc[c] = chain_init<T>(threadIdx.x * 1e-3 + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[c] = chain_fma(acc[c], a, b);
  }
  T s = chain_init<T>(0.0);
#pragma unroll
  for (int c = 0; c < 8; ++c) s = chain_add(s, acc[c]);
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
T chain_const(double v) { return (T)v; }
template <>
float2 chain_const<float2>(double v) { return make_float2((float)v, (float)v); }

// Fused multiply-adds per second (float32 lanes for T = float2: two per
// instruction).
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
    fma_chains<T><<<blocks, threads>>>(buf, iters, chain_const<T>(0.999), chain_const<T>(1e-7));
    cudaEventRecord(e1);
    if (cudaEventSynchronize(e1) != cudaSuccess) rc = AR_ERR_CUDA;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best) best = ms;  // first run is a warm-up
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(buf);
  const double lanes = std::is_same<T, float2>::value ? 2.0 : 1.0;
  if (rc == AR_OK) *out_rate = (double)blocks * threads * iters * 8 * lanes / (best * 1e-3);
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

extern "C" int ar_measure_fp32x2_rate(double* fp32_lane_fma_per_s) {
  if (!fp32_lane_fma_per_s) return AR_ERR_ARG;
  return ar::rate<float2>(8192, fp32_lane_fma_per_s);
}

namespace ar {
AR_CHECK_READER(chk_read_peaks)
}  // namespace ar
