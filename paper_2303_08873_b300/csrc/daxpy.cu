// daxpy variants: y <- a*x + y in float64 (the paper's vector-update region,
// Listings 1-5, adapted over threads per block as in Listing 4).
//
// Memory-bound: 24 bytes moved and one DFMA per element.  Variants differ in
// threads per block {64..1024} and elements per thread {1, 2, 4}; EPT >= 2
// moves 128-bit double2 words.  Each block covers BS*EPT consecutive
// elements with the EPT accesses of a thread spaced BS words apart, so every
// warp access is fully coalesced; all loads of a thread are issued before
// its first FMA to keep several 16-byte requests in flight.
#define AR_TU 1
#include <cstdio>

#include "common.cuh"

namespace ar {
namespace {

constexpr int kBlock[5] = {64, 128, 256, 512, 1024};
constexpr int kEpt[3] = {1, 2, 4};

__device__ __forceinline__ double2 ld_stream(const double2* p) {
  double2 v;
  asm volatile("ld.global.nc.L1::no_allocate.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "l"(p));
  return v;
}

template <int BS, int EPT>
__global__ void __launch_bounds__(BS) daxpy_kernel(int64_t n, double a, const double* __restrict__ x,
                                                   double* __restrict__ y) {
  if constexpr (EPT == 1) {
    const int64_t i = (int64_t)blockIdx.x * BS + threadIdx.x;
    if (i < n) y[i] = fma(a, __ldg(x + i), y[i]);
  } else {
    constexpr int W = EPT / 2;  // double2 words per thread
    const int64_t n2 = n >> 1;
    const double2* x2 = reinterpret_cast<const double2*>(x);
    double2* y2 = reinterpret_cast<double2*>(y);
    const int64_t base = (int64_t)blockIdx.x * (BS * W) + threadIdx.x;
    double2 xv[W], yv[W];
#pragma unroll
    for (int w = 0; w < W; ++w) {
      const int64_t i = base + (int64_t)w * BS;
      if (i < n2) {
        xv[w] = ld_stream(x2 + i);
        yv[w] = y2[i];
      }
    }
#pragma unroll
    for (int w = 0; w < W; ++w) {
      const int64_t i = base + (int64_t)w * BS;
      if (i < n2) {
        yv[w].x = fma(a, xv[w].x, yv[w].x);
        yv[w].y = fma(a, xv[w].y, yv[w].y);
        y2[i] = yv[w];
      }
    }
    // odd length: the last element is not part of any double2 word
    if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) y[n - 1] = fma(a, x[n - 1], y[n - 1]);
  }
}

template <int BS, int EPT>
int launch(int64_t n, double a, const double* x, double* y, cudaStream_t s) {
  const int64_t words = (EPT == 1) ? n : (n >> 1);
  const int64_t per_block = (EPT == 1) ? BS : (int64_t)BS * (EPT / 2);
  int64_t grid = ceil_div(words, per_block);
  if (grid == 0) grid = 1;  // n == 1 with EPT >= 2: only the odd tail
  if (grid > 0x7fffffffLL) return AR_ERR_ARG;
  daxpy_kernel<BS, EPT><<<(unsigned)grid, BS, 0, s>>>(n, a, x, y);
  return launch_status();
}

template <int BI>
int dispatch_ept(int e, int64_t n, double a, const double* x, double* y, cudaStream_t s) {
  switch (e) {
    case 0: return launch<kBlock[BI], 1>(n, a, x, y, s);
    case 1: return launch<kBlock[BI], 2>(n, a, x, y, s);
    default: return launch<kBlock[BI], 4>(n, a, x, y, s);
  }
}

}  // namespace

int daxpy_num_variants() { return kDaxpyVariants; }

int daxpy_variant_name(int v, char* buf, int len) {
  if (v < 0 || v >= kDaxpyVariants || !buf || len <= 0) return AR_ERR_ARG;
  snprintf(buf, (size_t)len, "daxpy_b%d_e%d", kBlock[v / 3], kEpt[v % 3]);
  return AR_OK;
}

int daxpy_launch(void* args, int variant, double, void* stream, void*) {
  const ar_daxpy_args* a = static_cast<const ar_daxpy_args*>(args);
  if (!a) return AR_ERR_ARG;
  return ar_daxpy(variant, a->n, a->a, a->x, a->y, stream);
}

}  // namespace ar

extern "C" int ar_daxpy(int variant, int64_t n, double a, const double* x, double* y, void* stream) {
  using namespace ar;
  if (variant < 0 || variant >= kDaxpyVariants || n < 0) return AR_ERR_ARG;
  if (n == 0) return AR_OK;
  if (!x || !y) return AR_ERR_ARG;
  const int bi = variant / 3, e = variant % 3;
  if (e > 0 && !(aligned16(x) && aligned16(y))) return AR_ERR_ARG;
  cudaStream_t s = as_stream(stream);
  switch (bi) {
    case 0: return dispatch_ept<0>(e, n, a, x, y, s);
    case 1: return dispatch_ept<1>(e, n, a, x, y, s);
    case 2: return dispatch_ept<2>(e, n, a, x, y, s);
    case 3: return dispatch_ept<3>(e, n, a, x, y, s);
    default: return dispatch_ept<4>(e, n, a, x, y, s);
  }
}

namespace ar {
AR_CHECK_READER(chk_read_daxpy)
}  // namespace ar
