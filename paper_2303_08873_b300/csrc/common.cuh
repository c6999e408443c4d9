// Shared helpers of the CUDA sources (internal; not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ar.h"
#include "ar_loops.h"

namespace ar {

constexpr int kNumSMs = 148;  // B300: 2 dies x 74 SMs

inline int launch_status() {
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? AR_OK : AR_ERR_CUDA;
}

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// Programmatic dependent launch, for chains of kernels on one stream (the
// sweeps of a stencil call): the kernel is launched as soon as every block of
// the kernel before it has started (each calls pdl_begin first), its blocks
// take the SM slots that the previous grid's last blocks free, and they wait
// in pdl_begin until that grid has completed and its writes are visible.  A
// kernel launched this way must call pdl_begin before touching global memory.
#ifdef __CUDACC__
__device__ __forceinline__ void pdl_begin() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

template <typename... P, typename... A>
int launch_pdl(void (*kernel)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, A&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at;
  at.id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at.val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = &at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<A&&>(args)...) == cudaSuccess ? AR_OK : AR_ERR_CUDA;
}
#endif

inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Bounds-check build.  Compiled with -DAR_CHECKED (build.py --checked), every
// AR_CHK(cond) evaluates cond; a false cond records the translation unit and
// source line of the first failing check and counts the failures in a device
// word of that translation unit, and the guarded access is skipped (a load
// yields 0, a store or copy does not happen; a skipped tensor copy leaves its
// bounded mbarrier wait to time out), so the kernels observe and never fault
// on a bad index.  In the normal build AR_CHK(cond) is the constant true and
// cond is not evaluated.  Each source file that uses it defines AR_TU (a
// small id) before including this header and instantiates AR_CHECK_READER
// once; ar_check_status (checked.cpp) reads and clears all of them.
#if defined(AR_CHECKED) && defined(__CUDACC__)
#ifndef AR_TU
#error "define AR_TU before including common.cuh"
#endif
static __device__ unsigned int g_ar_chk[2];  // first failure (AR_TU << 16 | line), failure count
__device__ __forceinline__ bool ar_chk(bool ok, unsigned line) {
  if (!ok) {
    atomicCAS(&g_ar_chk[0], 0u, ((unsigned)AR_TU << 16) | (line & 0xffffu));
    atomicAdd(&g_ar_chk[1], 1u);
  }
  return ok;
}
#define AR_CHK(c) ::ar::ar_chk(static_cast<bool>(c), __LINE__)
// reads (and with clear != 0 zeroes) this translation unit's word
#define AR_CHECK_READER(name)                                                             \
  int name(unsigned int* out2, int clear) {                                               \
    if (cudaMemcpyFromSymbol(out2, g_ar_chk, sizeof(g_ar_chk)) != cudaSuccess) return -1; \
    if (clear) {                                                                          \
      const unsigned int z[2] = {0u, 0u};                                                 \
      if (cudaMemcpyToSymbol(g_ar_chk, z, sizeof(z)) != cudaSuccess) return -1;           \
    }                                                                                     \
    return 0;                                                                             \
  }
#else
#define AR_CHK(c) true
#define AR_CHECK_READER(name) \
  int name(unsigned int* out2, int) {   \
    out2[0] = out2[1] = 0u;              \
    return 0;                            \
  }
#endif

#ifdef __CUDACC__
// AR_CHK helper: [p, p + bytes) lies inside the dynamic shared array that
// starts at `base` (the kernel's extern __shared__ array).
__device__ __forceinline__ bool in_dyn_smem(const void* base, const void* p, unsigned bytes) {
  unsigned dyn;
  asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
  const unsigned b = (unsigned)__cvta_generic_to_shared(base), q = (unsigned)__cvta_generic_to_shared(p);
  return q >= b && q - b + bytes <= dyn;
}
// AR_CHK helper: [p, p + bytes) lies inside the shared array [base, base + size).
__device__ __forceinline__ bool in_smem(const void* base, unsigned size, const void* p, unsigned bytes) {
  const unsigned b = (unsigned)__cvta_generic_to_shared(base), q = (unsigned)__cvta_generic_to_shared(p);
  return q >= b && q - b + bytes <= size;
}
#endif

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Number of SMs of the current device (cached per process; one GPU).
int device_sms();

// Variants per loop (the executor's device tables are sized by these).
constexpr int kDaxpyVariants = 15, kJacobiVariants = 16, kSpmvVariants = 9, kNbodyVariants = 9;
// The mixed-stream executor runs the first 8 SpMV variants (not the binned one).
constexpr int kExecSpmvVariants = 8;

// Per-loop launch hooks used by the builtin launcher table.
int daxpy_launch(void* args, int variant, double value, void* stream, void* user);
int jacobi7_launch(void* args, int variant, double value, void* stream, void* user);

int daxpy_num_variants();
int daxpy_variant_name(int v, char* buf, int len);
int jacobi7_num_variants();
int jacobi7_variant_name(int v, char* buf, int len);
int heat7_launch(void* args, int variant, double value, void* stream, void* user);
int heat7_num_variants();
int heat7_variant_name(int v, char* buf, int len);
int spmv_launch(void* args, int variant, double value, void* stream, void* user);
int spmv_num_variants();
int spmv_variant_name(int v, char* buf, int len);
int nbody_launch(void* args, int variant, double value, void* stream, void* user);
int nbody_num_variants();
int nbody_variant_name(int v, char* buf, int len);

}  // namespace ar
