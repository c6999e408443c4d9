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

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Number of SMs of the current device (cached per process; one GPU).
int device_sms();

// Variants per loop (the executor's device tables are sized by these).
constexpr int kDaxpyVariants = 15, kJacobiVariants = 16, kSpmvVariants = 8, kNbodyVariants = 9;

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
