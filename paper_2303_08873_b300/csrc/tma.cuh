// Inline-PTX wrappers for mbarriers and TMA tile loads (sm_90+ / sm_103a),
// and host creation of tiled tensor maps through the driver entry point.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace ar {

// Bounded spin on an mbarrier phase: each try_wait may suspend the thread
// for a hardware-defined interval; after kSpinLimit tries the wait gives up
// and returns false so the caller can flag AR_ERR_TIMEOUT and leave.
constexpr uint32_t kSpinLimit = 1u << 22;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0;
}

__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, uint32_t limit = kSpinLimit) {
  for (uint32_t it = 0; it < limit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// Order this thread's earlier generic-proxy shared-memory accesses before
// later async-proxy (TMA) accesses of the same memory.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// 3D tiled TMA load of one box at element coordinates (x, y, z) into shared
// memory, completing `bytes` on the mbarrier.  x must be a multiple of
// 16 bytes / element size; out-of-range elements are filled with zeros.
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y, int z,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}

// 2D tiled TMA load of one box at element coordinates (x, y); the same rules
// as tma_load_3d.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// Asynchronous 16-byte global -> shared copy (cp.async, L1 bypassed, so data
// written earlier in the same launch by other SMs is seen): src_bytes (0, 8
// or 16) are read, the rest of the 16 bytes is zero-filled.  Both addresses
// 16-byte aligned.
__device__ __forceinline__ void cp_async16(void* dst, const void* src, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int G>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(G) : "memory");
}

__device__ __forceinline__ void mbar_inval(uint32_t bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
}

// Order this thread's earlier generic-proxy global accesses (stores of a
// previous sweep, the acquire of a dependency counter) with later
// async-proxy (TMA) accesses of global memory.
__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}

// Device-side edits of a tensor map in global memory (64-byte aligned):
// tensormap.replace writes one field in the driver's encoding.  The writer
// then releases the map to the tensor-map proxy; a reader acquires it
// before its first tensor copy through it.
__device__ __forceinline__ void tmap_set_address(void* map, const void* addr) {
  asm volatile("tensormap.replace.tile.global_address.global.b1024.b64 [%0], %1;" ::"l"(map), "l"(addr)
               : "memory");
}
template <int ORD>
__device__ __forceinline__ void tmap_set_dim(void* map, int v) {
  asm volatile("tensormap.replace.tile.global_dim.global.b1024.b32 [%0], %1, %2;" ::"l"(map), "n"(ORD), "r"(v)
               : "memory");
}
template <int ORD>  // the byte stride of dimension ORD + 1
__device__ __forceinline__ void tmap_set_stride(void* map, unsigned long long bytes) {
  asm volatile("tensormap.replace.tile.global_stride.global.b1024.b64 [%0], %1, %2;" ::"l"(map), "n"(ORD),
               "l"(bytes)
               : "memory");
}
__device__ __forceinline__ void tmap_release() {
  asm volatile("fence.proxy.tensormap::generic.release.gpu;" ::: "memory");
}
__device__ __forceinline__ void tmap_acquire(const void* map) {
  asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(map) : "memory");
}

// Host: encode a 3D float64 tensor map over a dense (d2, d1, d0) array with
// d0 fastest.  Returns false if the driver entry point is missing or the
// encode call rejects the arguments.
bool encode_tensor_map_3d_f64(CUtensorMap* map, const void* base, uint64_t d0, uint64_t d1, uint64_t d2,
                              uint32_t b0, uint32_t b1, uint32_t b2);
// Host: the same for a dense 2D (d1, d0) float64 array with row pitch
// `pitch_bytes` (a multiple of 16).
bool encode_tensor_map_2d_f64(CUtensorMap* map, const void* base, uint64_t d0, uint64_t d1, uint64_t pitch_bytes,
                              uint32_t b0, uint32_t b1);

}  // namespace ar
