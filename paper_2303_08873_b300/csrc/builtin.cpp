// Built-in loop table: variant counts, defaults, names and region launchers
// for the region bodies (ar_loops.h).
#include <cuda_runtime.h>

#include <cstdio>

#include "common.cuh"

namespace ar {

int device_sms() {
  static const int sms = [] {  // initialised once, thread-safe
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
      return v;
    return kNumSMs;
  }();
  return sms;
}

}  // namespace ar

using namespace ar;

namespace {

struct LoopEntry {
  int (*count)();
  int (*name)(int, char*, int);
  ar_launch_fn launch;
  int def;
};

const LoopEntry* entry(int loop) {
  static const LoopEntry table[] = {
      {daxpy_num_variants, daxpy_variant_name, daxpy_launch, 6},
      {jacobi7_num_variants, jacobi7_variant_name, jacobi7_launch, 1},
      {spmv_num_variants, spmv_variant_name, spmv_launch, 0},
      {nbody_num_variants, nbody_variant_name, nbody_launch, 3},
      {heat7_num_variants, heat7_variant_name, heat7_launch, 1},
  };
  if (loop < 0 || loop >= (int)(sizeof table / sizeof table[0])) return nullptr;
  return &table[loop];
}

}  // namespace

extern "C" int ar_loop_num_variants(int loop) {
  const LoopEntry* e = entry(loop);
  return e ? e->count() : AR_ERR_ARG;
}

extern "C" int ar_loop_default_variant(int loop) {
  const LoopEntry* e = entry(loop);
  return e ? e->def : AR_ERR_ARG;
}

extern "C" int ar_loop_variant_name(int loop, int variant, char* buf, int len) {
  const LoopEntry* e = entry(loop);
  return e ? e->name(variant, buf, len) : AR_ERR_ARG;
}

extern "C" int ar_region_add_builtin(ar_region* r, int loop, int* out_count) {
  const LoopEntry* e = entry(loop);
  if (!r || !e) return AR_ERR_ARG;
  return ar_region_add_builtin_first(r, loop, e->count(), out_count);
}

extern "C" int ar_region_add_builtin_first(ar_region* r, int loop, int count, int* out_count) {
  const LoopEntry* e = entry(loop);
  if (!r || !e || count < 1 || count > e->count()) return AR_ERR_ARG;
  const int n = count;
  for (int v = 0; v < n; ++v) {
    char nm[64];
    e->name(v, nm, sizeof nm);
    const int rc = ar_variant_register(r, nm, (double)v, e->launch, nullptr, nullptr);
    if (rc != AR_OK) return rc;
  }
  if (out_count) *out_count = n;
  return AR_OK;
}
