// Confidence fallback of the mixed-stream executor: calls whose device-side
// selection was unsure are profiled exhaustively through the executor itself,
// and the profiled executions become records of the loop's region, which can
// then be trained again.  This is the adaptive region's record -> train loop
// (Section 2: the runtime records every execution's features, policy and
// time, and trains a model that maps features to the fastest policy; Table 1
// __apollo_region_train) driven by the learned selector's confidence.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "ar.h"
#include "ar_loops.h"
#include "model.h"

namespace {

constexpr int kExecNf[4] = {1, 3, 5, 1};  // the executor's features per loop
constexpr int kMaxVar = 16;               // most variants of an executor loop (Jacobi)
constexpr int kMaxReps = 16;
constexpr int kSlots = kMaxVar * (kMaxReps + 1);

size_t up256(size_t b) { return (b + 255) & ~size_t(255); }

// Workspace layout: the executor's one-call workspace, the one-call table,
// the forced-variant indices, per-execution output slots, and daxpy's saved y.
struct Layout {
  size_t exec_ws = 0, exec_bytes = 0, table = 0, force = 0, var = 0, conf = 0, feat = 0, t0 = 0, t1 = 0, st = 0,
         save = 0;
};

Layout layout() {
  Layout L;
  ar_exec_workspace_bytes(1, &L.exec_bytes);
  size_t o = 0;
  L.exec_ws = o;
  o = up256(o + L.exec_bytes);
  L.table = o;
  o = up256(o + sizeof(ar_exec_call));
  L.force = o;
  o = up256(o + sizeof(int32_t) * kMaxVar);
  L.var = o;
  o = up256(o + sizeof(int32_t) * kSlots);
  L.conf = o;
  o = up256(o + sizeof(float) * kSlots);
  L.feat = o;
  o = up256(o + sizeof(float) * 8 * kSlots);
  L.t0 = o;
  o = up256(o + sizeof(uint64_t) * kSlots);
  L.t1 = o;
  o = up256(o + sizeof(uint64_t) * kSlots);
  L.st = o;
  o = up256(o + sizeof(int32_t) * kSlots);
  L.save = o;
  return L;
}

int cuda_status(cudaError_t e) { return e == cudaSuccess ? AR_OK : AR_ERR_CUDA; }

template <class T>
T* at(void* base, size_t off) {
  return reinterpret_cast<T*>(static_cast<unsigned char*>(base) + off);
}

// Copy a retrained MLP of region r into the executor's device model buffers
// of loop L (same F, H and V).
int upload_mlp(ar_region* r, const ar_exec_models* m, int L, cudaStream_t s) {
  int F = 0, H = 0, V = 0;
  int rc = ar_mlp_export(r, nullptr, nullptr, nullptr, &F, &H, &V);
  if (rc != AR_OK) return rc;
  if (F != m->F[L] || V != m->V[L] || H != m->H || !m->theta[L] || !m->mu[L] || !m->sd[L]) return AR_ERR_STATE;
  std::vector<float> theta((size_t)ar_mlp_num_params(F, H, V)), mu(F), sd(F);
  rc = ar_mlp_export(r, theta.data(), mu.data(), sd.data(), &F, &H, &V);
  if (rc != AR_OK) return rc;
  cudaError_t e = cudaMemcpyAsync(const_cast<float*>(m->theta[L]), theta.data(), theta.size() * sizeof(float),
                                  cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(const_cast<float*>(m->mu[L]), mu.data(), mu.size() * sizeof(float), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(const_cast<float*>(m->sd[L]), sd.data(), sd.size() * sizeof(float), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // the host vectors go out of scope
  return cuda_status(e);
}

}  // namespace

extern "C" int ar_exec_fallback_workspace_bytes(int64_t max_daxpy_n, size_t* bytes) {
  if (max_daxpy_n < 0 || !bytes) return AR_ERR_ARG;
  *bytes = layout().save + up256(sizeof(double) * (size_t)max_daxpy_n);
  return AR_OK;
}

extern "C" int ar_exec_fallback(const ar_exec_call* calls, int ncalls, const float* features, const float* conf,
                                float tau, ar_region* const* regions, int reps, const ar_exec_models* models,
                                int retrain, void* workspace, size_t workspace_bytes, void* stream, int32_t* best,
                                int* num_profiled) {
  if (ncalls < 0 || ncalls > AR_EXEC_MAX_CALLS || (ncalls > 0 && (!calls || !features || !conf || !best)) ||
      !regions || reps < 1 || reps > kMaxReps || !(tau == tau) || !workspace)
    return AR_ERR_ARG;
  const Layout lay = layout();
  if (workspace_bytes < lay.save) return AR_ERR_ARG;
  const int64_t save_cap = (int64_t)((workspace_bytes - lay.save) / sizeof(double));
  // every region given must have the loop's variants and the executor's features
  for (int L = 0; L < 4; ++L) {
    if (!regions[L]) continue;
    int V = 0, nf = 0;
    if (ar_region_info(regions[L], &V, &nf, nullptr, nullptr, nullptr) != AR_OK) return AR_ERR_ARG;
    if (V != ar_exec_num_variants(L) || V > kMaxVar || nf != kExecNf[L]) return AR_ERR_STATE;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int32_t force_h[kMaxVar];
  for (int v = 0; v < kMaxVar; ++v) force_h[v] = v;
  int32_t* force = at<int32_t>(workspace, lay.force);
  cudaError_t e = cudaMemcpyAsync(force, force_h, sizeof(force_h), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return AR_ERR_CUDA;

  bool fed[4] = {false, false, false, false};
  int profiled = 0, result = AR_OK;
  std::vector<uint64_t> t0(kSlots), t1(kSlots);
  std::vector<int32_t> st(kSlots);
  std::vector<double> mean;
  for (int c = 0; c < ncalls && result == AR_OK; ++c) {
    best[c] = -1;
    const ar_exec_call& k = calls[c];
    if (k.loop < 0 || k.loop > 3 || !(conf[c] < tau) || !regions[k.loop]) continue;
    ar_region* r = regions[k.loop];
    const int L = k.loop, V = ar_exec_num_variants(L), nf = kExecNf[L];
    const float* f = features + 8 * c;
    // features recorded for every variant before: take the recorded best
    if (ar::region_key_means(r, f, nf, &mean) == V) {
      best[c] = ar::best_of_means(mean, ar::region_tie(r));
      continue;
    }
    if (L == AR_LOOP_DAXPY && k.n > save_cap) {
      result = AR_ERR_ARG;  // daxpy's y cannot be saved in this workspace
      break;
    }
    void* flush = nullptr;
    size_t flush_bytes = 0;
    ar::region_flush_buffer(r, &flush, &flush_bytes);
    ar_exec_call* table = at<ar_exec_call>(workspace, lay.table);
    double* saved = at<double>(workspace, lay.save);
    e = cudaMemcpyAsync(table, &k, sizeof(k), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && L == AR_LOOP_DAXPY && k.n > 0)
      e = cudaMemcpyAsync(saved, k.out0, sizeof(double) * (size_t)k.n, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) {
      result = AR_ERR_CUDA;
      break;
    }
    // each variant once untimed, then `reps` timed runs, each in its own slot
    int slot = 0;
    for (int v = 0; v < V && result == AR_OK; ++v)
      for (int t = 0; t <= reps && result == AR_OK; ++t, ++slot) {
        if (t > 0 && flush && flush_bytes) cudaMemsetAsync(flush, t & 0xff, flush_bytes, s);
        result = ar_exec_batch(table, 1, nullptr, force + v, at<int32_t>(workspace, lay.var) + slot,
                               at<float>(workspace, lay.conf) + slot, at<float>(workspace, lay.feat) + 8 * slot,
                               at<uint64_t>(workspace, lay.t0) + slot, at<uint64_t>(workspace, lay.t1) + slot,
                               at<int32_t>(workspace, lay.st) + slot, at<void>(workspace, lay.exec_ws),
                               lay.exec_bytes, stream);
      }
    if (result != AR_OK) break;
    e = cudaMemcpyAsync(t0.data(), at<uint64_t>(workspace, lay.t0), sizeof(uint64_t) * slot, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(t1.data(), at<uint64_t>(workspace, lay.t1), sizeof(uint64_t) * slot,
                          cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(st.data(), at<int32_t>(workspace, lay.st), sizeof(int32_t) * slot, cudaMemcpyDeviceToHost,
                          s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      result = AR_ERR_CUDA;
      break;
    }
    std::vector<double> m(V, 0.0);
    for (int v = 0, q = 0; v < V && result == AR_OK; ++v)
      for (int t = 0; t <= reps; ++t, ++q) {
        if (st[q] != AR_OK) {
          result = st[q];
          break;
        }
        if (t == 0) continue;  // warm-up
        const float ms = (float)((double)(t1[q] - t0[q]) * 1e-6);
        result = ar_add_record(r, f, nf, v, ms);
        if (result != AR_OK) break;
        m[v] += ms / reps;
      }
    if (result != AR_OK) break;
    best[c] = ar::best_of_means(m, ar::region_tie(r));
    fed[L] = true;
    ++profiled;
    // leave the call's outputs as its best variant computes them: daxpy's y
    // (updated in place by every run) goes back to its value before the
    // fallback, which every daxpy variant gives alike; the other loops
    // overwrite their outputs, so one more run of the best variant
    if (L == AR_LOOP_DAXPY) {
      if (k.n > 0) e = cudaMemcpyAsync(k.out0, saved, sizeof(double) * (size_t)k.n, cudaMemcpyDeviceToDevice, s);
      if (e != cudaSuccess) result = AR_ERR_CUDA;
      continue;
    }
    result = ar_exec_batch(table, 1, nullptr, force + best[c], at<int32_t>(workspace, lay.var),
                           at<float>(workspace, lay.conf), at<float>(workspace, lay.feat),
                           at<uint64_t>(workspace, lay.t0), at<uint64_t>(workspace, lay.t1),
                           at<int32_t>(workspace, lay.st), at<void>(workspace, lay.exec_ws), lay.exec_bytes, stream);
    if (result == AR_OK) {
      int32_t s0 = AR_OK;
      e = cudaMemcpyAsync(&s0, at<int32_t>(workspace, lay.st), sizeof(s0), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) result = AR_ERR_CUDA;
      else if (s0 != AR_OK) result = s0;
    }
  }
  // the daxpy restores (and every other enqueued copy) complete before return
  if (result == AR_OK && cudaStreamSynchronize(s) != cudaSuccess) result = AR_ERR_CUDA;
  if (result == AR_OK && retrain)
    for (int L = 0; L < 4 && result == AR_OK; ++L) {
      if (!fed[L]) continue;
      result = ar_train(regions[L]);
      int kind = -1;
      if (result == AR_OK) result = ar_region_info(regions[L], nullptr, nullptr, nullptr, nullptr, &kind);
      if (result == AR_OK && models && kind == 1) result = upload_mlp(regions[L], models, L, s);
    }
  if (num_profiled) *num_profiled = profiled;
  if (ar::log_level() >= 1) {
    int low = 0;
    for (int c = 0; c < ncalls; ++c) low += conf[c] < tau;
    ar::log_line("exec-fallback", "%d of %d calls below confidence %.3f: %d profiled, %d from records%s; status %d",
                 low, ncalls, (double)tau, profiled, low - profiled, retrain ? ", regions retrained" : "", result);
  }
  return result;
}
