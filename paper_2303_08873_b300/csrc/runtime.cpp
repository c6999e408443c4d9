// Adaptive-region runtime (C ABI of ar.h).
//
// Implements the region lifecycle of arXiv 2303.08873: create (Table 1
// region_create), begin / set_feature / get_policy / end around each
// execution (Table 1; Section 3.3 lowering), RoundRobin exploration until
// the number of unique (features, variant) points reaches min_train_data
// (Section 2, Apollo example), training on the fastest variant per feature
// vector (Section 2) and model-driven selection afterwards (Section 3.1).
// Elapsed times come from CUDA event pairs on the caller's stream, resolved
// without blocking as later calls arrive.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <set>
#include <string>
#include <vector>

#include "model.h"

namespace {

using ar::FKey;

enum Kind { K_DTREE = 0, K_MLP = 1, K_EXHAUSTIVE = 2, K_FIXED = 3, K_RFC = 4 };

struct Variant {
  std::string name;
  double value;
  ar_launch_fn fn;
  void* user;
  bool usable;
};

struct Pending {
  cudaEvent_t start, stop;
  FKey key;
  int variant;
};

}  // namespace

struct ar_region {
  std::string id;
  int nf = 0;
  Kind kind = K_DTREE;
  int depth = 2;
  int ntrees = 10;
  int hidden = 64;
  int fixed = 0;
  int reps = 5;
  float tau = 0.5f;
  double tie = ar::kTieRel;  // means within this fraction of the fastest tie (lowest index wins)
  int epochs = 200;
  uint64_t seed = 0x5eed;
  int min_train_req = 0;  // as passed; <= 0: number of variants
  int min_train = 0;      // effective, fixed at the first begin
  bool frozen = false;
  std::vector<Variant> variants;

  // current execution (begin .. end)
  bool open = false;
  bool have_policy = false;
  int ctx_nset = 0;
  float ctx_f[AR_MAX_FEATURES] = {};
  int ctx_policy = -1;
  cudaEvent_t ctx_start = nullptr;

  uint64_t explore_counter = 0;
  std::vector<ar::Record> records;
  // per exact feature vector: (sum of ms, count) of each variant's records
  std::map<FKey, std::vector<std::pair<double, int64_t>>> agg;
  std::deque<Pending> pending;
  std::vector<cudaEvent_t> event_pool;
  std::set<std::pair<FKey, int>> unique;
  bool trained = false;
  bool auto_trained = false;

  std::vector<ar::TreeNode> tree;
  std::vector<std::vector<ar::TreeNode>> forest;
  ar::MlpModel mlp;
  std::map<FKey, int> table;

  ar_fake_time_fn fake = nullptr;
  void* fake_user = nullptr;
  void* flush_buf = nullptr;
  size_t flush_bytes = 0;
  std::string err;
};

namespace {

int fail(ar_region* r, int code, const char* fmt, ...) __attribute__((format(printf, 3, 4)));
int fail(ar_region* r, int code, const char* fmt, ...) {
  if (r) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    r->err = buf;
  }
  return code;
}

int cuda_fail(ar_region* r, cudaError_t e, const char* what) {
  return fail(r, AR_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

bool parse_int(const std::string& s, long* out) {
  if (s.empty()) return false;
  char* end = nullptr;
  long v = strtol(s.c_str(), &end, 10);
  if (*end) return false;
  *out = v;
  return true;
}

int parse_spec(ar_region* r, const char* spec) {
  std::string s = spec ? spec : "";
  std::vector<std::string> tok;
  size_t p = 0;
  while (p <= s.size() && !s.empty()) {
    size_t q = s.find(',', p);
    if (q == std::string::npos) q = s.size();
    std::string t = s.substr(p, q - p);
    t.erase(0, t.find_first_not_of(" \t"));
    t.erase(t.find_last_not_of(" \t") + 1);
    tok.push_back(t);
    p = q + 1;
    if (q == s.size()) break;
  }
  size_t i = 0;
  if (!tok.empty() && tok[0].find('=') == std::string::npos) {
    const std::string& k = tok[0];
    long v = 0;
    if (k == "dtree" || k == "DecisionTree") {
      r->kind = K_DTREE;
      if (tok.size() > 1 && parse_int(tok[1], &v)) {
        if (v < 1 || v > 16) return fail(r, AR_ERR_ARG, "dtree depth %ld out of [1, 16]", v);
        r->depth = (int)v;
        ++i;
      }
    } else if (k == "rfc") {
      // Section 3.1: the number of trees and the depth are given together or not at all
      r->kind = K_RFC;
      long d = 0;
      const bool a1 = tok.size() > 1 && parse_int(tok[1], &v);
      const bool a2 = a1 && tok.size() > 2 && parse_int(tok[2], &d);
      if (a1 && !a2) return fail(r, AR_ERR_ARG, "rfc takes both ntrees and depth, or neither");
      if (a2) {
        if (v < 1 || v > 256 || d < 1 || d > 16) return fail(r, AR_ERR_ARG, "rfc ntrees in [1,256], depth in [1,16]");
        r->ntrees = (int)v;
        r->depth = (int)d;
        i += 2;
      }
    } else if (k == "mlp") {
      r->kind = K_MLP;
      if (tok.size() > 1 && parse_int(tok[1], &v)) {
        if (v != 32 && v != 64) return fail(r, AR_ERR_ARG, "mlp hidden width must be 32 or 64");
        r->hidden = (int)v;
        ++i;
      }
    } else if (k == "exhaustive") {
      r->kind = K_EXHAUSTIVE;
    } else if (k == "fixed") {
      r->kind = K_FIXED;
      if (tok.size() < 2 || !parse_int(tok[1], &v) || v < 0)
        return fail(r, AR_ERR_ARG, "fixed needs a variant index");
      r->fixed = (int)v;
      ++i;
    } else if (!k.empty()) {
      return fail(r, AR_ERR_ARG, "unknown model kind '%s'", k.c_str());
    }
    ++i;
  }
  for (; i < tok.size(); ++i) {
    const std::string& t = tok[i];
    if (t.empty()) continue;
    size_t eq = t.find('=');
    if (eq == std::string::npos) return fail(r, AR_ERR_ARG, "bad model option '%s'", t.c_str());
    std::string key = t.substr(0, eq), val = t.substr(eq + 1);
    long v = 0;
    if (key == "explore") {
      if (val != "roundrobin" && val != "RoundRobin") return fail(r, AR_ERR_ARG, "unknown explore '%s'", val.c_str());
    } else if (key == "reps") {
      if (!parse_int(val, &v) || v < 1 || v > 1000) return fail(r, AR_ERR_ARG, "bad reps");
      r->reps = (int)v;
    } else if (key == "conf") {
      char* end = nullptr;
      double d = strtod(val.c_str(), &end);
      if (*end || !(d >= 0.0 && d <= 1.0)) return fail(r, AR_ERR_ARG, "bad conf");
      r->tau = (float)d;
    } else if (key == "tie") {
      char* end = nullptr;
      double d = strtod(val.c_str(), &end);
      if (*end || !(d >= 0.0 && d < 1.0)) return fail(r, AR_ERR_ARG, "bad tie");
      r->tie = d;
    } else if (key == "epochs") {
      if (!parse_int(val, &v) || v < 1 || v > 100000) return fail(r, AR_ERR_ARG, "bad epochs");
      r->epochs = (int)v;
    } else if (key == "seed") {
      if (!parse_int(val, &v)) return fail(r, AR_ERR_ARG, "bad seed");
      r->seed = (uint64_t)v;
    } else {
      return fail(r, AR_ERR_ARG, "unknown model option '%s'", key.c_str());
    }
  }
  return AR_OK;
}

bool finite_all(const float* f, int n) {
  for (int i = 0; i < n; ++i)
    if (!std::isfinite(f[i])) return false;
  return true;
}

cudaEvent_t take_event(ar_region* r) {
  if (!r->event_pool.empty()) {
    cudaEvent_t e = r->event_pool.back();
    r->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

void give_event(ar_region* r, cudaEvent_t e) {
  if (e) r->event_pool.push_back(e);
}

void add_record(ar_region* r, const FKey& key, int variant, float ms) {
  ar::Record rec;
  for (int i = 0; i < AR_MAX_FEATURES; ++i) memcpy(&rec.f[i], &key[i], 4);
  rec.variant = variant;
  rec.ms = ms;
  r->records.push_back(rec);
  auto& a = r->agg[key];
  if (a.size() < r->variants.size()) a.resize(r->variants.size(), {0.0, 0});
  if (variant >= 0 && variant < (int)a.size()) {
    a[variant].first += ms;
    a[variant].second += 1;
  }
}

// Resolve completed pending executions in order; block on them if `wait`.
int resolve(ar_region* r, bool wait) {
  while (!r->pending.empty()) {
    Pending& p = r->pending.front();
    cudaError_t q = wait ? cudaEventSynchronize(p.stop) : cudaEventQuery(p.stop);
    if (q == cudaErrorNotReady) return AR_OK;
    if (q != cudaSuccess) return cuda_fail(r, q, "event");
    float ms = 0.f;
    cudaError_t e = cudaEventElapsedTime(&ms, p.start, p.stop);
    if (e != cudaSuccess) return cuda_fail(r, e, "cudaEventElapsedTime");
    add_record(r, p.key, p.variant, ms);
    give_event(r, p.start);
    give_event(r, p.stop);
    r->pending.pop_front();
  }
  return AR_OK;
}

int next_usable(const ar_region* r, int v) {
  const int V = (int)r->variants.size();
  for (int t = 0; t < V; ++t) {
    int c = (v + t) % V;
    if (r->variants[c].usable) return c;
  }
  return -1;
}

int explore_policy(ar_region* r) {
  const int V = (int)r->variants.size();
  const int v = (int)(r->explore_counter++ % (uint64_t)V);
  return next_usable(r, v);
}

// Model prediction; -1 when the model has no answer for these features.
int predict(const ar_region* r, const float* f, float* conf) {
  float c = 1.f;
  int v = -1;
  switch (r->kind) {
    case K_FIXED:
      v = r->fixed < (int)r->variants.size() ? r->fixed : -1;
      break;
    case K_DTREE:
      if (!r->tree.empty()) v = ar::tree_predict(r->tree, f, &c);
      break;
    case K_RFC:
      if (!r->forest.empty()) v = ar::forest_predict(r->forest, f, &c);
      break;
    case K_MLP:
      if (r->mlp.V > 0) v = ar::mlp_predict_host(r->mlp, f, &c);
      break;
    case K_EXHAUSTIVE: {
      auto it = r->table.find(ar::make_key(f, r->nf));
      if (it != r->table.end()) v = it->second;
      break;
    }
  }
  if (conf) *conf = c;
  return v;
}

int choose(ar_region* r, const float* f) {
  if (r->kind == K_FIXED) return next_usable(r, std::min(r->fixed, (int)r->variants.size() - 1));
  if (r->trained) {
    int v = predict(r, f, nullptr);
    if (v >= 0) {
      if (ar::log_level() >= 2) ar::log_line(r->id.c_str(), "policy %d from the model", next_usable(r, v));
      return next_usable(r, v);
    }
  }
  const int e = explore_policy(r);
  if (ar::log_level() >= 2) ar::log_line(r->id.c_str(), "policy %d from exploration", e);
  return e;
}

void freeze(ar_region* r) {
  if (r->frozen) return;
  r->frozen = true;
  r->min_train = r->min_train_req > 0 ? r->min_train_req : (int)r->variants.size();
}

}  // namespace

// ============================================================== C ABI
extern "C" {

int ar_region_create(const char* id, int num_features, const char* model_spec, int min_train_data,
                     ar_region** out) {
  if (!out || !id || !*id || num_features < 0 || num_features > AR_MAX_FEATURES) return AR_ERR_ARG;
  ar_region* r = new (std::nothrow) ar_region();
  if (!r) return AR_ERR_OOM;
  r->id = id;
  r->nf = num_features;
  r->min_train_req = min_train_data;
  int rc = parse_spec(r, model_spec);
  if (rc != AR_OK) {
    delete r;
    return rc;
  }
  *out = r;
  return AR_OK;
}

void ar_region_destroy(ar_region* r) {
  if (!r) return;
  for (auto& p : r->pending) {
    cudaEventDestroy(p.start);
    cudaEventDestroy(p.stop);
  }
  for (auto e : r->event_pool) cudaEventDestroy(e);
  if (r->ctx_start) cudaEventDestroy(r->ctx_start);
  delete r;
}

int ar_variant_register(ar_region* r, const char* name, double value, ar_launch_fn fn, void* user,
                        int* out_index) {
  if (!r) return AR_ERR_ARG;
  if (r->frozen) return fail(r, AR_ERR_STATE, "variants are closed after the first execution");
  if (!fn) return fail(r, AR_ERR_ARG, "NULL launcher");
  if ((int)r->variants.size() >= AR_MAX_VARIANTS) return fail(r, AR_ERR_ARG, "too many variants");
  Variant v;
  v.name = name ? name : std::to_string(value);
  v.value = value;
  v.fn = fn;
  v.user = user;
  v.usable = true;
  r->variants.push_back(v);
  if (out_index) *out_index = (int)r->variants.size() - 1;
  return AR_OK;
}

int ar_variant_register_range(ar_region* r, double begin, double end, double step, ar_launch_fn fn,
                              void* user, int* out_count) {
  if (!r) return AR_ERR_ARG;
  if (!(step > 0.0) || !(end >= begin) || !std::isfinite(begin) || !std::isfinite(end))
    return fail(r, AR_ERR_ARG, "range needs finite bounds, step > 0 and end >= begin");
  const double cnt = std::floor((end - begin) / step + 1e-9) + 1.0;
  if (cnt > AR_MAX_VARIANTS - (double)r->variants.size()) return fail(r, AR_ERR_ARG, "range too long");
  const int n = (int)cnt;
  for (int i = 0; i < n; ++i) {
    const double v = begin + i * step;
    char nm[64];
    snprintf(nm, sizeof nm, "%.17g", v);
    int rc = ar_variant_register(r, nm, v, fn, user, nullptr);
    if (rc != AR_OK) return rc;
  }
  if (out_count) *out_count = n;
  return AR_OK;
}

int ar_region_info(const ar_region* r, int* num_variants, int* num_features, int* min_train_data,
                   int* trained, int* model_kind) {
  if (!r) return AR_ERR_ARG;
  if (num_variants) *num_variants = (int)r->variants.size();
  if (num_features) *num_features = r->nf;
  if (min_train_data)
    *min_train_data = r->frozen ? r->min_train : (r->min_train_req > 0 ? r->min_train_req : (int)r->variants.size());
  if (trained) *trained = r->trained ? 1 : 0;
  if (model_kind) *model_kind = (int)r->kind;
  return AR_OK;
}

int ar_variant_info(const ar_region* r, int variant, double* value, char* name, int name_len, int* usable) {
  if (!r || variant < 0 || variant >= (int)r->variants.size()) return AR_ERR_ARG;
  const Variant& v = r->variants[variant];
  if (value) *value = v.value;
  if (name && name_len > 0) snprintf(name, (size_t)name_len, "%s", v.name.c_str());
  if (usable) *usable = v.usable ? 1 : 0;
  return AR_OK;
}

int ar_begin(ar_region* r, void* stream) {
  if (!r) return AR_ERR_ARG;
  if (r->open) return fail(r, AR_ERR_STATE, "begin inside an open execution");
  if (r->variants.empty()) return fail(r, AR_ERR_STATE, "region has no variants");
  if (next_usable(r, 0) < 0) return fail(r, AR_ERR_STATE, "no usable variant left");
  freeze(r);
  if (!r->fake) {
    int rc = resolve(r, false);
    if (rc != AR_OK) return rc;
    cudaEvent_t e = take_event(r);
    if (!e) return fail(r, AR_ERR_CUDA, "cudaEventCreate failed");
    cudaError_t ce = cudaEventRecord(e, reinterpret_cast<cudaStream_t>(stream));
    if (ce != cudaSuccess) {
      give_event(r, e);
      return cuda_fail(r, ce, "cudaEventRecord");
    }
    r->ctx_start = e;
  }
  r->open = true;
  r->have_policy = false;
  r->ctx_nset = 0;
  memset(r->ctx_f, 0, sizeof r->ctx_f);
  return AR_OK;
}

int ar_set_feature(ar_region* r, float value) {
  if (!r) return AR_ERR_ARG;
  if (!r->open || r->have_policy) return fail(r, AR_ERR_STATE, "set_feature outside begin/get_policy");
  if (r->ctx_nset >= r->nf) return fail(r, AR_ERR_STATE, "more than %d features", r->nf);
  if (!std::isfinite(value)) return fail(r, AR_ERR_ARG, "feature is NaN or inf");
  r->ctx_f[r->ctx_nset++] = value;
  return AR_OK;
}

int ar_get_policy(ar_region* r, int* out_variant) {
  if (!r || !out_variant) return AR_ERR_ARG;
  if (!r->open) return fail(r, AR_ERR_STATE, "get_policy outside begin/end");
  if (r->ctx_nset != r->nf) return fail(r, AR_ERR_STATE, "%d of %d features set", r->ctx_nset, r->nf);
  if (!r->have_policy) {
    int v = choose(r, r->ctx_f);
    if (v < 0) return fail(r, AR_ERR_STATE, "no usable variant left");
    r->ctx_policy = v;
    r->have_policy = true;
  }
  *out_variant = r->ctx_policy;
  return AR_OK;
}

static void close_ctx(ar_region* r) {
  if (r->ctx_start) give_event(r, r->ctx_start);
  r->ctx_start = nullptr;
  r->open = false;
  r->have_policy = false;
}

int ar_end(ar_region* r, void* stream) {
  if (!r) return AR_ERR_ARG;
  if (!r->open || !r->have_policy) return fail(r, AR_ERR_STATE, "end without begin and get_policy");
  const FKey key = ar::make_key(r->ctx_f, r->nf);
  const int v = r->ctx_policy;
  if (r->fake) {
    const double ms = r->fake(r->ctx_f, r->nf, v, r->fake_user);
    add_record(r, key, v, (float)ms);
    close_ctx(r);
  } else {
    cudaEvent_t stop = take_event(r);
    if (!stop) {
      close_ctx(r);
      return fail(r, AR_ERR_CUDA, "cudaEventCreate failed");
    }
    cudaError_t ce = cudaEventRecord(stop, reinterpret_cast<cudaStream_t>(stream));
    if (ce != cudaSuccess) {
      give_event(r, stop);
      close_ctx(r);
      return cuda_fail(r, ce, "cudaEventRecord");
    }
    r->pending.push_back(Pending{r->ctx_start, stop, key, v});
    r->ctx_start = nullptr;
    r->open = false;
    r->have_policy = false;
  }
  r->unique.insert({key, v});
  if (!r->auto_trained && !r->trained && r->kind != K_FIXED && (int)r->unique.size() >= r->min_train) {
    r->auto_trained = true;
    if (ar::log_level() >= 1)
      ar::log_line(r->id.c_str(), "%zu unique points reached min_train_data %d: training", r->unique.size(),
                   r->min_train);
    return ar_train(r);
  }
  return AR_OK;
}

int ar_invoke(ar_region* r, const float* features, int nf, void* args, void* stream, int* out_variant,
              double* out_value) {
  if (!r) return AR_ERR_ARG;
  if (nf != r->nf) return fail(r, AR_ERR_STATE, "expected %d features, got %d", r->nf, nf);
  if (nf > 0 && !features) return fail(r, AR_ERR_ARG, "NULL features");
  if (!finite_all(features, nf)) return fail(r, AR_ERR_ARG, "feature is NaN or inf");
  int rc = ar_begin(r, stream);
  if (rc != AR_OK) return rc;
  for (int i = 0; i < nf; ++i) ar_set_feature(r, features[i]);
  int v = -1;
  rc = ar_get_policy(r, &v);
  if (rc != AR_OK) {
    close_ctx(r);
    return rc;
  }
  Variant& var = r->variants[v];
  const int lrc = var.fn(args, v, var.value, stream, var.user);
  if (lrc != 0) {
    var.usable = false;
    if (ar::log_level() >= 1) ar::log_line(r->id.c_str(), "variant %d (%s) failed to launch: unusable", v, var.name.c_str());
    close_ctx(r);
    return fail(r, AR_ERR_CUDA, "variant %d (%s) launcher failed with %d", v, var.name.c_str(), lrc);
  }
  rc = ar_end(r, stream);
  if (rc != AR_OK) return rc;
  if (out_variant) *out_variant = v;
  if (out_value) *out_value = var.value;
  return AR_OK;
}

int ar_invoke_host(ar_region* r, const float* features, int nf, void* args, void* stream, const ar_host_copy* in,
                   int n_in, const ar_host_copy* out, int n_out, int* out_variant, double* out_value) {
  if (!r) return AR_ERR_ARG;
  // the checks of ar_invoke first, so that nothing is enqueued for a call it rejects
  if (nf != r->nf) return fail(r, AR_ERR_STATE, "expected %d features, got %d", r->nf, nf);
  if (nf > 0 && !features) return fail(r, AR_ERR_ARG, "NULL features");
  if (!finite_all(features, nf)) return fail(r, AR_ERR_ARG, "feature is NaN or inf");
  if (r->open) return fail(r, AR_ERR_STATE, "an execution is already open");
  if (r->variants.empty()) return fail(r, AR_ERR_STATE, "region has no variants");
  if (n_in < 0 || n_out < 0 || (n_in > 0 && !in) || (n_out > 0 && !out))
    return fail(r, AR_ERR_ARG, "bad copy list");
  for (int i = 0; i < n_in + n_out; ++i) {
    const ar_host_copy& c = i < n_in ? in[i] : out[i - n_in];
    if (c.bytes > 0 && (!c.host || !c.device)) return fail(r, AR_ERR_ARG, "copy %d has a NULL pointer", i);
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  for (int i = 0; i < n_in; ++i) {
    if (!in[i].bytes) continue;
    const cudaError_t e = cudaMemcpyAsync(in[i].device, in[i].host, in[i].bytes, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(r, e, "host-to-device copy");
  }
  int rc = ar_invoke(r, features, nf, args, stream, out_variant, out_value);
  if (rc != AR_OK) return rc;
  for (int i = 0; i < n_out; ++i) {
    if (!out[i].bytes) continue;
    const cudaError_t e = cudaMemcpyAsync(out[i].host, out[i].device, out[i].bytes, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_fail(r, e, "device-to-host copy");
  }
  return AR_OK;
}

int ar_select(ar_region* r, const float* features, int nf, int* out_variant, float* out_conf) {
  if (!r || !out_variant) return AR_ERR_ARG;
  if (nf != r->nf) return fail(r, AR_ERR_STATE, "expected %d features, got %d", r->nf, nf);
  if (nf > 0 && !features) return fail(r, AR_ERR_ARG, "NULL features");
  if (!finite_all(features, nf)) return fail(r, AR_ERR_ARG, "feature is NaN or inf");
  if (r->kind != K_FIXED && !r->trained) return fail(r, AR_ERR_NOMODEL, "no trained model");
  float f[AR_MAX_FEATURES] = {};
  for (int i = 0; i < nf; ++i) f[i] = features[i];
  float c = 1.f;
  int v = predict(r, f, &c);
  if (v < 0) return fail(r, AR_ERR_NOMODEL, "model has no entry for these features");
  if (ar::log_level() >= 2) ar::log_line(r->id.c_str(), "selected %d (%s), confidence %.3f", v, r->variants[v].name.c_str(), c);
  *out_variant = v;
  if (out_conf) *out_conf = c;
  return AR_OK;
}

int ar_profile(ar_region* r, const float* features, int nf, void* args, void* stream, int reps, float* out_ms,
               int* out_best) {
  if (!r) return AR_ERR_ARG;
  if (r->open) return fail(r, AR_ERR_STATE, "profile inside an open execution");
  if (nf != r->nf) return fail(r, AR_ERR_STATE, "expected %d features, got %d", r->nf, nf);
  if (nf > 0 && !features) return fail(r, AR_ERR_ARG, "NULL features");
  if (!finite_all(features, nf)) return fail(r, AR_ERR_ARG, "feature is NaN or inf");
  if (r->variants.empty()) return fail(r, AR_ERR_STATE, "region has no variants");
  if (reps <= 0) reps = r->reps;
  freeze(r);
  int rc = resolve(r, true);
  if (rc != AR_OK) return rc;
  float f[AR_MAX_FEATURES] = {};
  for (int i = 0; i < nf; ++i) f[i] = features[i];
  const FKey key = ar::make_key(f, nf);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int V = (int)r->variants.size();
  std::vector<double> mean(V, INFINITY);
  std::vector<cudaEvent_t> ev;
  if (!r->fake) {
    ev.resize(2 * (size_t)reps, nullptr);
    for (auto& e : ev)
      if (!(e = take_event(r))) {
        for (auto x : ev) give_event(r, x);
        return fail(r, AR_ERR_CUDA, "cudaEventCreate failed");
      }
  }
  int result = AR_OK;
  for (int v = 0; v < V && result == AR_OK; ++v) {
    Variant& var = r->variants[v];
    if (!var.usable) continue;
    if (var.fn(args, v, var.value, stream, var.user) != 0) {  // warm-up
      var.usable = false;
      cudaGetLastError();
      continue;
    }
    double sum = 0.0;
    bool ok = true;
    for (int t = 0; t < reps && ok; ++t) {
      if (!r->fake) {
        if (r->flush_buf && r->flush_bytes)
          cudaMemsetAsync(r->flush_buf, t & 0xff, r->flush_bytes, s);
        cudaEventRecord(ev[2 * t], s);
      }
      if (var.fn(args, v, var.value, stream, var.user) != 0) {
        ok = false;
        break;
      }
      if (!r->fake) {
        cudaEventRecord(ev[2 * t + 1], s);
      } else {
        const double ms = r->fake(f, nf, v, r->fake_user);
        add_record(r, key, v, (float)ms);
        sum += ms;
      }
    }
    if (!ok) {
      var.usable = false;
      cudaGetLastError();
      continue;
    }
    if (!r->fake) {
      cudaError_t ce = cudaEventSynchronize(ev[2 * reps - 1]);
      if (ce != cudaSuccess) {
        result = cuda_fail(r, ce, "profile");
        break;
      }
      for (int t = 0; t < reps; ++t) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev[2 * t], ev[2 * t + 1]);
        add_record(r, key, v, ms);
        sum += ms;
      }
    }
    mean[v] = sum / reps;
    r->unique.insert({key, v});
  }
  for (auto x : ev) give_event(r, x);
  if (result != AR_OK) return result;
  const int best = ar::best_of_means(mean, r->tie);
  if (best < 0) return fail(r, AR_ERR_STATE, "no variant could be profiled");
  if (ar::log_level() >= 2)
    ar::log_line(r->id.c_str(), "profiled %d variants x %d reps: best %d (%s) %.4g ms", V, reps, best,
                 r->variants[best].name.c_str(), mean[best]);
  if (r->kind == K_EXHAUSTIVE) {
    r->table[key] = best;
    r->trained = true;
  }
  if (out_ms)
    for (int v = 0; v < V; ++v) out_ms[v] = (float)mean[v];
  if (out_best) *out_best = best;
  return AR_OK;
}

int ar_flush_records(ar_region* r) {
  if (!r) return AR_ERR_ARG;
  return resolve(r, true);
}

int ar_train(ar_region* r) {
  if (!r) return AR_ERR_ARG;
  int rc = resolve(r, true);
  if (rc != AR_OK) return rc;
  if (r->kind == K_FIXED) {
    r->trained = true;
    return AR_OK;
  }
  if (r->records.empty()) return fail(r, AR_ERR_STATE, "no records to train on");
  std::vector<FKey> keys;
  std::vector<int> labels;
  ar::label_records(r->records, (int)r->variants.size(), &keys, &labels, r->tie);
  switch (r->kind) {
    case K_DTREE: {
      std::vector<std::array<float, AR_MAX_FEATURES>> X(keys.size());
      for (size_t i = 0; i < keys.size(); ++i) X[i] = ar::key_values(keys[i]);
      r->tree = ar::tree_fit(X, labels, r->nf, r->depth);
      break;
    }
    case K_RFC: {
      std::vector<std::array<float, AR_MAX_FEATURES>> X(keys.size());
      for (size_t i = 0; i < keys.size(); ++i) X[i] = ar::key_values(keys[i]);
      r->forest = ar::forest_fit(X, labels, r->nf, r->ntrees, r->depth, r->seed);
      break;
    }
    case K_EXHAUSTIVE:
      r->table.clear();
      for (size_t i = 0; i < keys.size(); ++i) r->table[keys[i]] = labels[i];
      break;
    case K_MLP: {
      std::vector<std::array<float, AR_MAX_FEATURES>> X(keys.size());
      for (size_t i = 0; i < keys.size(); ++i) X[i] = ar::key_values(keys[i]);
      std::string msg;
      rc = ar::mlp_fit(X, labels, r->nf, r->hidden, (int)r->variants.size(), r->epochs, r->seed, &r->mlp, &msg);
      if (rc != AR_OK) return fail(r, rc, "mlp training: %s", msg.c_str());
      break;
    }
    default:
      break;
  }
  r->trained = true;
  if (ar::log_level() >= 1)
    ar::log_line(r->id.c_str(), "trained %s on %zu labelled feature vectors from %zu records",
                 r->kind == K_DTREE ? "dtree" : r->kind == K_RFC ? "rfc" : r->kind == K_MLP ? "mlp" : "exhaustive",
                 keys.size(), r->records.size());
  return AR_OK;
}

int ar_add_record(ar_region* r, const float* features, int nf, int variant, float ms) {
  if (!r) return AR_ERR_ARG;
  if (nf != r->nf) return fail(r, AR_ERR_STATE, "expected %d features, got %d", r->nf, nf);
  if (nf > 0 && !features) return fail(r, AR_ERR_ARG, "NULL features");
  if (!finite_all(features, nf) || !std::isfinite(ms) || ms < 0) return fail(r, AR_ERR_ARG, "non-finite value");
  if (variant < 0 || variant >= (int)r->variants.size()) return fail(r, AR_ERR_ARG, "variant out of range");
  freeze(r);
  float f[AR_MAX_FEATURES] = {};
  for (int i = 0; i < nf; ++i) f[i] = features[i];
  const FKey key = ar::make_key(f, nf);
  add_record(r, key, variant, ms);
  r->unique.insert({key, variant});
  return AR_OK;
}

int ar_record_counts(const ar_region* r, int64_t* num_records, int64_t* num_unique) {
  if (!r) return AR_ERR_ARG;
  if (num_records) *num_records = (int64_t)r->records.size();
  if (num_unique) *num_unique = (int64_t)r->unique.size();
  return AR_OK;
}

int ar_get_records(const ar_region* r, int64_t first, int64_t count, float* features, int* variants, float* ms) {
  if (!r || first < 0 || count < 0 || first + count > (int64_t)r->records.size()) return AR_ERR_ARG;
  for (int64_t i = 0; i < count; ++i) {
    const ar::Record& rec = r->records[(size_t)(first + i)];
    if (features) memcpy(features + i * AR_MAX_FEATURES, rec.f, sizeof rec.f);
    if (variants) variants[i] = rec.variant;
    if (ms) ms[i] = rec.ms;
  }
  return AR_OK;
}

int ar_tree_export(const ar_region* r, int max_nodes, int* feat, double* thr, int* left, int* right, int* label,
                   int* out_nodes) {
  if (!r) return AR_ERR_ARG;
  if (r->kind != K_DTREE || r->tree.empty()) return AR_ERR_NOMODEL;
  const int n = (int)r->tree.size();
  if (out_nodes) *out_nodes = n;
  for (int i = 0; i < n && i < max_nodes; ++i) {
    const ar::TreeNode& t = r->tree[i];
    if (feat) feat[i] = t.feat;
    if (thr) thr[i] = t.thr;
    if (left) left[i] = t.left;
    if (right) right[i] = t.right;
    if (label) label[i] = t.label;
  }
  return AR_OK;
}

int ar_forest_size(const ar_region* r, int* ntrees) {
  if (!r || !ntrees) return AR_ERR_ARG;
  if (r->kind != K_RFC || r->forest.empty()) return AR_ERR_NOMODEL;
  *ntrees = (int)r->forest.size();
  return AR_OK;
}

int ar_forest_tree_export(const ar_region* r, int tree, int max_nodes, int* feat, double* thr, int* left, int* right,
                          int* label, int* out_nodes) {
  if (!r) return AR_ERR_ARG;
  if (r->kind != K_RFC || r->forest.empty()) return AR_ERR_NOMODEL;
  if (tree < 0 || tree >= (int)r->forest.size()) return AR_ERR_ARG;
  const auto& t = r->forest[tree];
  const int n = (int)t.size();
  if (out_nodes) *out_nodes = n;
  for (int i = 0; i < n && i < max_nodes; ++i) {
    if (feat) feat[i] = t[i].feat;
    if (thr) thr[i] = t[i].thr;
    if (left) left[i] = t[i].left;
    if (right) right[i] = t[i].right;
    if (label) label[i] = t[i].label;
  }
  return AR_OK;
}

int ar_mlp_export(const ar_region* r, float* theta, float* mu, float* sd, int* F, int* H, int* V) {
  if (!r) return AR_ERR_ARG;
  if (r->kind != K_MLP || r->mlp.V == 0) return AR_ERR_NOMODEL;
  if (F) *F = r->mlp.F;
  if (H) *H = r->mlp.H;
  if (V) *V = r->mlp.V;
  if (theta) memcpy(theta, r->mlp.theta.data(), r->mlp.theta.size() * sizeof(float));
  if (mu) memcpy(mu, r->mlp.mu.data(), r->mlp.mu.size() * sizeof(float));
  if (sd) memcpy(sd, r->mlp.sd.data(), r->mlp.sd.size() * sizeof(float));
  return AR_OK;
}

int ar_last_error(const ar_region* r, char* buf, int len) {
  if (!r || !buf || len <= 0) return AR_ERR_ARG;
  snprintf(buf, (size_t)len, "%s", r->err.c_str());
  return AR_OK;
}

int ar_set_fake_timer(ar_region* r, ar_fake_time_fn fn, void* user) {
  if (!r) return AR_ERR_ARG;
  if (r->open) return fail(r, AR_ERR_STATE, "timer change inside an open execution");
  r->fake = fn;
  r->fake_user = user;
  return AR_OK;
}

int ar_set_l2_flush(ar_region* r, void* device_buf, size_t bytes) {
  if (!r) return AR_ERR_ARG;
  r->flush_buf = bytes ? device_buf : nullptr;
  r->flush_bytes = device_buf ? bytes : 0;
  return AR_OK;
}

// ------------------------------------------------------------ persistence
int ar_region_save(const ar_region* r, const char* path) {
  if (!r || !path) return AR_ERR_ARG;
  ar_region* rw = const_cast<ar_region*>(r);
  int rc = resolve(rw, true);
  if (rc != AR_OK) return rc;
  ar::Blob b;
  b.put_bytes("ARREGION", 8);
  b.put_u32(2);
  b.put_u32((uint32_t)r->nf);
  b.put_u32((uint32_t)r->variants.size());
  b.put_u32((uint32_t)r->kind);
  b.put_u64(r->records.size());
  for (const auto& rec : r->records) {
    b.put_bytes(rec.f, sizeof rec.f);
    b.put_u32((uint32_t)rec.variant);
    b.put_f32(rec.ms);
  }
  b.put_u32(r->trained ? 1u : 0u);
  b.put_u32((uint32_t)r->tree.size());
  for (const auto& t : r->tree) {
    b.put_u32((uint32_t)t.feat);
    b.put_f64(t.thr);
    b.put_u32((uint32_t)t.left);
    b.put_u32((uint32_t)t.right);
    b.put_u32((uint32_t)t.label);
    b.put_f32(t.conf);
  }
  b.put_u32((uint32_t)r->forest.size());
  for (const auto& t : r->forest) {
    b.put_u32((uint32_t)t.size());
    for (const auto& nd : t) {
      b.put_u32((uint32_t)nd.feat);
      b.put_f64(nd.thr);
      b.put_u32((uint32_t)nd.left);
      b.put_u32((uint32_t)nd.right);
      b.put_u32((uint32_t)nd.label);
      b.put_f32(nd.conf);
    }
  }
  b.put_u32((uint32_t)r->mlp.F);
  b.put_u32((uint32_t)r->mlp.H);
  b.put_u32((uint32_t)r->mlp.V);
  b.put_u64(r->mlp.theta.size());
  b.put_bytes(r->mlp.theta.data(), r->mlp.theta.size() * 4);
  b.put_bytes(r->mlp.mu.data(), r->mlp.mu.size() * 4);
  b.put_bytes(r->mlp.sd.data(), r->mlp.sd.size() * 4);
  b.put_u32((uint32_t)r->table.size());
  for (const auto& kv : r->table) {
    b.put_bytes(kv.first.data(), sizeof(uint32_t) * AR_MAX_FEATURES);
    b.put_u32((uint32_t)kv.second);
  }
  b.put_u64(ar::fnv1a(b.data.data(), b.data.size()));
  FILE* f = fopen(path, "wb");
  if (!f) return fail(rw, AR_ERR_IO, "cannot open %s for writing", path);
  const size_t w = fwrite(b.data.data(), 1, b.data.size(), f);
  const int cl = fclose(f);
  if (w != b.data.size() || cl != 0) return fail(rw, AR_ERR_IO, "short write to %s", path);
  return AR_OK;
}

int ar_region_load(ar_region* r, const char* path) {
  if (!r || !path) return AR_ERR_ARG;
  if (r->open) return fail(r, AR_ERR_STATE, "load inside an open execution");
  FILE* f = fopen(path, "rb");
  if (!f) return fail(r, AR_ERR_IO, "cannot open %s", path);
  std::vector<uint8_t> data;
  uint8_t tmp[1 << 16];
  size_t got;
  while ((got = fread(tmp, 1, sizeof tmp, f)) > 0) data.insert(data.end(), tmp, tmp + got);
  fclose(f);
  if (data.size() < 8 + 16 + 8) return fail(r, AR_ERR_IO, "%s: truncated", path);
  uint64_t stored;
  memcpy(&stored, data.data() + data.size() - 8, 8);
  if (ar::fnv1a(data.data(), data.size() - 8) != stored) return fail(r, AR_ERR_IO, "%s: checksum mismatch", path);
  ar::Reader in{data.data(), data.size() - 8, 0, true};
  char magic[8];
  in.get_bytes(magic, 8);
  if (!in.ok || memcmp(magic, "ARREGION", 8) != 0) return fail(r, AR_ERR_IO, "%s: not a region file", path);
  const uint32_t version = in.get_u32();
  const uint32_t nf = in.get_u32(), V = in.get_u32(), kind = in.get_u32();
  if (!in.ok || version != 2) return fail(r, AR_ERR_IO, "%s: unsupported version", path);
  if ((int)nf != r->nf || (int)V != (int)r->variants.size())
    return fail(r, AR_ERR_STATE, "%s: region has %d features and %d variants, file %u and %u", path, r->nf,
                (int)r->variants.size(), nf, V);
  if ((int)kind != (int)r->kind) return fail(r, AR_ERR_STATE, "%s: model kind differs", path);
  const uint64_t nrec = in.get_u64();
  if (!in.ok || nrec > (in.size - in.pos) / (sizeof(float) * AR_MAX_FEATURES + 8))
    return fail(r, AR_ERR_IO, "%s: bad record count", path);
  std::vector<ar::Record> recs((size_t)nrec);
  for (auto& rec : recs) {
    in.get_bytes(rec.f, sizeof rec.f);
    rec.variant = (int)in.get_u32();
    rec.ms = in.get_f32();
    if (rec.variant < 0 || rec.variant >= (int)V) in.ok = false;
  }
  const uint32_t trained = in.get_u32();
  const uint32_t ntree = in.get_u32();
  if (!in.ok || ntree > 1u << 20) return fail(r, AR_ERR_IO, "%s: corrupt", path);
  std::vector<ar::TreeNode> tree(ntree);
  for (auto& t : tree) {
    t.feat = (int)in.get_u32();
    t.thr = in.get_f64();
    t.left = (int)in.get_u32();
    t.right = (int)in.get_u32();
    t.label = (int)in.get_u32();
    t.conf = in.get_f32();
    if (t.feat >= (int)nf || t.label < 0 || t.label >= (int)V) in.ok = false;
    if (t.feat >= 0 && (t.left <= 0 || t.right <= 0 || t.left >= (int)ntree || t.right >= (int)ntree)) in.ok = false;
  }
  auto read_nodes = [&](std::vector<ar::TreeNode>& nodes, uint32_t count) {
    nodes.resize(count);
    for (auto& t : nodes) {
      t.feat = (int)in.get_u32();
      t.thr = in.get_f64();
      t.left = (int)in.get_u32();
      t.right = (int)in.get_u32();
      t.label = (int)in.get_u32();
      t.conf = in.get_f32();
      if (t.feat >= (int)nf || t.label < 0 || t.label >= (int)V) in.ok = false;
      if (t.feat >= 0 && (t.left <= 0 || t.right <= 0 || t.left >= (int)count || t.right >= (int)count))
        in.ok = false;
    }
  };
  const uint32_t nforest = in.get_u32();
  if (!in.ok || nforest > 256) return fail(r, AR_ERR_IO, "%s: corrupt forest", path);
  std::vector<std::vector<ar::TreeNode>> forest(nforest);
  for (auto& t : forest) {
    const uint32_t cnt = in.get_u32();
    if (!in.ok || cnt > 1u << 20) return fail(r, AR_ERR_IO, "%s: corrupt forest", path);
    read_nodes(t, cnt);
  }
  ar::MlpModel m;
  m.F = (int)in.get_u32();
  m.H = (int)in.get_u32();
  m.V = (int)in.get_u32();
  const uint64_t np = in.get_u64();
  if (!in.ok || np > 1u << 24 || (m.V && np != (uint64_t)ar_mlp_num_params(m.F, m.H, m.V)))
    return fail(r, AR_ERR_IO, "%s: corrupt model", path);
  m.theta.resize((size_t)np);
  in.get_bytes(m.theta.data(), np * 4);
  m.mu.resize(m.V ? (size_t)m.F : 0);
  m.sd.resize(m.V ? (size_t)m.F : 0);
  in.get_bytes(m.mu.data(), m.mu.size() * 4);
  in.get_bytes(m.sd.data(), m.sd.size() * 4);
  const uint32_t ntab = in.get_u32();
  std::map<FKey, int> table;
  for (uint32_t i = 0; i < ntab && in.ok; ++i) {
    FKey k;
    in.get_bytes(k.data(), sizeof(uint32_t) * AR_MAX_FEATURES);
    const int v = (int)in.get_u32();
    if (v < 0 || v >= (int)V) in.ok = false;
    table[k] = v;
  }
  if (!in.ok || in.pos != in.size) return fail(r, AR_ERR_IO, "%s: corrupt", path);
  // commit
  resolve(r, true);
  freeze(r);
  r->records.swap(recs);
  r->unique.clear();
  r->agg.clear();
  for (const auto& rec : r->records) {
    const FKey k = ar::record_key(rec);
    r->unique.insert({k, rec.variant});
    auto& a = r->agg[k];
    if (a.size() < r->variants.size()) a.resize(r->variants.size(), {0.0, 0});
    a[rec.variant].first += rec.ms;
    a[rec.variant].second += 1;
  }
  r->tree.swap(tree);
  r->forest.swap(forest);
  r->mlp = std::move(m);
  r->table.swap(table);
  r->trained = trained != 0;
  r->auto_trained = r->trained;
  return AR_OK;
}

}  // extern "C"

namespace ar {

int region_key_means(const ar_region* r, const float* f, int nf, std::vector<double>* mean) {
  const int V = (int)r->variants.size();
  mean->assign(V, INFINITY);
  float g[AR_MAX_FEATURES] = {};
  for (int i = 0; i < nf && i < AR_MAX_FEATURES; ++i) g[i] = f[i];
  auto it = r->agg.find(make_key(g, nf));
  if (it == r->agg.end()) return 0;
  int have = 0;
  for (int v = 0; v < V && v < (int)it->second.size(); ++v)
    if (it->second[v].second > 0) {
      (*mean)[v] = it->second[v].first / (double)it->second[v].second;
      ++have;
    }
  return have;
}

double region_tie(const ar_region* r) { return r->tie; }

const char* region_id(const ar_region* r) { return r->id.c_str(); }

int log_level() {
  static const int level = [] {
    const char* e = getenv("AR_LOG");
    return e ? atoi(e) : 0;
  }();
  return level;
}

void log_line(const char* region_id, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  fprintf(stderr, "[ar] %s: %s\n", region_id ? region_id : "-", buf);
}

void region_flush_buffer(const ar_region* r, void** buf, size_t* bytes) {
  *buf = r->flush_buf;
  *bytes = r->flush_bytes;
}

}  // namespace ar
