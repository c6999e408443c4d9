// Internal model types of the runtime: records, labels, the CART decision
// tree, the MLP selector's host side, and a small binary serializer.
#pragma once

#include <array>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "ar.h"
#include "ar_loops.h"

namespace ar {

// Exact feature vector (bit patterns; -0 folded into +0; unused slots 0).
using FKey = std::array<uint32_t, AR_MAX_FEATURES>;

struct Record {
  float f[AR_MAX_FEATURES];
  int variant;
  float ms;
};

FKey make_key(const float* f, int nf);
FKey record_key(const Record& r);
std::array<float, AR_MAX_FEATURES> key_values(const FKey& k);

// Index of the fastest mean (non-finite means skipped): the lowest index whose
// mean is within a fraction `tie` (default 0.5 %) of the minimum; -1 if none
// is finite.
constexpr double kTieRel = 0.005;
int best_of_means(const std::vector<double>& mean, double tie = kTieRel);

// Training set from records: one sample per distinct feature vector (sorted
// by bit pattern), labelled with best_of_means of its per-variant means.
void label_records(const std::vector<Record>& recs, int num_variants, std::vector<FKey>* keys,
                   std::vector<int>* labels, double tie = kTieRel);

// CART decision tree (Gini; thresholds at midpoints of consecutive distinct
// values; x <= thr goes left; ties to the lowest feature, then the lowest
// threshold; leaves hold the majority label, ties to the lowest label).
struct TreeNode {
  int feat;    // -1 for a leaf
  double thr;
  int left, right;
  int label;   // majority label of the node's samples
  float conf;  // fraction of the node's samples carrying `label`
};
std::vector<TreeNode> tree_fit(const std::vector<std::array<float, AR_MAX_FEATURES>>& X,
                               const std::vector<int>& y, int nf, int max_depth);
int tree_predict(const std::vector<TreeNode>& t, const float* f, float* conf);

// Random forest (Section 3.1 model_type rfc, ntrees, depth): tree t is the
// CART above grown on a bootstrap sample of the training set (n draws with
// replacement) and, at every node it tries to split, on mtry =
// max(1, floor(sqrt(nf))) features drawn without replacement.  All draws come
// from one SplitMix64 stream seeded with `seed`, consumed tree by tree:
// n bootstrap indices (next() mod n), then per split attempt in depth-first
// preorder a partial Fisher-Yates shuffle (a + next() mod (nf - a)).
// Prediction: majority vote, ties to the lowest label; confidence = vote share.
std::vector<std::vector<TreeNode>> forest_fit(const std::vector<std::array<float, AR_MAX_FEATURES>>& X,
                                              const std::vector<int>& y, int nf, int ntrees, int max_depth,
                                              uint64_t seed);
int forest_predict(const std::vector<std::vector<TreeNode>>& forest, const float* f, float* conf);

// MLP selector (layout of ar_mlp_num_params): features -> signed log1p ->
// z-score -> Linear(F,H) ReLU Linear(H,H) ReLU Linear(H,V) -> softmax.
struct MlpModel {
  int F = 0, H = 0, V = 0;
  std::vector<float> theta, mu, sd;
};
int mlp_predict_host(const MlpModel& m, const float* f, float* conf);
// Train on the device with the fused kernels (ar_mlp_train); fills `out`.
int mlp_fit(const std::vector<std::array<float, AR_MAX_FEATURES>>& X, const std::vector<int>& y, int F, int H,
            int V, int epochs, uint64_t seed, MlpModel* out, std::string* msg);

// SplitMix64 (Steele, Lea & Flood 2014) for the runtime's own draws.
struct SplitMix64 {
  uint64_t s;
  uint64_t next() {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  double uniform() { return (next() >> 11) * (1.0 / 9007199254740992.0); }
};

uint64_t fnv1a(const uint8_t* p, size_t n);

// Log level from the environment variable AR_LOG (read once): 0 quiet
// (default), 1 training, automatic-training triggers, variants marked
// unusable and fallback summaries, 2 also every exhaustive profile and every
// model selection.  Lines go to stderr, prefixed "[ar] <region id>".
int log_level();
void log_line(const char* region_id, const char* fmt, ...) __attribute__((format(printf, 2, 3)));

// Region internals used by other parts of the library (runtime.cpp).
// Per-variant mean ms over the region's resolved records of one exact feature
// vector (+inf where a variant has none); returns the number of variants that
// have at least one record (0 if the vector was never recorded).
int region_key_means(const ar_region* r, const float* f, int nf, std::vector<double>* mean);
// The region's L2 flush buffer (ar_set_l2_flush), or nullptr / 0.
void region_flush_buffer(const ar_region* r, void** buf, size_t* bytes);
// The region's tie fraction for labels and exhaustive argmins (spec "tie=").
double region_tie(const ar_region* r);
// The region's id.
const char* region_id(const ar_region* r);

struct Blob {
  std::vector<uint8_t> data;
  void put_bytes(const void* p, size_t n) {
    const uint8_t* b = static_cast<const uint8_t*>(p);
    data.insert(data.end(), b, b + n);
  }
  void put_u32(uint32_t v) { put_bytes(&v, 4); }
  void put_u64(uint64_t v) { put_bytes(&v, 8); }
  void put_f32(float v) { put_bytes(&v, 4); }
  void put_f64(double v) { put_bytes(&v, 8); }
};

struct Reader {
  const uint8_t* p;
  size_t size, pos;
  bool ok;
  void get_bytes(void* dst, size_t n) {
    if (!ok || n > size - pos) {
      ok = false;
      if (n) memset(dst, 0, n);
      return;
    }
    memcpy(dst, p + pos, n);
    pos += n;
  }
  uint32_t get_u32() {
    uint32_t v = 0;
    get_bytes(&v, 4);
    return v;
  }
  uint64_t get_u64() {
    uint64_t v = 0;
    get_bytes(&v, 8);
    return v;
  }
  float get_f32() {
    float v = 0;
    get_bytes(&v, 4);
    return v;
  }
  double get_f64() {
    double v = 0;
    get_bytes(&v, 8);
    return v;
  }
};

}  // namespace ar
