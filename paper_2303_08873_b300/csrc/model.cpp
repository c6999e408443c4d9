// Host-side models of the runtime: labels from records (Section 2: the
// fastest policy per feature values), the CART decision tree (Section 3.1
// model_type dtree, default depth 2) and host inference of the MLP selector.
#include "model.h"

#include <algorithm>
#include <cmath>
#include <map>

namespace ar {

FKey make_key(const float* f, int nf) {
  FKey k{};
  for (int i = 0; i < nf && i < AR_MAX_FEATURES; ++i) {
    float v = f[i] == 0.0f ? 0.0f : f[i];  // fold -0 into +0
    memcpy(&k[i], &v, 4);
  }
  return k;
}

FKey record_key(const Record& r) {
  FKey k{};
  for (int i = 0; i < AR_MAX_FEATURES; ++i) memcpy(&k[i], &r.f[i], 4);
  return k;
}

std::array<float, AR_MAX_FEATURES> key_values(const FKey& k) {
  std::array<float, AR_MAX_FEATURES> v{};
  for (int i = 0; i < AR_MAX_FEATURES; ++i) memcpy(&v[i], &k[i], 4);
  return v;
}

int best_of_means(const std::vector<double>& mean, double tie) {
  double m = INFINITY;
  for (double t : mean)
    if (std::isfinite(t) && t < m) m = t;
  if (!std::isfinite(m)) return -1;
  for (size_t v = 0; v < mean.size(); ++v)
    if (std::isfinite(mean[v]) && mean[v] <= m * (1.0 + tie)) return (int)v;
  return -1;
}

void label_records(const std::vector<Record>& recs, int V, std::vector<FKey>* keys, std::vector<int>* labels,
                   double tie) {
  std::map<FKey, std::vector<std::pair<double, int>>> acc;
  for (const auto& r : recs) {
    auto& slot = acc[record_key(r)];
    if (slot.empty()) slot.assign((size_t)V, {0.0, 0});
    if (r.variant >= 0 && r.variant < V) {
      slot[r.variant].first += r.ms;
      slot[r.variant].second += 1;
    }
  }
  keys->clear();
  labels->clear();
  for (const auto& kv : acc) {
    std::vector<double> mean((size_t)V, INFINITY);
    for (int v = 0; v < V; ++v)
      if (kv.second[v].second > 0) mean[v] = kv.second[v].first / kv.second[v].second;
    const int b = best_of_means(mean, tie);
    if (b < 0) continue;
    keys->push_back(kv.first);
    labels->push_back(b);
  }
}

// ------------------------------------------------------------------ CART
namespace {

struct Fit {
  const std::vector<std::array<float, AR_MAX_FEATURES>>& X;
  const std::vector<int>& y;
  int nf, max_depth, nlab;
  std::vector<TreeNode> nodes;
  SplitMix64* rng = nullptr;  // random forest: per-node feature subsets
  int mtry = 0;

  void majority(const std::vector<int>& idx, int* label, float* conf) const {
    std::vector<int> cnt((size_t)nlab, 0);
    for (int i : idx) cnt[y[i]]++;
    int best = 0;
    for (int c = 1; c < nlab; ++c)
      if (cnt[c] > cnt[best]) best = c;
    *label = best;
    *conf = idx.empty() ? 0.f : (float)cnt[best] / (float)idx.size();
  }

  // score = A/nl + B/nr with A = sum cL^2, B = sum cR^2 (maximised); compared
  // exactly as fractions (A*nr + B*nl) / (nl*nr).
  struct Score {
    __int128 num, den;
  };
  static bool greater(const Score& a, const Score& b) { return a.num * b.den > b.num * a.den; }

  int grow(const std::vector<int>& idx, int depth) {
    const int me = (int)nodes.size();
    nodes.push_back(TreeNode{-1, 0.0, -1, -1, 0, 0.f});
    int lab;
    float conf;
    majority(idx, &lab, &conf);
    nodes[me].label = lab;
    nodes[me].conf = conf;
    bool pure = true;
    for (int i : idx)
      if (y[i] != y[idx[0]]) {
        pure = false;
        break;
      }
    if (depth >= max_depth || pure || idx.size() < 2) return me;

    bool have = false;
    Score best{0, 1};
    int bf = -1;
    double bthr = 0.0;
    std::vector<std::pair<double, int>> vals;
    // candidate features: all, or (forest) mtry distinct ones drawn by a
    // partial Fisher-Yates shuffle, visited in ascending order
    int feats[AR_MAX_FEATURES];
    int nfe = nf;
    for (int f = 0; f < nf; ++f) feats[f] = f;
    if (rng) {
      for (int a = 0; a < mtry; ++a) {
        const int b = a + (int)(rng->next() % (uint64_t)(nf - a));
        std::swap(feats[a], feats[b]);
      }
      nfe = mtry;
      std::sort(feats, feats + nfe);
    }
    for (int fi = 0; fi < nfe; ++fi) {
      const int f = feats[fi];
      vals.clear();
      for (int i : idx) vals.push_back({(double)X[i][f], y[i]});
      std::sort(vals.begin(), vals.end());
      std::vector<long long> lc((size_t)nlab, 0), rc((size_t)nlab, 0);
      for (auto& p : vals) rc[p.second]++;
      long long nl = 0, nr = (long long)vals.size();
      long long A = 0, B = 0;
      for (int c = 0; c < nlab; ++c) B += rc[c] * rc[c];
      for (size_t a = 0; a + 1 < vals.size(); ++a) {
        const int c = vals[a].second;
        A += 2 * lc[c] + 1;  // (l+1)^2 - l^2
        B -= 2 * rc[c] - 1;  // (r-1)^2 - r^2 = -(2r - 1)
        lc[c]++;
        rc[c]--;
        nl++;
        nr--;
        if (vals[a].first == vals[a + 1].first) continue;
        const double thr = (vals[a].first + vals[a + 1].first) / 2.0;
        Score s{(__int128)A * nr + (__int128)B * nl, (__int128)nl * nr};
        if (!have || greater(s, best)) {
          have = true;
          best = s;
          bf = f;
          bthr = thr;
        }
      }
    }
    if (!have) return me;
    std::vector<int> li, ri;
    for (int i : idx) ((double)X[i][bf] <= bthr ? li : ri).push_back(i);
    const int l = grow(li, depth + 1);
    const int r = grow(ri, depth + 1);
    nodes[me].feat = bf;
    nodes[me].thr = bthr;
    nodes[me].left = l;
    nodes[me].right = r;
    return me;
  }
};

}  // namespace

std::vector<TreeNode> tree_fit(const std::vector<std::array<float, AR_MAX_FEATURES>>& X, const std::vector<int>& y,
                               int nf, int max_depth) {
  int nlab = 1;
  for (int v : y) nlab = std::max(nlab, v + 1);
  Fit fit{X, y, nf, max_depth, nlab, {}};
  std::vector<int> idx(y.size());
  for (size_t i = 0; i < y.size(); ++i) idx[i] = (int)i;
  if (!idx.empty()) fit.grow(idx, 0);
  return fit.nodes;
}

std::vector<std::vector<TreeNode>> forest_fit(const std::vector<std::array<float, AR_MAX_FEATURES>>& X,
                                              const std::vector<int>& y, int nf, int ntrees, int max_depth,
                                              uint64_t seed) {
  int nlab = 1;
  for (int v : y) nlab = std::max(nlab, v + 1);
  SplitMix64 rng{seed};
  const int n = (int)y.size();
  int mtry = (int)std::floor(std::sqrt((double)nf));
  if (mtry < 1) mtry = 1;
  std::vector<std::vector<TreeNode>> forest;
  for (int t = 0; t < ntrees; ++t) {
    std::vector<int> idx((size_t)n);
    for (int i = 0; i < n; ++i) idx[i] = (int)(rng.next() % (uint64_t)n);  // bootstrap sample
    Fit fit{X, y, nf, max_depth, nlab, {}};
    fit.rng = &rng;
    fit.mtry = mtry;
    if (n > 0) fit.grow(idx, 0);
    forest.push_back(std::move(fit.nodes));
  }
  return forest;
}

int forest_predict(const std::vector<std::vector<TreeNode>>& forest, const float* f, float* conf) {
  if (forest.empty()) return -1;
  std::vector<int> votes;
  for (const auto& t : forest) {
    const int v = tree_predict(t, f, nullptr);
    if (v < 0) continue;
    if ((int)votes.size() <= v) votes.resize((size_t)v + 1, 0);
    votes[v]++;
  }
  int best = 0;
  for (int v = 1; v < (int)votes.size(); ++v)
    if (votes[v] > votes[best]) best = v;
  if (conf) *conf = (float)votes[best] / (float)forest.size();
  return best;
}

int tree_predict(const std::vector<TreeNode>& t, const float* f, float* conf) {
  if (t.empty()) return -1;
  int n = 0;
  while (t[n].feat >= 0) n = ((double)f[t[n].feat] <= t[n].thr) ? t[n].left : t[n].right;
  if (conf) *conf = t[n].conf;
  return t[n].label;
}

// ------------------------------------------------------------------ MLP host
int mlp_predict_host(const MlpModel& m, const float* f, float* conf) {
  const int F = m.F, H = m.H, V = m.V;
  const float* W1 = m.theta.data();
  const float* b1 = W1 + H * F;
  const float* W2 = b1 + H;
  const float* b2 = W2 + H * H;
  const float* W3 = b2 + H;
  const float* b3 = W3 + V * H;
  float x0[AR_MAX_FEATURES], h1[64], h2[64], lg[AR_MAX_VARIANTS];
  for (int i = 0; i < F; ++i) x0[i] = (copysignf(log1pf(fabsf(f[i])), f[i]) - m.mu[i]) / m.sd[i];
  for (int o = 0; o < H; ++o) {
    float s = b1[o];
    for (int i = 0; i < F; ++i) s = fmaf(W1[o * F + i], x0[i], s);
    h1[o] = s > 0.f ? s : 0.f;
  }
  for (int o = 0; o < H; ++o) {
    float s = b2[o];
    for (int i = 0; i < H; ++i) s = fmaf(W2[o * H + i], h1[i], s);
    h2[o] = s > 0.f ? s : 0.f;
  }
  int best = 0;
  for (int o = 0; o < V; ++o) {
    float s = b3[o];
    for (int i = 0; i < H; ++i) s = fmaf(W3[o * H + i], h2[i], s);
    lg[o] = s;
    if (s > lg[best]) best = o;
  }
  float z = 0.f;
  for (int o = 0; o < V; ++o) z += expf(lg[o] - lg[best]);
  if (conf) *conf = 1.0f / z;
  return best;
}

uint64_t fnv1a(const uint8_t* p, size_t n) {
  uint64_t h = 0xcbf29ce484222325ull;
  for (size_t i = 0; i < n; ++i) {
    h ^= p[i];
    h *= 0x100000001b3ull;
  }
  return h;
}

}  // namespace ar
