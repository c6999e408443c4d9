// Fused float32 kernels of the MLP selector: batched inference, the
// minibatch gradient of the mean cross-entropy, Adam, and a whole training
// run in one single-block launch (forward, backward and update per
// minibatch, activations kept in shared memory).
//
// The paper's model kinds are decision trees and random forests and it names
// neural networks as a further classifier (Section 3.1 model_type); this is
// that classifier, trained on the labels the region derives from its own
// profiling records (Section 2).
//
// Shared-memory layout of the training block (floats): theta [P], grad [P],
// x0 [8][BS+1], a1 [H][BS+1], a2 [H][BS+1], d3 [V][BS+1], loss [BS]; unit-major
// with a padded row so that per-sample writes (consecutive samples) and
// per-unit reductions (consecutive units) are both bank-conflict free.  Every
// reduction over samples runs s = 0 .. B-1 in order: results are
// deterministic.
#define AR_TU 6
#include <cmath>
#include <cstdio>
#include <string>
#include <vector>

#include "common.cuh"
#include "model.h"

namespace ar {
namespace {

constexpr int BS = 256;       // samples per minibatch = threads per block
constexpr int LD = BS + 1;    // padded row length
constexpr int MAXF = 8;
constexpr int MAXV = 32;
constexpr float B1 = 0.9f, B2 = 0.999f, EPS = 1e-8f;
// 1 - beta as separate constants: 1 - 0.999f rounds to 0.00099998713 in float32
constexpr float OMB1 = 0.1f, OMB2 = 0.001f;

__host__ __device__ inline int nparams(int F, int H, int V) { return H * F + H + H * H + H + V * H + V; }

__device__ __forceinline__ float slog1p(float f) { return copysignf(log1pf(fabsf(f)), f); }

// ---------------------------------------------------------------- inference
template <int H>
__global__ void __launch_bounds__(128) mlp_forward_kernel(const float* __restrict__ theta, const float* __restrict__ mu,
                                                          const float* __restrict__ sd, int F, int V, int64_t B,
                                                          const float* __restrict__ feats, float* __restrict__ probs,
                                                          int* __restrict__ variant, float* __restrict__ conf) {
  extern __shared__ float th[];
  const int P = nparams(F, H, V);
  for (int i = threadIdx.x; i < P; i += blockDim.x) th[i] = theta[i];
  __syncthreads();
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= B) return;
  const float* W1 = th;
  const float* b1 = W1 + H * F;
  const float* W2 = b1 + H;
  const float* b2 = W2 + H * H;
  const float* W3 = b2 + H;
  const float* b3 = W3 + V * H;
  float x0[MAXF];
#pragma unroll
  for (int f = 0; f < MAXF; ++f) x0[f] = f < F ? (slog1p(feats[s * F + f]) - mu[f]) / sd[f] : 0.f;
  float h1[H];
#pragma unroll
  for (int o = 0; o < H; ++o) {
    float a = b1[o];
#pragma unroll
    for (int f = 0; f < MAXF; ++f)
      if (f < F) a = fmaf(W1[o * F + f], x0[f], a);
    h1[o] = fmaxf(a, 0.f);
  }
  float lg[MAXV];
#pragma unroll
  for (int v = 0; v < MAXV; ++v) lg[v] = v < V ? b3[v] : 0.f;
  for (int o = 0; o < H; ++o) {
    float a = b2[o];
#pragma unroll
    for (int i = 0; i < H; ++i) a = fmaf(W2[o * H + i], h1[i], a);
    a = fmaxf(a, 0.f);
#pragma unroll
    for (int v = 0; v < MAXV; ++v)
      if (v < V) lg[v] = fmaf(W3[v * H + o], a, lg[v]);
  }
  int best = 0;
  float m = lg[0];
#pragma unroll
  for (int v = 1; v < MAXV; ++v)
    if (v < V && lg[v] > m) {
      m = lg[v];
      best = v;
    }
  float z = 0.f;
#pragma unroll
  for (int v = 0; v < MAXV; ++v)
    if (v < V) z += expf(lg[v] - m);
  if (probs) {
    const float iz = 1.f / z;
    for (int v = 0; v < V; ++v) probs[s * V + v] = expf(lg[v] - m) * iz;
  }
  if (variant) variant[s] = best;
  if (conf) conf[s] = 1.f / z;
}

// ---------------------------------------------------------------- training
struct Smem {
  float *th, *g, *x0, *a1, *a2, *d3, *loss;
};

__host__ __device__ inline size_t train_smem_floats(int F, int H, int V) {
  (void)F;
  return 2 * (size_t)nparams(MAXF, H, V) + (size_t)MAXF * LD + 2 * (size_t)H * LD + (size_t)V * LD + BS;
}

__device__ inline Smem carve(float* base, int H, int V) {
  Smem m;
  const int P = nparams(MAXF, H, V);
  m.th = base;
  m.g = m.th + P;
  m.x0 = m.g + P;
  m.a1 = m.x0 + MAXF * LD;
  m.a2 = m.a1 + H * LD;
  m.d3 = m.a2 + H * LD;
  m.loss = m.d3 + V * LD;
  return m;
}

// Gradient of the mean cross-entropy over rows idx[0..Bt) into m.g (and the
// loss into *loss_out if non-null).  Reads weights from m.th.  All BS threads
// of the block must call it.
template <int H>
__device__ void minibatch_grad(const Smem& m, int F, int V, int Bt, const float* __restrict__ feats,
                               const int* __restrict__ labels, const int* __restrict__ idx, const float* __restrict__ mu,
                               const float* __restrict__ sd, float* loss_out) {
  const int t = threadIdx.x;
  const float* W1 = m.th;
  const float* b1 = W1 + H * F;
  const float* W2 = b1 + H;
  const float* b2 = W2 + H * H;
  const float* W3 = b2 + H;
  const float* b3 = W3 + V * H;
  float* gW1 = m.g;
  float* gb1 = gW1 + H * F;
  float* gW2 = gb1 + H;
  float* gb2 = gW2 + H * H;
  float* gW3 = gb2 + H;
  float* gb3 = gW3 + V * H;
  const float inv_b = 1.f / (float)Bt;

  // ---- forward (thread t = sample t)
  if (t < Bt) {
    const int r = idx ? idx[t] : t;
    float x0[MAXF];
#pragma unroll
    for (int f = 0; f < MAXF; ++f) {
      x0[f] = f < F ? (slog1p(feats[(int64_t)r * F + f]) - mu[f]) / sd[f] : 0.f;
      if (f < F) m.x0[f * LD + t] = x0[f];
    }
    float h1[H];
#pragma unroll
    for (int o = 0; o < H; ++o) {
      float a = b1[o];
#pragma unroll
      for (int f = 0; f < MAXF; ++f)
        if (f < F) a = fmaf(W1[o * F + f], x0[f], a);
      h1[o] = fmaxf(a, 0.f);
      m.a1[o * LD + t] = h1[o];
    }
    float lg[MAXV];
#pragma unroll
    for (int v = 0; v < MAXV; ++v) lg[v] = v < V ? b3[v] : 0.f;
    for (int o = 0; o < H; ++o) {
      float a = b2[o];
#pragma unroll
      for (int i = 0; i < H; ++i) a = fmaf(W2[o * H + i], h1[i], a);
      a = fmaxf(a, 0.f);
      m.a2[o * LD + t] = a;
#pragma unroll
      for (int v = 0; v < MAXV; ++v)
        if (v < V) lg[v] = fmaf(W3[v * H + o], a, lg[v]);
    }
    float mx = lg[0];
#pragma unroll
    for (int v = 1; v < MAXV; ++v)
      if (v < V) mx = fmaxf(mx, lg[v]);
    float z = 0.f;
#pragma unroll
    for (int v = 0; v < MAXV; ++v)
      if (v < V) z += expf(lg[v] - mx);
    const int lab = min(max(labels[r], 0), V - 1);  // out-of-range labels are clamped
    float lgl = 0.f;
#pragma unroll
    for (int v = 0; v < MAXV; ++v)
      if (v == lab) lgl = lg[v];
    const float logz = logf(z);
    m.loss[t] = logz - (lgl - mx);  // -log softmax[lab]
    const float iz = 1.f / z;
#pragma unroll
    for (int v = 0; v < MAXV; ++v)
      if (v < V) m.d3[v * LD + t] = (expf(lg[v] - mx) * iz - (v == lab ? 1.f : 0.f)) * inv_b;
  }
  __syncthreads();

  // ---- layer 3 gradients: gW3[v][h] = sum_s d3[v][s] a2[h][s]; gb3
  for (int o = t; o < V * H + V; o += BS) {
    float acc = 0.f;
    if (o < V * H) {
      const int v = o / H, h = o % H;
      for (int s = 0; s < Bt; ++s) acc = fmaf(m.d3[v * LD + s], m.a2[h * LD + s], acc);
      gW3[o] = acc;
    } else {
      const int v = o - V * H;
      for (int s = 0; s < Bt; ++s) acc += m.d3[v * LD + s];
      gb3[v] = acc;
    }
  }
  if (loss_out && t == 0) {
    float L = 0.f;
    for (int s = 0; s < Bt; ++s) L += m.loss[s];
    *loss_out = L * inv_b;
  }
  __syncthreads();

  // ---- d2 = (W3^T d3) * [a2 > 0], in place of a2
  if (t < Bt) {
    float d3v[MAXV];
#pragma unroll
    for (int v = 0; v < MAXV; ++v) d3v[v] = v < V ? m.d3[v * LD + t] : 0.f;
    for (int h = 0; h < H; ++h) {
      float acc = 0.f;
#pragma unroll
      for (int v = 0; v < MAXV; ++v)
        if (v < V) acc = fmaf(W3[v * H + h], d3v[v], acc);
      m.a2[h * LD + t] = m.a2[h * LD + t] > 0.f ? acc : 0.f;
    }
  }
  __syncthreads();

  // ---- layer 2 gradients: gW2[o][i] = sum_s d2[o][s] a1[i][s] (4x4 tile per thread); gb2
  {
    constexpr int TI = H / 4;  // tiles per dimension
    for (int tile = t; tile < TI * TI; tile += BS) {
      const int o0 = (tile / TI) * 4, i0 = (tile % TI) * 4;
      float acc[4][4] = {};
      for (int s = 0; s < Bt; ++s) {
        float d[4], a[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          d[q] = m.a2[(o0 + q) * LD + s];
          a[q] = m.a1[(i0 + q) * LD + s];
        }
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[p][q] = fmaf(d[p], a[q], acc[p][q]);
      }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) gW2[(o0 + p) * H + i0 + q] = acc[p][q];
    }
    if (t < H) {
      float acc = 0.f;
      for (int s = 0; s < Bt; ++s) acc += m.a2[t * LD + s];
      gb2[t] = acc;
    }
  }
  __syncthreads();

  // ---- d1 = (W2^T d2) * [a1 > 0], in place of a1
  if (t < Bt) {
    float d2v[H];
#pragma unroll
    for (int o = 0; o < H; ++o) d2v[o] = m.a2[o * LD + t];
    for (int i = 0; i < H; ++i) {
      float acc = 0.f;
#pragma unroll
      for (int o = 0; o < H; ++o) acc = fmaf(W2[o * H + i], d2v[o], acc);
      m.a1[i * LD + t] = m.a1[i * LD + t] > 0.f ? acc : 0.f;
    }
  }
  __syncthreads();

  // ---- layer 1 gradients: gW1[h][f] = sum_s d1[h][s] x0[f][s]; gb1
  for (int o = t; o < H * F + H; o += BS) {
    float acc = 0.f;
    if (o < H * F) {
      const int h = o / F, f = o % F;
      for (int s = 0; s < Bt; ++s) acc = fmaf(m.a1[h * LD + s], m.x0[f * LD + s], acc);
      gW1[o] = acc;
    } else {
      const int h = o - H * F;
      for (int s = 0; s < Bt; ++s) acc += m.a1[h * LD + s];
      gb1[h] = acc;
    }
  }
  __syncthreads();
}

__device__ __forceinline__ void adam_one(float* th, float g, float* m, float* v, float c1, float c2, float lr) {
  const float mn = B1 * *m + OMB1 * g;
  const float vn = B2 * *v + OMB2 * g * g;
  *m = mn;
  *v = vn;
  *th -= lr * (mn / c1) / (sqrtf(vn / c2) + EPS);
}

template <int H>
__global__ void __launch_bounds__(BS, 1) mlp_grad_kernel(const float* __restrict__ theta, const float* __restrict__ mu,
                                                         const float* __restrict__ sd, int F, int V, int B,
                                                         const float* __restrict__ feats, const int* __restrict__ labels,
                                                         float* __restrict__ grad, float* __restrict__ loss) {
  extern __shared__ float smem[];
  Smem m = carve(smem, H, V);
  const int P = nparams(F, H, V);
  for (int i = threadIdx.x; i < P; i += BS) m.th[i] = theta[i];
  __syncthreads();
  minibatch_grad<H>(m, F, V, B, feats, labels, nullptr, mu, sd, loss);
  for (int i = threadIdx.x; i < P; i += BS) grad[i] = m.g[i];
}

template <int H>
__global__ void __launch_bounds__(BS, 1) mlp_train_kernel(float* __restrict__ theta, float* __restrict__ am,
                                                          float* __restrict__ av, const float* __restrict__ mu,
                                                          const float* __restrict__ sd, int F, int V, int n,
                                                          const float* __restrict__ feats, const int* __restrict__ labels,
                                                          const int* __restrict__ perm, int epochs, int batch, float lr,
                                                          float* __restrict__ loss) {
  extern __shared__ float smem[];
  Smem m = carve(smem, H, V);
  const int P = nparams(F, H, V);
  for (int i = threadIdx.x; i < P; i += BS) m.th[i] = theta[i];
  __syncthreads();
  int step = 0;
  float c1p = 1.f, c2p = 1.f;  // beta^t
  for (int e = 0; e < epochs; ++e) {
    for (int s0 = 0; s0 < n; s0 += batch) {
      const int Bt = min(batch, n - s0);
      ++step;
      c1p *= B1;
      c2p *= B2;
      minibatch_grad<H>(m, F, V, Bt, feats, labels, perm + (int64_t)e * n + s0, mu, sd, loss);
      const float c1 = 1.f - c1p, c2 = 1.f - c2p;
      for (int i = threadIdx.x; i < P; i += BS) adam_one(&m.th[i], m.g[i], &am[i], &av[i], c1, c2, lr);
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < P; i += BS) theta[i] = m.th[i];
}

__global__ void mlp_adam_kernel(float* __restrict__ th, const float* __restrict__ g, float* __restrict__ m,
                                float* __restrict__ v, int64_t n, float c1, float c2, float lr) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) adam_one(&th[i], g[i], &m[i], &v[i], c1, c2, lr);
}

bool valid_dims(int F, int H, int V) { return F >= 1 && F <= MAXF && (H == 32 || H == 64) && V >= 1 && V <= MAXV; }

template <typename K>
int set_smem(K kernel, size_t bytes) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) == cudaSuccess
             ? AR_OK
             : AR_ERR_CUDA;
}

}  // namespace

// ---------------------------------------------------------------- host fit
int mlp_fit(const std::vector<std::array<float, AR_MAX_FEATURES>>& X, const std::vector<int>& y, int F, int H, int V,
            int epochs, uint64_t seed, MlpModel* out, std::string* msg) {
  const int n = (int)y.size();
  if (n == 0 || !valid_dims(F, H, V)) {
    *msg = "bad dimensions";
    return AR_ERR_ARG;
  }
  // standardisation statistics of signed log1p features (float64 on the host)
  std::vector<float> mu(F), sd(F), feats((size_t)n * F);
  for (int f = 0; f < F; ++f) {
    double s = 0.0, ss = 0.0;
    for (int i = 0; i < n; ++i) s += std::copysign(std::log1p(std::fabs((double)X[i][f])), (double)X[i][f]);
    const double mean = s / n;
    for (int i = 0; i < n; ++i) {
      const double d = std::copysign(std::log1p(std::fabs((double)X[i][f])), (double)X[i][f]) - mean;
      ss += d * d;
    }
    const double dev = std::sqrt(ss / n);
    mu[f] = (float)mean;
    sd[f] = dev > 0 ? (float)dev : 1.f;
    for (int i = 0; i < n; ++i) feats[(size_t)i * F + f] = X[i][f];
  }
  // Glorot-uniform weights, zero biases; one permutation per epoch
  SplitMix64 rng{seed};
  const int P = nparams(F, H, V);
  std::vector<float> theta((size_t)P, 0.f);
  auto fill = [&](size_t off, int fo, int fi) {
    const double a = std::sqrt(6.0 / (fi + fo));
    for (int k = 0; k < fo * fi; ++k) theta[off + k] = (float)((2.0 * rng.uniform() - 1.0) * a);
  };
  fill(0, H, F);
  fill((size_t)H * F + H, H, H);
  fill((size_t)H * F + H + H * H + H, V, H);
  std::vector<int> perm((size_t)epochs * n);
  for (int e = 0; e < epochs; ++e) {
    int* p = perm.data() + (size_t)e * n;
    for (int i = 0; i < n; ++i) p[i] = i;
    for (int i = n - 1; i > 0; --i) {
      const int j = (int)(rng.next() % (uint64_t)(i + 1));
      std::swap(p[i], p[j]);
    }
  }
  float *d_th = nullptr, *d_m = nullptr, *d_v = nullptr, *d_mu = nullptr, *d_sd = nullptr, *d_f = nullptr,
        *d_loss = nullptr;
  int *d_y = nullptr, *d_perm = nullptr;
  cudaStream_t s = nullptr;
  int rc = AR_OK;
  auto ck = [&](cudaError_t e, const char* what) {
    if (e != cudaSuccess && rc == AR_OK) {
      rc = (e == cudaErrorMemoryAllocation) ? AR_ERR_OOM : AR_ERR_CUDA;
      *msg = std::string(what) + ": " + cudaGetErrorString(e);
    }
    return rc == AR_OK;
  };
  if (ck(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "stream") &&
      ck(cudaMalloc(&d_th, P * 4), "malloc") && ck(cudaMalloc(&d_m, P * 4), "malloc") &&
      ck(cudaMalloc(&d_v, P * 4), "malloc") && ck(cudaMalloc(&d_mu, F * 4), "malloc") &&
      ck(cudaMalloc(&d_sd, F * 4), "malloc") && ck(cudaMalloc(&d_f, feats.size() * 4), "malloc") &&
      ck(cudaMalloc(&d_loss, 4), "malloc") && ck(cudaMalloc(&d_y, (size_t)n * 4), "malloc") &&
      ck(cudaMalloc(&d_perm, perm.size() * 4), "malloc") &&
      ck(cudaMemcpyAsync(d_th, theta.data(), P * 4, cudaMemcpyHostToDevice, s), "copy") &&
      ck(cudaMemsetAsync(d_m, 0, P * 4, s), "memset") && ck(cudaMemsetAsync(d_v, 0, P * 4, s), "memset") &&
      ck(cudaMemcpyAsync(d_mu, mu.data(), F * 4, cudaMemcpyHostToDevice, s), "copy") &&
      ck(cudaMemcpyAsync(d_sd, sd.data(), F * 4, cudaMemcpyHostToDevice, s), "copy") &&
      ck(cudaMemcpyAsync(d_f, feats.data(), feats.size() * 4, cudaMemcpyHostToDevice, s), "copy") &&
      ck(cudaMemcpyAsync(d_y, y.data(), (size_t)n * 4, cudaMemcpyHostToDevice, s), "copy") &&
      ck(cudaMemcpyAsync(d_perm, perm.data(), perm.size() * 4, cudaMemcpyHostToDevice, s), "copy")) {
    const int lrc = ar_mlp_train(d_th, d_m, d_v, d_mu, d_sd, F, H, V, n, d_f, d_y, d_perm, epochs, BS, 1e-3f, d_loss, s);
    if (lrc != AR_OK && rc == AR_OK) {
      rc = lrc;
      *msg = "training launch failed";
    }
    if (rc == AR_OK && ck(cudaMemcpyAsync(theta.data(), d_th, P * 4, cudaMemcpyDeviceToHost, s), "copy"))
      ck(cudaStreamSynchronize(s), "sync");
  }
  cudaFree(d_th);
  cudaFree(d_m);
  cudaFree(d_v);
  cudaFree(d_mu);
  cudaFree(d_sd);
  cudaFree(d_f);
  cudaFree(d_loss);
  cudaFree(d_y);
  cudaFree(d_perm);
  if (s) cudaStreamDestroy(s);
  if (rc != AR_OK) return rc;
  out->F = F;
  out->H = H;
  out->V = V;
  out->theta.swap(theta);
  out->mu.swap(mu);
  out->sd.swap(sd);
  return AR_OK;
}

}  // namespace ar

// ---------------------------------------------------------------- C ABI
using namespace ar;

extern "C" int ar_mlp_num_params(int F, int H, int V) { return valid_dims(F, H, V) ? nparams(F, H, V) : AR_ERR_ARG; }

extern "C" int ar_mlp_forward(const float* theta, const float* mu, const float* sd, int F, int H, int V, int64_t B,
                              const float* feats, float* probs, int* variant, float* conf, void* stream) {
  if (!valid_dims(F, H, V) || B < 0) return AR_ERR_ARG;
  if (B == 0) return AR_OK;
  if (!theta || !mu || !sd || !feats) return AR_ERR_ARG;
  const size_t smem = (size_t)nparams(F, H, V) * 4;
  const unsigned grid = (unsigned)ceil_div(B, 128);
  cudaStream_t s = as_stream(stream);
  if (H == 64) {
    if (set_smem(mlp_forward_kernel<64>, smem) != AR_OK) return AR_ERR_CUDA;
    mlp_forward_kernel<64><<<grid, 128, smem, s>>>(theta, mu, sd, F, V, B, feats, probs, variant, conf);
  } else {
    if (set_smem(mlp_forward_kernel<32>, smem) != AR_OK) return AR_ERR_CUDA;
    mlp_forward_kernel<32><<<grid, 128, smem, s>>>(theta, mu, sd, F, V, B, feats, probs, variant, conf);
  }
  return launch_status();
}

extern "C" int ar_mlp_grad(const float* theta, const float* mu, const float* sd, int F, int H, int V, int B,
                           const float* feats, const int* labels, float* grad, float* loss, void* stream) {
  if (!valid_dims(F, H, V) || B < 1 || B > BS) return AR_ERR_ARG;
  if (!theta || !mu || !sd || !feats || !labels || !grad) return AR_ERR_ARG;
  const size_t smem = train_smem_floats(F, H, V) * 4;
  cudaStream_t s = as_stream(stream);
  if (H == 64) {
    if (set_smem(mlp_grad_kernel<64>, smem) != AR_OK) return AR_ERR_CUDA;
    mlp_grad_kernel<64><<<1, BS, smem, s>>>(theta, mu, sd, F, V, B, feats, labels, grad, loss);
  } else {
    if (set_smem(mlp_grad_kernel<32>, smem) != AR_OK) return AR_ERR_CUDA;
    mlp_grad_kernel<32><<<1, BS, smem, s>>>(theta, mu, sd, F, V, B, feats, labels, grad, loss);
  }
  return launch_status();
}

extern "C" int ar_mlp_adam(float* theta, const float* grad, float* m, float* v, int64_t n, int t, float lr,
                           void* stream) {
  if (n < 0 || t < 1) return AR_ERR_ARG;
  if (n == 0) return AR_OK;
  if (!theta || !grad || !m || !v) return AR_ERR_ARG;
  const float c1 = 1.f - powf(B1, (float)t), c2 = 1.f - powf(B2, (float)t);
  mlp_adam_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, as_stream(stream)>>>(theta, grad, m, v, n, c1, c2, lr);
  return launch_status();
}

extern "C" int ar_mlp_train(float* theta, float* adam_m, float* adam_v, const float* mu, const float* sd, int F, int H,
                            int V, int n, const float* feats, const int* labels, const int* perm, int epochs, int batch,
                            float lr, float* loss, void* stream) {
  if (!valid_dims(F, H, V) || n < 1 || epochs < 0 || batch < 1 || batch > BS) return AR_ERR_ARG;
  if (!theta || !adam_m || !adam_v || !mu || !sd || !feats || !labels || !perm) return AR_ERR_ARG;
  if (epochs == 0) return AR_OK;
  const size_t smem = train_smem_floats(F, H, V) * 4;
  cudaStream_t s = as_stream(stream);
  if (H == 64) {
    if (set_smem(mlp_train_kernel<64>, smem) != AR_OK) return AR_ERR_CUDA;
    mlp_train_kernel<64><<<1, BS, smem, s>>>(theta, adam_m, adam_v, mu, sd, F, V, n, feats, labels, perm, epochs,
                                             batch, lr, loss);
  } else {
    if (set_smem(mlp_train_kernel<32>, smem) != AR_OK) return AR_ERR_CUDA;
    mlp_train_kernel<32><<<1, BS, smem, s>>>(theta, adam_m, adam_v, mu, sd, F, V, n, feats, labels, perm, epochs,
                                             batch, lr, loss);
  }
  return launch_status();
}

namespace ar {
AR_CHECK_READER(chk_read_mlp)
}  // namespace ar
