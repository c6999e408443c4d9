// All-pairs n-body variants (FP32): the compute-bound region.
//
//   a_i = sum_j m_j (r_j - r_i) / (|r_j - r_i|^2 + eps^2)^(3/2),  G = 1,
//   j = i included (contributes exactly 0).
//
// Per interaction: 3 FADD + 3 FFMA (softened r^2) + 1 MUFU rsqrt + 3 FMUL +
// 3 FFMA = 12 FP32 lane operations and one MUFU.  The FP32 operations of two
// j bodies are issued together as packed pairs (FADD2 / FFMA2 / FMUL2 on
// sm_100+), so a thread issues ~7.5 instructions per interaction instead of
// ~14 and the FP32 pipe, not instruction issue, is the bound (nbody_math.cuh).
// Variants: shared-memory tile of T bodies (T = threads per block, 128 / 256 /
// 512) x unroll U (1 / 4 / 8) of the inner loop over j pairs; variant =
// 3*tile_index + unroll_index.  Each thread integrates two bodies (i and
// i + T) when that still leaves at least two blocks per SM, else one; its
// bodies share every shared-memory load.  Each thread sums one tile into
// local partials (even and odd j) before adding them to its running total,
// which keeps the float32 rounding error near sqrt(T) + sqrt(N/T) additions
// instead of N.  Small N, whose one-body-per-thread grid leaves fewer than
// two blocks per SM, splits each i-tile's j range over a thread-block
// cluster (nbody_tile_split).  The kernels declare a minimum of one
// resident block so the compiler keeps the unrolled interactions' operands
// in registers (92-110 a thread for unroll 4 and 8): held to 34-64
// registers, the same variants ran at half the rate for N <= 16k and 8 %
// slower at 64k.
//
// The batched form runs `count` independent systems of uneven size in one
// persistent launch: work items (system, i-tile) are ordered largest system
// first (an i-tile costs the system's size) and pulled from an atomic counter
// by resident blocks (as many as fit at the kernel's register count), so the
// long items start first and the tail is short.
#define AR_TU 4
#include <algorithm>
#include <atomic>
#include <cstdio>

#include "common.cuh"
#include "nbody_math.cuh"
#include "tma.cuh"

namespace ar {
namespace {

constexpr int kTiles[3] = {128, 256, 512};
constexpr int kUnroll[3] = {1, 4, 8};
constexpr int kBatchTile = 128;
constexpr int kMaxCluster = 8;  // portable thread-block cluster size

// Bodies base + i_first + r*T (r < R) of [base, base+n) against all bodies of
// the same range.  Padding bodies have zero mass and sit at the origin, so
// they add exactly 0.  `tile` holds two tiles of T bodies: each thread loads
// its body of the next tile into a register before the current tile's
// interactions and stores it into the other half after them, so the load's
// latency is hidden and one barrier per tile suffices (the half written in
// step k was last read in step k - 1, before the barrier that opens step k).
// The j range is [jb, je) within the n bodies (the whole range, or one
// cluster block's chunk); the partial sums are left in ax, ay, az.
template <int T, int U, int R>
__device__ __forceinline__ void body_partials(const float4* __restrict__ p, int64_t base, int64_t n,
                                              int64_t i_first, int64_t jb, int64_t je, float eps2, float4* tile,
                                              float (&ax)[R], float (&ay)[R], float (&az)[R]) {
  float2 npx[R], npy[R], npz[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int64_t i = i_first + (int64_t)r * T;
    const float4 pi = i < n ? p[base + i] : make_float4(0.f, 0.f, 0.f, 0.f);
    npx[r] = make_float2(-pi.x, -pi.x);
    npy[r] = make_float2(-pi.y, -pi.y);
    npz[r] = make_float2(-pi.z, -pi.z);
    ax[r] = ay[r] = az[r] = 0.f;
  }
  const float2 eps2v = make_float2(eps2, eps2);
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
  __syncthreads();  // the previous item's last tile has been read by every thread
  if (jb < je) tile_store(tile, threadIdx.x, jb + threadIdx.x < je ? p[base + jb + threadIdx.x] : zero);
  int cur = 0;
  for (int64_t j0 = jb; j0 < je; j0 += T) {
    __syncthreads();
    const int64_t j = j0 + T + threadIdx.x;
    const float4 q = j < je ? p[base + j] : zero;
    tile_accumulate<U, R>(tile + cur * T, T / 2, npx, npy, npz, eps2v, ax, ay, az);
    cur ^= 1;
    if (j0 + T < je) tile_store(tile + cur * T, threadIdx.x, q);
  }
}

template <int T, int U, int R>
__device__ __forceinline__ void body_tile(const float4* __restrict__ p, float4* __restrict__ a, int64_t base,
                                          int64_t n, int64_t i_first, float eps2, float4* tile) {
  float ax[R], ay[R], az[R];
  body_partials<T, U, R>(p, base, n, i_first, 0, n, eps2, tile, ax, ay, az);
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int64_t i = i_first + (int64_t)r * T;
    if (i < n) a[base + i] = make_float4(ax[r], ay[r], az[r], 0.f);
  }
}

template <int T, int U, int R>
__global__ void __launch_bounds__(T, 1) nbody_tile(int64_t N, const float4* __restrict__ p, float4* __restrict__ a,
                                                float eps2) {
  __shared__ float4 tile[2 * T];
  body_tile<T, U, R>(p, a, 0, N, (int64_t)blockIdx.x * (T * R) + threadIdx.x, eps2, tile);
}

__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// float4 at the same shared-memory offset in block `rank` of this cluster
__device__ __forceinline__ float4 ld_cluster_f4(const float4* local, unsigned rank) {
  uint32_t remote;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(smem_addr(local)), "r"(rank));
  float4 v;
  asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "r"(remote)
               : "memory");
  return v;
}

// Small N: the grid of i-tiles underfills the GPU, so each i-tile is split
// over a thread-block cluster of CS blocks (CS = gridDim.x / i-tiles, set at
// launch): block rank q takes the j bodies [q chunk, (q + 1) chunk), chunk a
// multiple of T, and leaves its partial sums in shared memory; after a
// cluster barrier rank 0 adds the CS partials in rank order from the other
// blocks' shared memory (distributed shared memory) and writes the result,
// and a second barrier keeps every block's shared memory alive until then.
// Both barriers are reached by every thread of every block.
template <int T, int U>
__global__ void __launch_bounds__(T, 1) nbody_tile_split(int64_t N, const float4* __restrict__ p,
                                                      float4* __restrict__ a, float eps2, int cs, int64_t chunk) {
  __shared__ float4 tile[2 * T];
  __shared__ float4 part[T];
  const unsigned q = cluster_rank();
  const int64_t i = (int64_t)(blockIdx.x / cs) * T + threadIdx.x;
  const int64_t jb = min((int64_t)q * chunk, N), je = min(jb + chunk, N);
  float ax[1], ay[1], az[1];
  body_partials<T, U, 1>(p, 0, N, i, jb, je, eps2, tile, ax, ay, az);
  part[threadIdx.x] = make_float4(ax[0], ay[0], az[0], 0.f);
  cluster_barrier();
  if (q == 0) {
    float4 s = part[threadIdx.x];
    for (int r = 1; r < cs; ++r) {
      const float4 o = ld_cluster_f4(&part[threadIdx.x], (unsigned)r);
      s.x += o.x;
      s.y += o.y;
      s.z += o.z;
    }
    if (i < N) a[i] = make_float4(s.x, s.y, s.z, 0.f);
  }
  cluster_barrier();
}

// ------------------------------------------------------------ batched
// One block: rank systems by size (descending, ties to the lower index),
// prefix-sum their i-tile counts in rank order, reset the work counter.
__global__ void nbody_batch_plan(int count, const int* __restrict__ offs, int* __restrict__ order,
                                 int* __restrict__ prefix, int* __restrict__ counter) {
  extern __shared__ int tiles_by_rank[];
  for (int b = threadIdx.x; b < count; b += blockDim.x) {
    const int nb = offs[b + 1] - offs[b];
    int rank = 0;
    for (int c = 0; c < count; ++c) {
      const int nc = offs[c + 1] - offs[c];
      rank += (nc > nb) || (nc == nb && c < b);
    }
    order[rank] = b;
    tiles_by_rank[rank] = (nb + kBatchTile - 1) / kBatchTile;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int r = 0; r < count; ++r) {
      prefix[r] = acc;
      acc += tiles_by_rank[r];
    }
    prefix[count] = acc;
    *counter = 0;
  }
}

__global__ void __launch_bounds__(kBatchTile, 1) nbody_batched(int count, const int* __restrict__ offs,
                                                            const float4* __restrict__ p, float4* __restrict__ a,
                                                            float eps2, const int* __restrict__ order,
                                                            const int* __restrict__ prefix, int* __restrict__ counter) {
  __shared__ float4 tile[2 * kBatchTile];
  __shared__ int item_s;
  const int total = prefix[count];
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) item_s = atomicAdd(counter, 1);
    __syncthreads();
    const int item = item_s;
    if (item >= total) break;
    int lo = 0, hi = count - 1;  // last rank with prefix <= item
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (prefix[mid] <= item)
        lo = mid;
      else
        hi = mid - 1;
    }
    const int b = order[lo];
    const int t = item - prefix[lo];
    const int64_t base = offs[b], n = offs[b + 1] - offs[b];
    body_tile<kBatchTile, 8, 1>(p, a, base, n, (int64_t)t * kBatchTile + threadIdx.x, eps2, tile);
  }
}

// Whether clusters of cs blocks of nbody_tile_split<T, U> fit on the device
// (asked once per cluster size).
template <int T, int U>
bool split_fits(int cs) {
  static std::atomic<int> known[kMaxCluster + 1];  // 0 not asked, 1 fits, 2 does not
  int k = known[cs].load(std::memory_order_relaxed);
  if (k == 0) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)cs);
    cfg.blockDim = dim3(T);
    cudaLaunchAttribute at;
    at.id = cudaLaunchAttributeClusterDimension;
    at.val.clusterDim.x = (unsigned)cs;
    at.val.clusterDim.y = at.val.clusterDim.z = 1;
    cfg.attrs = &at;
    cfg.numAttrs = 1;
    int n = 0;
    k = cudaOccupancyMaxActiveClusters(&n, nbody_tile_split<T, U>, &cfg) == cudaSuccess && n > 0 ? 1 : 2;
    (void)cudaGetLastError();
    known[cs].store(k, std::memory_order_relaxed);
  }
  return k == 1;
}

// Blocks per SM at the register count of nbody_tile_split<T, U> and of
// nbody_tile<T, U, B> (asked once per kernel).
template <int T, int U>
int resident_split() {
  static const int r = [] {
    int n = 0;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, nbody_tile_split<T, U>, T, 0) == cudaSuccess && n > 0
               ? n
               : 1;
  }();
  return r;
}
template <int T, int U, int B>
int resident_tile() {
  static const int r = [] {
    int n = 0;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, nbody_tile<T, U, B>, T, 0) == cudaSuccess && n > 0 ? n
                                                                                                             : 1;
  }();
  return r;
}

// Launch geometry of variant (T, U) at N bodies: two bodies per thread when
// the grid still fills the GPU twice over, otherwise one; and when even one
// body per thread leaves fewer than two blocks per SM, the j range is split
// over a cluster of up to kMaxCluster blocks per i-tile (nbody_tile_split):
// the largest cluster whose blocks still fit in one wave of resident slots,
// and when not even two do, enough clusters for two blocks per SM.
// `resident` (blocks per SM of the kernel that runs) is filled only when
// asked for.
struct Geom {
  int64_t grid;  // i-tiles (blocks, or clusters when split)
  int cs;        // cluster size; 1 when the j range is not split
  int bpt;       // bodies per thread
  int resident;
};
template <int T, int U>
Geom geometry(int64_t N, bool need_resident) {
  Geom g{};
  const int64_t want = 2LL * device_sms();
  const bool two = ceil_div(N, 2 * T) >= want;
  g.bpt = two ? 2 : 1;
  g.grid = ceil_div(N, two ? 2 * T : T);
  g.cs = 1;
  if (two) {
    if (need_resident) g.resident = resident_tile<T, U, 2>();
    return g;
  }
  const int resident = resident_split<T, U>();
  const int64_t fit = (int64_t)resident * device_sms() / g.grid;
  const int cs = fit >= 2 ? (int)std::min<int64_t>({(int64_t)kMaxCluster, fit, g.grid})
                          : (int)std::min<int64_t>({(int64_t)kMaxCluster, ceil_div(want, g.grid), g.grid});
  if (cs >= 2 && split_fits<T, U>(cs)) {
    g.cs = cs;
    g.resident = resident;
  } else if (need_resident) {
    g.resident = resident_tile<T, U, 1>();
  }
  return g;
}

template <int T, int U>
int launch_r(int64_t N, const float4* p, float4* a, float eps2, cudaStream_t s) {
  const Geom g = geometry<T, U>(N, false);
  if (g.grid > 0x7fffffffLL) return AR_ERR_ARG;
  if (g.bpt == 2) {
    nbody_tile<T, U, 2><<<(unsigned)g.grid, T, 0, s>>>(N, p, a, eps2);
    return launch_status();
  }
  if (g.cs >= 2) {
    const int cs = g.cs;
    const int64_t chunk = ceil_div(ceil_div(N, cs), T) * T;  // j bodies per block, whole tiles
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(g.grid * cs));
    cfg.blockDim = dim3(T);
    cfg.stream = s;
    cudaLaunchAttribute at;
    at.id = cudaLaunchAttributeClusterDimension;
    at.val.clusterDim.x = (unsigned)cs;
    at.val.clusterDim.y = at.val.clusterDim.z = 1;
    cfg.attrs = &at;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, nbody_tile_split<T, U>, N, p, a, eps2, cs, chunk) != cudaSuccess)
      return AR_ERR_CUDA;
    return launch_status();
  }
  nbody_tile<T, U, 1><<<(unsigned)g.grid, T, 0, s>>>(N, p, a, eps2);
  return launch_status();
}

template <int T>
Geom geometry_u(int u, int64_t N) {
  switch (u) {
    case 0: return geometry<T, 1>(N, true);
    case 1: return geometry<T, 4>(N, true);
    default: return geometry<T, 8>(N, true);
  }
}

template <int T>
int launch_u(int u, int64_t N, const float4* p, float4* a, float eps2, cudaStream_t s) {
  switch (u) {
    case 0: return launch_r<T, 1>(N, p, a, eps2, s);
    case 1: return launch_r<T, 4>(N, p, a, eps2, s);
    default: return launch_r<T, 8>(N, p, a, eps2, s);
  }
}

size_t batch_ws(int count) { return (size_t)(2 * count + 2) * sizeof(int) + 256; }

}  // namespace

int nbody_num_variants() { return kNbodyVariants; }

int nbody_variant_name(int v, char* buf, int len) {
  if (v < 0 || v >= kNbodyVariants || !buf || len <= 0) return AR_ERR_ARG;
  snprintf(buf, (size_t)len, "nbody_t%d_u%d", kTiles[v / 3], kUnroll[v % 3]);
  return AR_OK;
}

int nbody_launch(void* args, int variant, double, void* stream, void*) {
  const ar_nbody_args* a = static_cast<const ar_nbody_args*>(args);
  if (!a) return AR_ERR_ARG;
  return ar_nbody(variant, a->N, a->pos4, a->acc4, a->eps, stream);
}

}  // namespace ar

using namespace ar;

extern "C" int ar_nbody(int variant, int64_t N, const float* pos4, float* acc4, float eps, void* stream) {
  if (variant < 0 || variant >= kNbodyVariants || N < 0 || !(eps > 0.f)) return AR_ERR_ARG;
  if (N == 0) return AR_OK;
  if (!pos4 || !acc4 || !aligned16(pos4) || !aligned16(acc4)) return AR_ERR_ARG;
  const float4* p = reinterpret_cast<const float4*>(pos4);
  float4* a = reinterpret_cast<float4*>(acc4);
  const float eps2 = eps * eps;
  cudaStream_t s = as_stream(stream);
  switch (variant / 3) {
    case 0: return launch_u<128>(variant % 3, N, p, a, eps2, s);
    case 1: return launch_u<256>(variant % 3, N, p, a, eps2, s);
    default: return launch_u<512>(variant % 3, N, p, a, eps2, s);
  }
}

extern "C" int ar_nbody_geometry(int variant, int64_t N, int64_t* grid, int* cluster, int* bodies_per_thread,
                                 int* resident_per_sm, int* sms) {
  if (variant < 0 || variant >= kNbodyVariants || N < 1) return AR_ERR_ARG;
  Geom g;
  switch (variant / 3) {
    case 0: g = geometry_u<128>(variant % 3, N); break;
    case 1: g = geometry_u<256>(variant % 3, N); break;
    default: g = geometry_u<512>(variant % 3, N); break;
  }
  if (cudaGetLastError() != cudaSuccess) return AR_ERR_CUDA;
  if (grid) *grid = g.grid;
  if (cluster) *cluster = g.cs;
  if (bodies_per_thread) *bodies_per_thread = g.bpt;
  if (resident_per_sm) *resident_per_sm = g.resident;
  if (sms) *sms = device_sms();
  return AR_OK;
}

extern "C" int ar_nbody_batched_workspace_bytes(int count, size_t* bytes) {
  if (count < 0 || !bytes) return AR_ERR_ARG;
  *bytes = batch_ws(count);
  return AR_OK;
}

extern "C" int ar_nbody_batched(int count, const int32_t* offs, const float* pos4, float* acc4, float eps,
                                void* workspace, size_t workspace_bytes, void* stream) {
  if (count < 0 || count > 4096 || !(eps > 0.f)) return AR_ERR_ARG;
  if (count == 0) return AR_OK;
  if (!offs || !pos4 || !acc4 || !aligned16(pos4) || !aligned16(acc4)) return AR_ERR_ARG;
  if (!workspace || workspace_bytes < batch_ws(count)) return AR_ERR_ARG;
  cudaStream_t s = as_stream(stream);
  int* ws = reinterpret_cast<int*>((reinterpret_cast<uintptr_t>(workspace) + 255) & ~uintptr_t(255));
  int* order = ws;
  int* prefix = order + count;
  int* counter = prefix + count + 1;
  const int* o = reinterpret_cast<const int*>(offs);
  nbody_batch_plan<<<1, 256, count * sizeof(int), s>>>(count, o, order, prefix, counter);
  static const int resident = [] {  // blocks per SM at the kernel's register count
    int r = 0;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r, nbody_batched, kBatchTile, 0) == cudaSuccess && r > 0
               ? r
               : 1;
  }();
  const int grid = device_sms() * resident;
  nbody_batched<<<grid, kBatchTile, 0, s>>>(count, o, reinterpret_cast<const float4*>(pos4),
                                            reinterpret_cast<float4*>(acc4), eps * eps, order, prefix, counter);
  return launch_status();
}

namespace ar {
AR_CHECK_READER(chk_read_nbody)
}  // namespace ar
