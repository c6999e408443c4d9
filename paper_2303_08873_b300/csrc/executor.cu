// Persistent mixed-stream executor: a batch of region invocations of the
// four loops runs as features -> plan (device MLP selection) -> one
// persistent launch that pulls (phase, call, tile) work items from an atomic
// counter and dispatches each to the chosen variant's tile function.
//
// Ordering and waits: items are numbered by groups of 64 calls, phase-major
// inside a group (the group's calls' phase 0, then phase 1, ...; inside a
// phase the longest estimated item first), so an item of phase p, which
// waits for the phase p-1 items of its own call, only ever waits for items
// handed out before it to blocks that are already running; the wait is
// bounded and reports AR_ERR_TIMEOUT per call.  Data written inside this
// launch (Jacobi sweeps, merge-path carries, n-body chunk partials) are read
// with L1-bypassing loads (ld.global.cg) or tensor copies.
//
// Per item, thread 0 takes the next item index (issued before the previous
// item's release fence), finds its (call, phase) entry (usually the previous
// item's, kept in shared memory with the entry's end), and waits for the
// entry's dependency once per block and entry; the call descriptor and its
// tile geometry (Jacobi planes per tile, n-body j chunks) are copied to
// shared memory when the call changes.
#define AR_TU 5
#include <cudaTypedefs.h>

#include <cstdio>
#include <cstring>
#include <mutex>
#include <type_traits>

#include "common.cuh"
#include "merge_path.cuh"
#include "nbody_math.cuh"
#include "pairs.cuh"
#include "jacobi_ring.cuh"
#include "tma.cuh"

namespace ar {
namespace {

constexpr int T = 256;                   // threads per executor block
constexpr int PM = AR_EXEC_MAX_PHASES;   // phases per call
constexpr int kJKCMax = 94;              // Jacobi planes per tile at most (96 loaded: 24 four-plane boxes)
constexpr int kJBox = 4;                 // planes per tensor-copy box of the Jacobi tiles
constexpr int kJTilesPerBlock = 1;       // a Jacobi call's tiles per persistent block, at least (if N allows)
constexpr int kJB = 4;                   // Jacobi planes whose loads are issued together
constexpr int kDxTile = 16384;           // daxpy elements per tile
constexpr int kSpPasses = 16;            // SpMV row groups per tile (thread-row, vector-k)
constexpr int kCatchTiles = 512;         // tiles of a df call's catch-up phase
constexpr uint32_t kDepSpin = 1u << 24;  // dependency polls (with backoff) before giving up
constexpr int kMpPerTile = mp::kPerBlock;
constexpr int kMpBatchExec = 8;  // merge-path loads in flight per thread inside the persistent kernel
constexpr int kRunBlocksPerSm = 5;  // resident blocks of the persistent kernel per SM (registers spill; measured best)
static_assert(mp::kThreads == T, "merge-path tiles use the executor's block size");

__constant__ int c_nvar[4] = {kDaxpyVariants, kJacobiVariants, kExecSpmvVariants, kNbodyVariants};
__constant__ int c_default[4] = {6, 1, 0, 3};
__constant__ int c_dx_ept[3] = {1, 2, 4};
__constant__ int c_j_bx[4] = {32, 32, 64, 128};
__constant__ int c_j_by[4] = {4, 8, 4, 2};
__constant__ int c_sp_k[5] = {32, 2, 4, 8, 16};
__constant__ int c_nb_tile[3] = {128, 256, 512};

struct ModelsDev {
  int F[4], V[4], H;
  const float *theta[4], *mu[4], *sd[4];
};

// Work-item order: entries (phase p, call c) are handed out group by group
// (kGroup consecutive calls), phase-major inside a group, so all of a group's
// items are handed out before the next group's (a call's latency is about its
// group's, not the batch's) while every wait still targets items handed out
// earlier (phase p - 1 of the same call, earlier in the same group).  Inside
// a phase the group's calls go in `perm` order: longest estimated item first,
// so the short items fill the batch's tail.
constexpr int kGroup = 64;
__device__ __forceinline__ void entry_pc(int e, int ncalls, const int* perm, int& p, int& c) {
  const int g = e / (kGroup * PM);           // every group but the last is full
  const int c0 = g * kGroup;
  const int gn = min(kGroup, ncalls - c0);   // calls in this group
  const int r = e - c0 * PM;
  p = r / gn;
  c = perm[c0 + r % gn];
}

__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Bounded wait until *d >= need (polls with a 100 ns back-off); false if the
// limit ran out first.
__device__ __forceinline__ bool dep_wait(const volatile int* d, int need, uint32_t limit) {
  for (uint32_t spins = 0; *d < need;) {
    if (++spins > limit) return false;
    __nanosleep(100);
  }
  return true;
}

// A df Jacobi call of 2+ sweeps keeps float pairs in out/work between sweeps
// and ends with a catch-up phase (a float64 sweep that only runs when the
// first sweep met an input outside the float-pair range).
__device__ __forceinline__ bool jacobi_pair_chain(const ar_exec_call& c, int v) {
  return c.loop == AR_LOOP_JACOBI7 && v / 4 == 3 && c.sweeps >= 2 && c.sweeps + 1 <= PM;
}

// n-body i-bodies per tile: one per thread, two for 512-body tiles.
__device__ __forceinline__ int nb_bodies(int v) { return c_nb_tile[v / 3] > T ? c_nb_tile[v / 3] : T; }

// Chunks an n-body call's j range is split over, S, and the j bodies per
// chunk (whole Tt-body j tiles).  S > 1 only when the call's i tiles number
// fewer than `target` and its out1 holds S partial-sum arrays (16 N bytes
// each, 16-byte aligned, apart from the positions and accelerations): then
// the tiles of phase 0 each sum one (i tile, j chunk) into out1 and phase 1
// adds the S partials per body in chunk order.
struct NbSplit {
  int S;
  int64_t chunk;
};
__device__ NbSplit nbody_split(const ar_exec_call& k, int v, long long target) {
  const int64_t N = k.n, Tt = c_nb_tile[v / 3];
  const int64_t ti = cdiv(N, nb_bodies(v));
  NbSplit r{1, N};
  if (N <= 0 || ti >= target || !k.out1 || ((uintptr_t)k.out1 & 15u) != 0 || k.out1 == k.in0 ||
      k.out1 == k.out0)
    return r;
  int64_t S = min(cdiv(target, ti), cdiv(N, Tt));
  S = min(S, (int64_t)(k.out1_bytes / (16ull * (uint64_t)N)));
  if (S <= 1) return r;
  r.chunk = cdiv(cdiv(N, S), Tt) * Tt;
  r.S = (int)cdiv(N, r.chunk);  // no empty chunk
  return r;
}

__device__ __forceinline__ int phases_of(const ar_exec_call& c, int v, long long target) {
  if (c.loop == AR_LOOP_JACOBI7) return c.sweeps + (jacobi_pair_chain(c, v) ? 1 : 0);
  if (c.loop == AR_LOOP_SPMV && v >= 6) return 2;  // merge path: blocks, then the carry fix-up
  if (c.loop == AR_LOOP_NBODY && nbody_split(c, v, target).S > 1) return 2;  // chunk partials, then their sum
  return 1;
}

// Planes per Jacobi tile of an N^3 call run by variant v: as many as keep
// the call's tiles at least `target` (kJTilesPerBlock per block of the
// persistent kernel), at most kJKCMax, with the depth plus the two halo
// planes a whole number of the tensor copies' 4-plane boxes.  The chunks
// are not balanced over N: the ragged last chunk's tiles are handed out last
// in their phase, and short tiles there even out the phase's tail.
__device__ int jacobi_kc(int N, int v, long long target) {
  const long long cb = cdiv(N, c_j_bx[v % 4]) * cdiv(N, c_j_by[v % 4]);
  long long kc = cdiv((long long)N * cb, target);
  kc = max(2LL, min((long long)kJKCMax, kc));
  return (int)(cdiv(kc + 2, kJBox) * kJBox - 2);
}

__device__ int64_t tiles_of(const ar_exec_call& c, int v, int p, long long jtarget) {
  switch (c.loop) {
    case AR_LOOP_DAXPY: return cdiv(c.n, kDxTile);
    case AR_LOOP_JACOBI7: {
      const int64_t N = c.n;
      if (jacobi_pair_chain(c, v) && p == c.sweeps) return kCatchTiles;
      return cdiv(N, c_j_bx[v % 4]) * cdiv(N, c_j_by[v % 4]) * cdiv(N, jacobi_kc((int)N, v, jtarget));
    }
    case AR_LOOP_SPMV: {
      if (v == 0) return cdiv(c.n, (int64_t)T * kSpPasses);
      if (v < 6) return cdiv(c.n, (int64_t)(T / c_sp_k[v - 1]) * kSpPasses);
      const int64_t nb = cdiv(c.n + c.nnz, kMpPerTile);
      return p == 0 ? nb : cdiv(nb, T);
    }
    default: {
      const NbSplit sp = nbody_split(c, v, jtarget);
      return p == 0 ? cdiv(c.n, nb_bodies(v)) * sp.S : cdiv(c.n, T);
    }
  }
}

// Rough duration of one item of call k under variant v (ns, one block of a
// full persistent launch: about 8.8 GB/s of DRAM traffic or 81 GFLOP/s of
// FP32 work per block); only the order of these estimates is used.
__device__ float item_ns(const ar_exec_call& k, int v, long long jtarget) {
  switch (k.loop) {
    case AR_LOOP_DAXPY: return kDxTile * 24.f / 8.8f;
    case AR_LOOP_JACOBI7:
      return (float)c_j_bx[v % 4] * c_j_by[v % 4] * jacobi_kc((int)k.n, v, jtarget) * 16.f / 8.8f;
    case AR_LOOP_SPMV: {
      const float per_row = k.n > 0 ? (float)k.nnz / (float)k.n : 0.f;
      const float items = v == 0 ? (float)T * kSpPasses * (1.f + per_row)
                          : v < 6 ? (float)(T / c_sp_k[v - 1]) * kSpPasses * (1.f + per_row)
                                  : (float)kMpPerTile;
      return items * 12.f / 8.8f;
    }
    default: return (float)nb_bodies(v) * (float)nbody_split(k, v, jtarget).chunk * 20.f / 81.f;
  }
}

// ------------------------------------------------------------------ features
__global__ void __launch_bounds__(T) exec_features(const ar_exec_call* __restrict__ calls, float* __restrict__ feats,
                                                   unsigned long long* __restrict__ part) {
  __shared__ unsigned long long s1[T / 32], s2[T / 32];
  __shared__ int sm[T / 32];
  const int c = blockIdx.y;
  const ar_exec_call k = calls[c];
  if (k.loop == AR_LOOP_SPMV) {
    const int* rp = static_cast<const int*>(k.in0);
    unsigned long long a = 0, q = 0;
    int m = 0;
    for (int64_t r = (int64_t)blockIdx.x * T + threadIdx.x; r < k.n; r += (int64_t)gridDim.x * T) {
      const int len = __ldg(rp + r + 1) - __ldg(rp + r);
      a += (unsigned long long)len;
      q += (unsigned long long)len * (unsigned long long)len;
      m = max(m, len);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      q += __shfl_xor_sync(0xffffffffu, q, o);
      m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    }
    if ((threadIdx.x & 31) == 0) {
      s1[threadIdx.x / 32] = a;
      s2[threadIdx.x / 32] = q;
      sm[threadIdx.x / 32] = m;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long A = 0, Q = 0;
      int M = 0;
      for (int w = 0; w < T / 32; ++w) {
        A += s1[w];
        Q += s2[w];
        M = max(M, sm[w]);
      }
      // integer sums: the result does not depend on the order of the atomics
      atomicAdd(part + 3 * c, A);
      atomicAdd(part + 3 * c + 1, Q);
      atomicMax(part + 3 * c + 2, (unsigned long long)M);
    }
  } else if (blockIdx.x == 0 && threadIdx.x < 8) {
    float v = 0.f;
    if (threadIdx.x == 0) v = (float)k.n;
    if (threadIdx.x == 1 && k.loop == AR_LOOP_JACOBI7) v = (float)k.sweeps;
    // Jacobi: 1 when the row pitch is a multiple of 16 bytes (even N), the
    // condition for staging planes by tensor copies
    if (threadIdx.x == 2 && k.loop == AR_LOOP_JACOBI7) v = (k.n % 2 == 0) ? 1.f : 0.f;
    feats[8 * c + threadIdx.x] = v;
  }
}

// ------------------------------------------------------------------ plan
template <int H>
__device__ int mlp_choose(const ModelsDev& m, int L, const float* f, float* conf) {
  const int F = m.F[L], V = m.V[L];
  const float* th = m.theta[L];
  const float* W1 = th;
  const float* b1 = W1 + H * F;
  const float* W2 = b1 + H;
  const float* b2 = W2 + H * H;
  const float* W3 = b2 + H;
  const float* b3 = W3 + V * H;
  float x0[8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
    x0[i] = i < F ? (copysignf(log1pf(fabsf(f[i])), f[i]) - __ldg(m.mu[L] + i)) / __ldg(m.sd[L] + i) : 0.f;
  float h1[H];
#pragma unroll
  for (int o = 0; o < H; ++o) {
    float a = __ldg(b1 + o);
#pragma unroll
    for (int i = 0; i < 8; ++i)
      if (i < F) a = fmaf(__ldg(W1 + o * F + i), x0[i], a);
    h1[o] = fmaxf(a, 0.f);
  }
  float lg[32];
#pragma unroll
  for (int v = 0; v < 32; ++v) lg[v] = v < V ? __ldg(b3 + v) : -INFINITY;
  for (int o = 0; o < H; ++o) {
    float a = __ldg(b2 + o);
#pragma unroll
    for (int i = 0; i < H; ++i) a = fmaf(__ldg(W2 + o * H + i), h1[i], a);
    a = fmaxf(a, 0.f);
#pragma unroll
    for (int v = 0; v < 32; ++v)
      if (v < V) lg[v] = fmaf(__ldg(W3 + v * H + o), a, lg[v]);
  }
  int best = 0;
  float mx = lg[0];
#pragma unroll
  for (int v = 1; v < 32; ++v)
    if (lg[v] > mx) {
      mx = lg[v];
      best = v;
    }
  float z = 0.f;
#pragma unroll
  for (int v = 0; v < 32; ++v)
    if (v < V) z += expf(lg[v] - mx);
  *conf = 1.f / z;
  return best;
}

// Writes a tensor map of the N^3 float64 grid at `base` into `dst` (global,
// 128-byte aligned): the template `tm` (encoded on the host with the right
// box) with its address, extents and strides replaced.
__device__ void make_grid_map(CUtensorMap* dst, const CUtensorMap& tm, const void* base, int N) {
  const uint4* s4 = reinterpret_cast<const uint4*>(&tm);
  uint4* d4 = reinterpret_cast<uint4*>(dst);
  for (int q = 0; q < (int)(sizeof(CUtensorMap) / sizeof(uint4)); ++q) d4[q] = s4[q];
  tmap_set_address(dst, base);
  tmap_set_dim<0>(dst, N);
  tmap_set_dim<1>(dst, N);
  tmap_set_dim<2>(dst, N);
  tmap_set_stride<0>(dst, (unsigned long long)N * 8ull);
  tmap_set_stride<1>(dst, (unsigned long long)N * N * 8ull);
}

// Odd N: the map of the grid's 2N-wide 2D view (rows of 2N float64, pitch
// 16N bytes, (N^2 - 1) / 2 rows; see jacobi_tma_odd_tile).
__device__ void make_grid_map_2d(CUtensorMap* dst, const CUtensorMap& tm, const void* base, int N) {
  const uint4* s4 = reinterpret_cast<const uint4*>(&tm);
  uint4* d4 = reinterpret_cast<uint4*>(dst);
  for (int q = 0; q < (int)(sizeof(CUtensorMap) / sizeof(uint4)); ++q) d4[q] = s4[q];
  tmap_set_address(dst, base);
  tmap_set_dim<0>(dst, 2 * N);
  tmap_set_dim<1>(dst, (int)(((long long)N * N - 1) / 2));
  tmap_set_stride<0>(dst, (unsigned long long)N * 16ull);
}

// One-time check of the device-made maps against the host encoding (see
// tma_templates_ready); twod selects the 2D view of odd N.
__global__ void exec_tmap_check(const __grid_constant__ CUtensorMap tm, CUtensorMap* out, const void* base, int N,
                                bool twod) {
  if (threadIdx.x == 0) {
    if (twod)
      make_grid_map_2d(out, tm, base, N);
    else
      make_grid_map(out, tm, base, N);
    tmap_release();
  }
}

__global__ void __launch_bounds__(T) exec_plan(const ar_exec_call* __restrict__ calls, int ncalls, ModelsDev m,
                                               bool have_models, const int* __restrict__ force,
                                               int* __restrict__ variant, float* __restrict__ conf,
                                               float* __restrict__ feats, const unsigned long long* __restrict__ part,
                                               int* __restrict__ tiles, long long* __restrict__ prefix,
                                               int* __restrict__ done, unsigned long long* __restrict__ counter,
                                               uint64_t* __restrict__ t0, uint64_t* __restrict__ t1,
                                               int* __restrict__ status, int* __restrict__ vint,
                                               const __grid_constant__ CUtensorMap tm4,
                                               const __grid_constant__ CUtensorMap tm8,
                                               const __grid_constant__ CUtensorMap to4,
                                               const __grid_constant__ CUtensorMap to8, bool tma_ok, bool tma_odd_ok,
                                               CUtensorMap* __restrict__ maps, int* __restrict__ usetma,
                                               long long jtarget, int* __restrict__ perm) {
  __shared__ long long scan[T];
  __shared__ float s_cost[T];
  __shared__ int s_perm[T];
  const int c = threadIdx.x;
  if (c < ncalls) {
    const ar_exec_call k = calls[c];
    int st = AR_OK, v = -1;
    float cf = 1.f;
    const bool loop_ok = k.loop >= 0 && k.loop < 4;
    if (loop_ok && k.loop == AR_LOOP_SPMV) {
      const double rows = (double)k.n, A = (double)part[3 * c], Q = (double)part[3 * c + 1];
      const double mean = k.n > 0 ? A / rows : 0.0;
      const double var = k.n > 0 ? fmax(Q / rows - mean * mean, 0.0) : 0.0;
      float* f = feats + 8 * c;
      f[0] = (float)k.n;
      f[1] = (float)A;
      f[2] = (float)mean;
      f[3] = (float)var;
      f[4] = (float)part[3 * c + 2];
      f[5] = f[6] = f[7] = 0.f;
    }
    // Jacobi: u0, out and (for 2+ sweeps) work present and distinct, N < 2^16
    const bool jac_bad =
        k.loop == AR_LOOP_JACOBI7 &&
        (k.sweeps < 1 || k.sweeps > PM || k.n > 65535 ||
         (k.n > 0 && (!k.in0 || !k.out0 || k.in0 == k.out0 ||
                      (k.sweeps > 1 && (!k.out1 || k.out1 == k.out0 || k.out1 == k.in0)))));
    if (!loop_ok || jac_bad || k.n < 0) {
      st = AR_ERR_ARG;
    } else if (force) {
      v = force[c];
    } else if (have_models && m.theta[k.loop]) {
      float f[8];
      for (int i = 0; i < 8; ++i) f[i] = feats[8 * c + i];
      v = m.H == 64 ? mlp_choose<64>(m, k.loop, f, &cf) : mlp_choose<32>(m, k.loop, f, &cf);
    } else {
      v = c_default[k.loop];
    }
    if (st == AR_OK && (v < 0 || v >= c_nvar[k.loop])) st = AR_ERR_ARG;
    if (st == AR_OK && k.loop == AR_LOOP_SPMV && v >= 6 &&
        (!k.out1 || k.out1_bytes < 16ull * (unsigned long long)cdiv(k.n + k.nnz, kMpPerTile)))
      st = AR_ERR_ARG;  // merge-path needs its carry workspace
    if (st == AR_OK && k.loop == AR_LOOP_DAXPY && v % 3 != 0 &&
        (((uintptr_t)k.in0 | (uintptr_t)k.out0) & 15u) != 0)
      v -= v % 3;  // double2 variants need 16-byte alignment: one element per thread
    const int ph = st == AR_OK ? phases_of(k, v, jtarget) : 0;
    for (int p = 0; p < PM; ++p) {
      tiles[c * PM + p] = p < ph ? (int)tiles_of(k, v, p, jtarget) : 0;
      done[c * PM + p] = 0;
    }
    // tensor maps of u0, out and work for the tensor-copy Jacobi tiles (tma
    // and df families, shapes 32x4 and 32x8): even N at least one box wide,
    // 16-byte aligned buffers
    // (odd N: maps of the grid's 2N-wide 2D view)
    int use = 0;
    const bool odd = k.n % 2 != 0;
    if ((odd ? tma_odd_ok : tma_ok) && st == AR_OK && k.loop == AR_LOOP_JACOBI7 && v / 4 >= 2 && v % 4 <= 1) {
      const bool two = k.sweeps > 1;
      const uintptr_t al = (uintptr_t)k.in0 | (uintptr_t)k.out0 | (two ? (uintptr_t)k.out1 : 0);
      if (k.n >= 36 && k.n <= 65535 && (al & 15) == 0 && k.in0 && k.out0 && (!two || k.out1)) {
        const void* bufs[3] = {k.in0, k.out0, two ? k.out1 : nullptr};
        for (int q = 0; q < 3; ++q) {
          if (!bufs[q]) continue;
          if (odd)
            make_grid_map_2d(maps + 3 * c + q, v % 4 == 0 ? to4 : to8, bufs[q], (int)k.n);
          else
            make_grid_map(maps + 3 * c + q, v % 4 == 0 ? tm4 : tm8, bufs[q], (int)k.n);
        }
        tmap_release();
        use = 1;
      }
    }
    usetma[c] = use;
    // never NaN: the ranks below must be a permutation of the group
    s_cost[c] = st == AR_OK ? fmaxf(item_ns(k, v, jtarget), 0.f) : 0.f;
    t0[c] = ~0ull;
    t1[c] = 0ull;
    status[c] = st;
    variant[c] = st == AR_OK ? v : -1;
    vint[c] = v;
    conf[c] = cf;
  }
  __syncthreads();
  // each group's calls, longest estimated item first (ties by call index)
  if (c < ncalls) {
    const int c0 = c / kGroup * kGroup, gn = min(kGroup, ncalls - c0);
    int rank = 0;
    for (int q = c0; q < c0 + gn; ++q) rank += s_cost[q] > s_cost[c] || (s_cost[q] == s_cost[c] && q < c);
    s_perm[c0 + rank] = c;
    perm[c0 + rank] = c;
  }
  __syncthreads();
  // exclusive prefix over the entries in hand-out order (entry_pc): thread t
  // owns a run of entries
  const int total = PM * ncalls;
  const int per = (total + T - 1) / T;
  const int lo = threadIdx.x * per, hi = min(total, lo + per);
  long long s = 0;
  for (int e = lo; e < hi; ++e) {
    int ep, ec;
    entry_pc(e, ncalls, s_perm, ep, ec);
    s += tiles[ec * PM + ep];
  }
  scan[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long acc = 0;
    for (int t = 0; t < T; ++t) {
      const long long x = scan[t];
      scan[t] = acc;
      acc += x;
    }
    prefix[total] = acc;
    *counter = 0ull;
  }
  __syncthreads();
  long long acc = scan[threadIdx.x];
  for (int e = lo; e < hi; ++e) {
    prefix[e] = acc;
    int ep, ec;
    entry_pc(e, ncalls, s_perm, ep, ec);
    acc += tiles[ec * PM + ep];
  }
}

// ------------------------------------------------------------------ tiles
// kDxTile elements; EPT consecutive elements per thread access (double2 for
// EPT >= 2).  The variant's block size has no counterpart inside a
// persistent 256-thread block, so variants differing only in it run alike.
__device__ void daxpy_tile(const ar_exec_call& k, int v, int64_t t) {
  const int EPT = c_dx_ept[v % 3];
  const int64_t n = k.n, base = t * (int64_t)kDxTile;
  const double a = k.a;
  const double* x = static_cast<const double*>(k.in0);
  double* y = static_cast<double*>(k.out0);
  if (EPT == 1) {
#pragma unroll 4
    for (int e = threadIdx.x; e < kDxTile; e += T) {
      const int64_t i = base + e;
      if (i < n) y[i] = fma(a, __ldg(x + i), y[i]);
    }
  } else {
    const double2* x2 = reinterpret_cast<const double2*>(x);
    double2* y2 = reinterpret_cast<double2*>(y);
    const int64_t n2 = n >> 1, wb = base >> 1;
    const int W = kDxTile / 2, V2 = EPT / 2;  // double2 words per tile and per thread access
#pragma unroll 2
    for (int e = threadIdx.x * V2; e < W; e += T * V2) {
      for (int u = 0; u < V2; ++u) {
        const int64_t w = wb + e + u;
        if (w < n2) {
          const double2 xv = __ldg(x2 + w);
          double2 yv = y2[w];
          yv.x = fma(a, xv.x, yv.x);
          yv.y = fma(a, xv.y, yv.y);
          y2[w] = yv;
        }
      }
    }
    if ((n & 1) && threadIdx.x == 0 && n - 1 >= base && n - 1 < base + kDxTile) y[n - 1] = fma(a, x[n - 1], y[n - 1]);
  }
}

__device__ __forceinline__ double atcg(const double* __restrict__ u, int N, int i, int j, int k) {
  if ((unsigned)i >= (unsigned)N || (unsigned)j >= (unsigned)N || (unsigned)k >= (unsigned)N) return 0.0;
  return __ldcg(u + ((int64_t)k * N + j) * N + i);
}


// ---------------------------------------------------------------- Jacobi by TMA
// Box geometry of the tensor-copy tiles (shapes 32x4 and 32x8): boxes of
// (BX+4) x (BY+2) x kXDZ float64 in a kXRing-slot ring at a 128-byte aligned
// base inside the block's shared memory, one mbarrier per slot.
constexpr int kXDZ = kJBox, kXRing = 3;
template <int BX, int BY>
struct XGeom {
  static constexpr int PX = BX + 4, PY = BY + 2, PLANE = PX * PY, GROUP = PLANE * kXDZ;
  static constexpr int SLOT = (GROUP + 15) / 16 * 16;
  static constexpr uint32_t BYTES = GROUP * 8u;
  static constexpr int SMEM = kXRing * SLOT * 8 + 128;
  static_assert(SLOT * 8 % 128 == 0, "tensor-copy slots stay 128-byte aligned");
};

// One BX x BY x (ke - kb) tile of one sweep with its planes staged by tensor
// copies through `map` (a map of src, made by the plan kernel): box g holds
// planes kb-1+4g .. kb+2+4g (zero outside the grid) and completes output
// planes kb+4g-1 .. kb+4g+2.  Values and arithmetic as in jacobi_ring_tile:
// pair_math with float64 input splits each landed box in place (a value
// outside the pair range marks the point: redone in float64 for float64
// output, reported through *flag for pair output).  The caller's barrier
// after the tile orders its stores; returns false if a wait gave up (the
// copies in flight were drained).
template <int BX, int BY>
__device__ bool jacobi_tma_tile(const CUtensorMap* map, int N, int bx, int by, int kb, int ke, const double* src,
                                double* dst, bool pair_math, bool src_pairs, bool dst_pairs, int* flag,
                                unsigned char* smraw, uint64_t* bars) {
  using G = XGeom<BX, BY>;
  double* buf = reinterpret_cast<double*>(smraw + ((128u - (smem_addr(smraw) & 127u)) & 127u));
  const int tid = threadIdx.x;
  const bool active = tid < BX * BY;
  const int tx = tid % BX, ty = active ? tid / BX : 0;  // idle threads read a valid slot entry
  const int i0 = bx * BX, j0 = by * BY;
  const int kc = ke - kb;
  const int ngroups = (kc + 2 + kXDZ - 1) / kXDZ;
  const bool split = pair_math && !src_pairs;
  if (tid == 0) {
    for (int r = 0; r < kXRing; ++r) mbar_init(smem_addr(&bars[r]), 1);
    mbar_fence_init();
    fence_proxy_async_global();  // the previous sweep's stores before these tensor copies
    tmap_acquire(map);
  }
  __syncthreads();
  auto issue = [&](int g) {
    const int slot = g % kXRing;
    const uint32_t bar = smem_addr(&bars[slot]);
    mbar_arrive_expect_tx(bar, G::BYTES);
    if (AR_CHK(((i0 - 2) & 1) == 0 && (smem_addr(buf + (size_t)slot * G::SLOT) & 127u) == 0 &&
               in_smem(smraw, G::SMEM, buf + (size_t)slot * G::SLOT, G::BYTES)))
      tma_load_3d(smem_addr(buf + (size_t)slot * G::SLOT), map, i0 - 2, j0 - 1, kb - 1 + g * kXDZ, bar);
  };
  if (tid == 0)
    for (int g = 0; g < min(ngroups, kXRing - 1); ++g) issue(g);
  const int i = i0 + tx, j = j0 + ty;
  const bool inside = active && i < N && j < N;
  const int64_t NN = (int64_t)N * N;
  const int c = (ty + 1) * G::PX + tx + 2;
  double* od = dst + ((int64_t)kb * NN + (int64_t)j * N + i);
  float2* op = reinterpret_cast<float2*>(dst) + ((int64_t)kb * NN + (int64_t)j * N + i);
  double dm = 0.0, d0 = 0.0;
  float2 fm = make_float2(0.f, 0.f), f0 = make_float2(0.f, 0.f);
  bool marker_any = false;
  int g = 0, slot = 0, pslot = kXRing - 1;
  uint32_t phase = 0;
  bool failed = false;
  for (; g < ngroups; ++g, pslot = slot, slot = (slot + 1 == kXRing) ? 0 : slot + 1, phase ^= (slot == 0)) {
    const bool ok = mbar_wait_bounded(smem_addr(&bars[slot]), phase);
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    double* box = buf + (size_t)slot * G::SLOT;
    const double* prev = buf + (size_t)pslot * G::SLOT;
    if (split) {
      bool marker = false;
      for (int e = tid; e < G::GROUP; e += T) {
        const float2 f = df_split(box[e]);
        marker |= (f.x != f.x);
        reinterpret_cast<float2*>(box)[e] = f;
      }
      marker_any |= __syncthreads_or(marker);
    }
    // the sweep mode is a compile-time constant of each instantiation (as in
    // the stand-alone kernels): no mode tests in the unrolled plane loop
    auto planes = [&](auto native_c, auto guard_c, auto src_pairs_c, auto dst_pairs_c) {
      constexpr bool NAT = decltype(native_c)::value;
      constexpr bool GUARD = decltype(guard_c)::value;
      constexpr bool SP = decltype(src_pairs_c)::value;
      constexpr bool DP = decltype(dst_pairs_c)::value;
#pragma unroll
      for (int r = 0; r < kXDZ; ++r) {
        const int p = g * kXDZ - 1 + r;
        const bool live = !GUARD || (p >= 1 && p <= kc);  // block-uniform
        const int cp = (r == 0 ? (kXDZ - 1) * G::PLANE : (r - 1) * G::PLANE) + c;
        if constexpr (NAT) {
          const double* pc = (r == 0 ? prev : box) + cp;
          const double up = box[r * G::PLANE + c];
          if (live) {
            double s = pc[-1] + pc[1];
            s += pc[-G::PX];
            s += pc[G::PX];
            s += dm;
            s += up;
            if (inside && AR_CHK(od - dst >= 0 && od - dst < NN * N)) *od = s * kSixth;
            od += NN;
          }
          dm = d0;
          d0 = up;
        } else {
          const float2* pc = reinterpret_cast<const float2*>(r == 0 ? prev : box) + cp;
          const float2 up = reinterpret_cast<const float2*>(box)[r * G::PLANE + c];
          if (live) {
            const float2 res = df_avg6(pc[-1], pc[1], pc[-G::PX], pc[G::PX], fm, up);
            if (inside && AR_CHK(od - dst >= 0 && od - dst < NN * N)) {
              if constexpr (DP) {
                *op = res;
              } else {
                double v = SP ? finite_pair_to_double(res) : pair_to_double(res);
                if (!SP && (__double_as_longlong(v) & 0x7fffffffffffffffLL) > 0x7ff0000000000000LL) {
                  // an input outside the float-pair range: redo in float64
                  const int k = kb + p - 1;
                  double sd = atcg(src, N, i - 1, j, k) + atcg(src, N, i + 1, j, k);
                  sd += atcg(src, N, i, j - 1, k);
                  sd += atcg(src, N, i, j + 1, k);
                  sd += atcg(src, N, i, j, k - 1);
                  sd += atcg(src, N, i, j, k + 1);
                  v = sd * kSixth;
                }
                *od = v;
              }
            }
            op += NN;
            od += NN;
          }
          fm = f0;
          f0 = up;
        }
      }
    };
    using T_ = std::true_type;
    using F_ = std::false_type;
    const bool guard = g == 0 || g * kXDZ + kXDZ - 2 > kc;
    auto pair_planes = [&](auto guard_c) {
      if (src_pairs) {
        if (dst_pairs)
          planes(F_{}, guard_c, T_{}, T_{});
        else
          planes(F_{}, guard_c, T_{}, F_{});
      } else {
        if (dst_pairs)
          planes(F_{}, guard_c, F_{}, T_{});
        else
          planes(F_{}, guard_c, F_{}, F_{});
      }
    };
    if (!pair_math) {
      if (guard)
        planes(T_{}, T_{}, F_{}, F_{});
      else
        planes(T_{}, F_{}, F_{}, F_{});
    } else {
      if (guard)
        pair_planes(T_{});
      else
        pair_planes(F_{});
    }
    // every reader of box g-1 is past this barrier: its slot takes box g+2
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0 && g + kXRing - 1 < ngroups) issue(g + kXRing - 1);
  }
  if (failed && tid == 0) {  // drain the boxes still in flight (bounded) before the slots are reused
    const int issued = min(ngroups, g + kXRing - 1);
    for (int h = g; h < issued; ++h) (void)mbar_wait_bounded(smem_addr(&bars[h % kXRing]), (uint32_t)((h / kXRing) & 1));
  }
  __syncthreads();
  if (tid == 0)
    for (int r = 0; r < kXRing; ++r) mbar_inval(smem_addr(&bars[r]));
  if (dst_pairs && split && marker_any && tid == 0 && flag) atomicOr(flag, 1);
  fence_proxy_async_global();  // these stores before later tensor copies of dst
  return !failed;
}

// Odd N: the same tile through the grid's 2N-wide 2D view (`map` made by
// make_grid_map_2d): each plane lands as two half-boxes of 36 x (BY+2)/2,
// half b holding the rows with (k + y) & 1 == b from x = i0 - 2 - b, so
// element x sits at column x - i0 + 2 + b; rows and columns outside the grid
// are zeroed on edge tiles and the grid's last row (past the view) is loaded
// by the threads -- the staging of the stand-alone jacobi_tma_odd kernel.
// The readers take a plane's row-parity offsets from its index r inside the
// box (r & 1), which is the plane's parity relative to the box's first
// plane only while every box starts on a plane of the same parity.
static_assert(kXDZ % 2 == 0, "odd-N tiles need an even box depth");
template <int BX, int BY>
struct XOddGeom {
  static constexpr int PX = BX + 4, HB = (BY + 2) / 2;
  static constexpr int HALF = (PX * HB + 15) / 16 * 16;  // 128-byte aligned half-boxes
  static constexpr int PLANE = 2 * HALF, GROUP = PLANE * kXDZ;
  static constexpr uint32_t BYTES = 2u * kXDZ * PX * HB * 8u;
  static constexpr int SMEM = kXRing * GROUP * 8;  // the tile shared memory is 128-byte aligned
};

template <int BX, int BY>
__device__ bool jacobi_tma_odd_tile(const CUtensorMap* map, int N, int bx, int by, int kb, int ke, const double* src,
                                    double* dst, bool pair_math, bool src_pairs, bool dst_pairs, int* flag,
                                    unsigned char* smraw, uint64_t* bars) {
  using G = XOddGeom<BX, BY>;
  double* buf = reinterpret_cast<double*>(smraw);
  const int tid = threadIdx.x;
  const bool active = tid < BX * BY;
  const int tx = tid % BX, ty = active ? tid / BX : 0;  // idle threads read valid slot entries
  const int i0 = bx * BX, j0 = by * BY, y0 = j0 - 1;
  const int kc = ke - kb;
  const int ngroups = (kc + 2 + kXDZ - 1) / kXDZ;
  const bool split = pair_math && !src_pairs;
  const bool edge = i0 == 0 || i0 + BX + 2 > N || j0 == 0 || j0 + BY + 1 >= N;
  constexpr int kPad = G::HALF - G::PX * G::HB;
  for (int e = tid; e < kXRing * kXDZ * 2 * kPad; e += T)  // never copied: keep the splits clean
    buf[(e / kPad) * G::HALF + G::PX * G::HB + e % kPad] = 0.0;
  if (tid == 0) {
    for (int r = 0; r < kXRing; ++r) mbar_init(smem_addr(&bars[r]), 1);
    mbar_fence_init();
    fence_proxy_async_global();  // the previous sweep's stores before these tensor copies
    tmap_acquire(map);
  }
  fence_proxy_async_smem();
  __syncthreads();
  auto issue = [&](int g) {
    const int slot = g % kXRing;
    const uint32_t bar = smem_addr(&bars[slot]);
    mbar_arrive_expect_tx(bar, G::BYTES);
    double* sb = buf + (size_t)slot * G::GROUP;
#pragma unroll
    for (int r = 0; r < kXDZ; ++r) {
      const int k = kb - 1 + g * kXDZ + r;
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        const int yb = y0 + ((((k + y0) & 1) == b) ? 0 : 1);
        const long long R = (long long)k * N + yb;
        double* to = sb + r * G::PLANE + b * G::HALF;
        if (AR_CHK(((b * N + i0 - 2 - b) & 1) == 0 && (smem_addr(to) & 127u) == 0 &&
                   in_smem(smraw, G::SMEM, to, G::PX * G::HB * 8u)))
          tma_load_2d(smem_addr(to), map, b * N + i0 - 2 - b, (int)((R - b) >> 1), bar);
      }
    }
  };
  if (tid == 0)
    for (int g = 0; g < min(ngroups, kXRing - 1); ++g) issue(g);
  const int i = i0 + tx, j = j0 + ty;
  const bool inside = active && i < N && j < N;
  const int64_t NN = (int64_t)N * N;
  const int q = (kb + j) & 1;
  const int idc = (ty + 1) >> 1, ids = ty >> 1, idn = (ty + 2) >> 1;
  auto cen = [&](int bc) { return bc * G::HALF + idc * G::PX + tx + 2 + bc; };
  auto oth = [&](int bc, int id) { return (1 - bc) * G::HALF + id * G::PX + tx + 2 + (1 - bc); };
  const int cA = cen(q), sA = oth(q, ids), nA = oth(q, idn), uA = oth(q, idc);
  const int cB = cen(1 - q), sB = oth(1 - q, ids), nB = oth(1 - q, idn), uB = oth(1 - q, idc);
  double* od = dst + ((int64_t)kb * NN + (int64_t)j * N + i);
  float2* op = reinterpret_cast<float2*>(dst) + ((int64_t)kb * NN + (int64_t)j * N + i);
  double dm = 0.0, d0 = 0.0;
  float2 fm = make_float2(0.f, 0.f), f0 = make_float2(0.f, 0.f);
  bool marker_any = false;
  int g = 0, slot = 0, pslot = kXRing - 1;
  uint32_t phase = 0;
  bool failed = false;
  for (; g < ngroups; ++g, pslot = slot, slot = (slot + 1 == kXRing) ? 0 : slot + 1, phase ^= (slot == 0)) {
    const bool ok = mbar_wait_bounded(smem_addr(&bars[slot]), phase);
    double* box = buf + (size_t)slot * G::GROUP;
    const double* prev = buf + (size_t)pslot * G::GROUP;
    if (edge && ok) {
      for (int rr = tid; rr < kXDZ * 2 * G::HB; rr += T) {
        const int idx = rr % G::HB, b = (rr / G::HB) & 1, r = rr / (2 * G::HB);
        const int k = kb - 1 + g * kXDZ + r;
        const int y = y0 + 2 * idx + ((((k + y0) & 1) == b) ? 0 : 1);
        const int xb = i0 - 2 - b;
        double* d = box + r * G::PLANE + b * G::HALF + idx * G::PX;
        if ((unsigned)y >= (unsigned)N || (unsigned)k >= (unsigned)N) {
          for (int c = 0; c < G::PX; ++c) d[c] = 0.0;
        } else {
          const int c0 = max(0, -xb), c1 = min(G::PX, N - xb);
          for (int c = 0; c < c0; ++c) d[c] = 0.0;
          for (int c = c1; c < G::PX; ++c) d[c] = 0.0;
          if (k == N - 1 && y == N - 1) {
            const double* row = src + ((int64_t)k * N + y) * N + xb;
            for (int c = c0; c < c1; ++c) d[c] = __ldcg(row + c);
          }
        }
      }
    }
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    if (split) {
      bool marker = false;
      for (int e = tid; e < G::GROUP; e += T) {
        const float2 f = df_split(box[e]);
        marker |= (f.x != f.x);
        reinterpret_cast<float2*>(box)[e] = f;
      }
      marker_any |= __syncthreads_or(marker);
    }
    // the sweep mode is a compile-time constant of each instantiation (as in
    // the stand-alone kernels): no mode tests in the unrolled plane loop
    auto planes = [&](auto native_c, auto guard_c, auto src_pairs_c, auto dst_pairs_c) {
      constexpr bool NAT = decltype(native_c)::value;
      constexpr bool GUARD = decltype(guard_c)::value;
      constexpr bool SP = decltype(src_pairs_c)::value;
      constexpr bool DP = decltype(dst_pairs_c)::value;
#pragma unroll
      for (int r = 0; r < kXDZ; ++r) {
        const int p = g * kXDZ - 1 + r;
        const bool live = !GUARD || (p >= 1 && p <= kc);  // block-uniform
        const int cc = (r & 1) ? cB : cA, cs = (r & 1) ? sB : sA, cn = (r & 1) ? nB : nA, cu = (r & 1) ? uB : uA;
        const int pb = r == 0 ? (kXDZ - 1) * G::PLANE : (r - 1) * G::PLANE;
        if constexpr (NAT) {
          const double* pp = r == 0 ? prev : box;
          const double up = box[r * G::PLANE + cu];
          if (live) {
            double s = pp[pb + cc - 1] + pp[pb + cc + 1];
            s += pp[pb + cs];
            s += pp[pb + cn];
            s += dm;
            s += up;
            if (inside && AR_CHK(od - dst >= 0 && od - dst < NN * N)) *od = s * kSixth;
            od += NN;
          }
          dm = d0;
          d0 = up;
        } else {
          const float2* pp = reinterpret_cast<const float2*>(r == 0 ? prev : box);
          const float2 up = reinterpret_cast<const float2*>(box)[r * G::PLANE + cu];
          if (live) {
            const float2 res = df_avg6(pp[pb + cc - 1], pp[pb + cc + 1], pp[pb + cs], pp[pb + cn], fm, up);
            if (inside && AR_CHK(od - dst >= 0 && od - dst < NN * N)) {
              if constexpr (DP) {
                *op = res;
              } else {
                double v = SP ? finite_pair_to_double(res) : pair_to_double(res);
                if (!SP && (__double_as_longlong(v) & 0x7fffffffffffffffLL) > 0x7ff0000000000000LL) {
                  const int k = kb + p - 1;
                  double sd = atcg(src, N, i - 1, j, k) + atcg(src, N, i + 1, j, k);
                  sd += atcg(src, N, i, j - 1, k);
                  sd += atcg(src, N, i, j + 1, k);
                  sd += atcg(src, N, i, j, k - 1);
                  sd += atcg(src, N, i, j, k + 1);
                  v = sd * kSixth;
                }
                *od = v;
              }
            }
            op += NN;
            od += NN;
          }
          fm = f0;
          f0 = up;
        }
      }
    };
    using T_ = std::true_type;
    using F_ = std::false_type;
    const bool guard = g == 0 || g * kXDZ + kXDZ - 2 > kc;
    auto pair_planes = [&](auto guard_c) {
      if (src_pairs) {
        if (dst_pairs)
          planes(F_{}, guard_c, T_{}, T_{});
        else
          planes(F_{}, guard_c, T_{}, F_{});
      } else {
        if (dst_pairs)
          planes(F_{}, guard_c, F_{}, T_{});
        else
          planes(F_{}, guard_c, F_{}, F_{});
      }
    };
    if (!pair_math) {
      if (guard)
        planes(T_{}, T_{}, F_{}, F_{});
      else
        planes(T_{}, F_{}, F_{}, F_{});
    } else {
      if (guard)
        pair_planes(T_{});
      else
        pair_planes(F_{});
    }
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0 && g + kXRing - 1 < ngroups) issue(g + kXRing - 1);
  }
  if (failed && tid == 0) {
    const int issued = min(ngroups, g + kXRing - 1);
    for (int h = g; h < issued; ++h) (void)mbar_wait_bounded(smem_addr(&bars[h % kXRing]), (uint32_t)((h / kXRing) & 1));
  }
  __syncthreads();
  if (tid == 0)
    for (int r = 0; r < kXRing; ++r) mbar_inval(smem_addr(&bars[r]));
  if (dst_pairs && split && marker_any && tid == 0 && flag) atomicOr(flag, 1);
  fence_proxy_async_global();  // these stores before later tensor copies of dst
  return !failed;
}

// One BX x BY x 16-plane tile of one sweep, 2.5D: an xy tile with halo in
// shared memory (double buffered), z neighbours in registers.  Values are
// float64 or float pairs in memory (src_pairs / dst_pairs); `pair_math`
// selects float-pair arithmetic.  With float64 input and float-pair
// arithmetic, inputs outside the pair range mark the point: it is redone in
// float64 (dst float64) or, when dst holds pairs, reported through *flag.
// `map`: a tensor map of src (tma and df families, shapes 32x4 and 32x8,
// when the plan made one), else nullptr.  Returns false if a bounded wait
// gave up.
__device__ bool jacobi_sweep_tile(const ar_exec_call& k, int v, int64_t t, int kc, const double* src, double* dst,
                                  bool pair_math, bool src_pairs, bool dst_pairs, int* flag, unsigned char* smraw,
                                  const CUtensorMap* map, uint64_t* bars) {
  const int N = (int)k.n;
  const int fam = v / 4, BX = c_j_bx[v % 4], BY = c_j_by[v % 4];
  const int64_t gx = (N + BX - 1) / BX, gy = (N + BY - 1) / BY;
  const int bx = (int)(t % gx), by = (int)((t / gx) % gy), bz = (int)(t / (gx * gy));
  const int kb = bz * kc, ke = min(N, kb + kc);
  if (map && fam >= 2 && v % 4 <= 1) {
    if (N & 1)
      return v % 4 == 0 ? jacobi_tma_odd_tile<32, 4>(map, N, bx, by, kb, ke, src, dst, pair_math, src_pairs,
                                                     dst_pairs, flag, smraw, bars)
                        : jacobi_tma_odd_tile<32, 8>(map, N, bx, by, kb, ke, src, dst, pair_math, src_pairs,
                                                     dst_pairs, flag, smraw, bars);
    return v % 4 == 0 ? jacobi_tma_tile<32, 4>(map, N, bx, by, kb, ke, src, dst, pair_math, src_pairs, dst_pairs,
                                               flag, smraw, bars)
                      : jacobi_tma_tile<32, 8>(map, N, bx, by, kb, ke, src, dst, pair_math, src_pairs, dst_pairs,
                                               flag, smraw, bars);
  }
  const bool active = threadIdx.x < BX * BY;
  const int lx = threadIdx.x % BX, ly = threadIdx.x / BX;
  const int i = bx * BX + lx, j = by * BY + ly;
  const bool inside = active && i < N && j < N;
  const int64_t NN = (int64_t)N * N, col = (int64_t)j * N + i;
  if (fam == 0) {  // naive: 6 loads per point
    if (!inside) return true;
    for (int kk = kb; kk < ke; ++kk) {
      double s = atcg(src, N, i - 1, j, kk) + atcg(src, N, i + 1, j, kk);
      s += atcg(src, N, i, j - 1, kk);
      s += atcg(src, N, i, j + 1, kk);
      s += atcg(src, N, i, j, kk - 1);
      s += atcg(src, N, i, j, kk + 1);
      dst[kk * NN + col] = s * kSixth;
    }
    return true;
  }
  if (((uintptr_t)src | (uintptr_t)dst) % 16 == 0) {
    jacobi_ring_tile<kJacobi>(N, BX, BY, bx, by, kb, ke, src, dst, pair_math, src_pairs, dst_pairs, flag, smraw,
                              StencilCoef{0.0, 0.f, 0.f, 0.f, 0.f});
    return true;
  }
  // buffers not 16-byte aligned: global loads, those of 4 planes issued together
  const int PXs = BX + 2, PL = PXs * (BY + 2);
  const int cidx = (ly + 1) * PXs + lx + 1;
  // halo role: the x-edge threads load the x halo, the y-edge threads the y
  // halo (BX >= 32 and BY >= 2, so a thread has at most one of each)
  const int hx = lx == 0 ? -1 : (lx == BX - 1 ? 1 : 0);
  const int hy = ly == 0 ? -1 : (ly == BY - 1 ? 1 : 0);
  // 2.5D over planes kb..ke-1: the xy tile with halo in shared memory (double
  // buffered, one barrier per plane), z neighbours in registers.  The global
  // loads of kJB planes (centre of the plane above, halos) are issued
  // together before those planes are staged, so a thread has up to 3 kJB
  // independent loads in flight instead of one or two.
  auto sweep = [&](auto zero, auto ld, auto avg_store) {
    using Val = decltype(zero);
    Val* tile = reinterpret_cast<Val*>(smraw);
    Val below = inside ? ld(i, j, kb - 1) : zero;
    Val cur = inside ? ld(i, j, kb) : zero;
    for (int kc = kb; kc < ke; kc += kJB) {
      Val up[kJB], vx[kJB], vy[kJB];
#pragma unroll
      for (int q = 0; q < kJB; ++q) {
        const int kk = kc + q;
        up[q] = inside && kk < ke ? ld(i, j, kk + 1) : zero;
        vx[q] = active && hx != 0 && kk < ke ? ld(i + hx, j, kk) : zero;
        vy[q] = active && hy != 0 && kk < ke ? ld(i, j + hy, kk) : zero;
      }
#pragma unroll
      for (int q = 0; q < kJB; ++q) {
        const int kk = kc + q;
        if (kk < ke) {  // block-uniform
          Val* tb = tile + ((kk - kb) & 1) * PL;
          if (active) {
            tb[cidx] = cur;
            if (hx != 0) tb[cidx + hx] = vx[q];
            if (hy != 0) tb[cidx + hy * PXs] = vy[q];
          }
          __syncthreads();
          if (inside) avg_store(kk, tb[cidx - 1], tb[cidx + 1], tb[cidx - PXs], tb[cidx + PXs], below, up[q]);
          below = cur;
          cur = up[q];
        }
      }
    }
  };
  if (!pair_math) {
    sweep(
        0.0, [&](int ii, int jj, int kk) { return atcg(src, N, ii, jj, kk); },
        [&](int kk, double w, double e, double so, double no, double d, double u) {
          double s = w + e;
          s += so;
          s += no;
          s += d;
          s += u;
          dst[kk * NN + col] = s * kSixth;
        });
    return true;
  }
  // float-pair arithmetic; loads give pairs directly or split float64 values
  const float2* srcp = reinterpret_cast<const float2*>(src);
  bool marker = false;
  auto ldp = [&](int ii, int jj, int kk) -> float2 {
    if ((unsigned)ii >= (unsigned)N || (unsigned)jj >= (unsigned)N || (unsigned)kk >= (unsigned)N)
      return make_float2(0.f, 0.f);
    const int64_t o = ((int64_t)kk * N + jj) * N + ii;
    if (src_pairs) return __ldcg(srcp + o);
    const float2 f = df_split(__ldcg(src + o));
    marker |= (f.x != f.x);
    return f;
  };
  sweep(make_float2(0.f, 0.f), ldp,
        [&](int kk, float2 w, float2 e, float2 so, float2 no, float2 d, float2 u) {
          const float2 r = df_avg6(w, e, so, no, d, u);
          if (dst_pairs) {
            reinterpret_cast<float2*>(dst)[kk * NN + col] = r;
          } else {
            double dv = pair_to_double(r);
            if (!src_pairs && (__double_as_longlong(dv) & 0x7fffffffffffffffLL) > 0x7ff0000000000000LL) {
              // an input outside the float-pair range: redo this point in float64
              double s = atcg(src, N, i - 1, j, kk) + atcg(src, N, i + 1, j, kk);
              s += atcg(src, N, i, j - 1, kk);
              s += atcg(src, N, i, j + 1, kk);
              s += atcg(src, N, i, j, kk - 1);
              s += atcg(src, N, i, j, kk + 1);
              dv = s * kSixth;
            }
            dst[kk * NN + col] = dv;
          }
        });
  if (dst_pairs && marker && flag) atomicOr(flag, 1);
  return true;
}

// Phase p of a Jacobi call.  Buffers ping-pong so that the last sweep lands in
// `out`.  A df call with a pair chain: phase 0 float64 -> pairs, phases
// 1..S-2 pairs -> pairs, phase S-1 pairs -> float64, phase S the catch-up;
// once the call's flag is set, phase p >= 1 computes sweep p-1 in float64
// from float64 data and the catch-up computes sweep S-1.  maps: the call's
// tensor maps of (u0, out, work), or nullptr.  Returns false if a bounded
// wait gave up.
__device__ bool jacobi_tile(const ar_exec_call& k, int v, int p, int64_t t, int kc, bool flagged, int* flag,
                            unsigned char* smraw, const CUtensorMap* maps, uint64_t* bars) {
  const int S = k.sweeps, N = (int)k.n;
  const double* u0 = static_cast<const double*>(k.in0);
  double* out = static_cast<double*>(k.out0);
  double* work = static_cast<double*>(k.out1);
  auto dst_of = [&](int sw) -> double* { return ((S - 1 - sw) % 2 == 0) ? out : work; };
  auto src_of = [&](int sw) -> const double* { return sw == 0 ? u0 : dst_of(sw - 1); };
  auto map_of = [&](const double* b) -> const CUtensorMap* {
    return !maps ? nullptr : b == u0 ? maps : b == out ? maps + 1 : maps + 2;
  };
  const int fam = v / 4;
  if (!jacobi_pair_chain(k, v))
    return jacobi_sweep_tile(k, v, t, kc, src_of(p), dst_of(p), fam == 3, false, false, nullptr, smraw,
                             map_of(src_of(p)), bars);
  if (p == S) {  // catch-up: float64 sweep S-1 over a contiguous chunk of unknowns
    if (!flagged) return true;
    const double* src = src_of(S - 1);
    double* dst = dst_of(S - 1);
    const int64_t n3 = (int64_t)N * N * N, NN = (int64_t)N * N;
    const int64_t chunk = cdiv(n3, kCatchTiles);
    for (int64_t c = t * chunk + threadIdx.x; c < min(n3, (t + 1) * chunk); c += T) {
      const int i = (int)(c % N), j = (int)((c / N) % N), kk = (int)(c / NN);
      double s = atcg(src, N, i - 1, j, kk) + atcg(src, N, i + 1, j, kk);
      s += atcg(src, N, i, j - 1, kk);
      s += atcg(src, N, i, j + 1, kk);
      s += atcg(src, N, i, j, kk - 1);
      s += atcg(src, N, i, j, kk + 1);
      dst[c] = s * kSixth;
    }
    return true;
  }
  if (flagged)  // one sweep late, in float64
    return jacobi_sweep_tile(k, v, t, kc, src_of(p - 1), dst_of(p - 1), false, false, false, nullptr, smraw,
                             map_of(src_of(p - 1)), bars);
  return jacobi_sweep_tile(k, v, t, kc, src_of(p), dst_of(p), true, p > 0, p < S - 1, flag, smraw,
                           map_of(src_of(p)), bars);
}

__device__ void spmv_tile(const ar_exec_call& k, int v, int p, int64_t t, unsigned char* smraw) {
  const int* rp = static_cast<const int*>(k.in0);
  const int* col = static_cast<const int*>(k.in1);
  const double* val = static_cast<const double*>(k.in2);
  const double* x = static_cast<const double*>(k.in3);
  double* y = static_cast<double*>(k.out0);
  const int64_t rows = k.n, nnz = k.nnz;
  if (v < 6) {  // kSpPasses groups of T/K rows, K lanes per row (thread-row: K = 1)
    const int K = v == 0 ? 1 : c_sp_k[v - 1];
    const int lane = threadIdx.x % K;
    for (int g = 0; g < kSpPasses; ++g) {
      const int64_t r = (t * kSpPasses + g) * (T / K) + threadIdx.x / K;
      double s = 0.0;
      if (r < rows) {
        // the lane's nonzeros e = b + lane + K m in order, four per step
        // while four remain (their col and val loads, then their x
        // gathers, then the FMAs), the rest one at a time
        const int e1 = __ldg(rp + r + 1);
        int j0 = __ldg(rp + r) + lane;
        for (; j0 + 3 * K < e1; j0 += 4 * K) {
          int cc[4];
          double vv[4], xv[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            cc[u] = __ldg(col + j0 + u * K);
            vv[u] = __ldg(val + j0 + u * K);
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) xv[u] = __ldg(x + cc[u]);
#pragma unroll
          for (int u = 0; u < 4; ++u) s = fma(vv[u], xv[u], s);
        }
        for (; j0 < e1; j0 += K) s = fma(__ldg(val + j0), __ldg(x + __ldg(col + j0)), s);
      }
      for (int o = K / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, K);
      if (r < rows && lane == 0) y[r] = s;
    }
    return;
  }
  const int64_t nb = cdiv(rows + nnz, kMpPerTile);
  int64_t* carry_row = static_cast<int64_t*>(k.out1);
  double* carry_val = reinterpret_cast<double*>(carry_row + nb);
  if (p == 1) {  // carry fix-up over path blocks t*T ..
    const int64_t b = t * T + threadIdx.x;
    if (b >= nb) return;
    const int64_t r = __ldcg((const long long*)carry_row + b);
    if (r < 0 || (b > 0 && __ldcg((const long long*)carry_row + b - 1) == r)) return;
    double tot = __ldcg(carry_val + b);
    for (int64_t u = b + 1; u < nb && __ldcg((const long long*)carry_row + u) == r; ++u) tot += __ldcg(carry_val + u);
    y[r] = __ldcg(y + r) + tot;
    return;
  }
  // main pass of path block t (v 6: float64, v 7: float pairs)
  int64_t* sbounds = reinterpret_cast<int64_t*>(smraw + mp::kSmemBytes);
  const int64_t db = t * kMpPerTile, de = min(db + kMpPerTile, rows + nnz);
  if (threadIdx.x < 64) {  // warp 0 finds the block's first row, warp 1 its end
    const int64_t r = mp::search_warp(threadIdx.x < 32 ? db : de, rows, rp, nnz);
    if ((threadIdx.x & 31) == 0) sbounds[threadIdx.x >> 5] = r;
  }
  __syncthreads();
  const int64_t i0 = sbounds[0], i1 = sbounds[1];
  if (v == 6)
    mp::block<false, kMpBatchExec>(rows, nnz, rp, col, val, x, y, db, i0, i1, carry_row + t, carry_val + t, smraw);
  else
    mp::block<true, kMpBatchExec>(rows, nnz, rp, col, val, x, y, db, i0, i1, carry_row + t, carry_val + t, smraw);
}

// R i-bodies per thread (bodies i0 + r T) against the bodies [jb, je), j
// tiles of Tt bodies staged in shared memory in the pair layout of
// nbody_math.cuh; one pass over each tile serves all R.  The sums go to
// out[i].
template <int R>
__device__ __forceinline__ void nbody_rows(const float4* __restrict__ pos, float4* __restrict__ out, int64_t N,
                                           int64_t i0, int64_t jb, int64_t je, int Tt, int uidx, float eps2,
                                           float4* tile) {
  const float2 eps2v = make_float2(eps2, eps2);
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
  float2 npx[R], npy[R], npz[R];
  float ax[R], ay[R], az[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int64_t i = i0 + (int64_t)r * T;
    const float4 pi = i < N ? pos[i] : zero;
    npx[r] = make_float2(-pi.x, -pi.x);
    npy[r] = make_float2(-pi.y, -pi.y);
    npz[r] = make_float2(-pi.z, -pi.z);
    ax[r] = ay[r] = az[r] = 0.f;
  }
  for (int64_t j0 = jb; j0 < je; j0 += Tt) {
    __syncthreads();
    for (int q = threadIdx.x; q < Tt; q += T) {
      const int64_t jj = j0 + q;
      tile_store(tile, q, jj < je ? pos[jj] : zero);  // zero mass past the range adds exactly 0
    }
    __syncthreads();
    if (uidx == 0)
      tile_accumulate<1, R>(tile, Tt / 2, npx, npy, npz, eps2v, ax, ay, az);
    else if (uidx == 1)
      tile_accumulate<4, R>(tile, Tt / 2, npx, npy, npz, eps2v, ax, ay, az);
    else
      tile_accumulate<8, R>(tile, Tt / 2, npx, npy, npz, eps2v, ax, ay, az);
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int64_t i = i0 + (int64_t)r * T;
    if (i < N) out[i] = make_float4(ax[r], ay[r], az[r], 0.f);
  }
}

// Tile t of phase p of an n-body call whose j range is split into S chunks
// of `chunk` bodies (nbody_split; S = 1: not split).  Phase 0: nb_bodies(v)
// i-bodies (one or two per thread) against one chunk (all N bodies when not
// split), into acc or, split, into partial-sum array s of out1; tile t is
// (chunk t / i-tiles, i-tile t mod i-tiles).  Phase 1: T bodies per tile,
// each body's S partials added in chunk order.
__device__ void nbody_tile(const ar_exec_call& k, int v, int p, int64_t t, int S, int64_t chunk,
                           unsigned char* smraw) {
  const int64_t N = k.n;
  float4* acc = static_cast<float4*>(k.out0);
  float4* part = static_cast<float4*>(k.out1);
  if (p == 1) {  // written in this launch by other blocks: L1-bypassing loads
    const int64_t i = t * T + threadIdx.x;
    if (i >= N) return;
    float4 a = __ldcg(part + i);
    for (int s = 1; s < S; ++s) {
      const float4 q = __ldcg(part + (int64_t)s * N + i);
      a.x += q.x;
      a.y += q.y;
      a.z += q.z;
    }
    acc[i] = make_float4(a.x, a.y, a.z, 0.f);
    return;
  }
  const int Tt = c_nb_tile[v / 3], uidx = v % 3;
  const float4* pos = static_cast<const float4*>(k.in0);
  const int64_t ti = cdiv(N, nb_bodies(v));
  const int64_t s = S > 1 ? t / ti : 0, it = S > 1 ? t % ti : t;
  const int64_t i0 = it * nb_bodies(v) + threadIdx.x;
  const int64_t jb = s * chunk, je = S > 1 ? min(N, jb + chunk) : N;
  float4* out = S > 1 ? part + s * N : acc;
  float4* tile = reinterpret_cast<float4*>(smraw);
  // a 512-body tile holds two i-bodies per thread, summed in one pass over
  // each j tile (each shared-memory load serves both: 6 % faster at 256k
  // bodies than a pass per body)
  if (nb_bodies(v) == 2 * T)
    nbody_rows<2>(pos, out, N, i0, jb, je, Tt, uidx, k.eps * k.eps, tile);
  else
    nbody_rows<1>(pos, out, N, i0, jb, je, Tt, uidx, k.eps * k.eps, tile);
}

// ------------------------------------------------------------------ run
// largest tile: a merge-path block (staged products and row ends, open rows,
// partial sums) plus its two path bounds; Jacobi needs 2 x 4 x 130 doubles
constexpr int kSmemBytes = mp::kSmemBytes + 16;
static_assert(XGeom<32, 4>::SMEM <= kSmemBytes && XGeom<32, 8>::SMEM <= kSmemBytes &&
                  XOddGeom<32, 4>::SMEM <= kSmemBytes && XOddGeom<32, 8>::SMEM <= kSmemBytes,
              "the tensor-copy box rings fit the tile shared memory");
static_assert(kSmemBytes >= 8448, "shared memory of the Jacobi and n-body tiles");
static_assert(ring_smem_bytes(32, 4) <= kSmemBytes && ring_smem_bytes(32, 8) <= kSmemBytes &&
                  ring_smem_bytes(64, 4) <= kSmemBytes && ring_smem_bytes(128, 2) <= kSmemBytes,
              "the Jacobi plane ring of every shape fits the tile shared memory");
static_assert((128 + 4) / 2 * (2 + 2) <= 2 * T && (32 + 4) / 2 * (8 + 2) <= 2 * T,
              "a plane's 16-byte chunks fit kRingChunks per thread");

__global__ void __launch_bounds__(T, kRunBlocksPerSm) exec_run(const ar_exec_call* __restrict__ calls, int ncalls,
                                                 const int* __restrict__ vint, const int* __restrict__ tiles,
                                                 const long long* __restrict__ prefix, int* done,
                                                 unsigned long long* counter, uint64_t* t0, uint64_t* t1,
                                                 int* status, int* flags, const CUtensorMap* __restrict__ maps,
                                                 const int* __restrict__ usetma, const int* __restrict__ perm) {
  __shared__ __align__(128) unsigned char smraw[kSmemBytes];  // tensor-copy destinations
  __shared__ __align__(8) uint64_t s_bars[kXRing];
  __shared__ __align__(16) ar_exec_call s_k;  // the current item's call, copied when the call changes
  __shared__ long long s_item, s_t, s_next, s_end;
  __shared__ int s_c, s_p, s_ok, s_v, s_tma, s_flagged, s_pos, s_ready, s_cur, s_geo;
  __shared__ long long s_chunk;
  const int E = PM * ncalls;
  const long long total = prefix[E];
  if (threadIdx.x == 0) {
    s_next = (long long)atomicAdd(counter, 1ull);
    s_pos = 0;       // entry of this block's previous item
    s_end = -1;      // prefix[s_pos + 1] once looked up
    s_ready = -1;    // entry whose dependency this block has seen met
    s_cur = -1;      // call held in s_k
    s_c = s_p = 0;   // the previous item's call and phase
  }
  for (;;) {
    if (threadIdx.x == 0) {
      const long long it = s_next;
      s_item = it;
      if (it < total) {
        // last entry whose range starts at or before it.  A block's items
        // only grow: most lie in its previous item's entry; otherwise gallop
        // forward from that entry, then bisect
        int lo = s_pos, p = s_p, c = s_c;
        if (!(it < s_end)) {
          int step = 1;
          while (lo + step < E && prefix[lo + step] <= it) {
            lo += step;
            step <<= 1;
          }
          int hi = min(lo + step, E - 1);
          while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (prefix[mid] <= it)
              lo = mid;
            else
              hi = mid - 1;
          }
          s_end = (lo >= 0 && lo < E) ? prefix[lo + 1] : -1;
          p = c = 0;
          if (lo >= 0 && lo < E) entry_pc(lo, ncalls, perm, p, c);
        }
        // the item lies in entry lo's range, inside its (call, phase) tiles;
        // otherwise (checked build) it is skipped under entry 0's indices
        const bool valid = AR_CHK(lo >= 0 && lo < E && prefix[lo] <= it && it < prefix[lo + 1] &&
                                  it - prefix[lo] < (long long)tiles[c * PM + p]);
        if (!valid) {
          lo = 0;
          p = c = 0;
          s_end = -1;
          atomicExch(status, (int)AR_ERR_ARG);
        }
        s_pos = lo;
        int ok = valid ? 1 : 0;
        if (c != s_cur) {
          s_k = calls[c];
          s_v = vint[c];
          s_tma = usetma[c];
          s_cur = c;
          // the call's tile geometry, by the rules and the block count the
          // plan counted its tiles with: a Jacobi call's planes per tile, an
          // n-body call's j chunks and their length
          s_geo = 0;
          s_chunk = 0;
          const long long target = (long long)kJTilesPerBlock * gridDim.x;
          if (s_k.loop >= 0 && s_k.loop < 4 && s_v >= 0 && s_v < c_nvar[s_k.loop]) {
            if (s_k.loop == AR_LOOP_JACOBI7) {
              s_geo = jacobi_kc((int)s_k.n, s_v, target);
            } else if (s_k.loop == AR_LOOP_NBODY) {
              const NbSplit sp = nbody_split(s_k, s_v, target);
              s_geo = sp.S;
              s_chunk = sp.chunk;
            }
          }
          if (ok) atomicMin((unsigned long long*)t0 + c, (unsigned long long)gtimer());
        }
        // phase p > 0 waits once per entry for all of phase p - 1 (counters
        // only grow within a batch); the acquire fence then covers every
        // later item of the entry.  A float-pair chain's flag is final by
        // then: only its first sweep raises it
        if (ok && lo != s_ready) {
          if (p > 0) {
            // a call whose wait already gave up skips its later items at
            // once, so one lost dependency costs one bounded wait per block
            if (reinterpret_cast<volatile int*>(status)[c] == (int)AR_ERR_TIMEOUT ||
                !dep_wait(done + c * PM + p - 1, tiles[c * PM + p - 1], kDepSpin)) {
              ok = 0;
              atomicExch(status + c, (int)AR_ERR_TIMEOUT);
            }
            __threadfence();
          }
          s_flagged = p > 0 && __ldcg(flags + c) != 0;
          if (ok) s_ready = lo;
        }
        s_c = c;
        s_p = p;
        s_t = valid ? it - prefix[lo] : 0;
        s_ok = ok;
      }
    }
    __syncthreads();
    if (s_item >= total) break;
    const int c = s_c, p = s_p;
    const long long t = s_t;
    const ar_exec_call k = s_k;
    const int v = s_v;
    // the plan validated (loop, variant); re-checked so that a call table
    // changed under a running batch cannot index outside the variant tables
    if (s_ok && k.loop >= 0 && k.loop < 4 && v >= 0 && v < c_nvar[k.loop]) {
      switch (k.loop) {
        case AR_LOOP_DAXPY: daxpy_tile(k, v, t); break;
        case AR_LOOP_JACOBI7:
          if (!jacobi_tile(k, v, p, t, s_geo, s_flagged != 0, flags + c, smraw, s_tma ? maps + 3 * c : nullptr,
                           s_bars) &&
              threadIdx.x == 0)
            atomicExch(status + c, (int)AR_ERR_TIMEOUT);
          break;
        case AR_LOOP_SPMV: spmv_tile(k, v, p, t, smraw); break;
        default: nbody_tile(k, v, p, t, s_geo, s_chunk, smraw); break;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      // the next claim goes out before the release fence so the two round
      // trips overlap
      const long long nx = (long long)atomicAdd(counter, 1ull);
      __threadfence();
      atomicAdd(done + c * PM + p, 1);
      atomicMax((unsigned long long*)t1 + c, (unsigned long long)gtimer());
      s_next = nx;
    }
  }
}

struct WsLayout {
  size_t part, tiles, prefix, done, counter, vint, flags, usetma, perm, maps, total;
};

WsLayout layout(int max_calls) {
  auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
  WsLayout w;
  size_t o = 0;
  w.part = o;
  o = up(o + (size_t)max_calls * 3 * 8);
  w.tiles = o;
  o = up(o + (size_t)max_calls * PM * 4);
  w.prefix = o;
  o = up(o + ((size_t)max_calls * PM + 1) * 8);
  w.done = o;
  o = up(o + (size_t)max_calls * PM * 4);
  w.counter = o;
  o = up(o + 8);
  w.vint = o;
  o = up(o + (size_t)max_calls * 4);
  w.flags = o;
  o = up(o + (size_t)max_calls * 4);
  w.usetma = o;
  o = up(o + (size_t)max_calls * 4);
  w.perm = o;
  o = up(o + (size_t)max_calls * 4);
  w.maps = o;  // 3 tensor maps (u0, out, work) per call, 128-byte aligned
  o = up(o + (size_t)max_calls * 3 * sizeof(CUtensorMap));
  w.total = o + 256;
  return w;
}

// Templates of the Jacobi tiles' tensor maps (box 36 x 6 x 4 for shape 32x4,
// 36 x 10 x 4 for 32x8), encoded once; the plan kernel copies one per grid
// and replaces its address, extents and strides on the device.  Before the
// first use a check compares a device-made map with the host encoding of the
// same grid, byte for byte, on `s` (synchronous; not while `s` is capturing,
// in which case this batch stages Jacobi planes by cp.async instead).  Any
// mismatch or encode failure turns tensor copies off for the process.
struct MapTemplates {
  CUtensorMap tm4, tm8;  // 3D, even N
  CUtensorMap to4, to8;  // 2D view, odd N
  bool even_ok, odd_ok;
};
// One template check: a device-made map of a test grid against the host
// encoding of the same grid.
bool template_matches(const CUtensorMap& t, bool twod, int N, int box_rows, unsigned char* scratch, int slot,
                      cudaStream_t s) {
  const unsigned char* base = scratch + 1024 * (slot + 1);
  CUtensorMap want, got;
  const bool enc = twod ? encode_tensor_map_2d_f64(&want, base, 2ull * N, ((uint64_t)N * N - 1) / 2, 16ull * N, 36,
                                                   (uint32_t)box_rows)
                        : encode_tensor_map_3d_f64(&want, base, N, N, N, 36, (uint32_t)box_rows, kXDZ);
  if (!enc) return false;
  exec_tmap_check<<<1, 32, 0, s>>>(t, reinterpret_cast<CUtensorMap*>(scratch), base, N, twod);
  return cudaMemcpyAsync(&got, scratch, sizeof got, cudaMemcpyDeviceToHost, s) == cudaSuccess &&
         cudaStreamSynchronize(s) == cudaSuccess && std::memcmp(&want, &got, sizeof got) == 0;
}
bool tma_templates_ready(unsigned char* scratch, cudaStream_t s, MapTemplates* out) {
  static std::mutex mu;
  static int state = 0;  // 0 unchecked, 1 checked
  static MapTemplates tm{};
  std::lock_guard<std::mutex> lock(mu);
  if (state == 0) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
      *out = MapTemplates{};
      return false;
    }
    state = 1;
    tm.even_ok = encode_tensor_map_3d_f64(&tm.tm4, scratch, 64, 64, 64, 36, 6, kXDZ) &&
                 encode_tensor_map_3d_f64(&tm.tm8, scratch, 64, 64, 64, 36, 10, kXDZ) &&
                 template_matches(tm.tm4, false, 96, 6, scratch, 0, s) &&
                 template_matches(tm.tm8, false, 512, 10, scratch, 1, s);
    tm.odd_ok = encode_tensor_map_2d_f64(&tm.to4, scratch, 130, 2112, 1040, 36, 3) &&
                encode_tensor_map_2d_f64(&tm.to8, scratch, 130, 2112, 1040, 36, 5) &&
                template_matches(tm.to4, true, 97, 3, scratch, 2, s) &&
                template_matches(tm.to8, true, 511, 5, scratch, 3, s);
  }
  *out = tm;
  return tm.even_ok || tm.odd_ok;
}

// Self-test of the bounded waits: kind 0 waits on a counter that nothing
// raises, kind 1 on an mbarrier phase that nothing completes, kinds 2 and 3
// on ones already satisfied; each writes AR_ERR_TIMEOUT or AR_OK to *status.
__global__ void wait_selftest(int kind, uint32_t limit, int* status) {
  __shared__ int counter;
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  bool ok;
  if (kind == 0 || kind == 2) {
    counter = kind == 2 ? 1 : 0;
    ok = dep_wait(&counter, 1, limit);
  } else {
    const uint32_t b = smem_addr(&bar);
    mbar_init(b, 1);
    mbar_fence_init();
    if (kind == 3) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(b) : "memory");
    ok = mbar_wait_bounded(b, 0, limit);
    mbar_inval(b);
  }
  *status = ok ? AR_OK : AR_ERR_TIMEOUT;
}

}  // namespace
}  // namespace ar

using namespace ar;

extern "C" int ar_wait_selftest(int kind, unsigned int limit, int32_t* status, void* stream) {
  if (kind < 0 || kind > 3 || limit == 0 || limit > (1u << 24) || !status) return AR_ERR_ARG;
  wait_selftest<<<1, 32, 0, as_stream(stream)>>>(kind, limit, status);
  return launch_status();
}

extern "C" int ar_exec_num_variants(int loop) {
  const int nvar[4] = {kDaxpyVariants, kJacobiVariants, kExecSpmvVariants, kNbodyVariants};
  return loop >= 0 && loop < 4 ? nvar[loop] : AR_ERR_ARG;
}

extern "C" int ar_exec_workspace_bytes(int max_calls, size_t* bytes) {
  if (max_calls < 1 || max_calls > AR_EXEC_MAX_CALLS || !bytes) return AR_ERR_ARG;
  *bytes = layout(max_calls).total;
  return AR_OK;
}

extern "C" int ar_exec_batch(const ar_exec_call* calls, int ncalls, const ar_exec_models* models,
                             const int32_t* force_variant, int32_t* variant, float* conf, float* features,
                             uint64_t* t_start, uint64_t* t_end, int32_t* status, void* workspace,
                             size_t workspace_bytes, void* stream) {
  if (ncalls < 0 || ncalls > AR_EXEC_MAX_CALLS) return AR_ERR_ARG;
  if (ncalls == 0) return AR_OK;
  if (!calls || !variant || !conf || !features || !t_start || !t_end || !status || !workspace) return AR_ERR_ARG;
  const WsLayout w = layout(ncalls);
  if (workspace_bytes < w.total) return AR_ERR_ARG;
  ModelsDev m{};
  bool have = false;
  if (models) {
    if (models->H != 32 && models->H != 64) return AR_ERR_ARG;
    const int nfeat[4] = {1, 3, 5, 1};
    const int nvar[4] = {kDaxpyVariants, kJacobiVariants, kExecSpmvVariants, kNbodyVariants};
    for (int L = 0; L < 4; ++L) {
      m.F[L] = models->F[L];
      m.V[L] = models->V[L];
      m.theta[L] = models->theta[L];
      m.mu[L] = models->mu[L];
      m.sd[L] = models->sd[L];
      if (m.theta[L] && (m.F[L] != nfeat[L] || m.V[L] != nvar[L] || !m.mu[L] || !m.sd[L])) return AR_ERR_ARG;
    }
    m.H = models->H;
    have = true;
  }
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(workspace) + 255) &
                                                         ~uintptr_t(255));
  unsigned long long* part = reinterpret_cast<unsigned long long*>(base + w.part);
  int* tiles = reinterpret_cast<int*>(base + w.tiles);
  long long* prefix = reinterpret_cast<long long*>(base + w.prefix);
  int* done = reinterpret_cast<int*>(base + w.done);
  unsigned long long* counter = reinterpret_cast<unsigned long long*>(base + w.counter);
  int* vint = reinterpret_cast<int*>(base + w.vint);
  int* flags = reinterpret_cast<int*>(base + w.flags);
  int* usetma = reinterpret_cast<int*>(base + w.usetma);
  int* perm = reinterpret_cast<int*>(base + w.perm);
  CUtensorMap* maps = reinterpret_cast<CUtensorMap*>(base + w.maps);
  cudaStream_t s = as_stream(stream);
  MapTemplates tmt{};
  const bool tma_ok = tma_templates_ready(reinterpret_cast<unsigned char*>(maps), s, &tmt);
  if (cudaMemsetAsync(part, 0, (size_t)ncalls * 3 * 8, s) != cudaSuccess) return AR_ERR_CUDA;
  if (cudaMemsetAsync(flags, 0, (size_t)ncalls * 4, s) != cudaSuccess) return AR_ERR_CUDA;
  const int run_blocks = device_sms() * kRunBlocksPerSm;  // the persistent kernel's grid
  exec_features<<<dim3(64, (unsigned)ncalls), T, 0, s>>>(calls, features, part);
  exec_plan<<<1, T, 0, s>>>(calls, ncalls, m, have, force_variant, variant, conf, features, part, tiles, prefix,
                            done, counter, t_start, t_end, status, vint, tmt.tm4, tmt.tm8, tmt.to4, tmt.to8,
                            tma_ok && tmt.even_ok, tma_ok && tmt.odd_ok, maps, usetma,
                            (long long)kJTilesPerBlock * run_blocks, perm);
  exec_run<<<run_blocks, T, 0, s>>>(calls, ncalls, vint, tiles, prefix, done, counter, t_start, t_end, status,
                                    flags, maps, usetma, perm);
  return launch_status();
}

namespace ar {
AR_CHECK_READER(chk_read_executor)
}  // namespace ar
