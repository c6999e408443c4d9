// CSR SpMV variants, y = A x in float64 (the sparse region; stand-in for the
// paper's AMGMk relax benchmark, Table 3), and the device reduction of the
// row-length features the learned selector reads.
//
// Algorithmic traffic: 12 bytes per nonzero (val + col), 4 per row pointer,
// 8 per x entry (read once when it stays in L2) and 8 per output row.  One
// DFMA per nonzero; on B300 that float64 rate (~0.56e12/s) is of the same
// order as the HBM-limited nonzero rate, and a float64 instruction occupies
// the float64 pipe for its whole warp however many lanes are active, so the
// variants also differ in how many (partly masked) float64 instructions they
// spend per row.
//
// Variants: 0 thread-per-row; 1 warp-per-row (32-lane shuffle reduction);
// 2..5 vector-k with k = 2, 4, 8, 16 lanes per row; 6 merge-path
// (Merrill & Garland, SC'16) with the block's products staged in shared
// memory; 7 the same merge path in float-pair arithmetic (merge_path.cuh).
// Merge path cuts the merge of row ends and nonzero indices into equal chunks
// of 16 path items per thread, so every thread does the same work whatever
// the row lengths; rows that straddle threads are summed by a segmented scan
// inside the block, rows that straddle blocks by a second small kernel over
// the per-block carries.
#define AR_TU 3
#include <cstdio>
#include <mutex>

#include "common.cuh"
#include "merge_path.cuh"

namespace ar {
namespace {

using mp::ld_col;
using mp::ld_val;
constexpr int kMpThreads = mp::kThreads;
constexpr int kMpPerBlock = mp::kPerBlock;

// ------------------------------------------------------------ thread per row
__global__ void __launch_bounds__(256) spmv_thread_row(int64_t rows, const int* __restrict__ rowptr,
                                                       const int* __restrict__ col, const double* __restrict__ val,
                                                       const double* __restrict__ x, double* __restrict__ y) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rows) return;
  const int b = __ldg(rowptr + r), e = __ldg(rowptr + r + 1);
  double s = 0.0;
  for (int k = b; k < e; ++k) s = fma(ld_val(val + k), __ldg(x + ld_col(col + k)), s);
  y[r] = s;
}

// ------------------------------------------------------------ K lanes per row
template <int K>
__global__ void __launch_bounds__(256) spmv_vector(int64_t rows, const int* __restrict__ rowptr,
                                                   const int* __restrict__ col, const double* __restrict__ val,
                                                   const double* __restrict__ x, double* __restrict__ y) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t r = g / K;
  const int lane = threadIdx.x % K;
  double s = 0.0;
  if (r < rows) {
    const int b = __ldg(rowptr + r), e = __ldg(rowptr + r + 1);
    for (int k = b + lane; k < e; k += K) s = fma(ld_val(val + k), __ldg(x + ld_col(col + k)), s);
  }
#pragma unroll
  for (int o = K / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, K);
  if (r < rows && lane == 0) y[r] = s;
}

// ------------------------------------------------------------ merge path
__global__ void spmv_mp_partition(int64_t rows, int64_t nnz, int nblocks, const int* __restrict__ rowptr,
                                  int64_t* __restrict__ start_row) {
  pdl_begin();  // lets the main pass launch; the partition itself is launched in order
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b > nblocks) return;
  const int64_t L = rows + nnz;
  const int64_t d = min((int64_t)b * kMpPerBlock, L);
  start_row[b] = mp::search(d, 0, rows, rowptr, nnz);
}

// One path block per CTA (see merge_path.cuh); DF selects float-pair
// arithmetic.
template <bool DF>
__global__ void __launch_bounds__(kMpThreads, 5) spmv_mp_main(int64_t rows, int64_t nnz, const int* __restrict__ rowptr,
                                                           const int* __restrict__ col,
                                                           const double* __restrict__ val,
                                                           const double* __restrict__ x, double* __restrict__ y,
                                                           const int64_t* __restrict__ start_row,
                                                           int64_t* __restrict__ carry_row,
                                                           double* __restrict__ carry_val) {
  pdl_begin();  // the partition of this call is complete and visible
  __shared__ __align__(16) unsigned char smem[mp::kSmemBytes];
  const int b = blockIdx.x;
  mp::block<DF>(rows, nnz, rowptr, col, val, x, y, (int64_t)b * kMpPerBlock, start_row[b], start_row[b + 1],
                carry_row + b, carry_val + b, smem);
}

// Rows straddling blocks: the head of each run of equal carry rows adds the
// run's carries (block order) to y.  A block's carry row is always closed by
// a later block, which has already written y[row] in spmv_mp_main.
__global__ void spmv_mp_fixup(int nblocks, const int64_t* __restrict__ carry_row,
                              const double* __restrict__ carry_val, double* __restrict__ y) {
  pdl_begin();  // the main pass of this call is complete and visible
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nblocks) return;
  const int64_t r = carry_row[b];
  if (r < 0 || (b > 0 && carry_row[b - 1] == r)) return;
  double tot = carry_val[b];
  for (int u = b + 1; u < nblocks && carry_row[u] == r; ++u) tot += carry_val[u];
  y[r] += tot;
}

size_t mp_workspace(int64_t rows, int64_t nnz) {
  const int64_t nb = ceil_div(rows + nnz, kMpPerBlock);
  return (size_t)(nb + 1) * 8 + (size_t)nb * 8 + (size_t)nb * 8 + 256;
}

// ------------------------------------------------------------ length-binned
// Rows are grouped by length class and each class runs the decomposition that
// spends the fewest float64 lane-slots: a float64 instruction costs its whole
// warp whatever lanes are active, and on B300 the float64 pipe, not HBM,
// bounds CSR SpMV.  A row of length n on K lanes costs K (ceil(n / K) +
// log2 K) lane-slots (the FMAs plus the shuffle-reduction adds), which favours
// few lanes, but a row's latency grows with its passes, and the longest row
// bounds the kernel; so K grows with the length class (1 lane up to length 8,
// 2 up to 32, 4 up to 64, 8 up to 256, 16 up to 1024, 32 beyond), which keeps
// every row within 16 passes and spends ~1.1 lane-slots per nonzero on
// power-law rows against 1.6-2.6 for vector-k.  Each lane sums up to 8
// nonzeros per pass with all its column, value and x loads issued before the
// FMAs, over as many passes as the row needs (the last one trimmed to the
// row); rows of one class have similar lengths, so a warp's lanes finish
// together.
//
// Four launches: count (rows per class per block of kBinRows rows), scan
// (class offsets; units = warps of work per class), scatter (each row's id,
// first and end nonzero into the class's slots, in increasing row order) and
// a persistent kernel of one wave whose warps take units round-robin from
// the longest class down, loading the next unit's rows while they sum the
// current one.  Every row's sum has a fixed order (per lane in nonzero order,
// then a fixed lane tree), so results do not depend on the schedule.
constexpr int kBins = 10;
constexpr int kBinRows = 4096;  // rows per counting / scatter block
constexpr int kBinThreads = 256;
static_assert(2 * kBins + 2 <= kBinThreads, "the persistent kernel loads meta with one thread per entry");
// classes: lengths 0-2, 3-4, 5-8, 9-16, 17-32, 33-64, 65-128, 129-256,
// 257-1024, 1025+ (lanes per row; nonzeros per lane and pass)
__constant__ int kBinLanes[kBins] = {1, 1, 1, 2, 2, 4, 8, 8, 16, 32};
__constant__ int kBinU[kBins] = {2, 4, 8, 8, 8, 8, 8, 8, 8, 8};

__device__ __forceinline__ int bin_of(int len) {
  return len <= 2     ? 0
         : len <= 4    ? 1
         : len <= 8    ? 2
         : len <= 16   ? 3
         : len <= 32   ? 4
         : len <= 64   ? 5
         : len <= 128  ? 6
         : len <= 256  ? 7
         : len <= 1024 ? 8
                       : 9;
}

// Workspace: counts int32[nblk * kBins] (per block; exclusive offsets after
// the scan), meta int64[2 * kBins + 2] (class starts in the slot arrays;
// unit prefix, longest class first), and per slot the row id, first and end
// nonzero (int32[rows] each).
struct BinWs {
  int* counts;
  long long* meta;
  int *row, *beg, *end;
};
size_t bin_workspace(int64_t rows) {
  const int64_t nblk = ceil_div(rows, kBinRows);
  return (size_t)nblk * kBins * 4 + 256 + (size_t)(2 * kBins + 2) * 8 + 256 + 3 * ((size_t)rows * 4 + 256) + 256;
}
BinWs bin_ws(void* w, int64_t rows) {
  auto up = [](uintptr_t p) { return (p + 255) & ~uintptr_t(255); };
  const int64_t nblk = ceil_div(rows, kBinRows);
  BinWs b;
  uintptr_t p = up(reinterpret_cast<uintptr_t>(w));
  b.counts = reinterpret_cast<int*>(p);
  p = up(p + (size_t)nblk * kBins * 4);
  b.meta = reinterpret_cast<long long*>(p);
  p = up(p + (size_t)(2 * kBins + 2) * 8);
  b.row = reinterpret_cast<int*>(p);
  p = up(p + (size_t)rows * 4);
  b.beg = reinterpret_cast<int*>(p);
  p = up(p + (size_t)rows * 4);
  b.end = reinterpret_cast<int*>(p);
  return b;
}

// Block b counts the classes of rows [b kBinRows, (b+1) kBinRows).
__global__ void __launch_bounds__(kBinThreads) spmv_bin_count(int64_t rows, const int* __restrict__ rowptr,
                                                               int* __restrict__ counts) {
  pdl_begin();
  __shared__ int cnt[kBins];
  if (threadIdx.x < kBins) cnt[threadIdx.x] = 0;
  __syncthreads();
  const int64_t r0 = (int64_t)blockIdx.x * kBinRows, r1 = min(rows, r0 + kBinRows);
  int mine[kBins] = {};
  for (int64_t r = r0 + threadIdx.x; r < r1; r += kBinThreads) ++mine[bin_of(__ldg(rowptr + r + 1) - __ldg(rowptr + r))];
#pragma unroll
  for (int c = 0; c < kBins; ++c) {
    int v = mine[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(&cnt[c], v);  // integer sums: order-free
  }
  __syncthreads();
  if (threadIdx.x < kBins) counts[(int64_t)blockIdx.x * kBins + threadIdx.x] = cnt[threadIdx.x];
}

// One block: per class, exclusive offsets over the blocks (in place), the
// class starts, and the unit prefix (a unit = one warp: 32 / lanes rows of
// the class), longest class first.
__global__ void __launch_bounds__(kBinThreads) spmv_bin_scan(int nblk, int* __restrict__ counts,
                                                              long long* __restrict__ meta) {
  pdl_begin();
  __shared__ long long tot[kBins];
  const int w = threadIdx.x / 32, lane = threadIdx.x & 31;
  for (int c = w; c < kBins; c += kBinThreads / 32) {  // warp w scans classes w, w + 8, ...
    long long run = 0;
    for (int b0 = 0; b0 < nblk; b0 += 32) {
      const int b = b0 + lane;
      const int v = b < nblk ? counts[(int64_t)b * kBins + c] : 0;
      int incl = v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
      }
      if (b < nblk) counts[(int64_t)b * kBins + c] = (int)(run + incl - v);
      run += __shfl_sync(0xffffffffu, incl, 31);
    }
    if (lane == 0) tot[c] = run;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    long long s = 0;
    for (int c = 0; c < kBins; ++c) {
      meta[c] = s;
      s += tot[c];
    }
    meta[kBins] = s;
    long long u = 0;
    for (int q = 0; q < kBins; ++q) {
      const int c = kBins - 1 - q;
      meta[kBins + 1 + q] = u;
      const int rpw = 32 / kBinLanes[c];  // rows per warp
      u += (tot[c] + rpw - 1) / rpw;
    }
    meta[2 * kBins + 1] = u;
  }
}

// Block b writes its rows into their class's slots, in row order (ranks from
// warp ballots, warps in order).
__global__ void __launch_bounds__(kBinThreads) spmv_bin_scatter(int64_t rows, const int* __restrict__ rowptr,
                                                                 const int* __restrict__ counts,
                                                                 const long long* __restrict__ meta,
                                                                 int* __restrict__ srow, int* __restrict__ sbeg,
                                                                 int* __restrict__ send) {
  pdl_begin();
  __shared__ int base[kBins];
  __shared__ int wcnt[kBinThreads / 32][kBins];
  const int w = threadIdx.x / 32, lane = threadIdx.x & 31;
  if (threadIdx.x < kBins) base[threadIdx.x] = counts[(int64_t)blockIdx.x * kBins + threadIdx.x];
  const int64_t r0 = (int64_t)blockIdx.x * kBinRows, r1 = min(rows, r0 + kBinRows);
  for (int64_t c0 = r0; c0 < r1; c0 += kBinThreads) {
    const int64_t r = c0 + threadIdx.x;
    const int b = r < r1 ? __ldg(rowptr + r) : 0, e = r < r1 ? __ldg(rowptr + r + 1) : 0;
    const int c = r < r1 ? bin_of(e - b) : -1;
    const unsigned lt = (1u << lane) - 1u;
    int rank = 0;
#pragma unroll
    for (int q = 0; q < kBins; ++q) {
      const unsigned m = __ballot_sync(0xffffffffu, c == q);
      if (c == q) rank = __popc(m & lt);
      if (lane == 0) wcnt[w][q] = __popc(m);
    }
    __syncthreads();
    if (c >= 0) {
      int off = base[c] + rank;
      for (int v = 0; v < w; ++v) off += wcnt[v][c];
      const long long dst = meta[c] + off;
      if (AR_CHK(dst >= 0 && dst < rows)) {
        srow[dst] = (int)r;
        sbeg[dst] = b;
        send[dst] = e;
      }
    }
    __syncthreads();
    if (threadIdx.x < kBins) {
      int add = 0;
      for (int v = 0; v < kBinThreads / 32; ++v) add += wcnt[v][threadIdx.x];
      base[threadIdx.x] += add;
    }
    __syncthreads();
  }
}

// This lane's row of unit u: class, row id, nonzero range (r = -1: none).
struct BinRow {
  int c, r, b, e;
};
__device__ __forceinline__ BinRow bin_row(long long u, const long long* sm, const int* __restrict__ srow,
                                          const int* __restrict__ sbeg, const int* __restrict__ send) {
  int q = 0;  // position of the unit's class in the longest-first order
  while (q + 1 < kBins && sm[kBins + 2 + q] <= u) ++q;
  BinRow d;
  d.c = kBins - 1 - q;
  const int K = kBinLanes[d.c];
  const long long slot = (u - sm[kBins + 1 + q]) * (32 / K) + (threadIdx.x & 31) / K;
  if (slot < sm[d.c + 1] - sm[d.c]) {
    const long long s = sm[d.c] + slot;
    d.r = __ldg(srow + s);
    d.b = __ldg(sbeg + s);
    d.e = __ldg(send + s);
  } else {
    d.r = -1;
    d.b = d.e = 0;
  }
  return d;
}

// One row per group of K lanes, U nonzeros per lane per pass.
template <int K, int U>
__device__ __forceinline__ void binned_row(const BinRow& d, const int* __restrict__ col,
                                           const double* __restrict__ val, const double* __restrict__ x,
                                           double* __restrict__ y) {
  const int l = (threadIdx.x & 31) % K;
  double s = 0.0;
  for (int j0 = d.b; j0 < d.e; j0 += K * U) {
    const int nu = min(U, (d.e - j0 + K - 1) / K);  // passes this row still needs, uniform in the group
    int cc[U];
    double vv[U], xv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int j = j0 + l + u * K;
      const bool in = u < nu && j < d.e;
      cc[u] = in ? (K == 1 ? __ldg(col + j) : mp::ld_col(col + j)) : -1;
      vv[u] = in ? (K == 1 ? __ldg(val + j) : mp::ld_val(val + j)) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) xv[u] = cc[u] >= 0 ? __ldg(x + cc[u]) : 0.0;
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (u < nu && cc[u] >= 0) s = fma(vv[u], xv[u], s);
  }
  if constexpr (K > 1) {
#pragma unroll
    for (int o = K / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, K);
  }
  if (d.r >= 0 && l == 0) y[d.r] = s;
}

__global__ void __launch_bounds__(kBinThreads) spmv_binned(const int* __restrict__ col, const double* __restrict__ val,
                                                           const double* __restrict__ x, double* __restrict__ y,
                                                           const int* __restrict__ srow, const int* __restrict__ sbeg,
                                                           const int* __restrict__ send,
                                                           const long long* __restrict__ meta) {
  pdl_begin();
  __shared__ long long sm[2 * kBins + 2];
  if (threadIdx.x < 2 * kBins + 2) sm[threadIdx.x] = meta[threadIdx.x];
  __syncthreads();
  const long long units = sm[2 * kBins + 1];
  const long long nwarps = (long long)gridDim.x * (kBinThreads / 32);
  long long u = (long long)blockIdx.x * (kBinThreads / 32) + threadIdx.x / 32;
  BinRow d = u < units ? bin_row(u, sm, srow, sbeg, send) : BinRow{0, -1, 0, 0};
  for (; u < units; u += nwarps) {
    // the next unit's rows load while this one is summed
    const BinRow dn = u + nwarps < units ? bin_row(u + nwarps, sm, srow, sbeg, send) : BinRow{0, -1, 0, 0};
    switch (kBinLanes[d.c] * 16 + kBinU[d.c]) {  // (lanes, nonzeros per lane and pass)
      case 16 + 2: binned_row<1, 2>(d, col, val, x, y); break;
      case 16 + 4: binned_row<1, 4>(d, col, val, x, y); break;
      case 16 + 8: binned_row<1, 8>(d, col, val, x, y); break;
      case 32 + 8: binned_row<2, 8>(d, col, val, x, y); break;
      case 64 + 8: binned_row<4, 8>(d, col, val, x, y); break;
      case 128 + 8: binned_row<8, 8>(d, col, val, x, y); break;
      case 256 + 8: binned_row<16, 8>(d, col, val, x, y); break;
      default: binned_row<32, 8>(d, col, val, x, y); break;
    }
    d = dn;
  }
}

int launch_binned(int64_t rows, const int* rp, const int* c, const double* v, const double* x, double* y,
                  void* workspace, size_t workspace_bytes, cudaStream_t s) {
  if (!workspace || workspace_bytes < bin_workspace(rows)) return AR_ERR_ARG;
  if (rows > 0x7fffffffLL) return AR_ERR_ARG;
  static const int resident = [] {  // one wave of the persistent kernel
    int r = 0;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r, spmv_binned, kBinThreads, 0) == cudaSuccess && r > 0
               ? r
               : 1;
  }();
  const int64_t nblk = ceil_div(rows, kBinRows);
  const BinWs w = bin_ws(workspace, rows);
  spmv_bin_count<<<(unsigned)nblk, kBinThreads, 0, s>>>(rows, rp, w.counts);
  if (launch_status() != AR_OK) return AR_ERR_CUDA;
  int rc = launch_pdl(spmv_bin_scan, dim3(1), dim3(kBinThreads), 0, s, (int)nblk, w.counts, w.meta);
  if (rc == AR_OK)
    rc = launch_pdl(spmv_bin_scatter, dim3((unsigned)nblk), dim3(kBinThreads), 0, s, rows, rp,
                    (const int*)w.counts, (const long long*)w.meta, w.row, w.beg, w.end);
  if (rc != AR_OK) return rc;
  return launch_pdl(spmv_binned, dim3((unsigned)(device_sms() * resident)), dim3(kBinThreads), 0, s, c, v, x, y,
                    (const int*)w.row, (const int*)w.beg, (const int*)w.end, (const long long*)w.meta);
}

// ------------------------------------------------------------ features
constexpr int kFeatBlocks = 592;  // 4 per SM on B300

__global__ void __launch_bounds__(256) csr_stats_partial(int64_t rows, const int* __restrict__ rowptr,
                                                         long long* __restrict__ part) {
  __shared__ long long s1[8], s2[8];
  __shared__ int smax[8];
  long long a = 0, q = 0;
  int m = 0;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += (int64_t)gridDim.x * blockDim.x) {
    const int len = __ldg(rowptr + r + 1) - __ldg(rowptr + r);
    a += len;
    q += (long long)len * len;
    m = max(m, len);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    q += __shfl_xor_sync(0xffffffffu, q, o);
    m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  }
  const int w = threadIdx.x / 32;
  if ((threadIdx.x & 31) == 0) {
    s1[w] = a;
    s2[w] = q;
    smax[w] = m;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    long long A = 0, Q = 0;
    int M = 0;
    for (int k = 0; k < 8; ++k) {
      A += s1[k];
      Q += s2[k];
      M = max(M, smax[k]);
    }
    part[3 * blockIdx.x] = A;
    part[3 * blockIdx.x + 1] = Q;
    part[3 * blockIdx.x + 2] = M;
  }
}

// Integer sums are exact, so the result does not depend on the reduction
// order; mean and variance are formed once in float64.
__global__ void csr_stats_final(int64_t rows, int nparts, const long long* __restrict__ part,
                                float* __restrict__ out5) {
  __shared__ long long s1[256], s2[256], sm[256];
  long long a = 0, q = 0, m = 0;
  for (int k = threadIdx.x; k < nparts; k += blockDim.x) {
    a += part[3 * k];
    q += part[3 * k + 1];
    m = max(m, part[3 * k + 2]);
  }
  s1[threadIdx.x] = a;
  s2[threadIdx.x] = q;
  sm[threadIdx.x] = m;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      s1[threadIdx.x] += s1[threadIdx.x + o];
      s2[threadIdx.x] += s2[threadIdx.x + o];
      sm[threadIdx.x] = max(sm[threadIdx.x], sm[threadIdx.x + o]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double n = (double)rows;
    const double mean = rows > 0 ? (double)s1[0] / n : 0.0;
    const double var = rows > 0 ? fmax((double)s2[0] / n - mean * mean, 0.0) : 0.0;
    out5[0] = (float)rows;
    out5[1] = (float)s1[0];
    out5[2] = (float)mean;
    out5[3] = (float)var;
    out5[4] = (float)sm[0];
  }
}

constexpr int kNumVariants = kSpmvVariants;
const char* const kNames[kNumVariants] = {"spmv_thread_row", "spmv_warp_row", "spmv_vec2",
                                          "spmv_vec4",       "spmv_vec8",     "spmv_vec16",
                                          "spmv_merge_path", "spmv_df_merge_path", "spmv_binned"};

template <int K>
int launch_vector(int64_t rows, const int* rp, const int* c, const double* v, const double* x, double* y,
                  cudaStream_t s) {
  const int64_t grid = ceil_div(rows * K, 256);
  if (grid > 0x7fffffffLL) return AR_ERR_ARG;
  spmv_vector<K><<<(unsigned)grid, 256, 0, s>>>(rows, rp, c, v, x, y);
  return launch_status();
}

}  // namespace

int spmv_num_variants() { return kNumVariants; }

int spmv_variant_name(int v, char* buf, int len) {
  if (v < 0 || v >= kNumVariants || !buf || len <= 0) return AR_ERR_ARG;
  snprintf(buf, (size_t)len, "%s", kNames[v]);
  return AR_OK;
}

int spmv_launch(void* args, int variant, double, void* stream, void*) {
  const ar_spmv_args* a = static_cast<const ar_spmv_args*>(args);
  if (!a) return AR_ERR_ARG;
  return ar_spmv(variant, a->rows, a->nnz, a->rowptr, a->col, a->val, a->x, a->y, a->workspace,
                 a->workspace_bytes, stream);
}

}  // namespace ar

using namespace ar;

extern "C" int ar_spmv_workspace_bytes(int variant, int64_t rows, int64_t nnz, size_t* bytes) {
  if (variant < 0 || variant >= kNumVariants || rows < 0 || nnz < 0 || !bytes) return AR_ERR_ARG;
  *bytes = variant == 8 ? bin_workspace(rows) : variant >= 6 ? mp_workspace(rows, nnz) : 0;
  return AR_OK;
}

extern "C" int ar_spmv(int variant, int64_t rows, int64_t nnz, const int32_t* rowptr, const int32_t* col,
                       const double* val, const double* x, double* y, void* workspace, size_t workspace_bytes,
                       void* stream) {
  if (variant < 0 || variant >= kNumVariants || rows < 0 || nnz < 0 || nnz > 0x7fffffffLL) return AR_ERR_ARG;
  if (rows == 0) return AR_OK;
  if (!rowptr || !y || (nnz > 0 && (!col || !val || !x))) return AR_ERR_ARG;
  cudaStream_t s = as_stream(stream);
  const int* rp = reinterpret_cast<const int*>(rowptr);
  const int* c = reinterpret_cast<const int*>(col);
  switch (variant) {
    case 0: {
      spmv_thread_row<<<(unsigned)ceil_div(rows, 256), 256, 0, s>>>(rows, rp, c, val, x, y);
      return launch_status();
    }
    case 1: return launch_vector<32>(rows, rp, c, val, x, y, s);
    case 2: return launch_vector<2>(rows, rp, c, val, x, y, s);
    case 3: return launch_vector<4>(rows, rp, c, val, x, y, s);
    case 4: return launch_vector<8>(rows, rp, c, val, x, y, s);
    case 5: return launch_vector<16>(rows, rp, c, val, x, y, s);
    case 8: return launch_binned(rows, rp, c, val, x, y, workspace, workspace_bytes, s);
    default: {
      if (!workspace || workspace_bytes < mp_workspace(rows, nnz)) return AR_ERR_ARG;
      const int64_t nb = ceil_div(rows + nnz, kMpPerBlock);
      if (nb > 0x7ffffffeLL) return AR_ERR_ARG;
      uintptr_t p = (reinterpret_cast<uintptr_t>(workspace) + 255) & ~uintptr_t(255);
      int64_t* start_row = reinterpret_cast<int64_t*>(p);
      int64_t* carry_row = start_row + (nb + 1);
      double* carry_val = reinterpret_cast<double*>(carry_row + nb);
      spmv_mp_partition<<<(unsigned)ceil_div(nb + 1, 256), 256, 0, s>>>(rows, nnz, (int)nb, rp, start_row);
      if (launch_status() != AR_OK) return AR_ERR_CUDA;
      const int rc = launch_pdl(variant == 6 ? spmv_mp_main<false> : spmv_mp_main<true>, dim3((unsigned)nb),
                                dim3(kMpThreads), 0, s, rows, nnz, rp, c, val, x, y, start_row, carry_row, carry_val);
      if (rc != AR_OK) return rc;
      return launch_pdl(spmv_mp_fixup, dim3((unsigned)ceil_div(nb, 256)), dim3(256), 0, s, (int)nb, carry_row,
                        carry_val, y);
    }
  }
}

namespace ar {
namespace {

// Memory-side floor of a CSR SpMV: every nonzero's column and value are
// streamed and x[col] gathered, 8 nonzeros per thread in flight, with no row
// logic and no float64 arithmetic (the loaded bits are XORed into an integer
// that is stored only if it matches a constant, which keeps the loads live).
__global__ void __launch_bounds__(256) spmv_gather_floor(int64_t nnz, const int* __restrict__ col,
                                                         const double* __restrict__ val,
                                                         const double* __restrict__ x,
                                                         unsigned long long* __restrict__ sink) {
  unsigned long long acc = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
#pragma unroll 8
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nnz; j += stride) {
    const int c = __ldg(col + j);
    acc += (unsigned long long)__double_as_longlong(__ldg(val + j)) ^
           (unsigned long long)__double_as_longlong(__ldg(x + c));
  }
  if (acc == 0x5bd1e9955bd1e995ull) *sink = acc;
}

}  // namespace
}  // namespace ar

extern "C" int ar_spmv_gather_floor(int64_t nnz, const int32_t* col, const double* val, const double* x,
                                    void* sink8, void* stream) {
  using namespace ar;
  if (nnz < 0 || nnz > 0x7fffffffLL || (nnz > 0 && (!col || !val || !x || !sink8))) return AR_ERR_ARG;
  if (nnz == 0) return AR_OK;
  spmv_gather_floor<<<(unsigned)(device_sms() * 4), 256, 0, as_stream(stream)>>>(
      nnz, reinterpret_cast<const int*>(col), val, x, static_cast<unsigned long long*>(sink8));
  return launch_status();
}

extern "C" int ar_csr_features_workspace_bytes(int64_t rows, size_t* bytes) {
  if (rows < 0 || !bytes) return AR_ERR_ARG;
  *bytes = (size_t)kFeatBlocks * 3 * sizeof(long long);
  return AR_OK;
}

extern "C" int ar_csr_features(int64_t rows, const int32_t* rowptr, float* out5, void* workspace,
                               size_t workspace_bytes, void* stream) {
  if (rows < 0 || !rowptr || !out5) return AR_ERR_ARG;
  if (!workspace || workspace_bytes < (size_t)kFeatBlocks * 3 * sizeof(long long)) return AR_ERR_ARG;
  cudaStream_t s = as_stream(stream);
  long long* part = static_cast<long long*>(workspace);
  csr_stats_partial<<<kFeatBlocks, 256, 0, s>>>(rows, reinterpret_cast<const int*>(rowptr), part);
  csr_stats_final<<<1, 256, 0, s>>>(rows, kFeatBlocks, part, out5);
  return launch_status();
}

// ------------------------------------------------------------ no-allocation entry point
// Merge-path SpMV whose scratch (partition rows and per-block carries) lives
// in a fixed device array compiled into this library, for callers that must
// not allocate device memory.  The array exists on every GPU that loads the
// library and is held until the process exits.
namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)AR_SPMV_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_spmv_scratch[kNoAllocScratchBytes];
// Layout for nb path blocks: start_row int64[nb + 1], carry_row int64[nb],
// carry_val double[nb] = 24 nb + 8 bytes.  The header's capacity must be the
// largest path whose block count fits that layout in the array.
static_assert(AR_SPMV_NOALLOC_MAX_PATH ==
                  (long long)((kNoAllocScratchBytes - 8) / 24) * (long long)kMpPerBlock,
              "AR_SPMV_NOALLOC_MAX_PATH out of step with the merge-path block size or scratch layout");

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_spmv_scratch on the current device, looked up once per
// device (in host code the symbol names a host-side stand-in, not device
// memory).  Returns nullptr if the lookup fails.  The cached address belongs
// to the device's primary context: it does not survive cudaDeviceReset, after
// which this entry point must not be called again in the process.
void* scratch_on_current_device() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_spmv_scratch) != cudaSuccess) return nullptr;
    g_scratch_ptr[dev] = p;
  }
  return g_scratch_ptr[dev];
}

}  // namespace

extern "C" int ar_spmv_merge_path_noalloc(int64_t rows, int64_t nnz, const int32_t* rowptr, const int32_t* col,
                                          const double* val, const double* x, double* y, void* stream) {
  if (rows < 0 || nnz < 0 || nnz > 0x7fffffffLL) return AR_ERR_ARG;
  if (rows == 0) return AR_OK;
  if (!rowptr || !y || (nnz > 0 && (!col || !val || !x))) return AR_ERR_ARG;
  // bound each term before forming the sum, so the sum cannot overflow
  constexpr int64_t kMax = (int64_t)AR_SPMV_NOALLOC_MAX_PATH;
  if (rows > kMax || nnz > kMax - rows) {
    fprintf(stderr,
            "ar_spmv_merge_path_noalloc: rows + nnz >= %lld exceeds the fixed scratch limit %lld; "
            "use ar_spmv with a caller-provided workspace\n",
            (long long)(rows > kMax ? rows : rows + nnz), (long long)kMax);
    return AR_ERR_ARG;
  }
  void* base = scratch_on_current_device();
  if (!base) return AR_ERR_CUDA;
  const int64_t nb = ceil_div(rows + nnz, kMpPerBlock);
  // every scratch word the kernels read is written earlier in the same call:
  // no clearing is needed between calls
  int64_t* start_row = static_cast<int64_t*>(base);
  int64_t* carry_row = start_row + (nb + 1);
  double* carry_val = reinterpret_cast<double*>(carry_row + nb);
  cudaStream_t s = as_stream(stream);
  const int* rp = reinterpret_cast<const int*>(rowptr);
  const int* c = reinterpret_cast<const int*>(col);
  spmv_mp_partition<<<(unsigned)ceil_div(nb + 1, 256), 256, 0, s>>>(rows, nnz, (int)nb, rp, start_row);
  if (launch_status() != AR_OK) return AR_ERR_CUDA;
  const int rc = launch_pdl(spmv_mp_main<false>, dim3((unsigned)nb), dim3(kMpThreads), 0, s, rows, nnz, rp, c, val,
                            x, y, start_row, carry_row, carry_val);
  if (rc != AR_OK) return rc;
  return launch_pdl(spmv_mp_fixup, dim3((unsigned)ceil_div(nb, 256)), dim3(256), 0, s, (int)nb, carry_row, carry_val,
                    y);
}

namespace ar {
AR_CHECK_READER(chk_read_spmv)
}  // namespace ar
