// Merge-path CSR SpMV on one path block (internal): shared by the stand-alone
// merge-path variants and the mixed-stream executor.
//
// Merge path (Merrill & Garland, SC'16): the merge of the row-end list with
// the nonzero indices is a path of rows + nnz items; item d at path
// coordinate (i, d - i) either consumes the end of row i or nonzero d - i.
// The path is cut into blocks of kPerBlock items and each block into kItems
// items per thread, so every thread does the same work whatever the row
// lengths.
//
// One block runs in two phases.  Phase 1 (block-wide, coalesced, loads
// batched): the products val_j * x[col_j] of the block's nonzeros and its row
// ends go to shared memory.  Phase 2: each thread walks its items over shared
// memory only, in block-relative 32-bit coordinates, summing products and
// closing rows.  Threads that end inside the same open row form a run; a
// segmented scan leaves the run's total with its last thread, which adds it
// to the row, or hands it to the caller as the block's carry when the run
// reaches the end of the block.
//
// DF: the products are float pairs (operands split by prod_split, product by
// FMA without the lo x lo term) summed by pair_add, so the float64 pipe only
// converts finished rows; a block with an operand outside the split range or
// a non-finite pair sum redoes both phases in float64.
#pragma once

#include "common.cuh"
#include "pairs.cuh"

namespace ar {
namespace mp {

constexpr int kThreads = 256;
constexpr int kItems = 16;                    // path items per thread
constexpr int kPerBlock = kThreads * kItems;  // 4096
// Products (8 bytes each, float64 or a float pair) and the relative row ends
// (4 bytes each, plus a sentinel): nonzeros + rows of a block are at most
// kPerBlock, so 8 * kPerBlock + 8 bytes suffice.
constexpr int kStageBytes = 8 * kPerBlock + 16;
constexpr int kSmemBytes = kStageBytes + kThreads * 16;  // + open row and partial sum per thread
constexpr int kBatch = 8;                                // nonzeros whose loads a thread has in flight

__device__ __forceinline__ double ld_val(const double* p) {
  double v;
  asm volatile("ld.global.nc.L1::no_allocate.f64 %0, [%1];" : "=d"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ int ld_col(const int* p) {
  int v;
  asm volatile("ld.global.nc.L1::no_allocate.b32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}

// Rows consumed at path diagonal d (coordinate (i, d - i)), searched in [lo, hi].
__device__ __forceinline__ int64_t search(int64_t d, int64_t lo, int64_t hi, const int* __restrict__ rowptr,
                                          int64_t nnz) {
  lo = max(lo, d - nnz);
  hi = min(hi, d);
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if ((int64_t)__ldg(rowptr + mid + 1) <= d - mid - 1)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

// search(d, 0, rows, ...) by one warp (every lane returns the result): the
// rows consumed at path diagonal d, the smallest i in [max(0, d - nnz), min(rows, d)] with
// rowptr[i + 1] + i + 1 > d (the upper end if none).  Each step probes 32
// evenly spaced points of the range and keeps the part between the last
// probe below d and the first above, so a range of n rows takes about
// log_33 n dependent loads instead of log_2 n.
__device__ __forceinline__ int64_t search_warp(int64_t d, int64_t rows, const int* __restrict__ rowptr,
                                               int64_t nnz) {
  const int lane = threadIdx.x & 31;
  int64_t lo = max((int64_t)0, d - nnz), hi = min(rows, d);
  while (hi - lo > 32) {
    const int64_t n = hi - lo;
    const int64_t q = lo + (int64_t)(lane + 1) * n / 33;  // lo < q < hi
    const bool above = (int64_t)__ldg(rowptr + q + 1) > d - q - 1;
    const unsigned m = __ballot_sync(0xffffffffu, above);
    const int k = m ? __ffs(m) - 1 : 32;
    const int64_t qk = __shfl_sync(0xffffffffu, q, k & 31), qp = __shfl_sync(0xffffffffu, q, (k + 31) & 31);
    if (k == 32) {
      lo = qp + 1;  // every probe below: the answer lies past the last one
    } else {
      hi = qk;
      if (k > 0) lo = qp + 1;
    }
  }
  const int64_t q = lo + lane;
  const bool above = q < hi && (int64_t)__ldg(rowptr + q + 1) > d - q - 1;
  const unsigned m = __ballot_sync(0xffffffffu, above);
  return m ? lo + __ffs(m) - 1 : hi;
}

// Phase 1: products of nonzeros j0 + z, z < Z.  Thread t takes z = t,
// t + 256, ...; the column and value loads of a batch are issued together,
// then its x gathers.  Returns false if an operand is outside the float-pair
// split range (PAIRS only).
template <bool PAIRS, int B = kBatch>
__device__ __forceinline__ bool stage_products(int Z, int64_t j0, int64_t nnz, const int* __restrict__ col,
                                               const double* __restrict__ val, const double* __restrict__ x,
                                               double* sprod) {
  bool ok = true;
  const int t = threadIdx.x;
#pragma unroll
  for (int b0 = 0; b0 < kItems; b0 += B) {
    int cc[B];
    double vv[B];
#pragma unroll
    for (int u = 0; u < B; ++u) {
      const int z = t + (b0 + u) * kThreads;
      if (z < Z) {
        const bool in = AR_CHK(j0 + z >= 0 && j0 + z < nnz);
        cc[u] = in ? ld_col(col + j0 + z) : 0;
        vv[u] = in ? ld_val(val + j0 + z) : 0.0;
      }
    }
#pragma unroll
    for (int u = 0; u < B; ++u) {
      const int z = t + (b0 + u) * kThreads;
      if (z < Z && AR_CHK(cc[u] >= 0 && 8 * z + 8 <= kStageBytes)) {
        const double xv = __ldg(x + cc[u]);
        if constexpr (PAIRS) {
          float vh, vl, xh, xl;
          ok &= prod_split(vv[u], vh, vl);
          ok &= prod_split(xv, xh, xl);
          const float p = vh * xh;
          float pe = fmaf(vh, xh, -p);
          pe = fmaf(vh, xl, pe);
          pe = fmaf(vl, xh, pe);
          reinterpret_cast<float2*>(sprod)[z] = make_float2(p, pe);
        } else {
          sprod[z] = vv[u] * xv;
        }
      }
    }
  }
  return ok;
}

__device__ __forceinline__ bool pair_finite(float S, float C) {
  return (__float_as_uint(S) & 0x7f800000u) != 0x7f800000u && (__float_as_uint(C) & 0x7f800000u) != 0x7f800000u;
}

// Path block starting at diagonal db with i0 = rows consumed at db and
// i1 = rows consumed at its end; kThreads threads; smem: kSmemBytes of
// 16-byte aligned shared memory.  Writes y for every row closed in the block
// (the run totals included) and sets *carry_row / *carry_val to the open row
// continuing into the next block and its partial sum, or *carry_row = -1.
template <bool DF, int B = kBatch>
__device__ void block(int64_t rows, int64_t nnz, const int* __restrict__ rowptr, const int* __restrict__ col,
                      const double* __restrict__ val, const double* __restrict__ x, double* __restrict__ y,
                      int64_t db, int64_t i0, int64_t i1, int64_t* carry_row, double* carry_val,
                      unsigned char* smem) {
  int64_t* srow = reinterpret_cast<int64_t*>(smem + kStageBytes);
  double* sval = reinterpret_cast<double*>(smem + kStageBytes + 8 * kThreads);
  const int t = threadIdx.x;
  const int64_t de = min(db + kPerBlock, rows + nnz);
  const int64_t j0 = db - i0, j1 = de - i1;
  const int Z = (int)(j1 - j0);                                     // nonzeros of the block
  const int NR = i0 < rows ? (int)(min(i1, rows - 1) - i0 + 1) : 0;  // row ends of rows i0 .. min(i1, rows-1)
  double* sprod = reinterpret_cast<double*>(smem);
  int* send = reinterpret_cast<int*>(smem + 8 * (size_t)Z);
  // relative row ends rowptr[i0 + q + 1] - j0 >= 0; the sentinel stops the
  // walk at the last row of the matrix
  for (int q = t; q <= NR; q += kThreads)
    if (AR_CHK(8 * Z + 4 * (q + 1) <= kStageBytes && (q == NR || i0 + q + 1 <= rows)))
      send[q] = q < NR ? (int)(__ldg(rowptr + i0 + q + 1) - j0) : 0x7fffffff;
  bool native = !DF;
  if constexpr (!DF) {
    __syncthreads();  // the row ends are read by every thread's search below
  } else {
    native = __syncthreads_or(!stage_products<true, B>(Z, j0, nnz, col, val, x, sprod));  // also publishes the row ends
  }
  const int64_t d0 = min(db + (int64_t)t * kItems, de);
  const int n = (int)(min(d0 + kItems, de) - d0);
  // this thread's start on the path, searched over the staged row ends
  int64_t lo = max(i0, d0 - nnz), hi = min(i1, d0);
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if ((AR_CHK(mid - i0 >= 0 && mid - i0 <= NR) ? (int64_t)send[mid - i0] : 0) + j0 <= d0 - mid - 1)
      lo = mid + 1;
    else
      hi = mid;
  }
  const int ir0 = (int)(lo - i0), jr0 = (int)(d0 - lo - j0);
  for (int pass = 0; pass < 2; ++pass) {
    if (native) {
      if (DF) __syncthreads();  // the float-pair products are read no more
      stage_products<false, B>(Z, j0, nnz, col, val, x, sprod);
    }
    __syncthreads();
    int ir = ir0, jr = jr0;
    int re = AR_CHK(ir >= 0 && ir <= NR) ? send[ir] : 0x7fffffff;
    bool finite = true;
    if (native) {
      double s = 0.0;
      for (int it = 0; it < n; ++it) {
        if (jr >= re) {  // consume the end of row i0 + ir
          if (AR_CHK(i0 + ir < rows)) y[i0 + ir] = s;
          s = 0.0;
          ++ir;
          re = AR_CHK(ir <= NR) ? send[ir] : 0x7fffffff;
        } else {          // consume nonzero j0 + jr
          s += AR_CHK(jr >= 0 && jr < Z) ? sprod[jr] : 0.0;
          ++jr;
        }
      }
      sval[t] = s;
    } else {
      float S = 0.f, C = 0.f;
      for (int it = 0; it < n; ++it) {
        if (jr >= re) {  // the pair goes to y as is; converted below, by all threads at once
          finite &= pair_finite(S, C);
          if (AR_CHK(i0 + ir < rows)) reinterpret_cast<float2*>(y)[i0 + ir] = make_float2(S, C);
          S = C = 0.f;
          ++ir;
          re = AR_CHK(ir <= NR) ? send[ir] : 0x7fffffff;
        } else {
          const float2 pp =
              AR_CHK(jr >= 0 && jr < Z) ? reinterpret_cast<const float2*>(sprod)[jr] : make_float2(0.f, 0.f);
          ++jr;
          pair_add(S, C, pp.x, pp.y);
        }
      }
      finite &= pair_finite(S, C);
      sval[t] = f2d_bits(S) + f2d_bits(C);
    }
    // open row at the end of this thread's range
    srow[t] = (n > 0 && i0 + ir < rows) ? i0 + ir : -1;
    if (!DF || native || !__syncthreads_or(!finite)) break;
    native = true;  // a pair sum overflowed: redo the block in float64
  }
  if (DF && !native) {
    // rows i0 .. i1-1 closed in this block hold float pairs: convert them with
    // every lane busy (a float64 add costs its whole warp on the float64 pipe)
    __syncthreads();
    for (int64_t i = i0 + t; i < i1; i += kThreads) {
      if (!AR_CHK(i < rows)) continue;
      const float2 pp = reinterpret_cast<const float2*>(y)[i];
      y[i] = f2d_bits(pp.x) + f2d_bits(pp.y);
    }
  }
  // segmented inclusive scan of the partial sums over runs of equal open rows
  // (fixed tree order): each run's total ends in its last thread
  const int64_t r = srow[t];
  double v = sval[t];
#pragma unroll
  for (int off = 1; off < kThreads; off <<= 1) {
    __syncthreads();
    const double o = (t >= off && srow[t - off] == r) ? sval[t - off] : 0.0;
    __syncthreads();
    v += o;
    sval[t] = v;
  }
  if (t == 0) *carry_row = -1;
  __syncthreads();
  if (r >= 0 && (t == kThreads - 1 || srow[t + 1] != r)) {
    // the next thread consumed the row's end and wrote y[r] in phase 2
    const bool closed_here = t + 1 < kThreads && min(db + (int64_t)(t + 1) * kItems, de) < de;
    if (closed_here) {
      if (AR_CHK(r < rows)) y[r] += v;
    } else {
      *carry_row = r;
      *carry_val = v;
    }
  }
}

}  // namespace mp
}  // namespace ar
