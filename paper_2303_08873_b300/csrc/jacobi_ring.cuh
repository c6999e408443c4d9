// One Jacobi sweep over a BX x BY x (ke - kb) tile whose planes stream through
// a ring of shared-memory slots by 16-byte cp.async (internal): used by the
// stand-alone float-pair kernel when tensor copies cannot be used (odd N:
// rows are not 16-byte aligned) and by every Jacobi tile of the mixed-stream
// executor.
//
// Slot rows hold x from i0 - 2 - o to i0 + BX + 1 - o in 16-byte chunks that
// start at an even element index of the flat N^3 array; o = 0 for even N and
// o = (k + y) & 1 for odd N (the parity of row (k, y)'s first element), so
// element x of row (k, y) sits at column x - i0 + 2 + o.  A chunk half
// outside the grid reads as zero: chunks wholly outside are zero-filled by
// the copy, a chunk whose upper half lies past the row's end copies 8 bytes,
// and a chunk whose lower half lies before the row's start (only possible
// when o = 1, so that half is the previous row's last element, in bounds) is
// copied whole and that half zeroed by its copier after landing.  Float-pair
// sweeps with float64 input split every landed chunk in place the same way.
// Every value is loaded once per tile; the z neighbours come from the ring.
#pragma once

#include "common.cuh"
#include "pairs.cuh"
#include "tma.cuh"

namespace ar {

constexpr int kRingPlanes = 8;
constexpr int kRingChunks = 2;  // 16-byte chunks per thread and plane, at most (nchunk <= 2 * threads)

// Shared memory of the ring for a BX x BY tile.
__host__ __device__ constexpr int ring_smem_bytes(int BX, int BY) { return kRingPlanes * (BX + 4) * (BY + 2) * 8; }

// ST: the stencil (stencil_f64 / stencil_pair of pairs.cuh) with its
// coefficients cf.  src: float64 (pair_math false, or src_pairs false) or
// float pairs; dst: float pairs if dst_pairs, else float64.  Threads: blockDim.x >= BX * BY
// and 2 * blockDim.x >= (BX + 4) (BY + 2) / 2 (the chunks of one plane).
// A float-pair sweep with float64 input and float64 output redoes in float64
// every point whose inputs lie outside the float-pair range; with pairs out,
// such inputs set *flag instead.  Buffers 16-byte aligned.
template <int ST>
__device__ __forceinline__ void jacobi_ring_tile(int N, int BX, int BY, int bx, int by, int kb, int ke,
                                                 const double* src, double* dst, bool pair_math, bool src_pairs,
                                                 bool dst_pairs, int* flag, unsigned char* smraw,
                                                 const StencilCoef& cf) {
  const int nthr = blockDim.x;
  const int i0 = bx * BX, j0 = by * BY;
  const int PX = BX + 4, PL = PX * (BY + 2);
  const int chunks_row = PX / 2, nchunk = chunks_row * (BY + 2);
  double* ring = reinterpret_cast<double*>(smraw);
  const bool active = threadIdx.x < BX * BY;
  const int lx = threadIdx.x % BX, ly = threadIdx.x / BX;
  const int i = i0 + lx, j = j0 + ly;
  const bool inside = active && i < N && j < N;
  const int64_t NN = (int64_t)N * N;
  const bool odd = N & 1;
  const bool split = pair_math && !src_pairs;
  const bool may_zero = odd && i0 == 0;
  bool marker = false;
  // This thread's chunks (at most kRingChunks), fixed for the tile: slot
  // offset, row y, and for each row parity o the flat offset y*N + x0 and the
  // bytes to copy (16, 8 or 0 by which halves lie inside the row).
  // (per parity: suffix 0 / 1; selected by value, not by index, so the
  // arrays stay in registers)
  int soff[kRingChunks], cy[kRingChunks], cb0[kRingChunks], cb1[kRingChunks];
  bool z0[kRingChunks], z1[kRingChunks];  // a copied lower half to zero (x0 = -1)
  int64_t cxy0[kRingChunks];              // y*N + x0 for parity 0; parity 1 is one less
  int nmine = 0;
#pragma unroll
  for (int m = 0; m < kRingChunks; ++m) {
    const int c = threadIdx.x + m * nthr;
    const int row = c / chunks_row, cx = c - row * chunks_row;
    if (c < nchunk) nmine = m + 1;
    soff[m] = row * PX + 2 * cx;
    const int y = j0 - 1 + row;
    cy[m] = y;
    const bool yin = y >= 0 && y < N;
    const int x0 = i0 - 2 + 2 * cx;  // parity 0; parity 1 starts one element earlier
    const bool a0 = yin && x0 >= 0 && x0 < N, a1 = yin && x0 + 1 >= 0 && x0 + 1 < N;
    const bool b0 = yin && x0 - 1 >= 0 && x0 - 1 < N;  // parity 1: halves x0 - 1, x0
    cb0[m] = a1 ? 16 : (a0 ? 8 : 0);
    cb1[m] = a0 ? 16 : (b0 ? 8 : 0);
    z0[m] = !a0 && a1;
    z1[m] = !b0 && a0;
    cxy0[m] = (int64_t)y * N + x0;  // + kp * N^2
  }
  // plane kp (kb-1 <= kp) lives in slot (kp - kb + 1) % kRingPlanes
  auto slot_of = [&](int kp) { return (kp - kb + 1) % kRingPlanes; };
  // planes are issued in increasing order: kp * N^2 advances by N^2 per call
  const double* plane_src = src + (int64_t)(kb - 1) * NN;
  auto issue = [&](int kp) {
    if (kp <= ke) {
      const bool kin = kp >= 0 && kp < N;
      double* base = ring + slot_of(kp) * PL;
#pragma unroll
      for (int m = 0; m < kRingChunks; ++m) {
        if (m < nmine) {
          const bool o = odd && ((kp + cy[m]) & 1);
          const int bytes = kin ? (o ? cb1[m] : cb0[m]) : 0;
          const double* from = bytes ? plane_src + cxy0[m] - (o ? 1 : 0) : src;
          // destination inside the ring, source inside the grid for the bytes copied
          if (AR_CHK(slot_of(kp) * PL + soff[m] + 2 <= kRingPlanes * PL && soff[m] >= 0 &&
                     (from - src) >= 0 && (from - src) * 8 + bytes <= NN * N * 8))
            cp_async16(base + soff[m], from, bytes);
        }
      }
    }
    plane_src += NN;
    cp_async_commit();  // one group per plane, empty past ke, so the wait counts stay fixed
  };
  // after this thread's copies of plane kp have landed: zero a copied half
  // that lies before its row's start; split float64 values into pairs
  auto post = [&](int kp) {
    const bool kin = kp >= 0 && kp < N;
    double* base = ring + slot_of(kp) * PL;
#pragma unroll
    for (int m = 0; m < kRingChunks; ++m) {
      if (m < nmine && AR_CHK(slot_of(kp) * PL + soff[m] + 2 <= kRingPlanes * PL)) {
        double* e = base + soff[m];
        if (may_zero && kin && (((kp + cy[m]) & 1) ? z1[m] : z0[m])) e[0] = 0.0;
        if (split) {
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const float2 f = df_split(e[h]);
            marker |= (f.x != f.x);
            reinterpret_cast<float2*>(e)[h] = f;
          }
        }
      }
    }
  };
  const bool need_post = split || may_zero;
  for (int q = 0; q < kRingPlanes - 1; ++q) issue(kb - 1 + q);
  // running state of the compute: slots of planes kk-1, kk, kk+1, this row's
  // parity at plane kk, and the output offset of plane kk
  int sb = slot_of(kb - 1), sc = slot_of(kb), sa = slot_of(kb + 1);
  int o = odd ? ((kb + j) & 1) : 0;
  int64_t outo = (int64_t)kb * NN + (int64_t)j * N + i;
  const int rc = (ly + 1) * PX + lx + 2;
  for (int kk = kb; kk < ke; ++kk) {
    cp_async_wait<kRingPlanes - 4>();  // planes up to kk + 1 have landed (this thread's copies)
    if (need_post) {
      if (kk == kb) {
        post(kb - 1);
        post(kb);
      }
      post(kk + 1);
    }
    __syncthreads();
    issue(kk + kRingPlanes - 2);  // into the slot of plane kk - 2, read last in the previous step
    // every staged read inside the ring, the store inside the grid
    if (inside && AR_CHK(rc - PX - 1 >= 0 && rc + PX + 2 <= PL && outo >= 0 && outo < NN * N)) {
      // odd N: the neighbour rows (y +- 1 and planes k +- 1) have the other parity
      const int on = odd ? 1 - o : 0;
      const int c0 = sc * PL + rc + o;
      const int cs = sc * PL + rc - PX + on;
      const int cn = sc * PL + rc + PX + on;
      const int cb = sb * PL + rc + on;
      const int ca = sa * PL + rc + on;
      if (!pair_math) {
        const double* r = ring;
        double s = r[c0 - 1] + r[c0 + 1];
        s += r[cs];
        s += r[cn];
        s += r[cb];
        s += r[ca];
        dst[outo] = stencil_f64<ST>(r[c0], s, cf);
      } else {
        const float2* r = reinterpret_cast<const float2*>(ring);
        const float2 res = stencil_pair<ST>(r[c0], r[c0 - 1], r[c0 + 1], r[cs], r[cn], r[cb], r[ca], cf);
        if (dst_pairs) {
          reinterpret_cast<float2*>(dst)[outo] = res;
        } else {
          double dv = pair_to_double(res);
          if (split && (__double_as_longlong(dv) & 0x7fffffffffffffffLL) > 0x7ff0000000000000LL) {
            // an input outside the float-pair range: redo this point in float64
            // (L1-bypassing loads: src may have been written earlier in this launch)
            auto g = [&](int ii, int jj, int kq) {
              return ((unsigned)ii < (unsigned)N && (unsigned)jj < (unsigned)N && (unsigned)kq < (unsigned)N)
                         ? __ldcg(src + ((int64_t)kq * N + jj) * N + ii)
                         : 0.0;
            };
            double sd = g(i - 1, j, kk) + g(i + 1, j, kk);
            sd += g(i, j - 1, kk);
            sd += g(i, j + 1, kk);
            sd += g(i, j, kk - 1);
            sd += g(i, j, kk + 1);
            dv = stencil_f64<ST>(g(i, j, kk), sd, cf);
          }
          dst[outo] = dv;
        }
      }
    }
    sb = sc;
    sc = sa;
    sa = sa + 1 == kRingPlanes ? 0 : sa + 1;
    o ^= odd ? 1 : 0;
    outo += NN;
  }
  cp_async_wait<0>();  // no copy may land after the tile: the caller reuses the shared memory
  if (__syncthreads_or(dst_pairs && marker) && threadIdx.x == 0 && flag) atomicOr(flag, 1);
}

}  // namespace ar
