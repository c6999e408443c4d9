// 7-point 3D Jacobi variants (the stencil region; stand-in for the paper's
// Heat finite-difference benchmark, Table 3, adapted over block shapes as in
// Section 3.2.2).
//
//   out(i,j,k) = (W + E + S + N + D + U) / 6, zero outside [0,N)^3,
//   unknown (i,j,k) at (k*N + j)*N + i.
//
// Ideal traffic is 16 bytes per point per sweep (read once, write once).  On
// B300 the float64 pipe issues ~0.56e12 DFMA/s against 6.5e12 B/s of HBM, so
// the 6 float64 operations per point (5 adds, 1 multiply) bound the native
// families at ~1.5 TB/s.  The df family moves the arithmetic to the FP32 pipe
// in float-pair form (hi + lo, ~2^-46 relative) and keeps one float64 add per
// point.  Float64<->float32 conversions also issue on the float64 pipe on
// B300, so the df family converts with integer bit operations only.
//
// Families (variant = 4*family + shape; shapes 32x4, 32x8, 64x4, 128x2):
//   0 naive  one thread per point, 7 global loads through L1/L2
//   1 smem   2.5D: xy tile + halo in shared memory (double buffered, one
//            barrier per plane), z neighbours in a 3-register queue
//   2 tma    cp.async.bulk.tensor loads of (BX+4) x (BY+2) x 8-plane boxes
//            into a 3-slot ring with mbarrier completion; TMA zero fill
//            supplies the Dirichlet ghosts (also in z); two boxes in flight
//   3 df     as tma, plus an in-place conversion of each landed box from
//            float64 to float pairs; sums by TwoSum on the FP32 pipe
#define AR_TU 2
#include <cudaTypedefs.h>

#include <cstdio>
#include <mutex>
#include <type_traits>

#include "common.cuh"
#include "jacobi_ring.cuh"
#include "pairs.cuh"
#include "tma.cuh"

namespace ar {
namespace {

constexpr int kDZ = 4;     // planes per TMA box
// jacobi_tma_odd takes a plane's row-parity bundle from its index r inside
// the box (r & 1), which needs every box to start on a plane of the same
// parity: an even box depth.
static_assert(kDZ % 2 == 0, "odd-N tiles need an even box depth");
constexpr int kRing = 3;   // boxes resident per block
constexpr int kShapeX[4] = {32, 32, 64, 128};
constexpr int kShapeY[4] = {4, 8, 4, 2};
const char* const kFamily[4] = {"naive", "smem", "tma", "df"};

// ------------------------------------------------------------------ naive
template <int BX, int BY, int ST>
__global__ void __launch_bounds__(BX* BY) jacobi_naive(int N, const double* __restrict__ in,
                                                       double* __restrict__ out, StencilCoef cf) {
  pdl_begin();  // the previous sweep of the chain is complete and visible
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= N || j >= N) return;
  const int64_t NN = (int64_t)N * N;
  const int64_t c = k * NN + (int64_t)j * N + i;
  double s = (i > 0 ? in[c - 1] : 0.0) + (i < N - 1 ? in[c + 1] : 0.0);
  s += (j > 0 ? in[c - N] : 0.0);
  s += (j < N - 1 ? in[c + N] : 0.0);
  s += (k > 0 ? in[c - NN] : 0.0);
  s += (k < N - 1 ? in[c + NN] : 0.0);
  if (AR_CHK(c < NN * N)) out[c] = stencil_f64<ST>(ST == kHeat ? in[c] : 0.0, s, cf);
}

// ------------------------------------------------------------------ 2.5D smem
template <int BX, int BY, int ST>
__global__ void __launch_bounds__(BX* BY) jacobi_smem(int N, int KC, const double* __restrict__ in,
                                                      double* __restrict__ out, StencilCoef cf) {
  pdl_begin();  // the previous sweep of the chain is complete and visible
  __shared__ double tile[2][BY + 2][BX + 2];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int i = blockIdx.x * BX + tx, j = blockIdx.y * BY + ty;
  const int kb = blockIdx.z * KC;
  const int ke = min(N, kb + KC);
  const bool inside = i < N && j < N;
  const int64_t NN = (int64_t)N * N;
  const int64_t col = (int64_t)j * N + i;
  double below = (inside && kb > 0) ? in[(kb - 1) * NN + col] : 0.0;
  double cur = inside ? in[kb * NN + col] : 0.0;
  for (int k = kb; k < ke; ++k) {
    const int b = (k - kb) & 1;
    const double above = (inside && k + 1 < N) ? in[(k + 1) * NN + col] : 0.0;
    tile[b][ty + 1][tx + 1] = cur;
    if (tx == 0) tile[b][ty + 1][0] = at(in, N, i - 1, j, k);
    if (tx == BX - 1) tile[b][ty + 1][BX + 1] = at(in, N, i + 1, j, k);
    if (ty == 0) tile[b][0][tx + 1] = at(in, N, i, j - 1, k);
    if (ty == BY - 1) tile[b][BY + 1][tx + 1] = at(in, N, i, j + 1, k);
    __syncthreads();
    if (inside) {
      double s = tile[b][ty + 1][tx] + tile[b][ty + 1][tx + 2];
      s += tile[b][ty][tx + 1];
      s += tile[b][ty + 2][tx + 1];
      s += below;
      s += above;
      if (AR_CHK(k * NN + col < NN * N)) out[k * NN + col] = stencil_f64<ST>(cur, s, cf);
    }
    below = cur;
    cur = above;
  }
}

// ------------------------------------------------------------------ TMA ring
template <int BX, int BY>
struct TmaGeom {
  static constexpr int PX = BX + 4;              // x: 2 ghost columns each side (16-byte aligned x)
  static constexpr int PY = BY + 2;
  static constexpr int PLANE = PX * PY;          // elements per plane
  static constexpr int GROUP = PLANE * kDZ;      // elements per box
  static constexpr uint32_t BYTES = GROUP * 8u;
  // a tensor copy's shared-memory destination must be 128-byte aligned: slots
  // start at multiples of SLOT elements from the 128-byte aligned ring base
  static constexpr int SLOT = (GROUP + 15) / 16 * 16;
  static constexpr size_t SMEM = (size_t)kRing * SLOT * 8 + 128;
  static_assert(SLOT * 8 % 128 == 0, "TMA slots must stay 128-byte aligned");
};

// Sweep modes of the TMA kernel.  Buffers between the sweeps of one df call
// may hold float pairs (8 bytes per unknown, like a float64):
//   M_NATIVE  float64 in, float64 out, float64 arithmetic
//   M_DD      float64 in, float64 out, float-pair arithmetic; points whose
//             inputs are outside the float-pair range are redone in float64
//   M_DP      first sweep of a pair chain: float64 in, float pairs out; any
//             input outside the float-pair range sets *flag
//   M_PP      float pairs in, float pairs out  } when *flag is set these run
//   M_PD      float pairs in, float64 out      } the previous sweep in
//             float64 instead, from the alternate source (tmap_alt) to
//             out_alt, so the flagged chain ends one launch late (see the
//             catch-up kernel)
enum Mode { M_NATIVE = 0, M_DD = 1, M_DP = 2, M_PP = 3, M_PD = 4 };
// How a tma / df sweep stages its planes.
enum Staging { kStageSmem = 0, kStageTma = 1, kStageRing = 2, kStageTmaOdd = 3 };

template <int BX, int BY, int MODE, int ST>
__global__ void __launch_bounds__(BX* BY) jacobi_tma(const __grid_constant__ CUtensorMap tmap,
                                                     const __grid_constant__ CUtensorMap tmap_alt, int N, int KC,
                                                     const double* __restrict__ in, void* __restrict__ outv,
                                                     double* __restrict__ out_alt, int* status, int* flag,
                                                     StencilCoef cf) {
  pdl_begin();  // the previous sweep of the chain is complete and visible
  using G = TmaGeom<BX, BY>;
  extern __shared__ unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bars[kRing];
  // 128-byte aligned box ring; offsetting smem_raw itself (no integer round
  // trip) keeps the pointer in the shared window, so loads compile to LDS
  double* buf = reinterpret_cast<double*>(smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u));

  const int tid = threadIdx.x;
  const int tx = tid % BX, ty = tid / BX;
  const int i0 = blockIdx.x * BX, j0 = blockIdx.y * BY;
  const int kb = blockIdx.z * KC;
  const int kc = min(KC, N - kb);                 // output planes of this block
  const int ngroups = (kc + 2 + kDZ - 1) / kDZ;   // boxes covering planes kb-1 .. kb+kc
  // block-uniform: the flag was settled by an earlier launch on this stream
  const bool flagged = (MODE == M_PP || MODE == M_PD) && flag != nullptr && *flag != 0;
  const bool native = (MODE == M_NATIVE) || flagged;
  const bool split_boxes = !native && (MODE == M_DD || MODE == M_DP);
  const CUtensorMap* src_map = flagged ? &tmap_alt : &tmap;

  if (tid == 0) {
    for (int r = 0; r < kRing; ++r) mbar_init(smem_addr(&bars[r]), 1);
    mbar_fence_init();
  }
  __syncthreads();

  auto issue = [&](int g) {
    const int slot = g % kRing;
    const uint32_t bar = smem_addr(&bars[slot]);
    mbar_arrive_expect_tx(bar, G::BYTES);
    // float64 tensor copies: x even (16-byte start), a 128-byte aligned
    // destination inside the dynamic shared array
    if (AR_CHK(((i0 - 2) & 1) == 0 && (smem_addr(buf + (size_t)slot * G::SLOT) & 127u) == 0 &&
               in_dyn_smem(smem_raw, buf + (size_t)slot * G::SLOT, G::BYTES)))
      tma_load_3d(smem_addr(buf + (size_t)slot * G::SLOT), src_map, i0 - 2, j0 - 1, kb - 1 + g * kDZ, bar);
  };
  if (tid == 0)
    for (int g = 0; g < min(ngroups, kRing - 1); ++g) issue(g);

  const int i = i0 + tx, j = j0 + ty;
  const bool inside = i < N && j < N;
  const int64_t NN = (int64_t)N * N;
  const int64_t col = (int64_t)j * N + i;
  // the centre's neighbours +-1 and +-PX stay inside one staged plane
  const int c = AR_CHK(tx + 3 < G::PX && ty + 2 < G::PY) ? (ty + 1) * G::PX + tx + 2 : G::PX + 2;
  double* outd = flagged ? out_alt : static_cast<double*>(outv);
  float2* outp = static_cast<float2*>(outv);
  // z queue: the values of planes p-1 and p at this thread's column
  double dm = 0.0, d0 = 0.0;
  float2 fm = make_float2(0.f, 0.f), f0 = make_float2(0.f, 0.f);
  // output element of the next plane (one pointer per output format)
  double* od = outd + ((int64_t)kb * NN + col);
  float2* op = outp + ((int64_t)kb * NN + col);
  int g = 0;
  bool failed = false;
  // slot of box g and the mbarrier phase it completes, advanced per box
  int slot = 0, pslot = kRing - 1;
  uint32_t phase = 0;
  for (; g < ngroups; ++g, pslot = slot, slot = (slot + 1 == kRing) ? 0 : slot + 1, phase ^= (slot == 0)) {
    const bool ok = mbar_wait_bounded(smem_addr(&bars[slot]), phase);
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    double* box = buf + (size_t)slot * G::SLOT;
    const double* prev = buf + (size_t)pslot * G::SLOT;
    if (split_boxes) {
      bool marker = false;
#pragma unroll
      for (int e = tid; e < G::GROUP; e += BX * BY) {
        const float2 f = df_split(box[e]);
        marker |= (f.x != f.x);
        reinterpret_cast<float2*>(box)[e] = f;
      }
      if (__syncthreads_or(marker) && MODE == M_DP && tid == 0 && flag) atomicOr(flag, 1);
    }
    // Box g holds relative planes D*g .. D*g+D-1 (D = kDZ planes per box,
    // relative plane 0 = kb - 1), so it completes output planes
    // p = D*g-1 .. D*g+D-2; the centre plane of p is plane r-1 of this box, or
    // the last plane of the previous box for r = 0.  Unrolled, every
    // shared-memory offset below is a constant; the arithmetic kind and the
    // edge guards are hoisted out of the plane loop.
    auto planes = [&](auto native_c, auto guard_c) {
      constexpr bool NAT = decltype(native_c)::value;
      constexpr bool GUARD = decltype(guard_c)::value;
#pragma unroll
      for (int r = 0; r < kDZ; ++r) {
        const int p = g * kDZ - 1 + r;
        const bool live = !GUARD || (p >= 1 && p <= kc);  // block-uniform
        const int cp = (r == 0 ? (kDZ - 1) * G::PLANE : (r - 1) * G::PLANE) + c;
        if constexpr (NAT) {
          const double* pc = (r == 0 ? prev : box) + cp;
          const double up = box[r * G::PLANE + c];
          if (live) {
            double s = pc[-1] + pc[1];
            s += pc[-G::PX];
            s += pc[G::PX];
            s += dm;
            s += up;
            if (inside && AR_CHK(od - outd >= 0 && od - outd < NN * N)) *od = stencil_f64<ST>(pc[0], s, cf);
            od += NN;
          }
          dm = d0;
          d0 = up;
        } else {
          const float2* pc = reinterpret_cast<const float2*>(r == 0 ? prev : box) + cp;
          const float2 up = reinterpret_cast<const float2*>(box)[r * G::PLANE + c];
          if (live) {
            const float2 res = stencil_pair<ST>(pc[0], pc[-1], pc[1], pc[-G::PX], pc[G::PX], fm, up, cf);
            if (inside && AR_CHK(od - outd >= 0 && od - outd < NN * N && op - outp >= 0 && op - outp < NN * N)) {
              if constexpr (MODE == M_DP || MODE == M_PP) {  // pairs out (the native case is above)
                // stored unnormalised: the next sweep sums the hi parts exactly and
                // the lo parts in float, so |lo| of a few ulps of hi costs ~2^-46
                *op = res;
              } else {
                // a pairs -> float64 sweep only sees finite pairs (the first
                // sweep of the chain checked the range)
                double v = MODE == M_PD ? finite_pair_to_double(res) : pair_to_double(res);
                // NaN test on the bit pattern (a float64 compare would use the float64 pipe)
                if (MODE == M_DD && (__double_as_longlong(v) & 0x7fffffffffffffffLL) > 0x7ff0000000000000LL) {
                  // an input outside the float-pair range: redo in float64
                  const int k = kb + p - 1;
                  double sd = at(in, N, i - 1, j, k) + at(in, N, i + 1, j, k);
                  sd += at(in, N, i, j - 1, k);
                  sd += at(in, N, i, j + 1, k);
                  sd += at(in, N, i, j, k - 1);
                  sd += at(in, N, i, j, k + 1);
                  v = stencil_f64<ST>(at(in, N, i, j, k), sd, cf);
                }
                *od = v;
              }
            }
            if constexpr (MODE == M_DP || MODE == M_PP)
              op += NN;
            else
              od += NN;
          }
          fm = f0;
          f0 = up;
        }
      }
    };
    using T_ = std::true_type;
    using F_ = std::false_type;
    const bool guard = g == 0 || g * kDZ + kDZ - 2 > kc;
    if (native) {
      if (guard)
        planes(T_{}, T_{});
      else
        planes(T_{}, F_{});
    } else {
      if (guard)
        planes(F_{}, T_{});
      else
        planes(F_{}, F_{});
    }
    // every reader of box g-1 is past this barrier: its slot takes box g+2
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0 && g + kRing - 1 < ngroups) issue(g + kRing - 1);
  }
  if (failed) {
    if (tid == 0) {
      if (status) atomicExch(status, (int)AR_ERR_TIMEOUT);
      // drain the boxes still in flight (bounded) before the block exits
      const int issued = min(ngroups, g + kRing - 1);
      for (int h = g; h < issued; ++h) (void)mbar_wait_bounded(smem_addr(&bars[h % kRing]), (uint32_t)((h / kRing) & 1));
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ TMA, odd N
// Odd N: the row pitch N*8 is not a multiple of 16 bytes, so no 3D tensor map
// exists.  The grid is viewed instead as a 2D tensor of width 2N (pitch 16N
// bytes) and height (N^2 - 1) / 2: grid row R = kN + y (flat RN .. RN + N)
// sits in 2D row R >> 1 at columns (R & 1) N + x.  A tile's BY + 2 rows of
// one plane alternate between the two halves, so each plane is staged as two
// half-boxes of (BX + 4) x (BY + 2) / 2: half b holds the rows with
// (k + y) & 1 == b, copied from x = i0 - 2 - b (an even 2D column in both
// halves, as a tensor copy needs), so element x of such a row sits at column
// x - i0 + 2 + b.  TMA zero fill supplies the planes outside the grid; on
// edge tiles the rows outside [0, N) and the columns outside [0, N) hold
// neighbouring grid rows and are zeroed after landing, and the grid's last
// row (flat N^3 - N .. N^3, past the 2D view's last full row) is loaded by
// the threads.  Everything else is the jacobi_tma kernel: 4-plane groups in a
// 3-slot ring, the same sweep modes, flag and catch-up.
template <int BX, int BY>
struct OddGeom {
  static constexpr int PX = BX + 4;
  static constexpr int HB = (BY + 2) / 2;          // rows per half-box
  static constexpr int HALF = (PX * HB + 15) / 16 * 16;  // half-box stride: 128-byte aligned copies
  static constexpr int PLANE = 2 * HALF;
  static constexpr int GROUP = PLANE * kDZ;
  static constexpr uint32_t BYTES = 2u * kDZ * PX * HB * 8u;  // bytes landed per group
  static constexpr size_t SMEM = (size_t)kRing * GROUP * 8 + 128;
  static_assert((BY + 2) % 2 == 0, "tile rows split evenly between the halves");
  static_assert(HALF * 8 % 128 == 0 && GROUP * 8 % 128 == 0, "tensor-copy destinations stay 128-byte aligned");
};

template <int BX, int BY, int MODE, int ST>
__global__ void __launch_bounds__(BX* BY) jacobi_tma_odd(const __grid_constant__ CUtensorMap tmap,
                                                         const __grid_constant__ CUtensorMap tmap_alt, int N, int KC,
                                                         const double* __restrict__ in, void* __restrict__ outv,
                                                         const double* __restrict__ in_alt,
                                                         double* __restrict__ out_alt, int* status, int* flag,
                                                         StencilCoef cf) {
  pdl_begin();  // the previous sweep of the chain is complete and visible
  using G = OddGeom<BX, BY>;
  extern __shared__ unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bars[kRing];
  double* buf = reinterpret_cast<double*>(smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u));

  const int tid = threadIdx.x;
  const int tx = tid % BX, ty = tid / BX;
  const int i0 = blockIdx.x * BX, j0 = blockIdx.y * BY, y0 = j0 - 1;
  const int kb = blockIdx.z * KC;
  const int kc = min(KC, N - kb);
  const int ngroups = (kc + 2 + kDZ - 1) / kDZ;
  const bool flagged = (MODE == M_PP || MODE == M_PD) && flag != nullptr && *flag != 0;
  const bool native = (MODE == M_NATIVE) || flagged;
  const bool split_boxes = !native && (MODE == M_DD || MODE == M_DP);
  const CUtensorMap* src_map = flagged ? &tmap_alt : &tmap;
  const double* src = flagged ? in_alt : in;  // the staged data (for the edge fix-ups)
  // block-uniform: a tile that meets the grid's x or y faces holds copied
  // values of neighbouring grid rows to zero (and maybe the last row to load)
  const bool edge = i0 == 0 || i0 + BX + 2 > N || j0 == 0 || j0 + BY + 1 >= N;

  if (tid == 0) {
    for (int r = 0; r < kRing; ++r) mbar_init(smem_addr(&bars[r]), 1);
    mbar_fence_init();
  }
  // the padding after each half-box is never copied: zero it once, so that
  // splitting a landed group in place reads no garbage (which would mark it)
  constexpr int kPad = G::HALF - G::PX * G::HB;
  for (int e = tid; e < kRing * kDZ * 2 * kPad; e += BX * BY)
    if (AR_CHK((e / kPad) * G::HALF + G::PX * G::HB + e % kPad < kRing * G::GROUP))
      buf[(e / kPad) * G::HALF + G::PX * G::HB + e % kPad] = 0.0;
  fence_proxy_async_smem();
  __syncthreads();

  auto issue = [&](int g) {
    const int slot = g % kRing;
    const uint32_t bar = smem_addr(&bars[slot]);
    mbar_arrive_expect_tx(bar, G::BYTES);
    double* sb = buf + (size_t)slot * G::GROUP;
#pragma unroll
    for (int r = 0; r < kDZ; ++r) {
      const int k = kb - 1 + g * kDZ + r;
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        const int yb = y0 + ((((k + y0) & 1) == b) ? 0 : 1);  // first tile row of parity b
        const long long R = (long long)k * N + yb;
        const int yrow = (int)((R - b) >> 1);                  // R - b is even: exact, also below 0
        double* dst = sb + r * G::PLANE + b * G::HALF;
        if (AR_CHK(((b * N + i0 - 2 - b) & 1) == 0 && (smem_addr(dst) & 127u) == 0 &&
                   in_dyn_smem(smem_raw, dst, G::PX * G::HB * 8u)))
          tma_load_2d(smem_addr(dst), src_map, b * N + i0 - 2 - b, yrow, bar);
      }
    }
  };
  if (tid == 0)
    for (int g = 0; g < min(ngroups, kRing - 1); ++g) issue(g);

  const int i = i0 + tx, j = j0 + ty;
  const bool inside = i < N && j < N;
  const int64_t NN = (int64_t)N * N;
  const int64_t col = (int64_t)j * N + i;
  // offsets in a plane: the centre row lies in half bc = (k + j) & 1 at
  // column tx + 2 + bc; the rows j -+ 1 and the centres of the planes k -+ 1
  // lie in the other half.  Output plane p of group g has its centre in
  // group plane r - 1 with bc = q ^ (r & 1), q = (kb + j) & 1: bundle A (bc = q)
  // for even r, bundle B (bc = 1 - q) for odd r.
  const int q = (kb + j) & 1;
  const int idc = (ty + 1) >> 1, ids = ty >> 1, idn = (ty + 2) >> 1;
  auto cen = [&](int bc) { return bc * G::HALF + idc * G::PX + tx + 2 + bc; };
  auto oth = [&](int bc, int id) { return (1 - bc) * G::HALF + id * G::PX + tx + 2 + (1 - bc); };
  const int cA = cen(q), sA = oth(q, ids), nA = oth(q, idn), uA = oth(q, idc);
  const int cB = cen(1 - q), sB = oth(1 - q, ids), nB = oth(1 - q, idn), uB = oth(1 - q, idc);
  double* outd = flagged ? out_alt : static_cast<double*>(outv);
  float2* outp = static_cast<float2*>(outv);
  double dm = 0.0, d0 = 0.0;
  float2 fm = make_float2(0.f, 0.f), f0 = make_float2(0.f, 0.f);
  double* od = outd + ((int64_t)kb * NN + col);
  float2* op = outp + ((int64_t)kb * NN + col);
  int g = 0;
  bool failed = false;
  int slot = 0, pslot = kRing - 1;
  uint32_t phase = 0;
  for (; g < ngroups; ++g, pslot = slot, slot = (slot + 1 == kRing) ? 0 : slot + 1, phase ^= (slot == 0)) {
    const bool ok = mbar_wait_bounded(smem_addr(&bars[slot]), phase);
    double* box = buf + (size_t)slot * G::GROUP;
    const double* prev = buf + (size_t)pslot * G::GROUP;
    if (edge && ok) {
      // one staged row per thread: zero it if it lies outside the grid, else
      // zero its columns outside [0, N); load the grid's last row
      for (int rr = tid; rr < kDZ * 2 * G::HB; rr += BX * BY) {
        const int idx = rr % G::HB, b = (rr / G::HB) & 1, r = rr / (2 * G::HB);
        const int k = kb - 1 + g * kDZ + r;
        const int y = y0 + 2 * idx + ((((k + y0) & 1) == b) ? 0 : 1);
        const int xb = i0 - 2 - b;  // x of the row's first column
        double* d = box + r * G::PLANE + b * G::HALF + idx * G::PX;
        if (!AR_CHK(d - box >= 0 && d - box + G::PX <= G::GROUP)) continue;
        if ((unsigned)y >= (unsigned)N || (unsigned)k >= (unsigned)N) {
          for (int c = 0; c < G::PX; ++c) d[c] = 0.0;
        } else {
          const int c0 = max(0, -xb), c1 = min(G::PX, N - xb);  // columns inside the grid
          for (int c = 0; c < c0; ++c) d[c] = 0.0;
          for (int c = c1; c < G::PX; ++c) d[c] = 0.0;
          if (k == N - 1 && y == N - 1) {
            const double* row = src + ((int64_t)k * N + y) * N + xb;
            for (int c = c0; c < c1; ++c)
              d[c] = AR_CHK(row + c - src >= 0 && row + c - src < NN * N) ? __ldcg(row + c) : 0.0;
          }
        }
      }
    }
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    if (split_boxes) {
      bool marker = false;
#pragma unroll
      for (int e = tid; e < G::GROUP; e += BX * BY) {
        const float2 f = df_split(box[e]);
        marker |= (f.x != f.x);
        reinterpret_cast<float2*>(box)[e] = f;
      }
      if (__syncthreads_or(marker) && MODE == M_DP && tid == 0 && flag) atomicOr(flag, 1);
    }
    auto planes = [&](auto native_c, auto guard_c) {
      constexpr bool NAT = decltype(native_c)::value;
      constexpr bool GUARD = decltype(guard_c)::value;
#pragma unroll
      for (int r = 0; r < kDZ; ++r) {
        const int p = g * kDZ - 1 + r;
        const bool live = !GUARD || (p >= 1 && p <= kc);  // block-uniform
        const int cc = (r & 1) ? cB : cA, cs = (r & 1) ? sB : sA, cn = (r & 1) ? nB : nA;
        const int cu = (r & 1) ? uB : uA;
        const int pb = r == 0 ? (kDZ - 1) * G::PLANE : (r - 1) * G::PLANE;
        if constexpr (NAT) {
          const double* pp = r == 0 ? prev : box;
          const double up = box[r * G::PLANE + cu];
          if (live) {
            double s = pp[pb + cc - 1] + pp[pb + cc + 1];
            s += pp[pb + cs];
            s += pp[pb + cn];
            s += dm;
            s += up;
            if (inside && AR_CHK(od - outd >= 0 && od - outd < NN * N)) *od = stencil_f64<ST>(pp[pb + cc], s, cf);
            od += NN;
          }
          dm = d0;
          d0 = up;
        } else {
          const float2* pp = reinterpret_cast<const float2*>(r == 0 ? prev : box);
          const float2 up = reinterpret_cast<const float2*>(box)[r * G::PLANE + cu];
          if (live) {
            const float2 res =
                stencil_pair<ST>(pp[pb + cc], pp[pb + cc - 1], pp[pb + cc + 1], pp[pb + cs], pp[pb + cn], fm, up, cf);
            if (inside && AR_CHK(od - outd >= 0 && od - outd < NN * N && op - outp >= 0 && op - outp < NN * N)) {
              if constexpr (MODE == M_DP || MODE == M_PP) {
                *op = res;
              } else {
                double v = MODE == M_PD ? finite_pair_to_double(res) : pair_to_double(res);
                if (MODE == M_DD && (__double_as_longlong(v) & 0x7fffffffffffffffLL) > 0x7ff0000000000000LL) {
                  const int k = kb + p - 1;
                  double sd = at(in, N, i - 1, j, k) + at(in, N, i + 1, j, k);
                  sd += at(in, N, i, j - 1, k);
                  sd += at(in, N, i, j + 1, k);
                  sd += at(in, N, i, j, k - 1);
                  sd += at(in, N, i, j, k + 1);
                  v = stencil_f64<ST>(at(in, N, i, j, k), sd, cf);
                }
                *od = v;
              }
            }
            if constexpr (MODE == M_DP || MODE == M_PP)
              op += NN;
            else
              od += NN;
          }
          fm = f0;
          f0 = up;
        }
      }
    };
    using T_ = std::true_type;
    using F_ = std::false_type;
    const bool guard = g == 0 || g * kDZ + kDZ - 2 > kc;
    if (native) {
      if (guard)
        planes(T_{}, T_{});
      else
        planes(T_{}, F_{});
    } else {
      if (guard)
        planes(F_{}, T_{});
      else
        planes(F_{}, F_{});
    }
    // every reader of group g-1 is past this barrier: its slot takes group g+2
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0 && g + kRing - 1 < ngroups) issue(g + kRing - 1);
  }
  if (failed) {
    if (tid == 0) {
      if (status) atomicExch(status, (int)AR_ERR_TIMEOUT);
      const int issued = min(ngroups, g + kRing - 1);
      for (int h = g; h < issued; ++h) (void)mbar_wait_bounded(smem_addr(&bars[h % kRing]), (uint32_t)((h / kRing) & 1));
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ cp.async ring
// The df family when tensor copies cannot be used (odd N): each block streams
// its column's planes through a shared-memory ring (jacobi_ring.cuh), in the
// same sweep modes as jacobi_tma.
template <int BX, int BY, int MODE, int ST>
__global__ void __launch_bounds__(BX* BY) jacobi_ring(int N, int KC, const double* __restrict__ in, void* outv,
                                                      const double* __restrict__ in_alt, double* out_alt, int* flag,
                                                      StencilCoef cf) {
  pdl_begin();  // the previous sweep of the chain is complete and visible
  extern __shared__ __align__(16) unsigned char ring_smem[];
  const int kb = blockIdx.z * KC, ke = min(N, kb + KC);
  // block-uniform: the flag was settled by an earlier launch on this stream
  const bool flagged = (MODE == M_PP || MODE == M_PD) && flag != nullptr && *flag != 0;
  if (flagged) {  // the previous sweep in float64, from the float64 data
    jacobi_ring_tile<ST>(N, BX, BY, blockIdx.x, blockIdx.y, kb, ke, in_alt, out_alt, false, false, false, nullptr,
                         ring_smem, cf);
    return;
  }
  constexpr bool src_pairs = MODE == M_PP || MODE == M_PD;
  constexpr bool dst_pairs = MODE == M_DP || MODE == M_PP;
  jacobi_ring_tile<ST>(N, BX, BY, blockIdx.x, blockIdx.y, kb, ke, in, static_cast<double*>(outv), MODE != M_NATIVE,
                       src_pairs, dst_pairs, MODE == M_DP ? flag : nullptr, ring_smem, cf);
}

// ------------------------------------------------------------------ host side
template <int BX, int BY, int ST>
int launch_naive(int N, const double* in, double* out, const StencilCoef& cf, cudaStream_t s) {
  dim3 grid((unsigned)ceil_div(N, BX), (unsigned)ceil_div(N, BY), (unsigned)N);
  return launch_pdl(jacobi_naive<BX, BY, ST>, grid, dim3(BX, BY), 0, s, N, in, out, cf);
}

inline int chunk_planes(int N, int64_t colblocks, int resident_per_sm, int lo, int hi) {
  const int64_t target = 2LL * device_sms() * resident_per_sm;
  int64_t kc = ceil_div((int64_t)N * colblocks, target);
  if (kc < lo) kc = lo;
  if (kc > hi) kc = hi;
  if (kc > N) kc = N;
  return (int)kc;
}

template <int BX, int BY, int ST>
int launch_smem(int N, const double* in, double* out, const StencilCoef& cf, cudaStream_t s) {
  const int64_t cb = ceil_div(N, BX) * ceil_div(N, BY);
  const int KC = chunk_planes(N, cb, 2048 / (BX * BY), 4, 1 << 30);
  dim3 grid((unsigned)ceil_div(N, BX), (unsigned)ceil_div(N, BY), (unsigned)ceil_div(N, KC));
  return launch_pdl(jacobi_smem<BX, BY, ST>, grid, dim3(BX, BY), 0, s, N, KC, in, out, cf);
}

// TMA staging needs a 16-byte row pitch (even N), a grid at least one box wide
// and 16-byte aligned buffers; decided once per call so that every sweep of a
// call uses the same buffer format.
bool tma_usable(int shape, int N, const void* a, const void* b, const void* c) {
  const int PX = kShapeX[shape] + 4, PY = kShapeY[shape] + 2;
  return !(N & 1) && N >= PX && N >= PY && N >= kDZ && aligned16(a) && (!b || aligned16(b)) && (!c || aligned16(c));
}

// Odd N: tensor copies through the 2N-wide view (jacobi_tma_odd).
bool tma_odd_usable(int shape, int N, const void* a, const void* b, const void* c) {
  const int PX = kShapeX[shape] + 4;
  return (N & 1) && N >= PX && N >= 5 && aligned16(a) && (!b || aligned16(b)) && (!c || aligned16(c));
}

// Float64 sweep of the flagged pair chain's last step: does nothing unless
// the first sweep flagged an input outside the float-pair range.
template <int ST>
__global__ void __launch_bounds__(256) jacobi_catchup(int N, const int* __restrict__ flag,
                                                      const double* __restrict__ in, double* __restrict__ out,
                                                      StencilCoef cf) {
  pdl_begin();  // the previous sweep of the chain is complete and visible
  if (*flag == 0) return;
  const int64_t n3 = (int64_t)N * N * N, NN = (int64_t)N * N;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n3; c += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(c % N), j = (int)((c / N) % N), k = (int)(c / NN);
    double s = at(in, N, i - 1, j, k) + at(in, N, i + 1, j, k);
    s += at(in, N, i, j - 1, k);
    s += at(in, N, i, j + 1, k);
    s += at(in, N, i, j, k - 1);
    s += at(in, N, i, j, k + 1);
    out[c] = stencil_f64<ST>(in[c], s, cf);
  }
}

template <int BX, int BY, int MODE, int ST>
int launch_tma(int N, const double* in, void* out, const double* in_alt, double* out_alt, int* status, int* flag,
               const StencilCoef& cf, cudaStream_t s) {
  using G = TmaGeom<BX, BY>;
  static std::once_flag once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(once, [] {
    attr_err = cudaFuncSetAttribute(jacobi_tma<BX, BY, MODE, ST>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)G::SMEM);
  });
  if (attr_err != cudaSuccess) return AR_ERR_CUDA;
  CUtensorMap map, map_alt;
  if (!encode_tensor_map_3d_f64(&map, in, (uint64_t)N, (uint64_t)N, (uint64_t)N, G::PX, G::PY, kDZ) ||
      !encode_tensor_map_3d_f64(&map_alt, in_alt ? in_alt : in, (uint64_t)N, (uint64_t)N, (uint64_t)N, G::PX, G::PY,
                                kDZ))
    return AR_ERR_CUDA;
  const int64_t cb = ceil_div(N, BX) * ceil_div(N, BY);
  int resident = (int)((227 * 1024) / G::SMEM);
  if (resident > 2048 / (BX * BY)) resident = 2048 / (BX * BY);
  if (resident < 1) resident = 1;
  // KC + 2 a multiple of the box depth wastes no loaded plane
  int KC = chunk_planes(N, cb, resident, kDZ - 2, 8 * kDZ - 2);
  KC = (int)(ceil_div(KC + 2, kDZ) * kDZ - 2);
  dim3 grid((unsigned)ceil_div(N, BX), (unsigned)ceil_div(N, BY), (unsigned)ceil_div(N, KC));
  return launch_pdl(jacobi_tma<BX, BY, MODE, ST>, grid, dim3(BX * BY), G::SMEM, s, map, map_alt, N, KC, in, out,
                    out_alt, status, flag, cf);
}

template <int BX, int BY, int MODE, int ST>
int launch_tma_odd(int N, const double* in, void* out, const double* in_alt, double* out_alt, int* status,
                   int* flag, const StencilCoef& cf, cudaStream_t s) {
  using G = OddGeom<BX, BY>;
  static std::once_flag once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(once, [] {
    attr_err = cudaFuncSetAttribute(jacobi_tma_odd<BX, BY, MODE, ST>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)G::SMEM);
  });
  if (attr_err != cudaSuccess) return AR_ERR_CUDA;
  // the grid as 2N-wide rows: (N^2 - 1) / 2 full rows (the last grid row is
  // loaded by the kernel)
  const uint64_t W = 2ull * (uint64_t)N, H = ((uint64_t)N * N - 1) / 2;
  CUtensorMap map, map_alt;
  if (!encode_tensor_map_2d_f64(&map, in, W, H, W * 8, G::PX, G::HB) ||
      !encode_tensor_map_2d_f64(&map_alt, in_alt ? in_alt : in, W, H, W * 8, G::PX, G::HB))
    return AR_ERR_CUDA;
  const int64_t cb = ceil_div(N, BX) * ceil_div(N, BY);
  int resident = (int)((227 * 1024) / G::SMEM);
  if (resident > 2048 / (BX * BY)) resident = 2048 / (BX * BY);
  if (resident < 1) resident = 1;
  int KC = chunk_planes(N, cb, resident, kDZ - 2, 8 * kDZ - 2);
  KC = (int)(ceil_div(KC + 2, kDZ) * kDZ - 2);
  dim3 grid((unsigned)ceil_div(N, BX), (unsigned)ceil_div(N, BY), (unsigned)ceil_div(N, KC));
  return launch_pdl(jacobi_tma_odd<BX, BY, MODE, ST>, grid, dim3(BX * BY), G::SMEM, s, map, map_alt, N, KC, in, out,
                    in_alt, out_alt, status, flag, cf);
}

template <int BX, int BY, int MODE, int ST>
int launch_ring(int N, const double* in, void* out, const double* in_alt, double* out_alt, int* flag,
                const StencilCoef& cf, cudaStream_t s) {
  constexpr int smem = ring_smem_bytes(BX, BY);
  static_assert(smem <= 48 * 1024, "ring fits the default dynamic shared memory");
  static_assert((BX + 4) / 2 * (BY + 2) <= kRingChunks * BX * BY, "a plane's chunks fit kRingChunks per thread");
  const int64_t cb = ceil_div(N, BX) * ceil_div(N, BY);
  int resident = (227 * 1024) / smem;
  if (resident > 2048 / (BX * BY)) resident = 2048 / (BX * BY);
  const int KC = chunk_planes(N, cb, resident, 8, 64);
  dim3 grid((unsigned)ceil_div(N, BX), (unsigned)ceil_div(N, BY), (unsigned)ceil_div(N, KC));
  return launch_pdl(jacobi_ring<BX, BY, MODE, ST>, grid, dim3(BX * BY), smem, s, N, KC, in, out, in_alt, out_alt,
                    flag, cf);
}

template <int BX, int BY, int ST>
int launch_family(int fam, int mode, int staging, int N, const double* in, double* out, const double* in_alt,
                  double* out_alt, int* status, int* flag, const StencilCoef& cf, cudaStream_t s) {
  if (fam == 0) return launch_naive<BX, BY, ST>(N, in, out, cf, s);
  if (fam == 3 && staging == kStageRing) {
    switch (mode) {
      case M_DD: return launch_ring<BX, BY, M_DD, ST>(N, in, out, nullptr, nullptr, nullptr, cf, s);
      case M_DP: return launch_ring<BX, BY, M_DP, ST>(N, in, out, nullptr, nullptr, flag, cf, s);
      case M_PP: return launch_ring<BX, BY, M_PP, ST>(N, in, out, in_alt, out_alt, flag, cf, s);
      default: return launch_ring<BX, BY, M_PD, ST>(N, in, out, in_alt, out_alt, flag, cf, s);
    }
  }
  if (staging == kStageTmaOdd) {
    switch (mode) {
      case M_NATIVE: return launch_tma_odd<BX, BY, M_NATIVE, ST>(N, in, out, nullptr, nullptr, status, nullptr, cf, s);
      case M_DD: return launch_tma_odd<BX, BY, M_DD, ST>(N, in, out, nullptr, nullptr, status, nullptr, cf, s);
      case M_DP: return launch_tma_odd<BX, BY, M_DP, ST>(N, in, out, nullptr, nullptr, status, flag, cf, s);
      case M_PP: return launch_tma_odd<BX, BY, M_PP, ST>(N, in, out, in_alt, out_alt, status, flag, cf, s);
      default: return launch_tma_odd<BX, BY, M_PD, ST>(N, in, out, in_alt, out_alt, status, flag, cf, s);
    }
  }
  if (fam == 1 || staging != kStageTma) return launch_smem<BX, BY, ST>(N, in, out, cf, s);
  switch (mode) {
    case M_NATIVE: return launch_tma<BX, BY, M_NATIVE, ST>(N, in, out, nullptr, nullptr, status, nullptr, cf, s);
    case M_DD: return launch_tma<BX, BY, M_DD, ST>(N, in, out, nullptr, nullptr, status, nullptr, cf, s);
    case M_DP: return launch_tma<BX, BY, M_DP, ST>(N, in, out, nullptr, nullptr, status, flag, cf, s);
    case M_PP: return launch_tma<BX, BY, M_PP, ST>(N, in, out, in_alt, out_alt, status, flag, cf, s);
    default: return launch_tma<BX, BY, M_PD, ST>(N, in, out, in_alt, out_alt, status, flag, cf, s);
  }
}

template <int ST>
int sweep(int variant, int mode, int staging, int N, const double* in, double* out, const double* in_alt,
          double* out_alt, int* status, int* flag, const StencilCoef& cf, cudaStream_t s) {
  const int fam = variant / 4;
  switch (variant % 4) {
    case 0: return launch_family<32, 4, ST>(fam, mode, staging, N, in, out, in_alt, out_alt, status, flag, cf, s);
    case 1: return launch_family<32, 8, ST>(fam, mode, staging, N, in, out, in_alt, out_alt, status, flag, cf, s);
    case 2: return launch_family<64, 4, ST>(fam, mode, staging, N, in, out, in_alt, out_alt, status, flag, cf, s);
    default: return launch_family<128, 2, ST>(fam, mode, staging, N, in, out, in_alt, out_alt, status, flag, cf, s);
  }
}

}  // namespace

namespace {
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  });
  return encode;
}
}  // namespace

bool encode_tensor_map_3d_f64(CUtensorMap* map, const void* base, uint64_t d0, uint64_t d1, uint64_t d2,
                              uint32_t b0, uint32_t b1, uint32_t b2) {
  auto encode = tensor_map_encoder();
  if (!encode) return false;
  cuuint64_t dims[3] = {d0, d1, d2};
  cuuint64_t strides[2] = {d0 * 8, d0 * d1 * 8};
  cuuint32_t box[3] = {b0, b1, b2};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, const_cast<void*>(base), dims, strides, box, estr,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

bool encode_tensor_map_2d_f64(CUtensorMap* map, const void* base, uint64_t d0, uint64_t d1, uint64_t pitch_bytes,
                              uint32_t b0, uint32_t b1) {
  auto encode = tensor_map_encoder();
  if (!encode) return false;
  cuuint64_t dims[2] = {d0, d1};
  cuuint64_t strides[1] = {pitch_bytes};
  cuuint32_t box[2] = {b0, b1};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<void*>(base), dims, strides, box, estr,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

int jacobi7_num_variants() { return kJacobiVariants; }

int jacobi7_variant_name(int v, char* buf, int len) {
  if (v < 0 || v >= kJacobiVariants || !buf || len <= 0) return AR_ERR_ARG;
  snprintf(buf, (size_t)len, "jacobi7_%s_%dx%d", kFamily[v / 4], kShapeX[v % 4], kShapeY[v % 4]);
  return AR_OK;
}

int jacobi7_launch(void* args, int variant, double, void* stream, void*) {
  const ar_jacobi7_args* a = static_cast<const ar_jacobi7_args*>(args);
  if (!a) return AR_ERR_ARG;
  return ar_jacobi7(variant, a->N, a->sweeps, a->u0, a->out, a->work, a->status, stream);
}

int heat7_num_variants() { return kJacobiVariants; }

int heat7_variant_name(int v, char* buf, int len) {
  if (v < 0 || v >= kJacobiVariants || !buf || len <= 0) return AR_ERR_ARG;
  snprintf(buf, (size_t)len, "heat7_%s_%dx%d", kFamily[v / 4], kShapeX[v % 4], kShapeY[v % 4]);
  return AR_OK;
}

int heat7_launch(void* args, int variant, double, void* stream, void*) {
  const ar_heat7_args* a = static_cast<const ar_heat7_args*>(args);
  if (!a) return AR_ERR_ARG;
  return ar_heat7(variant, a->N, a->steps, a->alpha, a->u0, a->out, a->work, a->status, stream);
}

namespace {

// `sweeps` applications of stencil ST from u0, the last one landing in out.
template <int ST>
int stencil_run(int variant, int N, int sweeps, const StencilCoef& cf, const double* u0, double* out, double* work,
                int* status, void* stream) {
  if (variant < 0 || variant >= kJacobiVariants || N < 0 || sweeps < 0 || N > 65535) return AR_ERR_ARG;
  if (N == 0) return AR_OK;
  if (!u0 || !out || (sweeps > 1 && !work)) return AR_ERR_ARG;
  if (u0 == out || u0 == work || out == work) return AR_ERR_ARG;
  cudaStream_t s = as_stream(stream);
  const int64_t n3 = (int64_t)N * N * N;
  if (sweeps == 0) {
    return cudaMemcpyAsync(out, u0, (size_t)n3 * sizeof(double), cudaMemcpyDeviceToDevice, s) == cudaSuccess
               ? AR_OK
               : AR_ERR_CUDA;
  }
  const int fam = variant / 4;
  // tma and df stage planes by tensor copies when the grid allows it; the df
  // family otherwise (odd N) streams them by cp.async; 16-byte aligned
  // buffers are needed either way, else the shared-memory tile runs
  const double* w = sweeps > 1 ? work : nullptr;
  const int staging = fam < 2                                    ? kStageSmem
                      : tma_usable(variant % 4, N, u0, out, w)     ? kStageTma
                      : tma_odd_usable(variant % 4, N, u0, out, w) ? kStageTmaOdd
                      : (fam == 3 && aligned16(u0) && aligned16(out) && (!w || aligned16(w))) ? kStageRing
                                                                                               : kStageSmem;
  const bool staged = staging != kStageSmem;
  auto dst_of = [&](int j) -> double* { return ((sweeps - 1 - j) % 2 == 0) ? out : work; };
  // df calls of 2+ sweeps keep float pairs between sweeps; status[1] records
  // whether the first sweep met an input outside the float-pair range, in
  // which case every later launch computes the previous sweep in float64 from
  // the float64 data and a final catch-up launch computes the last one
  int* flag = (fam == 3 && staged && sweeps >= 2 && status) ? status + 1 : nullptr;
  if (flag && cudaMemsetAsync(flag, 0, sizeof(int), s) != cudaSuccess) return AR_ERR_CUDA;
  for (int sw = 0; sw < sweeps; ++sw) {
    const double* src = sw == 0 ? u0 : dst_of(sw - 1);
    double* dst = dst_of(sw);
    int mode = M_NATIVE;
    const double* alt_src = nullptr;
    double* alt_dst = nullptr;
    if (fam == 3) {
      if (!flag) {
        mode = M_DD;
      } else if (sw == 0) {
        mode = M_DP;
      } else {
        mode = (sw == sweeps - 1) ? M_PD : M_PP;
        alt_src = sw == 1 ? u0 : dst_of(sw - 2);
        alt_dst = dst_of(sw - 1);
      }
    }
    const int rc = sweep<ST>(variant, mode, staging, N, src, dst, alt_src, alt_dst, status, flag, cf, s);
    if (rc != AR_OK) return rc;
  }
  if (flag) {
    const double* src = sweeps >= 2 ? dst_of(sweeps - 2) : u0;
    return launch_pdl(jacobi_catchup<ST>, dim3(device_sms() * 4), dim3(256), 0, s, N, flag, src, dst_of(sweeps - 1),
                      cf);
  }
  return AR_OK;
}

}  // namespace
}  // namespace ar

extern "C" int ar_jacobi7(int variant, int N, int sweeps, const double* u0, double* out, double* work,
                          int* status, void* stream) {
  return ar::stencil_run<ar::kJacobi>(variant, N, sweeps, ar::StencilCoef{0.0, 0.f, 0.f, 0.f, 0.f}, u0, out, work,
                                      status, stream);
}

extern "C" int ar_heat7(int variant, int N, int steps, double alpha, const double* u0, double* out, double* work,
                        int* status, void* stream) {
  if (!(alpha >= 0.0 && alpha <= 1.0)) return AR_ERR_ARG;  // NaN fails too
  const double beta = 1.0 - 6.0 * alpha;
  const float ahi = (float)alpha, bhi = (float)beta;
  const ar::StencilCoef cf{alpha, ahi, (float)(alpha - (double)ahi), bhi, (float)(beta - (double)bhi)};
  return ar::stencil_run<ar::kHeat>(variant, N, steps, cf, u0, out, work, status, stream);
}

namespace ar {
AR_CHECK_READER(chk_read_jacobi7)
}  // namespace ar
