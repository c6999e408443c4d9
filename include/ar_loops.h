/*
 * ar_loops.h -- the region bodies and their variants, C ABI.
 *
 * The paper adapts loop regions by choosing among code variants at run time;
 * its GPU use case picks the number of threads per team for each region
 * (Section 3.2.2, Listing 4: variants([64:1024:64]), default 256 threads).
 * The variants here are hand-written CUDA kernels (sm_103a) for four loops:
 * daxpy (the paper's vector-update example, Listings 1-5), a 7-point 3D
 * Jacobi stencil (stand-in for Heat, Table 3), CSR SpMV (stand-in for AMGMk
 * relax, Table 3) and all-pairs n-body.
 *
 * Conventions for every call below:
 *  - Pointers are DEVICE pointers unless stated; the caller owns them.
 *  - `stream` is a cudaStream_t passed as void* (NULL = default stream).
 *    Calls only enqueue work; they do not synchronise.
 *  - Return AR_OK (0) or a negative ar_status from ar.h: AR_ERR_ARG for a bad
 *    variant index, size or alignment (nothing is launched), AR_ERR_CUDA if
 *    the launch failed.  Empty problems (n = 0, N = 0, rows = 0) launch
 *    nothing and return AR_OK.
 *  - Variant names are "<loop>_<family>_<shape>", see *_variant_name.
 */
#ifndef AR_LOOPS_H
#define AR_LOOPS_H

#include <stddef.h>
#include <stdint.h>

#include "ar.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Loop ids for ar_region_add_builtin.  The mixed-stream executor below runs
 * the first four; AR_LOOP_HEAT7 is stand-alone and region use only. */
enum { AR_LOOP_DAXPY = 0, AR_LOOP_JACOBI7 = 1, AR_LOOP_SPMV = 2, AR_LOOP_NBODY = 3, AR_LOOP_HEAT7 = 4 };

/* Number of variants of a loop, its default variant (the fixed baseline the
 * selection is compared with) and a variant's name. */
int ar_loop_num_variants(int loop);
int ar_loop_default_variant(int loop);
int ar_loop_variant_name(int loop, int variant, char *buf, int len);

/* Register all variants of a built-in loop on a region, in index order, with
 * launchers that read `args` as the loop's ar_*_args block below.  Variant
 * values are the variant indices. */
int ar_region_add_builtin(ar_region *r, int loop, int *out_count);
/* The same for the loop's first `count` variants only (1 .. the loop's
 * count; AR_ERR_ARG otherwise), e.g. the variants the mixed-stream executor
 * runs (ar_exec_num_variants), for a region that learns the executor's
 * choices. */
int ar_region_add_builtin_first(ar_region *r, int loop, int count, int *out_count);

/* ---------------------------------------------------------------- daxpy ---
 * y[i] <- a*x[i] + y[i] for i in [0, n), float64, one fused multiply-add per
 * element.  15 variants: threads per block {64,128,256,512,1024} x elements
 * per thread {1,2,4}; variant = 3*block_index + ept_index.  EPT 2 and 4 use
 * 128-bit (double2) accesses and need x and y 16-byte aligned (AR_ERR_ARG
 * otherwise).  Default: 256 threads x 1 element (variant 6), the paper's
 * 256-thread default (Section 4.2).  x and y must not overlap. */
typedef struct ar_daxpy_args {
  int64_t n;
  double a;
  const double *x;
  double *y;
} ar_daxpy_args;
int ar_daxpy(int variant, int64_t n, double a, const double *x, double *y, void *stream);

/* -------------------------------------------------------------- Jacobi ---
 * `sweeps` sweeps of u'(i,j,k) = (u(i-1)+u(i+1)+u(j-1)+u(j+1)+u(k-1)+u(k+1))/6
 * over N^3 float64 unknowns stored at (k*N + j)*N + i, zero outside the cube.
 * Reads u0 (unchanged), writes the result to `out`, uses `work` (N^3
 * doubles) as the ping-pong partner; u0, out and work must be distinct.
 * Variants: family {naive, smem (2.5D shared-memory z-march), tma
 * (cp.async.bulk.tensor tiles with mbarrier completion), df (tma staging plus
 * float-pair arithmetic on the FP32 pipe, ~2^-46 relative; points whose
 * inputs lie outside [2^-74, 2^118) in magnitude are recomputed in float64)}
 * x block shape {32x4, 32x8,
 * 64x4, 128x2}; variant = 4*family + shape.  The tma family needs N >= BX+4
 * and 16-byte aligned buffers (odd N: tensor copies through a 2N-wide view of
 * the grid); otherwise the tma family runs the smem kernel of the same shape
 * and the df family a cp.async plane ring (aligned buffers) or the smem
 * kernel.  Default: naive 32x8 (variant 1).
 * `status` (device int[2], may be NULL): status[0] receives AR_ERR_TIMEOUT if
 * a bounded wait inside a tma/df kernel gave up (the caller zeroes it);
 * status[1] is scratch for the df family (calls that may run at the same
 * time on different streams need their own status arrays), which with a
 * status array and 2+ sweeps keeps float pairs (8 bytes per unknown) in
 * out/work between sweeps and, when an input lies outside the float-pair
 * range, recomputes the whole call in float64 (one extra launch at the end, which otherwise exits at
 * once).  Without a status array every df sweep converts from and to
 * float64 and redoes out-of-range points in float64.  The sweeps of one call
 * are chained by programmatic dependent launch (each waits for the previous
 * one before its first global access), so a caller's next operation on
 * `stream` is ordered after the whole call as usual; a kernel the caller
 * itself launches next with programmatic dependent launch must execute
 * griddepcontrol.wait before reading the output (the last kernel of the
 * call lets dependents launch early).  The merge-path SpMV variants chain
 * their launches the same way. */
typedef struct ar_jacobi7_args {
  int N;
  int sweeps;
  const double *u0;
  double *out;
  double *work;
  int *status;
} ar_jacobi7_args;
int ar_jacobi7(int variant, int N, int sweeps, const double *u0, double *out, double *work,
               int *status, void *stream);

/* ---------------------------------------------------------------- Heat ---
 * `steps` explicit (forward Euler) steps of the heat equation on the same
 * grid: u'(i,j,k) = u + alpha (u(i-1)+u(i+1)+u(j-1)+u(j+1)+u(k-1)+u(k+1) -
 * 6u), zero outside the cube, alpha = kappa dt / h^2 with 0 <= alpha <= 1
 * (AR_ERR_ARG otherwise, NaN included; the scheme is stable for alpha <=
 * 1/6).  The finite-difference scheme of the paper's Heat benchmark
 * (Table 3) on a 3D grid.  Layout, buffers, the 16 variants (same families
 * and shapes as ar_jacobi7, named heat7_*), the tma/df requirements and the
 * status array behave exactly as for ar_jacobi7; the df family carries
 * alpha as a float pair and u + alpha (sum - 6u) to ~2^-46 of |u| +
 * alpha sum|neighbours|.  Default: naive 32x8 (variant 1).  Not accepted by
 * ar_exec_batch. */
typedef struct ar_heat7_args {
  int N;
  int steps;
  double alpha;
  const double *u0;
  double *out;
  double *work;
  int *status;
} ar_heat7_args;
int ar_heat7(int variant, int N, int steps, double alpha, const double *u0, double *out, double *work,
             int *status, void *stream);

/* ---------------------------------------------------------------- SpMV ---
 * y = A x for a CSR matrix of `rows` rows and nnz nonzeros: rowptr int32
 * [rows+1] (rowptr[0] = 0, non-decreasing, rowptr[rows] = nnz < 2^31), col
 * int32 [nnz] (column indices, any order within a row, each < length of x),
 * val float64 [nnz], x float64, y float64 [rows] (written, not accumulated).
 * Each row's products are summed in float64 in a variant-specific order,
 * except variant 7.  Variants: 0 thread-per-row, 1 warp-per-row, 2..5
 * vector-k (k = 2, 4, 8, 16 lanes per row), 6 merge-path (equal path work
 * per thread, products staged in shared memory; rows crossing threads and
 * blocks summed in a fixed order), 7 merge-path in float-pair arithmetic
 * (operands split into float pairs, products and row sums carried to
 * ~2^-46 relative of the sum of |val x|; the rows of a path block holding a
 * nonzero operand of magnitude outside [2^-62, 2^62), or a sum that
 * overflows a float, are redone in float64), 8 length-binned (rows grouped
 * by length class, 0-2, 3-4, 5-8, 9-16, 17-32, 33-64, 65-128, 129-256,
 * 257-1024, 1025+, with 1, 1, 1, 2, 2, 4, 8, 8, 16, 32 lanes per row and up
 * to 8 nonzeros per lane per pass: few float64 lane-slots per nonzero while
 * no row takes more than 16 passes; four launches: count, scan, scatter of
 * the rows into class order, one persistent pass, longest class first).
 * Default: thread-per-row.  Merge-path (6, 7) and binned (8) use the
 * caller's workspace (ar_spmv_workspace_bytes; device memory, contents need
 * no initialisation; AR_ERR_ARG if too small).  Results are deterministic. */
typedef struct ar_spmv_args {
  int64_t rows;
  int64_t nnz;
  const int32_t *rowptr;
  const int32_t *col;
  const double *val;
  const double *x;
  double *y;
  void *workspace;
  size_t workspace_bytes;
} ar_spmv_args;
int ar_spmv_workspace_bytes(int variant, int64_t rows, int64_t nnz, size_t *bytes);
int ar_spmv(int variant, int64_t rows, int64_t nnz, const int32_t *rowptr, const int32_t *col, const double *val,
            const double *x, double *y, void *workspace, size_t workspace_bytes, void *stream);

/* Merge-path SpMV (variant 6 above) for callers that cannot allocate device
 * memory: its scratch is a fixed array of AR_SPMV_NOALLOC_SCRATCH_BYTES
 * compiled into this library, so the caller passes only inputs and outputs.
 * This entry point has no counterpart in the paper; it exists for callers
 * such as plug-ins handed a device whose memory another allocator already
 * owns, or latency-critical loops that must not pay the device-wide
 * synchronisation cudaMalloc/cudaFree imply.
 *  - Capacity: rows + nnz <= AR_SPMV_NOALLOC_MAX_PATH (about 1.43e9, enough
 *    for every matrix of the workload); larger problems return AR_ERR_ARG
 *    with a message on stderr and launch nothing.
 *  - Memory: every GPU that loads the library holds the 8 MiB array until the
 *    process exits.  The first call on a device looks up the array's device
 *    address (cudaGetSymbolAddress, once per device, with that device
 *    current); make that first call before any stream capture.  The cached
 *    address does not survive cudaDeviceReset: do not call this entry point
 *    after resetting the device in the same process.
 *  - No allocation: calls no cudaMalloc, cudaFree or allocating routine.
 *  - Sharing: all calls on a device use the same array; the kernels write
 *    every scratch word before reading it, so nothing needs clearing, but two
 *    calls that overlap on the GPU (different streams, no ordering) race on
 *    the scratch and give wrong results.  Order them on one stream.
 * Returns AR_OK, AR_ERR_ARG (bad arguments or over capacity) or AR_ERR_CUDA. */
#define AR_SPMV_NOALLOC_SCRATCH_BYTES (8u << 20)
/* 24 bytes per 4096-item path block plus 8 (checked against the kernels'
 * block size by a static_assert in the library's source) */
#define AR_SPMV_NOALLOC_MAX_PATH ((long long)(((AR_SPMV_NOALLOC_SCRATCH_BYTES - 8u) / 24u) * 4096u))
int ar_spmv_merge_path_noalloc(int64_t rows, int64_t nnz, const int32_t *rowptr, const int32_t *col,
                               const double *val, const double *x, double *y, void *stream);

/* Row-length features of a CSR matrix, the learned selector's inputs: out5 =
 * (rows, nnz, mean, population variance, max) of rowptr[r+1] - rowptr[r], as
 * float32 in device memory.  Integer sums are exact; mean and variance are
 * formed in float64.  workspace: ar_csr_features_workspace_bytes of device
 * memory (no initialisation needed). */
int ar_csr_features_workspace_bytes(int64_t rows, size_t *bytes);

/* Measurement kernel, not an SpMV: streams col and val of all nnz nonzeros
 * and gathers x[col[j]], 8 nonzeros in flight per thread, with no row logic
 * and no float64 arithmetic, so its time is the memory-side floor of any
 * CSR SpMV variant on the matrix (for power-law rows, random 8-byte gathers
 * that each cost a 32-byte sector, not HBM bytes, set it).  sink8: 8 bytes
 * of device memory that the kernel may write (its result is meaningless).
 * Returns AR_OK, AR_ERR_ARG (nnz outside [0, 2^31), NULL pointers) or
 * AR_ERR_CUDA. */
int ar_spmv_gather_floor(int64_t nnz, const int32_t *col, const double *val, const double *x, void *sink8,
                         void *stream);
int ar_csr_features(int64_t rows, const int32_t *rowptr, float *out5, void *workspace, size_t workspace_bytes,
                    void *stream);

/* --------------------------------------------------------------- n-body ---
 * acc4[i] = (sum_j m_j d_ij / (|d_ij|^2 + eps^2)^(3/2), 0), d_ij = r_j - r_i,
 * over all N bodies (j = i adds 0), float32.  pos4 holds (x, y, z, m) per
 * body; both arrays 16-byte aligned.  eps > 0.  Variants: shared-memory tile
 * {128, 256, 512} bodies x inner unroll {1, 4, 8}; variant = 3*tile + unroll.
 * Default: tile 256, unroll 1 (variant 3).  Small N (fewer than two blocks
 * per SM even at one body per thread) splits each tile's j range over a
 * thread-block cluster of up to 8 blocks and adds the partial sums in a
 * fixed order: results are bit-identical from run to run at every N. */
typedef struct ar_nbody_args {
  int64_t N;
  const float *pos4;
  float *acc4;
  float eps;
} ar_nbody_args;
int ar_nbody(int variant, int64_t N, const float *pos4, float *acc4, float eps, void *stream);

/* Launch geometry of n-body variant `variant` at N >= 1 bodies on the
 * current device, as ar_nbody would launch it: i-tiles (*grid), the
 * thread-block cluster size over which each i-tile's j range is split (1 =
 * not split), bodies per thread, resident blocks per SM of the kernel that
 * runs (occupancy API) and the SM count.  grid x cluster / (resident x sms)
 * is the number of waves the launch takes, the quantity that decides which
 * variant is fastest near the split thresholds; it is a pure function of N
 * and the device, so a selector can use it as a feature.  Host-only (no
 * kernel runs); AR_ERR_ARG for a bad variant or N < 1. */
int ar_nbody_geometry(int variant, int64_t N, int64_t *grid, int *cluster, int *bodies_per_thread,
                      int *resident_per_sm, int *sms);

/* `count` independent systems in one persistent launch: system b is bodies
 * [offs[b], offs[b+1]) of pos4/acc4 (offs: device int32 [count+1],
 * non-decreasing).  Work items (system, 256-body tile) run largest system
 * first, pulled from a device counter.  workspace: device memory of
 * ar_nbody_batched_workspace_bytes (no initialisation needed); count <= 4096. */
int ar_nbody_batched_workspace_bytes(int count, size_t *bytes);
int ar_nbody_batched(int count, const int32_t *offs, const float *pos4, float *acc4, float eps, void *workspace,
                     size_t workspace_bytes, void *stream);

/* ------------------------------------------------ host data: GPU / host split ---
 * Loops whose data live in HOST memory, with the iteration space split
 * between the GPU and the host cores: the paper's co-scheduling use case
 * (Section 3.2, Listing 5: numeric variants [0.0:1.0:0.1] are the fraction
 * of the loop run on the GPU, the GPU part runs asynchronously while the host
 * cores run the rest, and the region waits for both) and, with fractions 0
 * and 1 only, its device-selection use case (Section 3.2, Listing 3: variants
 * cpu and gpu).  For fraction f the GPU takes the first m = round(f n)
 * elements (daxpy) or rows (SpMV): their inputs are copied host -> device
 * (one cudaMemcpyAsync per array), one of the loop's CUDA variants
 * (gpu_variant) runs on them, and the result slice is copied back, all on
 * `stream`; meanwhile an OpenMP loop of this library computes the rest on
 * the host cores (daxpy: the same fused multiply-add as the device, so every
 * split gives the same bits; SpMV: each row's products summed by fused
 * multiply-add in nonzero order).  The call blocks until both parts are done
 * (host memory pinned for the copies to overlap the host loop).  Device
 * buffers: caller-owned, at least the GPU part's size (the whole arrays for
 * f = 1); unused when m = 0.  AR_ERR_ARG for f outside [0, 1], bad sizes or
 * pointers, a bad gpu_variant or workspace (SpMV: the variant's
 * ar_spmv_workspace_bytes for the GPU's rows); AR_ERR_CUDA if a copy or
 * launch fails (the stream is synchronised before returning, the host part
 * is not run, and the output's contents are undefined). */
typedef struct ar_daxpy_split_args {
  int64_t n;
  double a;
  const double *x; /* host */
  double *y;       /* host, updated in place */
  double *x_dev, *y_dev;
  int gpu_variant; /* ar_daxpy variant of the GPU part */
} ar_daxpy_split_args;
int ar_daxpy_split(double gpu_fraction, const ar_daxpy_split_args *args, void *stream);

typedef struct ar_spmv_split_args {
  int64_t rows, nnz, cols;   /* cols: length of x */
  const int32_t *rowptr;     /* host CSR, as for ar_spmv */
  const int32_t *col;
  const double *val, *x;     /* host */
  double *y;                 /* host, written */
  int32_t *rowptr_dev, *col_dev;
  double *val_dev, *x_dev, *y_dev;
  void *workspace;           /* device, for the GPU variant */
  size_t workspace_bytes;
  int gpu_variant;           /* ar_spmv variant of the GPU part */
} ar_spmv_split_args;
int ar_spmv_split(double gpu_fraction, const ar_spmv_split_args *args, void *stream);

/* Register the GPU fractions [begin:end:step] (inclusive, 0 <= begin,
 * end <= 1) as variants of a region whose executions run ar_daxpy_split
 * (loop AR_LOOP_DAXPY) or ar_spmv_split (AR_LOOP_SPMV) on an args block of
 * the matching type; each variant's value is its fraction.  [0.0:1.0:0.1]
 * is the co-scheduling region, [0:1:1] the device-selection region (variant
 * 0 = host cores, 1 = GPU).  The region's timing (CUDA events around the
 * blocking call) covers both parts and the copies. */
int ar_region_add_split(ar_region *r, int loop, double begin, double end, double step, int *out_count);

/* Host threads the split loops' OpenMP part uses. */
int ar_split_threads(void);

/* ------------------------------------------------------------ mixed stream ---
 * Persistent execution of a batch of region invocations of the four loops
 * (up to AR_EXEC_MAX_CALLS per batch) in three launches on `stream`:
 *   1. features: per call, the selector's features (daxpy: n; Jacobi: N,
 *      sweeps, 1 if N is even else 0 (a 16-byte row pitch, which tensor
 *      copies need); SpMV: rows, nnz, mean, variance, max of the row
 *      lengths, reduced from rowptr on the device; n-body: N);
 *   2. plan (one block): per call, the variant -- force_variant[c] if given,
 *      else the argmax of the loop's MLP (models->theta[loop]; the loop's
 *      default variant if that is NULL) with its confidence -- and the
 *      table of work items (one phase per Jacobi sweep; two for merge-path
 *      SpMV, main pass and carry fix-up; one otherwise), ordered by groups
 *      of 64 consecutive calls and phase-major inside a group, a group's
 *      calls inside a phase longest estimated item first (an n-body item
 *      of a large N before the short memory-bound items);
 *   3. run: a persistent kernel whose blocks pull work items from an atomic
 *      counter and run the chosen variant's tile of that call.  An item of
 *      phase p waits (bounded) until every item of phase p-1 of its call is
 *      done (a wait that gives up sets the call's status to AR_ERR_TIMEOUT,
 *      and the call's later items are then skipped without waiting); every awaited item was handed out earlier, and all of a
 *      group's items are handed out before the next group's, so a call's
 *      latency is about its group's rather than the whole batch's.
 * The tiles compute exactly what the stand-alone variants compute (same
 * data, same tolerances).  An n-body call whose tiles of i-bodies are
 * fewer than the persistent kernel's blocks may hand its j range out in
 * chunks: when out1 is 16-byte aligned, distinct from in0 and out0, and
 * holds S >= 2 arrays of N float4 (out1_bytes >= 32 N), each tile sums one
 * (i tile, j chunk) into array s and a second phase adds each body's S
 * partials in chunk order into out0 (S at most what out1_bytes holds, one
 * j tile per chunk at least; deterministic, the sum order differs from the
 * unsplit call's).  Without such an out1 the call runs unsplit.  Jacobi tiles of the tma and df families with
 * shapes 32x4 and 32x8 stage their planes by tensor copies when N is even,
 * N >= 36 and u0/out/work are 16-byte aligned (through tensor maps the plan
 * kernel makes on the device from host-encoded templates; the first batch
 * of a process checks, once and synchronously on `stream`, that a
 * device-made map equals the host encoding, and uses the cp.async plane ring
 * instead while the check fails or while `stream` is capturing before it
 * ran); the other Jacobi tiles stream planes by cp.async.  EPT 2/4 daxpy
 * variants on buffers that are not 16-byte aligned run with one element per
 * thread.
 * All arrays are device memory.  Per call c: variant[c], conf[c] (1 when
 * forced or defaulted), features[8c..8c+7], t_start[c] / t_end[c] (%globaltimer
 * ns of the first tile's start and the last tile's end), status[c] (AR_OK,
 * AR_ERR_ARG for a bad loop/variant or, for Jacobi, sweeps outside [1,
 * AR_EXEC_MAX_PHASES], N > 65535 or u0/out/work missing or not distinct
 * (work only for 2+ sweeps), AR_ERR_TIMEOUT if a dependency wait gave
 * up).  The call table and models must stay valid until the work completes.
 * workspace: ar_exec_workspace_bytes(max_calls) bytes, no initialisation
 * needed.  Two batches that share a workspace (or a call table) must not
 * overlap on the GPU: order them on one stream.  The launches contain no host
 * synchronisation and can be captured in a CUDA graph together with the copy
 * that refreshes `calls` (a captured graph replays on the stream it is
 * launched on, which must be the one other batches using the workspace run
 * on); the one exception is the first batch's tensor-map check above. */
#define AR_EXEC_MAX_CALLS 256
#define AR_EXEC_MAX_PHASES 64
typedef struct ar_exec_call {
  int32_t loop;   /* AR_LOOP_* */
  int32_t sweeps; /* Jacobi sweeps, 1 .. AR_EXEC_MAX_PHASES */
  int64_t n;      /* daxpy n | Jacobi N | SpMV rows | n-body N */
  int64_t nnz;    /* SpMV nonzeros */
  double a;       /* daxpy a */
  float eps;      /* n-body softening */
  int32_t reserved;
  const void *in0, *in1, *in2, *in3; /* daxpy x | Jacobi u0 | SpMV rowptr, col, val, x | n-body pos4 */
  void *out0, *out1;                 /* daxpy y | Jacobi out, work | SpMV y, merge-path workspace |
                                        n-body acc4, optional partial-sum workspace (see below) */
  uint64_t out1_bytes;               /* SpMV: merge-path workspace bytes (16 per 4096 rows+nnz);
                                        n-body: partial-sum workspace bytes */
} ar_exec_call;
typedef struct ar_exec_models {
  int32_t F[4], V[4], H; /* per loop: features (1, 3, 5, 1), variants (must match the loop); hidden 32/64 */
  const float *theta[4], *mu[4], *sd[4];
} ar_exec_models;
int ar_exec_workspace_bytes(int max_calls, size_t *bytes);
/* Variants the executor runs for a loop (AR_ERR_ARG for another loop): all
 * of daxpy, Jacobi and n-body, and SpMV variants 0-7 (not spmv_binned). */
int ar_exec_num_variants(int loop);

/* Self-test of the bounded device waits that every kernel here uses (the
 * executor's dependency wait and the tensor-copy mbarrier wait): kind 0
 * waits on a counter that nothing raises and kind 1 on an mbarrier phase
 * that nothing completes, each for at most `limit` polls (1 .. 2^24), then
 * gives up; kinds 2 and 3 wait on ones already satisfied.  status: one
 * device int32, set to AR_ERR_TIMEOUT (kinds 0, 1) or AR_OK (kinds 2, 3).
 * One block, no fault, no hang; AR_ERR_ARG for a bad kind or limit. */
int ar_wait_selftest(int kind, unsigned int limit, int32_t *status, void *stream);
int ar_exec_batch(const ar_exec_call *calls, int ncalls, const ar_exec_models *models, const int32_t *force_variant,
                  int32_t *variant, float *conf, float *features, uint64_t *t_start, uint64_t *t_end,
                  int32_t *status, void *workspace, size_t workspace_bytes, void *stream);

/* Confidence fallback of a mixed-stream batch.  The region learns from its
 * profiled executions (Section 2: every execution's features, policy and time
 * are recorded, and the model trained on them maps features to the fastest
 * policy; Table 1, __apollo_region_train); a call the device MLP was unsure
 * of is profiled exhaustively and its executions join the records of its
 * loop's region.  For each call c in [0, ncalls) with conf[c] < tau:
 *  - if the loop's region already holds records of every variant for the
 *    call's exact feature vector, nothing runs: best[c] is the fastest mean
 *    of those records (ties within the region's tie fraction, 0.5 % by
 *    default, to the lowest index);
 *  - otherwise every variant runs as a one-call ar_exec_batch forced to it,
 *    once untimed and `reps` times timed by the executor's own per-call time
 *    (t_end - t_start), each timed run preceded by the region's L2 flush
 *    (ar_set_l2_flush) if it has one; each timed run is appended to the
 *    region as a record (features, variant, ms), so a profiled call adds
 *    exactly V x reps records, and best[c] is the fastest mean.  The call's
 *    outputs end as its best variant computes them: one more untimed run of
 *    best[c], except for daxpy, whose y (updated in place by every run) is
 *    saved in the workspace before profiling and restored after (every daxpy
 *    variant computes the same fused multiply-add per element, so the saved
 *    y is the best variant's result too).
 * Other calls get best[c] = -1.  With retrain != 0 every region that received
 * records is trained again (ar_train) and, when `models` is given and the
 * region's model is an MLP, its new parameters are copied into that loop's
 * device buffers models->theta/mu/sd (same F, H and V), ready for the next
 * batch.
 *  calls, features (8 floats per call, as ar_exec_batch writes them), conf:
 *    HOST copies of the batch's table and outputs; the calls' device buffers
 *    must still be valid.
 *  regions[4]: one region per loop (NULL skips that loop's calls) with the
 *    executor's variant count (ar_exec_num_variants) and feature count
 *    (1, 3, 5, 1);
 *    AR_ERR_STATE otherwise.  reps: 1 .. 16.
 *  workspace: device memory of ar_exec_fallback_workspace_bytes(n), n the
 *    largest daxpy n that may fall back (AR_ERR_ARG for a larger one).
 *  best: HOST int32[ncalls]; *num_profiled (may be NULL): calls profiled.
 * Blocking: synchronises `stream` once per profiled call and before return.
 * Returns AR_OK, AR_ERR_ARG, AR_ERR_STATE, AR_ERR_CUDA, or the first failing
 * execution's status (e.g. AR_ERR_TIMEOUT); after an error the outputs of
 * the call being profiled are undefined (earlier calls keep theirs) and the
 * records appended so far stay in the regions. */
int ar_exec_fallback_workspace_bytes(int64_t max_daxpy_n, size_t *bytes);
int ar_exec_fallback(const ar_exec_call *calls, int ncalls, const float *features, const float *conf, float tau,
                     ar_region *const *regions, int reps, const ar_exec_models *models, int retrain, void *workspace,
                     size_t workspace_bytes, void *stream, int32_t *best, int *num_profiled);

/* ------------------------------------------------------------ MLP selector ---
 * The learned selector of the adaptive region: the paper's model kinds are
 * decision trees and random forests and it names neural networks as a
 * classifier the design admits (Section 3.1 model_type).  Network:
 *   x0 = (sign(f) log(1+|f|) - mu) / sd          (F raw features)
 *   h1 = relu(W1 x0 + b1), h2 = relu(W2 h1 + b2), logits = W3 h2 + b3,
 *   p = softmax(logits), loss = mean_s -log p_s[label_s]
 * Parameters theta (float32, ar_mlp_num_params of them) in the order W1 (H x F,
 * row major), b1 (H), W2 (H x H), b2 (H), W3 (V x H), b3 (V).  Limits:
 * 1 <= F <= 8, H in {32, 64}, 1 <= V <= 32, minibatch <= 256.  All pointers
 * are device pointers; features are row-major (rows x F). */
int ar_mlp_num_params(int F, int H, int V);

/* Inference for B rows: probs (B x V, may be NULL), argmax variant (ties to
 * the lowest index) and confidence = max probability (either may be NULL). */
int ar_mlp_forward(const float *theta, const float *mu, const float *sd, int F, int H, int V, int64_t B,
                   const float *feats, float *probs, int *variant, float *conf, void *stream);

/* Gradient of the mean cross-entropy over one minibatch of B <= 256 rows
 * (fixed-order sums, deterministic) into grad (ar_mlp_num_params floats) and
 * the loss into *loss (device float, may be NULL).  Labels outside [0, V) are
 * clamped into it. */
int ar_mlp_grad(const float *theta, const float *mu, const float *sd, int F, int H, int V, int B,
                const float *feats, const int *labels, float *grad, float *loss, void *stream);

/* One Adam step (Kingma & Ba; beta1 0.9, beta2 0.999, eps 1e-8) at step t >= 1
 * on n parameters: m, v updated in place, theta -= lr m_hat / (sqrt(v_hat)+eps). */
int ar_mlp_adam(float *theta, const float *grad, float *m, float *v, int64_t n, int t, float lr, void *stream);

/* Whole training run in one single-block launch: for each epoch e and each
 * minibatch of `batch` consecutive entries of perm[e*n .. e*n+n) (the last one
 * may be partial): forward, cross-entropy backward and an Adam step.  theta is
 * updated in place; adam_m and adam_v (n_params floats each) must be zeroed
 * by the caller; *loss receives the last minibatch's loss. */
int ar_mlp_train(float *theta, float *adam_m, float *adam_v, const float *mu, const float *sd, int F, int H,
                 int V, int n, const float *feats, const int *labels, const int *perm, int epochs, int batch,
                 float lr, float *loss, void *stream);

/* ------------------------------------------------------------ bounds check ---
 * The library also builds as a bounds-check flavour (compiled with
 * AR_CHECKED; libadaptive_region_checked.so): every index check written into
 * the kernels (tensor-copy coordinates, alignment and shared-memory ranges
 * of the stencil rings, the edge fix-ups, global stores of the stencils,
 * every shared and global index of the merge-path blocks, the executor's
 * work-item lookup) is compiled in; a failing check records itself and its
 * access is skipped, so a bad index shows up as a status, never as a fault.
 * ar_check_status reports *enabled (1 in that flavour, 0 otherwise), the
 * first failing check (source-file id << 16 | source line, 0 if none) and
 * the number of failures since the last clear; clear != 0 resets them.
 * Blocking (reads device memory). */
int ar_check_status(int *enabled, uint32_t *first_failure, uint32_t *failures, int clear);

/* ---------------------------------------------------------------- peaks ---
 * Issue-rate microbenchmarks (blocking, for roofline denominators): run a
 * dependent-chain FMA kernel on every SM and return fused multiply-adds per
 * second for float64 and float32. */
int ar_measure_fma_rates(double *fp64_fma_per_s, double *fp32_fma_per_s);

/* The same microbenchmark with packed float32 pairs (one FFMA2 instruction =
 * two float32 lanes' FMAs): float32 lane FMAs per second, the ceiling of the
 * n-body kernels' packed arithmetic.  AR_ERR_ARG if the pointer is null. */
int ar_measure_fp32x2_rate(double *fp32_lane_fma_per_s);

#ifdef __cplusplus
}
#endif
#endif /* AR_LOOPS_H */
