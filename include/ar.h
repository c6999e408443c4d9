/*
 * ar.h -- adaptive-region runtime, C ABI.
 *
 * An adaptive region (arXiv 2303.08873, Section 3.1 "adaptation" directive;
 * Section 2 and Table 1, the Apollo calls it lowers to) is a code region that
 * owns an ordered list of variants, a list of float features describing each
 * execution, a store of profiling records, and a model that maps features to
 * the variant expected to run fastest.  Its lifecycle (Section 3, "lifecycle
 * of adaptation"; Section 3.3 lowering): create once -> per execution begin,
 * set the features, get the policy, run that variant, end (record the elapsed
 * time) -> once enough unique data exist, train -> later executions use the
 * model's choice.
 *
 * Conventions for every call below:
 *  - Return value: AR_OK (0) or a negative ar_status; no call aborts or exits.
 *    Out-parameters are left untouched when an error is returned.
 *    ar_last_error() gives a one-line description of the last error.
 *  - Ownership: the library owns the region object, a copy of `id`, the
 *    records and the models.  The caller owns every device buffer and stream
 *    and every `args` block (borrowed for the duration of the call only).
 *  - Streams are passed as `void *` holding a cudaStream_t (NULL = legacy
 *    default stream).  Region executions are enqueued on that stream without
 *    host synchronisation; elapsed times come from CUDA events and are
 *    resolved lazily.  Only ar_profile, ar_train, ar_flush_records,
 *    ar_region_save and ar_region_load block the host.
 *  - Threads: a region object must not be used by two threads at once.
 *  - Logging: the environment variable AR_LOG (read once per process) sets a
 *    log level for stderr lines "[ar] <region id>: ...": 0 or unset quiet,
 *    1 training, automatic-training triggers, variants marked unusable and
 *    confidence-fallback summaries, 2 also every exhaustive profile, model
 *    selection and execution policy.
 */
#ifndef AR_H
#define AR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define AR_MAX_FEATURES 8  /* features per execution context            */
#define AR_MAX_VARIANTS 64 /* variants per region                        */

typedef enum ar_status {
  AR_OK = 0,
  AR_ERR_ARG = -1,     /* bad argument (NULL, out of range, NaN/inf feature) */
  AR_ERR_STATE = -2,   /* call not valid in the region's current state      */
  AR_ERR_CUDA = -3,    /* a CUDA call or a variant's launcher failed         */
  AR_ERR_NOMODEL = -4, /* a prediction was asked of a region with no model   */
  AR_ERR_IO = -5,      /* file missing, truncated, corrupt or unwritable     */
  AR_ERR_TIMEOUT = -6, /* a bounded device-side wait gave up                 */
  AR_ERR_OOM = -7      /* host or device allocation failed                   */
} ar_status;

typedef struct ar_region ar_region;

/* A variant's body.  `args` is the caller's argument block passed through
 * ar_invoke/ar_profile unchanged; `variant` is the variant index and `value`
 * its numeric value (Section 3.1 model_output).  Must enqueue its work on
 * `stream` and return 0, or return a non-zero code if the launch failed
 * (the runtime then marks this variant unusable and returns AR_ERR_CUDA). */
typedef int (*ar_launch_fn)(void *args, int variant, double value, void *stream, void *user);

/* Test hook: a deterministic cost model replacing the CUDA-event timer.
 * Returns the elapsed milliseconds to record for one execution. */
typedef double (*ar_fake_time_fn)(const float *features, int nf, int variant, void *user);

/* Create a region (Table 1 __apollo_region_create).
 *   id              copied; any non-empty string.
 *   num_features    0..AR_MAX_FEATURES features per execution (Section 3.1
 *                   features clause; the region itself is implicit).
 *   model_spec      NULL/"" for the default, else comma-separated:
 *                     "dtree[,<depth>]"  decision tree, default depth 2
 *                                        (Section 3.1 model_type)
 *                     "rfc[,<ntrees>,<depth>]"  random forest: both
 *                                        numbers or neither (Section 3.1);
 *                                        default 10 trees of depth 2
 *                     "mlp[,<hidden>]"   3-layer MLP selector, hidden 64
 *                     "exhaustive"       per-feature-vector table of the
 *                                        fastest profiled variant
 *                     "fixed,<index>"    always the given variant
 *                   options: "explore=roundrobin" (default), "reps=<n>"
 *                   (ar_profile repetitions, default 5), "conf=<tau>" (MLP
 *                   confidence threshold, default 0.5), "epochs=<n>"
 *                   (MLP training epochs, default 200), "seed=<n>",
 *                   "tie=<f>" (0 <= f < 1: variants whose mean time is
 *                   within a fraction f of the fastest tie, the lowest
 *                   index wins, in labels and exhaustive argmins; default
 *                   0.005 - a larger f keeps labels steady among variants
 *                   that run alike).
 *   min_train_data  unique (features, variant) points needed before the
 *                   automatic training; <= 0 means "number of variants"
 *                   (Section 3.1 default), fixed when the first execution
 *                   begins.
 * Errors: AR_ERR_ARG for a bad spec or count; AR_ERR_OOM. */
int ar_region_create(const char *id, int num_features, const char *model_spec, int min_train_data,
                     ar_region **out);

/* Destroy a region and every resource it holds; NULL is ignored.  Pending
 * CUDA events are released without waiting for them. */
void ar_region_destroy(ar_region *r);

/* Append one categorical or numeric variant (Section 3.1 variants clause).
 * Its index is its registration order, starting at 0 (Section 3.3: the
 * leftmost variant is 0).  Registration closes when the first execution
 * begins (AR_ERR_STATE afterwards).  AR_ERR_ARG if fn is NULL or the region
 * already has AR_MAX_VARIANTS variants. */
int ar_variant_register(ar_region *r, const char *name, double value, ar_launch_fn fn, void *user,
                        int *out_index);

/* Append the numeric range [begin:end:step], end inclusive (Section 3.1:
 * [10:20:2] is 10,12,...,20).  Value i is begin + i*step computed from i;
 * count = floor((end-begin)/step + 1e-9) + 1.  All share one launcher. */
int ar_variant_register_range(ar_region *r, double begin, double end, double step, ar_launch_fn fn,
                              void *user, int *out_count);

/* Region facts: variant count, feature count, effective min_train_data,
 * whether a model is trained (1) and the model kind (0 dtree, 1 mlp,
 * 2 exhaustive, 3 fixed, 4 rfc).  Any out pointer may be NULL. */
int ar_region_info(const ar_region *r, int *num_variants, int *num_features, int *min_train_data,
                   int *trained, int *model_kind);

/* Variant facts: numeric value, name (NUL-terminated, truncated to
 * name_len), usable flag (0 once its launcher failed).  Pointers may be NULL. */
int ar_variant_info(const ar_region *r, int variant, double *value, char *name, int name_len,
                    int *usable);

/* ---- Apollo-shaped execution calls (Table 1) ---------------------------- */

/* Begin a profiled execution (__apollo_region_begin): records a start event
 * on `stream` and clears the feature context.  AR_ERR_STATE if an execution
 * is already open or the region has no variant. */
int ar_begin(ar_region *r, void *stream);

/* Append one feature value (__apollo_region_set_feature).  AR_ERR_ARG for
 * NaN/inf, AR_ERR_STATE outside begin/end or beyond num_features. */
int ar_set_feature(ar_region *r, float value);

/* Variant to run for the current features (__apollo_region_get_policy),
 * in [0, num_variants-1]: the model's prediction once trained, else the
 * exploration policy (RoundRobin cycles the usable variants).  AR_ERR_STATE
 * unless all num_features features are set inside begin/end. */
int ar_get_policy(ar_region *r, int *out_variant);

/* End the execution (__apollo_region_end): records the stop event and a
 * pending record (features, variant, elapsed ms), then trains the model
 * automatically if this execution made the count of unique points reach
 * min_train_data (once).  AR_ERR_STATE without a matching begin/get_policy. */
int ar_end(ar_region *r, void *stream);

/* ---- Convenience execution calls ---------------------------------------- */

/* begin + set_feature x nf + get_policy + run the variant's launcher on
 * `args` + end.  nf must equal num_features (AR_ERR_STATE).  Returns the
 * variant index and value.  If the launcher fails the execution is dropped
 * (no record), the variant is marked unusable, and AR_ERR_CUDA is returned. */
int ar_invoke(ar_region *r, const float *features, int nf, void *args, void *stream,
              int *out_variant, double *out_value);

/* One block of host memory and its device counterpart, for ar_invoke_host. */
typedef struct ar_host_copy {
  void *host;   /* host address; pinned (cudaHostAlloc / cudaHostRegister)
                   for the copy to run asynchronously */
  void *device; /* device address (caller-owned) */
  size_t bytes;
} ar_host_copy;

/* End-to-end execution on host data (the region's execution of Table 1 with
 * its inputs and results in host memory): on `stream`, copy every `in`
 * block host -> device (one cudaMemcpyAsync each, in order), then ar_invoke
 * (features -> the model's or the exploration's variant -> its launcher ->
 * the profiling record, which times the variant only), then copy every `out`
 * block device -> host.  `args` holds the device addresses the variant
 * reads and writes (the `device` sides of the copies and any scratch the
 * caller owns).  Nothing blocks the host when the host blocks are pinned;
 * the results are in host memory once `stream` completes (pageable host
 * memory also works, with copies that block the host).  Independent
 * invocations on different streams overlap their copies with each other's
 * kernels.  Errors: as ar_invoke; AR_ERR_ARG for a bad copy list (NULL
 * pointer with a non-zero size, negative count) before anything is
 * enqueued; AR_ERR_CUDA if a copy cannot be enqueued. */
int ar_invoke_host(ar_region *r, const float *features, int nf, void *args, void *stream,
                   const ar_host_copy *in, int n_in, const ar_host_copy *out, int n_out, int *out_variant,
                   double *out_value);

/* Prediction only (no execution): the trained model's variant and its
 * confidence (MLP: max softmax probability; dtree: fraction of training
 * labels agreeing in the leaf; exhaustive/fixed: 1).  AR_ERR_NOMODEL if
 * no model is trained (an exhaustive table without this feature vector
 * also gives AR_ERR_NOMODEL). */
int ar_select(ar_region *r, const float *features, int nf, int *out_variant, float *out_conf);

/* Exhaustive profiling of one feature vector (blocking): for each usable
 * variant, one untimed warm-up then `reps` (<= 0: the spec's reps) timed
 * executions, each preceded by an L2 flush if a flush buffer is set.  The
 * launcher runs (reps+1) x num_variants times on the same `args`, so the
 * variant bodies must be repeatable on them.  Appends every timed execution
 * as a record.  out_ms (num_variants floats, may be NULL) receives each
 * variant's mean (+inf for unusable ones); out_best the fastest, means
 * within the region's tie fraction (0.5 % by default) tying to the lowest
 * index. */
int ar_profile(ar_region *r, const float *features, int nf, void *args, void *stream, int reps,
               float *out_ms, int *out_best);

/* Train the region's model on all records so far (__apollo_region_train).
 * Resolves pending events first (blocking).  Labels: for each distinct
 * feature vector, the variant with the lowest mean time (ties within the
 * region's tie fraction, 0.5 % by default, to the lowest index).  AR_ERR_STATE with no records; AR_ERR_CUDA if MLP
 * training on the device fails. */
int ar_train(ar_region *r);

/* Block until every pending record is resolved. */
int ar_flush_records(ar_region *r);

/* Insert an externally measured record (e.g. gathered in earlier runs). */
int ar_add_record(ar_region *r, const float *features, int nf, int variant, float ms);

/* Number of resolved records, and of unique (features, variant) points
 * (pending executions included). */
int ar_record_counts(const ar_region *r, int64_t *num_records, int64_t *num_unique);

/* Copy resolved records [first, first+count): features as count rows of
 * AR_MAX_FEATURES floats (unused slots 0), variants, elapsed ms. */
int ar_get_records(const ar_region *r, int64_t first, int64_t count, float *features, int *variants,
                   float *ms);

/* Export the decision tree: up to max_nodes nodes; feat[i] = -1 marks a
 * leaf.  A sample goes to left[i] when (double)x[feat[i]] <= thr[i].
 * AR_ERR_NOMODEL if the region has no trained tree. */
int ar_tree_export(const ar_region *r, int max_nodes, int *feat, double *thr, int *left, int *right,
                   int *label, int *out_nodes);

/* Random forest: number of trees, and one tree in the layout of
 * ar_tree_export.  Each tree is CART grown on a bootstrap sample of the
 * training set with max(1, floor(sqrt(num_features))) candidate features per
 * split; all draws come from one SplitMix64 stream (the spec's seed, default
 * 0x5eed) consumed tree by tree: the n bootstrap indices (next() mod n), then
 * per split attempt in depth-first preorder a partial Fisher-Yates shuffle
 * (a + next() mod (F - a)).  Prediction: majority vote, ties to the lowest
 * variant; confidence = vote share.  AR_ERR_NOMODEL without a trained forest. */
int ar_forest_size(const ar_region *r, int *ntrees);
int ar_forest_tree_export(const ar_region *r, int tree, int max_nodes, int *feat, double *thr, int *left,
                          int *right, int *label, int *out_nodes);

/* Export the trained MLP: theta (ar_mlp_num_params floats, layout of
 * ar_loops.h), mu and sd (F floats each).  Any pointer may be NULL to query
 * the dimensions only.  AR_ERR_NOMODEL if no MLP is trained. */
int ar_mlp_export(const ar_region *r, float *theta, float *mu, float *sd, int *F, int *H, int *V);

/* Persist / restore records and model (Section 2: records persist across
 * runs in a per-region store; Section 3: a model trained in one run serves
 * later runs).  Versioned binary file with a checksum.  Load replaces the
 * region's records and model; it needs the same feature and variant counts
 * (AR_ERR_STATE) and a well-formed file (AR_ERR_IO otherwise). */
int ar_region_save(const ar_region *r, const char *path);
int ar_region_load(ar_region *r, const char *path);

/* Copy the last error message (NUL-terminated, truncated to len). */
int ar_last_error(const ar_region *r, char *buf, int len);

/* Replace CUDA-event timing by a deterministic host cost model (tests).
 * NULL restores event timing. */
int ar_set_fake_timer(ar_region *r, ar_fake_time_fn fn, void *user);

/* Device buffer overwritten before every timed ar_profile execution so that
 * memory-bound variants are timed from HBM rather than L2 (NULL/0 disables).
 * Borrowed: must outlive the region or be reset. */
int ar_set_l2_flush(ar_region *r, void *device_buf, size_t bytes);

#ifdef __cplusplus
}
#endif
#endif /* AR_H */
