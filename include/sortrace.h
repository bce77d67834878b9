/*
 * sortrace.h -- C ABI of a GB300 (sm_103a) comparison sort.
 *
 * The operation is the one the paper ("Sort Race", arXiv 1609.04471) races its
 * methods on: order an array of items under one comparison, in place, with the
 * caller owning the array -- the C library's qsort(base, n, size, cmp) model
 * that every method of the paper implements (Section 5; Appendix A's
 * mergesort6 has exactly that signature).  Here the comparison is fixed by a
 * key type instead of a function pointer:
 *
 *   SR_KEY_I32 / SR_KEY_I64   two's-complement signed order
 *   SR_KEY_U32 / SR_KEY_U64   unsigned order
 *   SR_KEY_F32                IEEE-754 totalOrder on the bit patterns
 *                             (-0.0 < +0.0; NaNs, if any, by their patterns)
 *
 * "Sorted" means non-decreasing (Section 2, the definition of Run(A)).  Output
 * bit patterns are the input bit patterns, permuted.
 *
 * Memory and streams.  Every pointer named d_* is a device pointer on the
 * current CUDA device, aligned to its element size; the caller owns it.  The
 * library allocates its scratch stream-ordered on `stream` from a pool it owns
 * and frees it on the same stream.  Calls are asynchronous: results are valid
 * once `stream` completes.  `stream` is a cudaStream_t passed as void*; NULL
 * means the legacy default stream.
 *
 * Errors.  Argument errors are reported before anything is launched and leave
 * the memory untouched.  n <= 1 is a no-op that returns SR_OK.  A failed launch
 * or allocation returns SR_ERR_CUDA or SR_ERR_OOM (the data may then be
 * partially permuted).  Errors found on the device (bad segment offsets) are
 * recorded in a per-device status word and returned by sr_stream_status().
 * No C++ exception crosses this interface.  Thread safety: calls may come from
 * several host threads; each call's device work is ordered on its stream.
 */
#ifndef SORTRACE_H
#define SORTRACE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SR_ABI_VERSION 2

typedef enum {
    SR_KEY_I32 = 0,
    SR_KEY_U32 = 1,
    SR_KEY_F32 = 2,
    SR_KEY_U64 = 3,
    SR_KEY_I64 = 4
} sr_key_type;

typedef enum {
    SR_OK = 0,
    SR_ERR_INVALID_ARG = 1,  /* null pointer with n > 0, unknown key type, bad option */
    SR_ERR_UNSUPPORTED = 2,  /* valid request this build does not serve */
    SR_ERR_OOM = 3,          /* scratch allocation failed */
    SR_ERR_CUDA = 4,         /* a CUDA call or launch failed */
    SR_ERR_TIMEOUT = 5,      /* a bounded device-side wait ran out */
    SR_ERR_INTERNAL = 6,     /* a device-side consistency check failed */
    SR_ERR_BAD_SEGMENTS = 7  /* segment offsets not non-decreasing within [0, total] */
} sr_status;

typedef void *sr_stream;     /* a cudaStream_t */

/*
 * sr_sort_keys -- sorts d_keys[0..n) in place, ascending under the order of kt.
 *   d_keys  device array of n keys of type kt (4-byte keys: 4-byte aligned;
 *           8-byte keys: 8-byte aligned).
 * The result is unique (equal keys are indistinguishable).  Inputs that are
 * already sorted are left untouched, and strictly descending inputs are
 * reversed in one pass: the adaptivity the paper credits for its mergesort
 * and quicksort wins (Section 4, the remark that with techniques (e) and (f)
 * quicksort takes O(n) on sorted and reversely sorted lists; Section 3,
 * technique (a)).  Inputs with few keys out of place (k-exchange lists,
 * Section 2) take the few-displaced-keys path: the keys left in order stay in
 * order and only the others are sorted on the side.  Cites: Section 1 (the
 * race's operation), Section 5 (qsort interface), Section 2 (sortedness).
 * Asynchronous on `stream`.  A call repeated with the same arguments (key type,
 * n, buffer) on any stream replays a CUDA graph the library builds on the
 * second such call; the graph and its scratch stay with the library (at most
 * 16 argument sets per process, least recently used dropped).  Calls inside a
 * stream capture launch their kernels into the capture instead.
 */
sr_status sr_sort_keys(void *d_keys, size_t n, sr_key_type kt, sr_stream stream);

/*
 * sr_release_cached -- drops the graphs (and their scratch) that the library
 * keeps for repeated sr_sort_keys / sr_sort_pairs calls on the current device,
 * after waiting for their last replays.  Later calls build them again.
 */
sr_status sr_release_cached(void);

/*
 * sr_sort_pairs -- stable sort of (d_keys[i], d_vals[i]) by key, in place.
 *   d_keys  n keys of type kt;  d_vals  n uint32 payloads moved with their keys.
 * Equal keys keep their input order: the mergesort's stability (Section 6,
 * where stability is what decides for mergesort; Section 3, technique (a),
 * the stable treatment of equal items in reversed runs).  With payload =
 * original index the output is unique.  Repeated calls replay a graph as for
 * sr_sort_keys.
 */
sr_status sr_sort_pairs(void *d_keys, uint32_t *d_vals, size_t n, sr_key_type kt,
                        sr_stream stream);

/*
 * sr_sort_segmented -- sorts every segment d_keys[off[s] .. off[s+1]) on its own,
 * s = 0 .. num_segments-1, in one batched launch sequence.
 *   d_offsets  device array of num_segments + 1 int64 offsets (CSR); must be
 *              non-decreasing with d_offsets[0] >= 0.  Empty segments are allowed.
 * Offsets are read on the device; offsets that fail the check set the device
 * status word to SR_ERR_BAD_SEGMENTS (see sr_stream_status) and no key is moved.
 * The total length d_offsets[num_segments] is read back first (the call waits
 * for `stream` once); use sr_sort_segmented_ex to avoid that.
 * The paper sorts one array per call; the batch is each of those calls side by
 * side (Section 1: the same operation on many instances).
 */
sr_status sr_sort_segmented(void *d_keys, const int64_t *d_offsets, size_t num_segments,
                            sr_key_type kt, sr_stream stream);

/*
 * sr_sort_segmented_ex -- sr_sort_segmented with the key array's length given:
 *   n_keys  length of d_keys; every offset must lie in [0, n_keys].
 * sr_sort_segmented reads d_offsets[num_segments] back to the host once (it
 * waits for `stream`) to size its scratch; this form reads nothing back, so a
 * sequence of calls can be captured in a CUDA graph (the first call on a
 * device must come before any capture).  Small segments are sorted many to a
 * CTA, medium ones one per CTA, and long ones by merge passes, all from one
 * persistent work queue (see stats.big_segments).
 */
sr_status sr_sort_segmented_ex(void *d_keys, size_t n_keys, const int64_t *d_offsets,
                               size_t num_segments, sr_key_type kt, sr_stream stream);

/*
 * Launch configurations of the segmented sort.  Each key width has a fixed
 * list (sr_segmented_num_configs); sr_segmented_config_info describes entry
 * `config`:
 *   strategy       0: small segments (<= small_keys) are sorted many to a CTA
 *                  as (segment, key) composites ("packs"); 1: one CTA of the
 *                  smallest of five fixed shapes per small segment (<= 3840
 *                  keys), from ladder `ladder`: 0 = 128x9, 128x15, 256x9,
 *                  256x11, 256x15 (threads x keys per thread); 1 = 64x9,
 *                  128x9, 128x15, 256x11, 256x15; 2 = 128x13, 128x17,
 *                  128x19, 128x23, 256x15.
 *   sort_threads   threads of the persistent sort CTA.
 *   pack_items     composite keys per thread of a pack (strategy 0; else 0).
 *   tile_items     keys per thread of a block-sort tile; tile_keys =
 *                  sort_threads * tile_items.
 *   fan_in         merge fan-in: block-sort tiles one CTA merges in shared
 *                  memory, so one CTA sorts a segment of up to cta_keys =
 *                  fan_in * tile_keys keys; longer segments go through global
 *                  merge passes starting from runs of cta_keys keys.
 *   merge_threads  threads of a global merge tile (tile_items keys each).
 * Every configuration gives the same (unique) result; they differ in speed
 * with the segment-length mix.  The package's autotuner times them on a
 * workload and keeps the fastest.  SR_SEG_CONFIG_DEFAULT (-1) selects the
 * library default (entry 0).  sr_segmented_config_info returns
 * SR_ERR_INVALID_ARG for an unknown key type or entry or a null `out`.
 */
#define SR_SEG_CONFIG_DEFAULT (-1)
typedef struct sr_segmented_config {
    int32_t strategy;
    int32_t sort_threads;
    int32_t pack_items;
    int32_t tile_items;
    int32_t fan_in;
    int32_t merge_threads;
    int64_t tile_keys;
    int64_t cta_keys;
    int64_t small_keys;         /* longest segment sorted as a small one */
    int32_t ladder;             /* strategy 1: small-shape ladder; else -1 */
    int32_t reserved;
} sr_segmented_config;

int sr_segmented_num_configs(sr_key_type kt);
sr_status sr_segmented_config_info(sr_key_type kt, int config, sr_segmented_config *out);

/*
 * sr_sort_segmented_cfg -- sr_sort_segmented_ex under launch configuration
 * `config` (0 .. sr_segmented_num_configs(kt) - 1, or SR_SEG_CONFIG_DEFAULT);
 * SR_ERR_INVALID_ARG for any other value.  Reads nothing back to the host
 * (graph-capturable like sr_sort_segmented_ex, which is this call with
 * SR_SEG_CONFIG_DEFAULT).
 */
sr_status sr_sort_segmented_cfg(void *d_keys, size_t n_keys, const int64_t *d_offsets,
                                size_t num_segments, sr_key_type kt, int config, sr_stream stream);

/*
 * sr_sort_keys_host -- sr_sort_keys on a HOST array: copies h_keys[0..n) to the
 * device, sorts it there and copies it back, then waits for `stream`.  Pinned
 * host memory gives the fastest copies; pageable memory also works.
 */
sr_status sr_sort_keys_host(void *h_keys, size_t n, sr_key_type kt, sr_stream stream);

/*
 * sr_sort_keys_host_async -- sr_sort_keys_host without the final wait: the
 * copy in, the sort and the copy out are queued on `stream` and the call
 * returns at once.  h_keys must be page-locked host memory (cudaHostAlloc /
 * cudaHostRegister; SR_ERR_INVALID_ARG otherwise) and must not be touched
 * until the stream completes.  Calls on different streams overlap one
 * array's copies with another's sort.
 */
sr_status sr_sort_keys_host_async(void *h_keys, size_t n, sr_key_type kt, sr_stream stream);

/*
 * sr_sort_keys_host_many -- sorts `count` host arrays h_keys[i][0..n[i]) of key
 * type kt in place, as a pipeline: array i+1 is copied in while earlier ones
 * are sorted and copied out (the library's streams: one for the copies in, in
 * array order, and two lanes of sort + copy out that take the arrays in turn).  Queued after the caller's earlier work on `stream`; the caller's
 * later work on `stream` waits for all of it; the call returns at once.
 * Every array with n[i] > 1 must be page-locked host memory (else
 * SR_ERR_INVALID_ARG before anything is queued) and left alone until the
 * stream completes.  Same result per array as sr_sort_keys.
 */
sr_status sr_sort_keys_host_many(void *const *h_keys, const size_t *n, int count, sr_key_type kt,
                                 sr_stream stream);

/*
 * sr_sort_keys_noalloc -- sr_sort_keys for callers that must not allocate device
 * memory while they sort (a service that reserves all of its memory up front
 * so it can never hit out-of-memory mid-request, a framework that forbids
 * allocations behind its back, a latency-critical path where an allocation
 * could stall).  It allocates nothing: its scratch is one fixed device array
 * inside this library, present on every GPU that loads the library until the
 * process exits.  The paper has no counterpart; it is an interface variant.
 *   n        at most SR_NOALLOC_MAX_KEYS keys (any key type); a larger n returns
 *            SR_ERR_INVALID_ARG and leaves the keys untouched.
 * Same result as sr_sort_keys.  All calls on a device share the one scratch
 * array, which keeps the previous call's contents (each call clears what it
 * needs zeroed): calls whose device work overlaps in time race and give wrong
 * results -- keep them ordered on one stream.  The first call on each device
 * looks up the array's device address and should come before any stream
 * capture.  sr_get_stats does not report on these calls.
 */
#define SR_NOALLOC_MAX_KEYS (1u << 20)
sr_status sr_sort_keys_noalloc(void *d_keys, size_t n, sr_key_type kt, sr_stream stream);

/* Options of the learned-partition sort; zero fields take the defaults. */
typedef struct {
    uint32_t num_buckets;    /* power of two in [2^4, 2^20]; default 2^16 */
    uint32_t sample_stride;  /* one key in sample_stride is sampled; default 100 */
    uint32_t train_points;   /* points of the sorted sample used in training; default 2048 */
    uint32_t train_steps;    /* full-batch Adam steps; default 16 */
    float learning_rate;     /* Adam step size; default 1e-3 */
    uint32_t model;          /* SR_MODEL_* */
    uint32_t bucket_config;  /* 1 + the segmented-sort configuration that sorts the
                                buckets (sr_segmented_config_info); 0: the default */
} sr_learned_opts;

enum {
    SR_MODEL_TRAINED = 0,      /* the trained monotone network */
    SR_MODEL_EQUAL_WIDTH = 1,  /* ablation: equal-width buckets over [min, max] */
    SR_MODEL_UNTRAINED = 2,    /* the quantile start, no training steps */
    SR_MODEL_FORCE_BAD = 3     /* test hook: a non-monotone router; the check must fail */
};

/*
 * sr_sort_keys_learned -- same result as sr_sort_keys (bit for bit), computed by
 * routing keys to buckets with a small monotone network trained on a sorted
 * sample of the input, scattering them, sorting each bucket, and checking
 * that every bucket's largest key is <= the next bucket's smallest; if the
 * check fails the plain sort runs instead (the fallback is in stats.fallback).
 * The call reads the check's outcome back, so it waits for `stream` once;
 * inside a stream capture it reads nothing back: the plain sort becomes the
 * body of a conditional (IF) graph node whose condition the check sets on the
 * device, so the whole call can be captured and replayed (the first call on a
 * device must come before any capture).
 * The paper has no learned component; this is the partition-then-sort form of
 * its quicksort (Section 4: split by pivots, then sort the parts), with the
 * pivots read off a learned CDF.
 */
sr_status sr_sort_keys_learned(void *d_keys, size_t n, sr_key_type kt,
                               const sr_learned_opts *opts, sr_stream stream);

/*
 * Presortedness of the input as the run-detection scan sees it (Section 2):
 * runs = Run(A) = descents + 1; sorted = (runs == 1); strictly_descending = every
 * neighbour pair descends.  Tile counts refer to the scan's tiles of `tile` keys.
 */
typedef struct {
    uint64_t n;
    uint64_t runs;
    int32_t sorted;
    int32_t strictly_descending;
    uint64_t tile;
    uint64_t tiles;
    uint64_t tiles_ascending;   /* tiles with no descent inside */
    uint64_t tiles_descending;  /* tiles strictly descending inside */
} sr_run_info;

/* sr_detect_runs -- runs the scan on d_keys and waits for it; fills *out. */
sr_status sr_detect_runs(const void *d_keys, size_t n, sr_key_type kt, sr_run_info *out,
                         sr_stream stream);

/* What the last sort call on this host thread did. */
typedef struct {
    uint32_t abi_version;
    int32_t call;               /* 1 keys, 2 pairs, 3 segmented, 4 learned */
    uint64_t n;
    int32_t key_type;
    int32_t tile;               /* keys per block-sort tile */
    int32_t merge_tile;         /* output keys per merge CTA */
    int32_t passes_planned;     /* merge steps launched (each a 4-way or 2-way merge pass over the data) */
    int32_t passes_skipped;     /* steps found already in order (no bytes moved) */
    int32_t input_class;        /* 0 unsorted, 1 sorted, 2 strictly descending,
                                   3 at most 64 distinct keys (4-byte keys, keys only:
                                   counted per distinct key and written as runs),
                                   4 few displaced keys (keys only: the keys left in
                                   order merged with the displaced ones, sorted on
                                   the side) */
    int32_t fallback;           /* learned: 1 if the bucket check failed */
    uint64_t runs;              /* Run(A) of the input, from the scan */
    uint64_t bytes_moved;       /* DRAM bytes the executed passes read + wrote */
    uint64_t max_bucket;        /* learned: largest bucket */
    uint64_t big_segments;      /* segmented: segments longer than one tile */
    float model_loss;           /* learned: training loss after the last step */
    float bucket_imbalance;     /* learned: B * sum(c_b^2) / n^2 over bucket sizes c_b; 1 = even */
    uint64_t displaced;         /* input class 4: keys sorted on the side (at least Rem(A),
                                   Section 2: the kept ones are in order); 0 otherwise */
} sr_stats;

/* sr_get_stats -- waits for the last call's stream and fills *out. */
sr_status sr_get_stats(sr_stats *out);

/* sr_stream_status -- waits for `stream`, returns the device status word of the
 * current device (SR_OK if clean) and clears it. */
sr_status sr_stream_status(sr_stream stream);

/* sr_status_string -- a static, human-readable name for s. */
const char *sr_status_string(sr_status s);

/* ---------------------------------------------------------------------------
 * Instrumentation.  Every kernel the library launches belongs to one of these
 * kinds.  sr_launch_count() is the number of kernels the library has launched
 * in this process (graph replays included: once a replay has run on the
 * current device, the call waits for that device's queued work to read the
 * kernels the replays' branches ran).  Between sr_profile_begin() and sr_profile_end() the calls
 * made by this host thread bracket each launch with CUDA events on the
 * launch's own stream; sr_profile_end() waits for them and returns, per kind,
 * the launch count and the summed device time (ms).  Profiling cannot be
 * used inside a stream capture.
 * ------------------------------------------------------------------------- */
enum {
    SR_KERNEL_DETECT = 0,     /* run-detection scan */
    SR_KERNEL_REVERSE = 1,    /* whole-input reversal */
    SR_KERNEL_BLOCK_SORT = 2, /* shared-memory tile sort */
    SR_KERNEL_PARTITION = 3,  /* merge pass planning (which passes have pairs out of order) */
    SR_KERNEL_MERGE = 4,      /* global merge pass */
    SR_KERNEL_COPY = 5,       /* copy-back / gather */
    SR_KERNEL_SEGMENTED = 6,  /* segmented / bucket sorts */
    SR_KERNEL_MODEL = 7,      /* learned router: train, predict, histogram, scatter */
    SR_KERNEL_DISPLACED = 8,  /* keys out of place: the few-displaced-keys path (bounds, split, bucket
                                 sorts, merge) and the in-place merges of the neighbour repair */
    SR_KERNEL_KINDS = 9
};

typedef struct {
    uint64_t launches;
    double ms;
} sr_kernel_time;

uint64_t sr_launch_count(void);
sr_status sr_profile_begin(void);
sr_status sr_profile_end(sr_kernel_time *out, int count);

/* ---------------------------------------------------------------------------
 * The learned partitioner's model, exposed for tests and reuse.
 *
 * Network (H = SR_MODEL_HIDDEN hidden units, one input x = normalised key):
 *   d_j = softplus(delta_j),  x_j = x0 + sum_{i<j} d_i   (knots, j = 0..H)
 *   h_j = min(max((x - x_j) / d_j, 0), 1)                (hidden layer)
 *   w = softmax(beta),  y = sum_j w_j h_j                (predicted CDF)
 * theta = [x0, delta[H], beta[H]] (SR_MODEL_PARAMS floats).
 * Loss over samples (x_i, t_i): L = mean (y(x_i) - t_i)^2.
 * ------------------------------------------------------------------------- */
#define SR_MODEL_HIDDEN 32
#define SR_MODEL_PARAMS 65

/* sr_model_loss_grad -- forward and backward pass on the device over m points
 * d_x[i], d_t[i] (float32); writes L to *h_loss and dL/dtheta to h_grad[65].
 * Synchronous. */
sr_status sr_model_loss_grad(const float *d_x, const float *d_t, size_t m,
                             const float *h_theta, float *h_loss, float *h_grad,
                             sr_stream stream);

/* sr_model_train -- `steps` full-batch Adam steps on the device starting from
 * h_theta (updated in place); the final loss goes to *h_loss.  Synchronous. */
sr_status sr_model_train(const float *d_x, const float *d_t, size_t m, float *h_theta,
                         uint32_t steps, float learning_rate, float *h_loss,
                         sr_stream stream);

/* sr_model_buckets -- bucket of every key: x = (ord(key) - lo) / (hi - lo) with
 * ord the key's order-preserving unsigned image (lo, hi given in that image),
 * bucket = min(floor(y(x) * num_buckets), num_buckets - 1) into d_out[n]. */
sr_status sr_model_buckets(const void *d_keys, size_t n, sr_key_type kt, const float *h_theta,
                           uint64_t lo, uint64_t hi, uint32_t num_buckets, uint32_t *d_out,
                           sr_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* SORTRACE_H */
