/*
 * rsort.h -- C ABI of librsort, a single-GPU (GB300, sm_103a) implementation of
 * the robust sample-sort partition step of Axtmann & Sanders, "Robust Massively
 * Parallel Sorting" (arXiv 1606.08766), and the sorts built on it.
 *
 * The paper's processing elements become virtual partitions of one GPU's HBM:
 * virtual partition i of p holds the positions [floor(i*n/p), floor((i+1)*n/p))
 * of the input and, after partitioning, the i-th bucket of the output.
 *
 * Conventions shared by every entry point
 *   - Every function returns an rsort_status and never throws or aborts.
 *   - "d_" pointers are DEVICE pointers on the context's device; the caller owns
 *     them.  Host pointers are named without the prefix.
 *   - stream: a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Work is enqueued on it and the call returns without waiting, unless the
 *     function says otherwise.
 *   - Keys are 64-bit patterns: RSORT_KEY_U64 orders them as unsigned
 *     integers; RSORT_KEY_F64 orders IEEE-754 binary64 values by their bit
 *     pattern mapped to an unsigned integer (negative: all bits flipped,
 *     non-negative: sign bit flipped), so -0.0 < +0.0 and NaNs sit beyond the
 *     infinities of their sign.  Outputs always hold the original bits.
 *   - Ties are broken by the original position (Section 2: unique identifiers
 *     compared lexicographically), so every result below is unique: it does not
 *     depend on the seed, the plan, the batch or the device schedule.
 *   - n <= 2^32 - 1 (positions are 32-bit); larger n gives RSORT_EINVAL.
 *   - Errors raised asynchronously on the device (a capacity check, an expired
 *     bounded wait) are latched in the context and returned by rsort_check(),
 *     by a stats read-back, and by the next call.
 */
#ifndef RSORT_H
#define RSORT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t rsort_status;
#define RSORT_OK 0
#define RSORT_PENDING 1
#define RSORT_EINVAL (-1)
#define RSORT_ENOMEM (-2)
#define RSORT_ECUDA (-3)
#define RSORT_ETIMEOUT (-4)
#define RSORT_ECANCELLED (-5)
#define RSORT_EUNSUPPORTED (-6)
#define RSORT_EDEVICE (-7)

typedef int32_t rsort_key_type;
#define RSORT_KEY_U64 0
#define RSORT_KEY_F64 1

typedef struct rsort_ctx rsort_ctx;

/* Statistics of one rsort_sort call (read back on request). */
typedef struct {
    uint64_t n;              /* elements sorted                                  */
    uint32_t p;              /* virtual partitions = level-1 buckets             */
    uint32_t levels;         /* partition levels that had work                   */
    uint32_t path;           /* 0: direct in-SM sort, 1: sample-sort levels       */
    uint32_t max_bucket;     /* largest level-1 bucket (virtual partition)       */
    double max_over_mean;    /* max_bucket / (n/p): the imbalance of Section 2    */
    uint64_t final_buckets;  /* buckets handed to the in-SM sort                 */
    uint64_t bytes_moved;    /* algorithmic HBM bytes of the whole call          */
    uint64_t level_elems[4]; /* elements partitioned at levels 1..4 (0: unused)  */
    uint64_t class_elems[5]; /* elements handed to the in-SM sort by size class:
                                copy-through, <= 1024, <= 2048, <= 4096, larger */
    uint64_t algo_elems[6];  /* elements finished by each in-SM algorithm (the
                                size-dependent choice of Section 6): [0]
                                rank-by-counting, [1] equal-width bins, [2]
                                bitonic (clustered keys), [3] quicksort
                                (medium_sort = 1), [4] oversize merge sort, [5]
                                all keys equal and already in position order.
                                Copy-through buckets (class_elems[0]) are not
                                sorted and are not counted here.             */
} rsort_stats;

/* Creates a context on CUDA device `device`.  hbm_budget_bytes caps the scratch
 * the context may hold (0 = no cap).  tune_table_path: NULL for the built-in
 * plan table, else a text file of "name value" lines overriding tunables.
 * The context owns its scratch pool; the caller owns *out and must call
 * rsort_destroy.  Errors: EINVAL (bad device / unreadable table), ECUDA. */
rsort_status rsort_create(rsort_ctx **out, int device, uint64_t hbm_budget_bytes,
                          const char *tune_table_path);

/* Waits for the context's outstanding work, frees its scratch and the
 * context.  NULL is accepted and ignored. */
rsort_status rsort_destroy(rsort_ctx *ctx);

/* Static, human-readable text for a status code. */
const char *rsort_strerror(rsort_status status);

/* Synchronises the context's last stream and returns the first latched device
 * or CUDA error (RSORT_OK if none), clearing it. */
rsort_status rsort_check(rsort_ctx *ctx);

/* ONE level of the robust sample-sort partition step (Appendix "Robust
 * Multi-Level Sample Sort"; splitters every S/k-th sample, Appendix
 * "Generalizing Quicksort"):
 *   1. S = min(n, 16*ceil(log2 k)*k) samples, sample j drawn from positions
 *      [floor(j*n/S), floor((j+1)*n/S)) at offset splitmix64(seed, j) modulo
 *      the stratum size, each carrying its position as tie-breaker;
 *   2. the sample is sorted by (key, position);
 *   3. splitter j (j = 1..k-1) is sorted sample floor(j*S/k);
 *   4. element (x, i) goes to bucket #{splitters lexicographically < (x, i)};
 *   5. buckets are written in order, each in increasing position.
 * d_keys_in [n] (read only, must not alias the outputs), d_keys_out [n],
 * d_pos_out [n] (original positions), d_offsets_out [k+1] (bucket starts,
 * d_offsets_out[k] = n).  1 <= k <= 2048.  Errors: EINVAL, ENOMEM, ECUDA. */
rsort_status rsort_partition(rsort_ctx *ctx, rsort_key_type type, const void *d_keys_in,
                             uint64_t n, uint32_t k, uint64_t seed, void *d_keys_out,
                             uint32_t *d_pos_out, uint64_t *d_offsets_out, void *stream);

/* Options of rsort_partition_ex (NULL = the plain robust step). */
typedef struct rsort_partition_opts {
    /* 1: classify (key, position) pairs lexicographically -- the robust step;
     * 0: classify by key only, #{splitter keys < x}, so all copies of a key
     *    land in one partition: the "no tie-breaking" ablation the paper
     *    measures against its robust AMS-sort (NTB-AMS, Section 6). */
    uint32_t tie_break;
    /* b >= 1.  b > 1: AMS-sort overpartitioning (Section 3 on AMS-sort;
     * Appendix "Implementation Details" picks b = 2 / ((1+eps)^(1/l) - 1), so
     * b = 10 for eps = 0.2 with one level).  The same sample gives b*k - 1
     * fine splitters (sorted sample floor(j*S/(b*k)), j = 1..b*k-1); the exact
     * sizes of the b*k fine partitions are counted, and consecutive fine
     * partitions are assigned to the k outputs by an in-order greedy scan
     * under the smallest load bound L that needs at most k groups (this
     * minimises the largest output; L <= ceil(n/k) + largest fine partition).
     * Requires b*k <= 10240.  b = 1: no overpartitioning. */
    uint32_t overpartition;
} rsort_partition_opts;

/* rsort_partition with the options above.  Same arguments, layout and errors
 * as rsort_partition, plus two optional device outputs (NULL to skip):
 *   d_fine_sizes_out  [b*k] u64: size of every fine partition (b = 1: of
 *                     every output);
 *   d_group_first_out [k+1] u32: first fine partition of every output
 *                     (output g holds fine partitions [first[g], first[g+1]);
 *                     empty trailing outputs start at b*k).
 * Output g holds, in increasing position, the elements whose fine partition
 * lies in its range.  Errors: EINVAL (also tie_break > 1, overpartition == 0,
 * b*k > 10240), ENOMEM, ECUDA. */
rsort_status rsort_partition_ex(rsort_ctx *ctx, rsort_key_type type, const void *d_keys_in,
                                uint64_t n, uint32_t k, uint64_t seed,
                                const rsort_partition_opts *opts, void *d_keys_out,
                                uint32_t *d_pos_out, uint64_t *d_offsets_out,
                                uint64_t *d_fine_sizes_out, uint32_t *d_group_first_out,
                                void *stream);

/* Binary-tree median approximation (Section 3, "Approximate Median Selection
 * with a Single Reduction"; the pivot rule of the paper's robust quicksort).
 * Leaf i holds element i (in the order given; shuffle first for the paper's
 * randomly permuted input), the leaves are padded with empty ones to a power
 * of two P, and every node forwards a window of k entries:
 *   - a leaf with one element: its element with k/2 entries below it and
 *     k/2 - 1 above (coin 0) or k/2 - 1 below and k/2 above (coin 1);
 *   - an empty leaf: k/2 entries below and k/2 above every element;
 *   - an internal node: the middle k of its children's 2k merged entries.
 * The root returns its window entry k/2 (coin 0) or k/2 + 1 (coin 1, 1-based),
 * moving to the nearest element when that entry is not one.
 *   - Coins: bit 0 of splitmix64(seed, i) for leaf i, of splitmix64(seed, P)
 *     at the root.
 *   - Elements are ordered by (key, position); float64 keys by their mapped
 *     IEEE bit pattern.
 * d_keys [n] (1 <= n <= 2^24, device); k in {2, 4, 8, 16, 32}; *d_pos_out
 * (device u64) receives the position of the chosen element.  One CTA
 * reduces the tree through the context's scratch (24 bytes per leaf).
 * Errors: EINVAL, ENOMEM, ECUDA. */
rsort_status rsort_approx_median(rsort_ctx *ctx, rsort_key_type type, const void *d_keys,
                                 uint64_t n, uint32_t k, uint64_t seed, uint64_t *d_pos_out,
                                 void *stream);

/* Plain sort (Section 2's output contract): keys_out[j] = keys_in[perm[j]] with
 * (key, perm[j]) strictly increasing.  Large inputs run the multi-level robust
 * sample sort (level 1 with k = p_virtual buckets, deeper levels until buckets
 * fit one SM, then an in-shared-memory sort per bucket: rank-by-counting for
 * tiny buckets, bitonic for medium ones -- the paper's size-dependent choice,
 * Section 6 and Appendix "Parameter Tuning").  d_keys_in may alias d_keys_out.
 * p_virtual: 1 (choose automatically) or 2..2048.  seed: sampling seed (does
 * not change the result).  opt_stats: NULL, or a host struct filled after a
 * synchronising read-back.  Errors: EINVAL, ENOMEM, ECUDA, EDEVICE. */
rsort_status rsort_sort(rsort_ctx *ctx, rsort_key_type type, const void *d_keys_in,
                        void *d_keys_out, uint32_t *d_perm_out, uint64_t n,
                        uint32_t p_virtual, uint64_t seed, void *stream,
                        rsort_stats *opt_stats);

/* Batched segmented sort in one launch sequence: every segment
 * s = [d_offsets[s], d_offsets[s+1]) of the n keys is sorted on its own, with
 * segment-LOCAL positions in d_perm_out (the same bytes as sorting that
 * segment alone with rsort_sort).  All segments share every launch: segments
 * of at most 4096 keys go straight to the in-shared-memory sort
 * (rank-by-counting when tiny), larger ones run the robust sample-sort levels
 * with a per-segment bucket count; the choice by segment size is the paper's
 * size-dependent algorithm choice (Section 6, Appendix "Parameter Tuning").
 * d_offsets: device array of num_segments + 1 nondecreasing u64 values with
 * d_offsets[num_segments] <= n; keys outside the segments are left untouched.
 * Offsets are checked on the device: a violation skips that segment and is
 * reported as RSORT_EDEVICE by rsort_check.  d_keys_in must not alias
 * d_keys_out.  No host synchronisation: once the context's scratch has been
 * sized by a first call of the same n, the call can be captured in a CUDA
 * graph.  Errors: EINVAL, ENOMEM, ECUDA (EDEVICE via rsort_check). */
rsort_status rsort_segmented(rsort_ctx *ctx, rsort_key_type type, const void *d_keys_in,
                             void *d_keys_out, uint32_t *d_perm_out, uint64_t n,
                             const uint64_t *d_offsets, uint32_t num_segments, uint64_t seed,
                             void *stream);

/* Allocation-free variant of rsort_partition (the paper has no counterpart;
 * this is a library-level convenience).  It exists for callers that cannot
 * allocate device memory at the moment they partition: frameworks whose
 * device memory must all come from their own allocator (which would not see
 * an allocation made here), and real-time loops that forbid allocation after
 * start-up because an allocation can block.  It needs no context.
 *   - Same arguments and result as rsort_partition (caller-owned inputs and
 *     outputs), on the CURRENT device and the given stream.
 *   - Scratch comes from one fixed 8 MiB device array inside librsort that
 *     every GPU loading the library holds until the process exits.  Limit:
 *     k <= 1024 (any n <= 2^32 - 1); larger k returns RSORT_EINVAL.
 *   - The first call on a device looks up that array's device address and
 *     sets kernel attributes (runtime calls that later calls skip).
 *   - Every call uses the same array (its contents persist between calls and
 *     are re-initialised by each call), so calls whose work overlaps on the
 *     GPU (other streams, other host threads) race: serialise them.
 *   - It calls no cudaMalloc, cudaFree or other allocating routine.
 *   - Errors: EINVAL (arguments, k > 1024), ECUDA (a launch failed).  It
 *     reads nothing back from the device, so device-side capacity flags are
 *     not reported; none can be raised, because the host sizes every scratch
 *     region for the largest plan the device computes from (n, k). */
rsort_status rsort_partition_noalloc(rsort_key_type type, const void *d_keys_in, uint64_t n,
                                     uint32_t k, uint64_t seed, void *d_keys_out,
                                     uint32_t *d_pos_out, uint64_t *d_offsets_out,
                                     void *stream);

/* ---------------------------------------------------------------------------
 * Serving: continuous batching of sort requests (no counterpart in the paper;
 * the sorts are the same robust sample sort).
 *
 * rsort_submit queues a request and returns at once with a ticket.  A runtime
 * thread of the context keeps up to `serve_slots` batches in flight on their
 * own CUDA streams and scratch workspaces.  Requests of at most
 * `serve_alone_min` keys (default 2^20) are grouped -- same key type, arrival
 * order, up to `serve_batch_keys` keys -- and sorted together as the segments
 * of one segmented sort; larger ones run alone.  A batch starts when a slot is
 * free and its scratch fits the context's HBM budget next to the batches in
 * flight, so requests arriving while others run are admitted as slots and
 * memory free up and overlap with them on the device.  Each result is the
 * same as sorting that request alone with rsort_sort (segment-local
 * permutation), whatever it was batched with.
 *
 * The caller owns the request's device buffers; they must stay valid and
 * untouched until the ticket reports a final status.  p_virtual only matters
 * for requests that run alone (it does not change results).
 *
 * The runtime keeps the final status and latency of the last `serve_history`
 * finished requests (default 2^20); an older ticket is forgotten and then
 * reads as unknown (EINVAL), so a long-running server holds bounded host
 * memory.
 * ------------------------------------------------------------------------- */
typedef struct {
    rsort_key_type type;
    const void *d_keys_in;   /* n keys, must not alias d_keys_out            */
    void *d_keys_out;        /* n keys                                       */
    uint32_t *d_perm_out;    /* n positions                                  */
    uint64_t n;              /* <= 2^32 - 1                                  */
    uint32_t p_virtual;      /* 0/1: automatic; 2..2048                      */
    uint64_t seed;
} rsort_request;

/* Queues a request.  *ticket_out identifies it.  Errors: EINVAL (bad
 * arguments), ENOMEM (its scratch alone exceeds the context budget), ECUDA
 * (the runtime could not start). */
rsort_status rsort_submit(rsort_ctx *ctx, const rsort_request *req, uint64_t *ticket_out);

/* Non-blocking status: RSORT_PENDING (queued or running), RSORT_OK (done;
 * *latency_ns_out, if not NULL, gets submit-to-completion nanoseconds),
 * RSORT_ECANCELLED, or the request's error.  EINVAL for an unknown ticket
 * (never issued, or finished more than `serve_history` requests ago). */
rsort_status rsort_poll(rsort_ctx *ctx, uint64_t ticket, uint64_t *latency_ns_out);

/* Blocks until the request has a final status or timeout_ns passes
 * (RSORT_ETIMEOUT).  Returns the final status otherwise, or EINVAL if the
 * ticket is unknown (as for rsort_poll). */
rsort_status rsort_wait(rsort_ctx *ctx, uint64_t ticket, uint64_t timeout_ns);

/* Cancels a request that has not started: RSORT_OK, its buffers are left
 * untouched and its status becomes RSORT_ECANCELLED.  A running or finished
 * request cannot be cancelled (RSORT_EINVAL). */
rsort_status rsort_cancel(rsort_ctx *ctx, uint64_t ticket);

typedef struct {
    uint64_t submitted, completed, cancelled, failed, queued;
    uint32_t inflight_batches;
    uint64_t batches;
    uint64_t keys_completed;
    double mean_batch_requests;
    double p50_us, p99_us, max_us;   /* submit-to-completion latency */
    double elapsed_s;                /* first submit to last completion */
} rsort_serve_stats;

/* Counters since the runtime started (or the last reset), and latency
 * percentiles over the last `serve_history` completions in that time.  All
 * zero before the first submit. */
rsort_status rsort_get_serve_stats(rsort_ctx *ctx, rsort_serve_stats *out);
rsort_status rsort_reset_serve_stats(rsort_ctx *ctx);

/* Profiling (tracing): when enabled, the library records CUDA events around
 * every kernel it launches on the call's stream.  rsort_phase_times copies up
 * to max entries of {kernel name, accumulated milliseconds, launches} into the
 * caller's arrays (names are static strings) after synchronising, and resets
 * the accumulators.  *count receives the number of distinct kernels. */
rsort_status rsort_set_profiling(rsort_ctx *ctx, int enable);
rsort_status rsort_phase_times(rsort_ctx *ctx, const char **names, double *ms,
                               uint64_t *launches, int max, int *count);

/* Tunables of a context (also settable from the tune table file given to
 * rsort_create, one "name value" per line).  They change speed, never
 * results.
 *   classifier   0: the splitter tree of Super Scalar Sample Sort;
 *                1 (default): a lookup table over the keys' leading bits
 *                into the same sorted splitters, then a binary search inside
 *                the bin.
 *   serve_slots, serve_batch_keys, serve_alone_min, serve_history
 *                serving runtime (see rsort_submit); fixed once the runtime
 *                has started.
 *   target_bucket  automatic fan-outs aim at final buckets of this many keys
 *                (64..4096, default 1536).
 *   level1_stable  level 1 of rsort_sort / rsort_segmented: 1 keeps input
 *                order inside buckets; 0 ranks elements by shared-memory
 *                atomics (faster on distinct keys); 2 (default) decides on
 *                the device per call: input order when at least 1/16 of the
 *                level's buckets are equality buckets (both bounding
 *                splitters hold one key, as with many copies of a key), whose
 *                elements, kept in position order, are final at once.
 *                rsort_partition always keeps input order.
 *   deep_levels_stable  1: the partition levels of rsort_sort /
 *                rsort_segmented after the first keep input order inside
 *                buckets; 0 (default): they rank elements by shared-memory
 *                atomics.  The result is the same either way (the in-SM sort
 *                orders (key, position) pairs).
 *   max_levels   at most this many partition levels of rsort_sort /
 *                rsort_segmented (1..3, default 3); a call launches fewer
 *                when its sizes bound every bucket within 4096 keys sooner
 *                (n / p, the fan-out targets and the 512-bucket cap of a
 *                deeper level: 2^28 keys at p = 1024 take two).  A bucket
 *                still above 4096 keys after the last level is merge-sorted
 *                through global memory by one CTA (slow; rare).
 *   The in-SM sort of a bucket is chosen by its size (Section 6's
 *   size-dependent choice, applied per bucket; paper_1606_08766_gb300.autotune
 *   measures these on the device and writes a table of them):
 *   small_cap, mid_cap  buckets of at most small_cap keys (64..1024, default
 *                1024) are sorted by 128-thread CTAs of 8 slots a thread, of
 *                at most mid_cap (64..2048, default 2048) by 128-thread CTAs
 *                of 16 slots, larger ones (up to 4096) by 256-thread CTAs of
 *                16 slots.
 *   rank_max     buckets of at most this many keys (0..128, default 64) are
 *                sorted by rank-by-counting (Appendix "Fast Work-Inefficient
 *                Ranking").
 *   sort_small, sort_mid, sort_medium  the algorithm of each of the three
 *                classes above: 0 (default) equal-width bins with ranking
 *                inside the bins (bitonic when keys cluster), 2 bitonic sort
 *                (Appendix "Bitonic Sort"), and for the mid and medium
 *                classes 1: in-SM quicksort whose pivots are the binary-tree
 *                median approximation (see rsort_approx_median) of a
 *                256-element stratified sample of each segment.
 *   medium_sort  1 sets sort_mid and sort_medium to quicksort, 0 to bins.
 *   target_bucket@c  (c = 1..32) the fan-out target of segments of
 *                ceil(log2 m) = c keys (64..4096; 0 falls back to
 *                target_bucket): the bucket count of such a segment is
 *                ceil(m / target).
 *   unit_scatter  1 (default): a level with 33..1024 buckets stores every
 *                element's bucket id when it classifies, and its scatter
 *                writes whole 8-element units (64 bytes of keys, 32 bytes of
 *                positions), holding each bucket's incomplete last unit in
 *                shared memory; 0: the staged scatter, which classifies
 *                again.
 *   atomic_scatter  1: levels of rsort_sort / rsort_segmented that may
 *                leave buckets in any order and do not take the unit scatter
 *                keep the ids of their classify pass and scatter with a
 *                small-footprint kernel that ranks by shared-memory atomics;
 *                0 (default): the staged scatter.
 *   bulk_classify  1: the classify pass that stores bucket ids stages its
 *                keys through bulk copies (cp.async.bulk on shared-memory
 *                barriers) into a 4-stage ring when the key array is 16-byte
 *                aligned; 0 (default): 16-byte loads into registers.
 *   wide_scatter_k  levels with at least this many buckets stage 4096-key
 *                sub-tiles with 512 threads when shared memory allows
 *                (default 1024).
 *   warp_direct_max_k  partition levels with at most this many buckets per
 *                segment classify and scatter per warp sub-chunk straight to
 *                HBM; larger levels stage every sub-tile through shared
 *                memory (default 0: always staged).
 * Errors: EINVAL for an unknown name or an out-of-range value. */
rsort_status rsort_set_tunable(rsort_ctx *ctx, const char *name, int64_t value);
rsort_status rsort_get_tunable(rsort_ctx *ctx, const char *name, int64_t *value);

/* Number of kernels this context has launched since creation. */
rsort_status rsort_launch_count(rsort_ctx *ctx, uint64_t *out);

#ifdef __cplusplus
}
#endif

#endif /* RSORT_H */
