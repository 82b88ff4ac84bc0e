/*
 * oracle.c -- plain, slow, obviously correct CPU oracle for robust sample sort.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file.  Only tests/, __graft_entry__.smoke() and the cpu_baseline /
 * reference leg of bench.py may load it.  It shares no code, header, table or
 * constant generator with the CUDA path: every definition below is written out
 * again here from the paper (Axtmann & Sanders, "Robust Massively Parallel
 * Sorting", arXiv 1606.08766).
 *
 * What it computes
 *   oracle_sort        The output contract of Section 2 ("Preliminaries"): the
 *                      globally sorted sequence.  Ties are broken by the
 *                      original position, the "append a unique identifier and
 *                      compare lexicographically" semantics of Section 2 that
 *                      the robust algorithms simulate implicitly (Section 5,
 *                      Appendix "Robust Multi-Level Sample Sort").  Because
 *                      positions are distinct the result is unique:
 *                      perm is the permutation with (phi(x[perm[j]]), perm[j])
 *                      strictly increasing in j.  Textbook top-down merge sort.
 *   oracle_sort_parallel  The same result on several host threads: the index
 *                      array is cut into equal chunks that the threads
 *                      merge-sort at once, then adjacent sorted runs are
 *                      merged pairwise, the merges of a round running at
 *                      once.  Used to time the oracle on all host cores.
 *   oracle_segmented   The same contract applied to each segment on its own
 *                      (segment-local positions).
 *   oracle_partition   One level of the robust sample-sort partition step
 *                      (Appendix "Robust Multi-Level Sample Sort"), step by
 *                      step in the paper's order: draw samples and attach their
 *                      input positions as tie-breakers, rank (sort) the sample,
 *                      take every S/k-th sample as a splitter (Appendix
 *                      "Generalizing Quicksort"), assign every element to the
 *                      partition given by the number of splitters that are
 *                      lexicographically smaller than (key, position), and lay
 *                      the partitions out in order.
 *
 *   oracle_partition_ex  The same step with the two switches the paper
 *                      measures around it: classification by key only (the
 *                      NTB ablation of Section 6) and AMS-sort
 *                      overpartitioning (b*k fine partitions assigned to the
 *                      k outputs by a greedy scan that minimises the largest
 *                      output; Section 3 "AMS-sort", Appendix "Implementation
 *                      Details").
 *
 *   oracle_tree_median The binary-tree median approximation of Section 3
 *                      ("Approximate Median Selection with a Single
 *                      Reduction"): leaves forward k-entry windows around
 *                      their median, internal nodes merge and forward the
 *                      middle k, the root flips a coin between its two middle
 *                      entries.
 *
 * Readings where the paper is silent:
 *   - phi: 64-bit floating-point elements (Appendix "Experimental Results") are
 *     ordered by their IEEE-754 bit pattern mapped to an unsigned integer
 *     (negative: all bits flipped; non-negative: sign bit flipped), so
 *     -0.0 < +0.0.  Unsigned 64-bit keys use the identity.
 *   - sample size S = min(n, a*k) with a = 16 * ceil(log2 k) samples per
 *     partition (the 16 log p samples per PE of Appendix "Implementation
 *     Details").
 *   - sampling: stratified, sample j drawn from positions
 *     [floor(j*n/S), floor((j+1)*n/S)) at offset h(seed, j) mod (stratum
 *     size), with h the splitmix64 generator
 *     (Steele, Lea & Flood 2014): h(s, j) = mix(s + (j+1) * 0x9e3779b97f4a7c15).
 *   - splitter j (j = 1..k-1) is the sorted sample's element floor(j*S/k).
 *   - NTB: an element equal to a splitter key goes below it (the search counts
 *     splitter keys strictly smaller than x, as the Super Scalar Sample Sort
 *     descent does).
 *   - overpartitioning: the sample is the plain step's (the paper sorts
 *     O(k log k) samples per level whatever b is); fine splitter j
 *     (j = 1..b*k-1) is sorted sample floor(j*S/(b*k)); "a greedy algorithm
 *     ... minimizing the load imbalance" is read as: the smallest bound L for
 *     which the in-order greedy scan needs at most k groups, then that scan.
 *   - tree median: leaves are the elements in input order (callers shuffle
 *     if they need randomly permuted input), padded with empty leaves to a
 *     power of two; an empty leaf forwards k/2 entries below and k/2 above
 *     every element (its undefined positions); coins are bit 0 of
 *     splitmix64(seed, leaf) and, at the root, splitmix64(seed, leaves); an
 *     undefined root choice moves to the nearest element of the root window.
 *
 * parity pins: see tests/test_oracle_pins.py.  All functions are pinned.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------------- */
/* Key order                                                                */
/* ---------------------------------------------------------------------- */

/* Order-preserving map of the raw 64-bit pattern to an unsigned key.
 * key_type 0: unsigned 64-bit integer, identity.
 * key_type 1: IEEE-754 binary64: flip every bit of a negative pattern, flip
 *             only the sign bit of a non-negative one. */
static uint64_t phi(uint64_t bits, int key_type)
{
    if (key_type == 0)
        return bits;
    if (bits >> 63)                 /* sign bit set: negative number */
        return ~bits;
    return bits | 0x8000000000000000ULL;
}

/* Lexicographic order on (key, position): the unique-identifier order of
 * Section 2. */
static int pair_less(uint64_t ka, uint64_t pa, uint64_t kb, uint64_t pb)
{
    if (ka != kb)
        return ka < kb;
    return pa < pb;
}

/* ---------------------------------------------------------------------- */
/* Textbook top-down merge sort of an index array                           */
/* ---------------------------------------------------------------------- */

/* Sorts idx[lo, hi) by (key[idx], idx); scratch has the same extent. */
static void merge_sort(uint32_t *idx, uint32_t *scratch, uint64_t lo, uint64_t hi,
                       const uint64_t *key)
{
    if (hi - lo < 2)
        return;
    uint64_t mid = lo + (hi - lo) / 2;
    merge_sort(idx, scratch, lo, mid, key);
    merge_sort(idx, scratch, mid, hi, key);
    /* merge the two sorted halves into scratch, then copy back */
    uint64_t i = lo, j = mid, o = lo;
    while (i < mid && j < hi) {
        uint32_t a = idx[i], b = idx[j];
        if (pair_less(key[b], b, key[a], a))
            scratch[o++] = idx[j++];
        else
            scratch[o++] = idx[i++];
    }
    while (i < mid)
        scratch[o++] = idx[i++];
    while (j < hi)
        scratch[o++] = idx[j++];
    memcpy(idx + lo, scratch + lo, (size_t)(hi - lo) * sizeof(uint32_t));
}

/* Sorted output contract of Section 2 with position tie-breaking.
 * keys_bits: n raw 64-bit patterns.  Writes keys_out[j] = keys_bits[perm[j]]
 * and perm_out.  Returns 0, or -1 on bad arguments / allocation failure. */
int oracle_sort(const uint64_t *keys_bits, uint64_t n, int key_type,
                uint64_t *keys_out, uint32_t *perm_out)
{
    if (n > 0xFFFFFFFFULL || (key_type != 0 && key_type != 1))
        return -1;
    if (n == 0)
        return 0;
    uint64_t *key = (uint64_t *)malloc(n * sizeof(uint64_t));
    uint32_t *scratch = (uint32_t *)malloc(n * sizeof(uint32_t));
    if (!key || !scratch) {
        free(key);
        free(scratch);
        return -1;
    }
    for (uint64_t i = 0; i < n; ++i) {
        key[i] = phi(keys_bits[i], key_type);
        perm_out[i] = (uint32_t)i;
    }
    merge_sort(perm_out, scratch, 0, n, key);
    for (uint64_t j = 0; j < n; ++j)
        keys_out[j] = keys_bits[perm_out[j]];
    free(key);
    free(scratch);
    return 0;
}

/* ---------------------------------------------------------------------- */
/* The same merge sort on several threads                                  */
/* ---------------------------------------------------------------------- */

typedef struct {
    uint32_t *idx, *scratch;
    const uint64_t *key;
    uint64_t lo, mid, hi;   /* chunk [lo, hi), or runs [lo, mid) and [mid, hi) */
} par_task;

static void *sort_chunk(void *arg)
{
    par_task *t = (par_task *)arg;
    merge_sort(t->idx, t->scratch, t->lo, t->hi, t->key);
    return NULL;
}

/* Merges the sorted runs idx[lo, mid) and idx[mid, hi) into scratch[lo, hi). */
static void *merge_runs(void *arg)
{
    par_task *t = (par_task *)arg;
    uint64_t i = t->lo, j = t->mid, o = t->lo;
    while (i < t->mid && j < t->hi) {
        uint32_t a = t->idx[i], b = t->idx[j];
        if (pair_less(t->key[b], b, t->key[a], a))
            t->scratch[o++] = t->idx[j++];
        else
            t->scratch[o++] = t->idx[i++];
    }
    while (i < t->mid)
        t->scratch[o++] = t->idx[i++];
    while (j < t->hi)
        t->scratch[o++] = t->idx[j++];
    return NULL;
}

/* oracle_sort's result computed by nthreads threads (1..256): chunk c of the
 * positions is [c*n/T, (c+1)*n/T); each is merge-sorted by its own thread, then
 * every round merges runs 2r and 2r+1 (one thread per merge) until one run is
 * left.  Returns 0, or -1 on bad arguments / allocation or thread failure. */
int oracle_sort_parallel(const uint64_t *keys_bits, uint64_t n, int key_type, int nthreads,
                         uint64_t *keys_out, uint32_t *perm_out)
{
    if (n > 0xFFFFFFFFULL || (key_type != 0 && key_type != 1) || nthreads < 1 ||
        nthreads > 256)
        return -1;
    if (n == 0)
        return 0;
    uint64_t T = (uint64_t)nthreads < n ? (uint64_t)nthreads : n;
    uint64_t *key = (uint64_t *)malloc(n * sizeof(uint64_t));
    uint32_t *scratch = (uint32_t *)malloc(n * sizeof(uint32_t));
    uint64_t *bound = (uint64_t *)malloc((T + 1) * sizeof(uint64_t));
    par_task *task = (par_task *)malloc(T * sizeof(par_task));
    pthread_t *th = (pthread_t *)malloc(T * sizeof(pthread_t));
    int rc = -1;
    if (!key || !scratch || !bound || !task || !th)
        goto done;
    for (uint64_t i = 0; i < n; ++i) {
        key[i] = phi(keys_bits[i], key_type);
        perm_out[i] = (uint32_t)i;
    }
    for (uint64_t c = 0; c <= T; ++c)
        bound[c] = c * n / T;
    for (uint64_t c = 0; c < T; ++c) {
        task[c] = (par_task){perm_out, scratch, key, bound[c], bound[c], bound[c + 1]};
        if (pthread_create(&th[c], NULL, sort_chunk, &task[c]) != 0) {
            for (uint64_t d = 0; d < c; ++d)
                pthread_join(th[d], NULL);
            goto done;
        }
    }
    for (uint64_t c = 0; c < T; ++c)
        pthread_join(th[c], NULL);
    /* pairwise merges: runs are bound[0..runs]; each round halves the runs */
    uint32_t *src = perm_out, *dst = scratch;
    uint64_t runs = T;
    while (runs > 1) {
        uint64_t pairs = runs / 2, started = 0;
        for (uint64_t r = 0; r < pairs; ++r) {
            task[r] = (par_task){src, dst, key, bound[2 * r], bound[2 * r + 1],
                                 bound[2 * r + 2]};
            if (pthread_create(&th[r], NULL, merge_runs, &task[r]) != 0)
                break;
            ++started;
        }
        for (uint64_t r = 0; r < started; ++r)
            pthread_join(th[r], NULL);
        if (started < pairs)
            goto done;
        if (runs % 2)   /* the odd run out is carried over unchanged */
            memcpy(dst + bound[runs - 1], src + bound[runs - 1],
                   (size_t)(bound[runs] - bound[runs - 1]) * sizeof(uint32_t));
        /* run r of the next round starts where run 2r started (the carried
         * odd run included); the last bound stays n */
        for (uint64_t r = 0; r <= pairs; ++r)
            bound[r] = bound[2 * r];
        runs = pairs + (runs % 2);
        bound[runs] = n;
        uint32_t *t = src;
        src = dst;
        dst = t;
    }
    if (src != perm_out)
        memcpy(perm_out, src, (size_t)n * sizeof(uint32_t));
    for (uint64_t j = 0; j < n; ++j)
        keys_out[j] = keys_bits[perm_out[j]];
    rc = 0;
done:
    free(key);
    free(scratch);
    free(bound);
    free(task);
    free(th);
    return rc;
}

/* The same contract applied to every segment [offsets[s], offsets[s+1]) on its
 * own; perm_out holds segment-local positions. */
int oracle_segmented(const uint64_t *keys_bits, const uint64_t *offsets, uint32_t nseg,
                     int key_type, uint64_t *keys_out, uint32_t *perm_out)
{
    for (uint32_t s = 0; s < nseg; ++s) {
        uint64_t a = offsets[s], b = offsets[s + 1];
        if (b < a)
            return -1;
        int rc = oracle_sort(keys_bits + a, b - a, key_type, keys_out + a, perm_out + a);
        if (rc)
            return rc;
    }
    return 0;
}

/* ---------------------------------------------------------------------- */
/* splitmix64 (Steele, Lea & Flood 2014), counter form                      */
/* ---------------------------------------------------------------------- */

/* Output number c (0-based) of the splitmix64 stream whose state starts at s:
 * the state advances by the golden gamma before each output, and the output is
 * the state passed through the two xor-shift-multiply rounds and a final
 * xor-shift. */
uint64_t oracle_splitmix64_at(uint64_t s, uint64_t c)
{
    uint64_t z = s + (c + 1) * 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

/* ---------------------------------------------------------------------- */
/* One level of the robust sample-sort partition step                       */
/* ---------------------------------------------------------------------- */

static uint32_t ceil_log2_u32(uint32_t k)
{
    uint32_t l = 0;
    while ((1ULL << l) < k)
        ++l;
    return l;
}

/* Number of samples drawn for n elements and k partitions. */
uint64_t oracle_sample_count(uint64_t n, uint32_t k)
{
    uint64_t a = 16ULL * ceil_log2_u32(k);
    uint64_t s = a * k;
    return s < n ? s : n;
}

/* Partitions n keys into k >= 1 buckets (Appendix "Robust Multi-Level Sample
 * Sort").  Outputs (each may be NULL except where noted):
 *   sample_pos  [S]    the sampled input positions, in draw order
 *   spl_key     [k-1]  splitter keys (mapped by phi), spl_pos [k-1] positions
 *   bucket      [n]    partition of every input element
 *   keys_out    [n]    raw key bits laid out partition by partition, each
 *   pos_out     [n]    partition in increasing input position
 *   offsets     [k+1]  start of every partition; offsets[k] = n
 * Returns 0, or -1 on bad arguments / allocation failure. */
int oracle_partition(const uint64_t *keys_bits, uint64_t n, int key_type, uint32_t k,
                     uint64_t seed, uint64_t *sample_pos, uint64_t *spl_key,
                     uint32_t *spl_pos, uint32_t *bucket, uint64_t *keys_out,
                     uint32_t *pos_out, uint64_t *offsets)
{
    if (k == 0 || n > 0xFFFFFFFFULL || (key_type != 0 && key_type != 1))
        return -1;
    uint64_t S = oracle_sample_count(n, k);
    uint64_t *key = (uint64_t *)malloc((n ? n : 1) * sizeof(uint64_t));
    uint32_t *b = (uint32_t *)malloc((n ? n : 1) * sizeof(uint32_t));
    uint64_t *skey = (uint64_t *)malloc((S ? S : 1) * sizeof(uint64_t));
    uint32_t *sidx = (uint32_t *)malloc((S ? S : 1) * sizeof(uint32_t));
    uint32_t *sscr = (uint32_t *)malloc((S ? S : 1) * sizeof(uint32_t));
    uint64_t *tk = (uint64_t *)malloc((k ? k : 1) * sizeof(uint64_t));
    uint32_t *ti = (uint32_t *)malloc((k ? k : 1) * sizeof(uint32_t));
    uint64_t *cnt = (uint64_t *)calloc((size_t)k + 1, sizeof(uint64_t));
    int rc = -1;
    if (!key || !b || !skey || !sidx || !sscr || !tk || !ti || !cnt)
        goto done;
    for (uint64_t i = 0; i < n; ++i)
        key[i] = phi(keys_bits[i], key_type);

    /* Step 1: random samples of the data, each carrying its input position as
     * tie-breaker.  Stratified: sample j comes from stratum
     * [floor(j*n/S), floor((j+1)*n/S)), so the strata tile the whole input. */
    uint32_t *sample_order = sidx; /* sample number -> input position */
    if (S > 0) {
        for (uint64_t j = 0; j < S; ++j) {
            uint64_t lo = (j * n) / S, hi = ((j + 1) * n) / S;
            uint64_t pos = lo + oracle_splitmix64_at(seed, j) % (hi - lo);
            sample_order[j] = (uint32_t)pos;
            if (sample_pos)
                sample_pos[j] = pos;
        }
    }

    /* Step 2: rank the samples by (key, position): sort the sample positions
     * with the same textbook merge sort (the key array is indexed by input
     * position, so sorting positions sorts the pairs). */
    merge_sort(sample_order, sscr, 0, S, key);
    for (uint64_t j = 0; j < S; ++j)
        skey[j] = key[sample_order[j]];

    /* Step 3: every S/k-th sample becomes a splitter: splitter j (1-based,
     * j = 1..k-1) is sorted sample floor(j*S/k).  With S = 0 there are no
     * elements and no splitters are needed. */
    for (uint32_t j = 1; j < k && S > 0; ++j) {
        uint64_t r = ((uint64_t)j * S) / k;
        tk[j - 1] = skey[r];
        ti[j - 1] = sample_order[r];
        if (spl_key)
            spl_key[j - 1] = skey[r];
        if (spl_pos)
            spl_pos[j - 1] = sample_order[r];
    }

    /* Step 4: classify.  An element (x, i) goes to partition
     * b = #{ splitters (s.key, s.pos) lexicographically smaller than (x, i) }:
     * the search on the key alone, repeated with positions as tie-breakers when
     * the key equals the bounding splitter's key, counts exactly these. */
    for (uint64_t i = 0; i < n; ++i) {
        uint32_t c = 0;
        for (uint32_t j = 0; j + 1 < k; ++j)
            if (pair_less(tk[j], ti[j], key[i], i))
                ++c;
        b[i] = c;
        if (bucket)
            bucket[i] = c;
        cnt[c + 1] += 1;
    }

    /* Step 5: lay the partitions out in order, each in increasing position. */
    for (uint32_t j = 0; j < k; ++j)
        cnt[j + 1] += cnt[j];
    if (offsets)
        for (uint32_t j = 0; j <= k; ++j)
            offsets[j] = cnt[j];
    if (keys_out || pos_out) {
        for (uint64_t i = 0; i < n; ++i) {
            uint64_t o = cnt[b[i]]++;
            if (keys_out)
                keys_out[o] = keys_bits[i];
            if (pos_out)
                pos_out[o] = (uint32_t)i;
        }
    }
    rc = 0;
done:
    free(key);
    free(b);
    free(skey);
    free(sidx);
    free(sscr);
    free(tk);
    free(ti);
    free(cnt);
    return rc;
}

/* ---------------------------------------------------------------------- */
/* Partition-step variants: NTB ablation and AMS overpartitioning           */
/* ---------------------------------------------------------------------- */

/* Greedy assignment of consecutive fine partitions (sizes c[0..K)) to groups
 * under a load bound L >= max c: the fine partitions are visited in order and
 * a new group is opened whenever adding the next one would lift the current
 * group above L.  Returns the number of groups used; if first != NULL (room
 * for kmax entries) first[g] receives the fine partition group g starts at. */
static uint64_t greedy_groups(const uint64_t *c, uint32_t K, uint64_t L, uint32_t *first,
                              uint32_t kmax)
{
    uint64_t groups = 1, load = 0;
    if (first && kmax > 0)
        first[0] = 0;
    for (uint32_t j = 0; j < K; ++j) {
        if (load + c[j] > L) {
            if (first && groups < kmax)
                first[groups] = j;
            ++groups;
            load = 0;
        }
        load += c[j];
    }
    return groups;
}

/* The partition step with the two switches the paper evaluates around it.
 *
 *   tie_break = 1  the robust classification of oracle_partition:
 *                  fine partition of (x, i) = #{ splitters lexicographically
 *                  smaller than (x, i) }.
 *   tie_break = 0  the "no tie-breaking" ablation (NTB-AMS, Section 6,
 *                  figure "RAMS vs NTB-AMS"): the same splitters, but the
 *                  classification looks at keys only,
 *                  #{ splitters whose key is smaller than x }, so every copy
 *                  of a key lands in one partition.
 *   over = b >= 1  AMS-sort overpartitioning (Section 3, AMS-sort; Appendix
 *                  "Implementation Details": b = 2 / ((1 + eps)^(1/l) - 1)):
 *                  the same sample yields K = b*k partitions (splitter j,
 *                  j = 1..K-1, is sorted sample floor(j*S/K)); their exact
 *                  sizes are counted and consecutive fine partitions are
 *                  assigned to the k outputs by the greedy scan above, with
 *                  the smallest bound L for which k groups suffice, which
 *                  minimises the largest output.  b = 1 is the plain step
 *                  (no grouping: output g is partition g).
 *
 * The sample is the one of oracle_partition (S = oracle_sample_count(n, k),
 * stratified, sorted by (key, position)).  Outputs (NULL to skip):
 *   fine_sizes  [b*k]  exact size of every fine partition
 *   group_first [k+1]  first fine partition of every output; K past the end
 *   keys_out, pos_out [n], offsets [k+1]  as in oracle_partition.
 * Returns 0, or -1 on bad arguments / allocation failure. */
int oracle_partition_ex(const uint64_t *keys_bits, uint64_t n, int key_type, uint32_t k,
                        uint64_t seed, int tie_break, uint32_t over, uint64_t *fine_sizes,
                        uint32_t *group_first, uint64_t *keys_out, uint32_t *pos_out,
                        uint64_t *offsets)
{
    if (k == 0 || over == 0 || n > 0xFFFFFFFFULL || (key_type != 0 && key_type != 1) ||
        (uint64_t)k * over > 0xFFFFFFFFULL)
        return -1;
    const uint32_t K = k * over;
    uint64_t S = oracle_sample_count(n, k);
    uint64_t *key = (uint64_t *)malloc((n ? n : 1) * sizeof(uint64_t));
    uint32_t *fb = (uint32_t *)malloc((n ? n : 1) * sizeof(uint32_t));
    uint32_t *grp = (uint32_t *)malloc((n ? n : 1) * sizeof(uint32_t));
    uint32_t *order = (uint32_t *)malloc((S ? S : 1) * sizeof(uint32_t));
    uint32_t *sscr = (uint32_t *)malloc((S ? S : 1) * sizeof(uint32_t));
    uint64_t *tk = (uint64_t *)malloc((size_t)K * sizeof(uint64_t));
    uint32_t *ti = (uint32_t *)malloc((size_t)K * sizeof(uint32_t));
    uint64_t *c = (uint64_t *)calloc((size_t)K, sizeof(uint64_t));
    uint32_t *first = (uint32_t *)malloc(((size_t)k + 1) * sizeof(uint32_t));
    uint64_t *cnt = (uint64_t *)calloc((size_t)k + 1, sizeof(uint64_t));
    int rc = -1;
    if (!key || !fb || !grp || !order || !sscr || !tk || !ti || !c || !first || !cnt)
        goto done;
    for (uint64_t i = 0; i < n; ++i)
        key[i] = phi(keys_bits[i], key_type);

    /* sample and rank it exactly as oracle_partition does */
    for (uint64_t j = 0; j < S; ++j) {
        uint64_t lo = (j * n) / S, hi = ((j + 1) * n) / S;
        order[j] = (uint32_t)(lo + oracle_splitmix64_at(seed, j) % (hi - lo));
    }
    merge_sort(order, sscr, 0, S, key);

    /* K - 1 fine splitters: every S/K-th sample.  Without a sample (S = 0,
     * which the sample-size rule gives for k = 1) there are no splitters and
     * every element is in fine partition 0. */
    const uint32_t nfs = S > 0 ? K - 1 : 0;
    for (uint32_t j = 1; j <= nfs; ++j) {
        uint64_t r = ((uint64_t)j * S) / K;
        tk[j - 1] = key[order[r]];
        ti[j - 1] = order[r];
    }

    /* fine classification, with or without positions as tie-breakers */
    for (uint64_t i = 0; i < n; ++i) {
        uint32_t f = 0;
        for (uint32_t j = 0; j < nfs; ++j) {
            int smaller = tie_break ? pair_less(tk[j], ti[j], key[i], i) : (tk[j] < key[i]);
            if (smaller)
                ++f;
        }
        fb[i] = f;
        c[f] += 1;
    }

    /* groups: the smallest bound L with at most k greedy groups.  Every group
     * holds at least ceil(n/k) elements in the worst case and at least the
     * largest fine partition; the bound ceil(n/k) + max c always suffices
     * (each closed group then exceeds n/k, so k of them would exceed n). */
    uint64_t maxc = 0;
    for (uint32_t j = 0; j < K; ++j)
        if (c[j] > maxc)
            maxc = c[j];
    uint64_t lo = (n + k - 1) / k;
    if (maxc > lo)
        lo = maxc;
    uint64_t hi = (n + k - 1) / k + maxc;
    if (hi < lo)
        hi = lo;
    while (lo < hi) {
        uint64_t mid = lo + (hi - lo) / 2;
        if (greedy_groups(c, K, mid, NULL, 0) <= k)
            hi = mid;
        else
            lo = mid + 1;
    }
    for (uint32_t g = 0; g <= k; ++g)
        first[g] = K;
    if (over == 1) {
        /* no overpartitioning: output g is fine partition g */
        for (uint32_t g = 0; g < k; ++g)
            first[g] = g;
    } else {
        greedy_groups(c, K, lo, first, k);
    }
    for (uint64_t i = 0; i < n; ++i) {
        uint32_t g = 0;
        while (g + 1 < k && first[g + 1] <= fb[i])
            ++g;
        grp[i] = g;
        cnt[g + 1] += 1;
    }

    /* lay the outputs out in order, each in increasing position */
    for (uint32_t g = 0; g < k; ++g)
        cnt[g + 1] += cnt[g];
    if (offsets)
        for (uint32_t g = 0; g <= k; ++g)
            offsets[g] = cnt[g];
    if (fine_sizes)
        for (uint32_t j = 0; j < K; ++j)
            fine_sizes[j] = c[j];
    if (group_first)
        for (uint32_t g = 0; g <= k; ++g)
            group_first[g] = first[g];
    for (uint64_t i = 0; i < n; ++i) {
        uint64_t o = cnt[grp[i]]++;
        if (keys_out)
            keys_out[o] = keys_bits[i];
        if (pos_out)
            pos_out[o] = (uint32_t)i;
    }
    rc = 0;
done:
    free(key);
    free(fb);
    free(grp);
    free(order);
    free(sscr);
    free(tk);
    free(ti);
    free(c);
    free(first);
    free(cnt);
    return rc;
}

/* ---------------------------------------------------------------------- */
/* Binary-tree median approximation (Section 3, "Approximate Median         */
/* Selection with a Single Reduction")                                      */
/* ---------------------------------------------------------------------- */

/* A window entry: tag -1 is "undefined on the left" (below every element),
 * +1 "undefined on the right" (above every element), 0 an element (key,
 * position).  Entries are ordered by tag, then (key, position). */
typedef struct {
    int tag;
    uint64_t key;
    uint32_t pos;
} tm_entry;

static int tm_less(const tm_entry *a, const tm_entry *b)
{
    if (a->tag != b->tag)
        return a->tag < b->tag;
    if (a->tag != 0)
        return 0;
    return pair_less(a->key, a->pos, b->key, b->pos);
}

/* Window that a leaf holding m in {0, 1} elements forwards: its sorted data
 * a[1..m] read at positions c-k/2+1 .. c+k/2, c = floor(m/2) or (for odd m,
 * by the coin) ceil(m/2), undefined positions left of 1 as -inf and right of
 * m as +inf. */
static void tm_leaf(tm_entry *w, uint32_t k, int m, uint64_t key, uint32_t pos, int coin)
{
    long c = (m % 2 == 1 && coin) ? (m + 1) / 2 : m / 2;
    for (uint32_t t = 0; t < k; ++t) {
        long at = c - (long)(k / 2) + 1 + (long)t; /* 1-based position */
        if (at < 1) {
            w[t].tag = -1;
        } else if (at > m) {
            w[t].tag = 1;
        } else {
            w[t].tag = 0;
            w[t].key = key;
            w[t].pos = pos;
        }
    }
}

/* Approximate median of keys[0..n) (n >= 1) with even window size k >= 2.
 * Leaf i (i < P = next power of two >= n) holds element i, or nothing when
 * i >= n.  Internal nodes merge their children's k-entry windows and forward
 * the middle k of the 2k merged entries; the root returns entry k/2 or k/2+1
 * (1-based) of its window.  Coins: leaf i uses bit 0 of splitmix64(seed, i),
 * the root bit 0 of splitmix64(seed, P).  When the chosen entry is undefined
 * (possible only when n is tiny next to k), the defined entry of the root
 * window nearest to the middle is returned.  Returns the position of the
 * chosen element, or -1 on bad arguments. */
int64_t oracle_tree_median(const uint64_t *keys_bits, uint64_t n, int key_type, uint32_t k,
                           uint64_t seed)
{
    if (n == 0 || n > 0xFFFFFFFFULL || k < 2 || (k & 1) || (key_type != 0 && key_type != 1))
        return -1;
    uint64_t P = 1;
    while (P < n)
        P <<= 1;
    tm_entry *lvl = (tm_entry *)malloc(P * k * sizeof(tm_entry));
    tm_entry *nxt = (tm_entry *)malloc((P / 2 + 1) * k * sizeof(tm_entry));
    tm_entry *mrg = (tm_entry *)malloc(2 * (size_t)k * sizeof(tm_entry));
    int64_t res = -1;
    if (!lvl || !nxt || !mrg)
        goto done;
    for (uint64_t i = 0; i < P; ++i) {
        int m = i < n ? 1 : 0;
        uint64_t key = i < n ? phi(keys_bits[i], key_type) : 0;
        tm_leaf(lvl + i * k, k, m, key, (uint32_t)i, (int)(oracle_splitmix64_at(seed, i) & 1));
    }
    for (uint64_t cnt = P; cnt > 1; cnt /= 2) {
        for (uint64_t j = 0; j < cnt / 2; ++j) {
            /* merge the two sorted windows of children 2j and 2j+1 */
            const tm_entry *a = lvl + (2 * j) * k, *b = lvl + (2 * j + 1) * k;
            uint32_t ia = 0, ib = 0;
            for (uint32_t t = 0; t < 2 * k; ++t) {
                if (ib >= k || (ia < k && !tm_less(&b[ib], &a[ia])))
                    mrg[t] = a[ia++];
                else
                    mrg[t] = b[ib++];
            }
            /* middle k of the 2k merged entries: positions k/2+1 .. 3k/2 */
            for (uint32_t t = 0; t < k; ++t)
                nxt[j * k + t] = mrg[k / 2 + t];
        }
        tm_entry *tmp = lvl;
        lvl = nxt;
        nxt = tmp;
    }
    {
        int coin = (int)(oracle_splitmix64_at(seed, P) & 1);
        long pick = coin ? (long)(k / 2) : (long)(k / 2) - 1; /* 0-based */
        for (long d = 0; d < (long)k; ++d) {
            long cand[2] = {pick - d, pick + d};
            for (int s = 0; s < 2; ++s) {
                if (cand[s] >= 0 && cand[s] < (long)k && lvl[cand[s]].tag == 0) {
                    res = (int64_t)lvl[cand[s]].pos;
                    goto done;
                }
            }
        }
        res = 0;
    }
done:
    free(lvl);
    free(nxt);
    free(mrg);
    return res;
}
