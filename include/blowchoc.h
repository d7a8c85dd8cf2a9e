/*
 * blowchoc.h -- C ABI of a GPU (sm_103a) Blocked Bloom filter with choices.
 *
 * The data structure is the "BlowChoc" filter of J. E. Schmitz, J. Zentgraf
 * and S. Rahmann, "Blocked Bloom Filters with Choices" (arXiv 2501.18977):
 * M blocks of 512 bits; a key x has c candidate blocks h_1(x)..h_c(x) and a
 * bit set F(x) = {f_1(x)..f_k(x)} inside a block (Section 3.1, Eq. 3).
 *
 * Conventions shared by every entry point:
 *  - Return value: BLOWCHOC_OK (0) or a negative BLOWCHOC_E* code. No
 *    exception crosses the ABI. blowchoc_last_error() describes the last
 *    failure of the calling thread.
 *  - Pointers named d_* are DEVICE pointers (global memory of the current
 *    CUDA device), 8-byte aligned. The caller owns them and keeps them alive
 *    until the work queued on the given stream has finished.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream). Insert and query are asynchronous and stream-ordered; the
 *    caller orders calls on different streams (events) if one must see the
 *    other's result.
 *  - There is no CPU fallback: without a usable CUDA device every call that
 *    needs one fails with BLOWCHOC_ECUDA. The host-only calls
 *    (blowchoc_cost_ranks, blowchoc_fpr_estimate,
 *    blowchoc_derive_multipliers, blowchoc_shard_layout,
 *    blowchoc_shard_partition_scratch, and blowchoc_stats_decode of an
 *    existing filter) compute host-side preparation and statistics only; no
 *    insert or query runs without a device.
 */
#ifndef BLOWCHOC_H
#define BLOWCHOC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BLOWCHOC_OK 0
#define BLOWCHOC_EINVAL (-1)   /* bad argument */
#define BLOWCHOC_ENOMEM (-2)   /* device allocation failed */
#define BLOWCHOC_ECUDA (-3)    /* CUDA runtime error (or no device) */
#define BLOWCHOC_ETIMEOUT (-4) /* a bounded device-side wait gave up */
#define BLOWCHOC_EBUDGET (-5)  /* request exceeds a memory budget */

#define BLOWCHOC_BLOCK_BITS 512
#define BLOWCHOC_MAX_K 32
#define BLOWCHOC_MAX_CHOICES 3

/* Block-selection costs, with j = set bits of the block after insertion and
 * a = bits the key would newly set there (Section 3.2, Appendix A):
 *   MIX (Eq. 5): sigma k (j/256)^k + a        cost_param = sigma >= 0
 *   LA  (Eq. 6): k ((j + mu k)/256)^k + a     cost_param = mu >= 0
 *   EXP (Eq. 4): beta^(j/128) + a/k           cost_param = beta > 0
 * Costs are evaluated once per filter on the host in IEEE double and turned
 * into an exact integer rank table; ties go to the lowest choice index. */
typedef enum {
    BLOWCHOC_COST_MIX = 0,
    BLOWCHOC_COST_LA = 1,
    BLOWCHOC_COST_EXP = 2
} blowchoc_cost;

typedef struct {
    uint64_t nblocks;   /* M >= 1 blocks of 512 bits (m = 512 M bits), M <= 2^32 */
    uint32_t k;         /* bit-address hashes, 1..32 */
    uint32_t choices;   /* c, 1..3 (c = 1 is a Blocked Bloom filter, no cost) */
    int32_t cost;       /* blowchoc_cost */
    uint32_t bitsel;    /* bit selection (Section 3.3): 0 = random, 1 = distinct (Appendix B) */
    double cost_param;  /* sigma | mu | beta */
    uint64_t hash_seed; /* seeds the hash multipliers (see blowchoc_multipliers) */
    uint64_t batch;     /* B >= 1: batch size of the batch-synchronous insertion */
} blowchoc_params;

typedef struct blowchoc_filter blowchoc_filter;

typedef struct {
    uint64_t inserted;  /* keys whose bits were OR-ed into a block */
    uint64_t skipped;   /* keys already contained in a candidate block (Section 3.2) */
    uint64_t set_bits;  /* total 1-bits of the filter */
    uint64_t hist[BLOWCHOC_BLOCK_BITS + 1]; /* hist[L] = blocks with L set bits (Fig. 8) */
    double fpr_est;     /* 1 - (1 - q)^c, q from the histogram, see blowchoc_stats */
} blowchoc_filter_stats;

/*
 * blowchoc_create -- allocate a filter of params->nblocks zeroed blocks on the
 * current device (Section 3.1; the block layout of Section 2.2).
 *   params  in, host pointer, read during the call only.
 *   stream  the filter's home stream: zeroing is queued there, and
 *           blowchoc_stats / blowchoc_destroy order themselves on it.
 *   out     out, receives the handle; the library owns the device memory
 *           (filter words, rank table, counters, scratch) until destroy.
 * Hash multipliers (Section 3.4: "a random large integer" coprime to the
 * range b) are drawn from splitmix64 seeded with hash_seed, forced odd and
 * redrawn until coprime: first a_1..a_c for the block hashes (range M), then
 * a'_1..a'_k for the bit hashes (range 512; with distinct selection the
 * range of a'_i is 512 - i + 1).
 * Layout: bit p of block b is bit (p mod 64) of the little-endian 64-bit
 * word 8b + p/64; blocks are contiguous and 64-byte aligned.
 * Errors: EINVAL (M = 0 or > 2^32, k not in 1..32, c not in 1..3, bad cost
 * kind or parameter, bitsel > 1, batch = 0, out NULL), ENOMEM, ECUDA.
 */
int blowchoc_create(const blowchoc_params *params, void *stream, blowchoc_filter **out);

/*
 * blowchoc_insert -- insert d_keys[0..n) (Section 3.2, Fig. 2B), in batches
 * of B = params.batch keys. Every key of a batch decides against the bits
 * present when its batch starts: if some candidate block already holds all
 * of F(x), the key is skipped; otherwise it goes to the candidate of least
 * cost (lowest index on ties). The batch's bits are OR-ed in after all its
 * choices. B = 1 is the paper's one-key-at-a-time insertion. The result
 * depends only on (params, key sequence), never on launch configuration.
 *   d_keys  device, n uint64 keys (any values; u = 64-bit keys).
 *   n       may be 0 (no-op).
 * May grow an internal device scratch buffer (up to 2 min(B, n) bytes: a
 * choice byte per key, and a byte of word flags in the persistent insert).
 * Errors: EINVAL (NULL filter, NULL keys with n > 0), ENOMEM, ECUDA.
 */
int blowchoc_insert(blowchoc_filter *f, const uint64_t *d_keys, uint64_t n, void *stream);

/*
 * blowchoc_insert_noalloc -- blowchoc_insert that allocates no device memory.
 * The paper has no counterpart: this is a library service for callers that
 * cannot let a library call cudaMalloc, such as applications whose device
 * memory is entirely handed out by their own allocator or fixed budget, and
 * latency-critical loops (a request-serving loop, host code between CUDA
 * graph replays) where an allocation may synchronise the device.
 * Same arguments, semantics and results as blowchoc_insert (bit-identical
 * filter words and counters). Batches that run over the whole grid (more
 * than 2048 keys with the persistent insert on, the default; more than 16384
 * with it off) keep their per-key choices in one fixed array inside the
 * library's device image (4 MiB, held by every GPU that loads the library
 * until the process exits) instead of a buffer the filter allocates, and run
 * as a choose/set launch pair per batch rather than one persistent launch,
 * so they are somewhat slower than blowchoc_insert; smaller batches and
 * B = 1 need no scratch at all.
 *  - Limit: min(B, n) <= 4,194,304 keys for batches on the fixed array;
 *    larger batches are rejected with EINVAL and a message naming the limit.
 *  - B = 1 runs the one-warp sequential kernel and 2 <= B <= 16 the one-CTA
 *    batch loop: the tuning's seq_window is not used, because the exact
 *    reservation kernels need a reservation buffer (one word per block) that
 *    would have to be allocated. Results are the same.
 *  - The first call on a device looks the array's device address up
 *    (cudaGetSymbolAddress) with that device current; make that first call
 *    before any stream capture. Call with the filter's device current. The
 *    address is kept for the life of the process: after a device reset
 *    (cudaDeviceReset) it is stale, and this call must not be used again.
 *  - Calls no cudaMalloc, cudaFree or allocating library routine.
 *  - All calls on a device share the one array: two of these calls whose
 *    work overlaps on the GPU (different streams, no ordering between them)
 *    race and give wrong results. Every choice byte of a batch is written
 *    before it is read, so nothing needs clearing between calls.
 * Errors: EINVAL (NULL filter, NULL keys with n > 0, batch over the limit,
 * wrong current device), ECUDA.
 */
int blowchoc_insert_noalloc(blowchoc_filter *f, const uint64_t *d_keys, uint64_t n, void *stream);

/*
 * blowchoc_insert_host / blowchoc_query_host -- blowchoc_insert and
 * blowchoc_query on HOST buffers. Keys move to the device in chunks through
 * a device staging ring on the filter's own copy stream, so the copies of
 * the next chunks overlap the kernels of earlier ones on `stream`. Chunks
 * grow within a call from 2^20 keys to 2^24 (at most a quarter of the ring;
 * 2^22 for a query call issued while the device is idle, which the copies
 * bound), one insert or query launch each. The ring position continues across
 * calls, so a query's first copies overlap the kernels of the insert before
 * it. Insert chunks are whole multiples of the batch size B, so the words and
 * counters equal those of one blowchoc_insert over all n keys. Query chunks
 * are multiples of 64 keys, and the bitmap layout is that of blowchoc_query.
 *   h_keys    host, in, n uint64. Pinned (page-locked) memory lets copies run
 *             asynchronously; pageable memory works but copies synchronously.
 *   h_bitmap  host, out, ceil(n/64) uint64 words.
 * Both calls are ordered on `stream` and return once the work is queued. The
 * caller keeps both buffers alive and unchanged until `stream` completes;
 * the bitmap is complete when it does. The ring is owned by the filter: it
 * holds up to the tuning's host_ring_keys (default 2^27 keys, 1 GiB, plus
 * one bitmap word per 64 keys), no more than the largest call needs, and two
 * chunks at least (two batches if B is larger than a chunk). It grows on
 * demand and never shrinks; growing synchronises the device. Host-buffer
 * calls on one filter share that staging: issue them from one host thread at
 * a time (any streams may be used; per-chunk events order the ring between
 * them).
 * Errors: EINVAL (NULL filter, NULL buffers with n > 0), ENOMEM, ECUDA.
 */
int blowchoc_insert_host(blowchoc_filter *f, const uint64_t *h_keys, uint64_t n, void *stream);
int blowchoc_query_host(blowchoc_filter *f, const uint64_t *h_keys, uint64_t n, uint64_t *h_bitmap,
                        void *stream);

/*
 * blowchoc_query -- membership of d_keys[0..n) (Section 3.1): key t is
 * reported present iff all bits of F(x) are set in at least one of its c
 * candidate blocks. No false negatives for inserted keys.
 *   d_bitmap  device, out, ceil(n/64) uint64 words: bit (t mod 64) of word
 *             t/64 (least significant first) is key t; bits past n are 0.
 * Errors: EINVAL (NULL filter, NULL pointers with n > 0), ECUDA.
 */
int blowchoc_query(blowchoc_filter *f, const uint64_t *d_keys, uint64_t n,
                   uint64_t *d_bitmap, void *stream);

/*
 * blowchoc_stats -- load statistics (Appendix C, Fig. 8): the histogram of
 * set bits per block, the total, and the insert/skip counters. Runs on the
 * filter's home stream and synchronises it before returning (host result).
 * fpr_est is the false-positive rate implied by the histogram for ideal
 * hashing, q = mean_b (L_b/512)^k (exact in expectation for c = 1; with
 * distinct bit selection mean_b C(L_b, k) / C(512, k)), combined over c
 * candidates as if independent: 1 - (1 - q)^c.
 * Errors: EINVAL (NULL pointers), ECUDA, ETIMEOUT (an earlier bounded
 * device wait of this filter gave up; its result is not trustworthy).
 */
int blowchoc_stats(blowchoc_filter *f, blowchoc_filter_stats *out);

/*
 * blowchoc_stats_async / blowchoc_stats_decode -- the same statistics without
 * a host wait, for pipelined callers. stats_async recomputes the histogram
 * on `stream` and copies the filter's raw counters to h_raw
 * (BLOWCHOC_STATS_RAW_WORDS uint64: [0] inserted, [1] skipped, [2] error
 * word, [3 + L] blocks of load L for L = 0..512) on the same stream; it
 * returns once the work is queued. With pinned h_raw the copy is
 * asynchronous; the caller keeps h_raw alive until `stream` completes. The
 * histogram scratch belongs to the filter: order its stats calls (one stream,
 * or streams the caller orders). stats_decode is host-only: it fills `out`
 * from a completed h_raw exactly as blowchoc_stats does.
 * Errors: EINVAL (NULL pointers), ECUDA; decode: ETIMEOUT when the error
 * word is set (an earlier bounded device wait of this filter gave up).
 */
#define BLOWCHOC_STATS_RAW_WORDS 516
int blowchoc_stats_async(blowchoc_filter *f, uint64_t *h_raw, void *stream);
int blowchoc_stats_decode(const blowchoc_filter *f, const uint64_t *h_raw, blowchoc_filter_stats *out);

/*
 * blowchoc_destroy -- synchronise the home stream and free the filter's
 * device memory. NULL is accepted (no-op). The memory is freed even when the
 * synchronisation reports an error. Errors: ECUDA (an earlier asynchronous
 * failure surfaced by the synchronisation).
 */
int blowchoc_destroy(blowchoc_filter *f);

/*
 * blowchoc_words -- the device address and length (8 M words) of the filter
 * words. The library keeps ownership; the pointer is valid until destroy.
 * Reading or writing it must be ordered with the filter's other work.
 * Errors: EINVAL (NULL argument).
 */
int blowchoc_words(blowchoc_filter *f, uint64_t **d_words, uint64_t *nwords);

/*
 * blowchoc_multipliers -- the hash multipliers in use (Section 3.4):
 * a_block[0..c) for h_1..h_c and a_bit[0..k) for f_1..f_k (host arrays of at
 * least 3 and 32 entries). Errors: EINVAL.
 */
int blowchoc_multipliers(blowchoc_filter *f, uint64_t *a_block, uint64_t *a_bit);

/*
 * blowchoc_derive_multipliers -- the multipliers a filter created with
 * `params` will use, without creating it: successive splitmix64 outputs of
 * params->hash_seed, forced odd and redrawn until coprime to the hash's range
 * (Section 3.4); first a_block[0..c) for the range M, then a_bit[0..k) for
 * the range 512 (random bits) or 512 - i for the (i+1)-th (distinct bits,
 * Appendix B). a_block and a_bit are host arrays of at least 3 and 32
 * entries. Host-only: needs no device.
 * Errors: EINVAL (NULL, the parameters blowchoc_create rejects).
 */
int blowchoc_derive_multipliers(const blowchoc_params *params, uint64_t *a_block, uint64_t *a_bit);

/*
 * ---- Sub-arrays (Section 3.4, parallelization) ----------------------------
 * A filter of M blocks can be split into T sub-arrays of ceil(M / T) blocks
 * each, one writer per sub-array (one GPU per sub-array, or all of them on
 * one GPU): an additional linear hash h_0 : U -> [T] with multiplier a_0
 * (same range rules as the block hashes) routes a key to its sub-array, and
 * the block hashes h_1..h_c address [ceil(M / T)] inside it. A sub-array is
 * an ordinary filter (blowchoc_create) of ceil(M / T) blocks whose hash seed
 * is the generator state after a_0 was drawn; each inserts the keys routed
 * to it in their order, in its own batches of B. T = 1 is the unsplit filter.
 */

/* blowchoc_shard_layout -- host-only: a_0 (the first odd splitmix64 output
 * of hash_seed coprime to T; 0 for T = 1), the sub-array size ceil(nblocks /
 * T) and the hash seed of the sub-arrays (the generator state after a_0; the
 * seed itself for T = 1). Errors: EINVAL (NULL, nblocks = 0, T outside
 * 1..1024). */
int blowchoc_shard_layout(uint64_t nblocks, uint32_t T, uint64_t hash_seed, uint64_t *a0, uint64_t *sub_nblocks,
                          uint64_t *sub_seed);

/* blowchoc_shard_partition_scratch -- *words = uint64 words of scratch that
 * blowchoc_shard_partition needs for n keys and T sub-arrays. Host-only.
 * Errors: EINVAL (NULL, T outside 1..1024). */
int blowchoc_shard_partition_scratch(uint64_t n, uint32_t T, uint64_t *words);

/*
 * blowchoc_shard_partition -- stable partition of d_keys[0..n) by sub-array
 * h_0(x) (Section 3.4: the main thread that distributes keys to the
 * sub-arrays' writers).
 *   d_out_keys   device, out, n uint64: the keys of sub-array 0, then of
 *                sub-array 1, ..., each in input order.
 *   d_out_index  device, out, n uint64: input index of each output key.
 *   d_offsets    device, out, T + 1 uint64: sub-array t's keys are output
 *                positions d_offsets[t] .. d_offsets[t + 1] - 1; d_offsets[T] = n.
 *   d_scratch    device, scratch_words uint64 (blowchoc_shard_partition_scratch),
 *                owned by the caller, overwritten.
 * Stream-ordered, asynchronous; three kernels. Errors: EINVAL (NULL buffers
 * with n > 0, T outside 1..1024, even a0 with T > 1, scratch too small), ECUDA.
 */
int blowchoc_shard_partition(const uint64_t *d_keys, uint64_t n, uint32_t T, uint64_t a0, uint64_t *d_out_keys,
                             uint64_t *d_out_index, uint64_t *d_offsets, uint64_t *d_scratch, uint64_t scratch_words,
                             void *stream);

/*
 * blowchoc_shard_unpermute -- the query bitmap in input order from the
 * sub-arrays' answers in partition order.
 *   d_seg_bits  device, in: per sub-array t, an LSB-first bitmap of its
 *               d_offsets[t + 1] - d_offsets[t] keys (as blowchoc_query writes
 *               it), segments of ceil(count / 64) words in order of t.
 *   d_offsets, d_index  device, in: from blowchoc_shard_partition.
 *   d_bitmap    device, out, ceil(n / 64) words: bit d_index[j] set iff the
 *               j-th partitioned key was reported present; other bits 0.
 * Stream-ordered. Errors: EINVAL (NULL buffers with n > 0, T outside
 * 1..1024), ECUDA.
 */
int blowchoc_shard_unpermute(const uint64_t *d_seg_bits, const uint64_t *d_offsets, const uint64_t *d_index,
                             uint64_t n, uint32_t T, uint64_t *d_bitmap, void *stream);

/*
 * blowchoc_set_cost_table -- replace the filter's cost by a table (a learned
 * cost, or any cost outside Eq. 4-6): costs[L * (k + 1) + a] for block load
 * L = 0..512 and new bits a = 0..k; entries with L + a > 512 are never used.
 * Not in the paper. Choices stay exact: the table is ranked on the host like
 * the built-in costs (equal values share a rank; ties go to the lowest
 * choice index). Takes effect for inserts queued after the call.
 * Errors: EINVAL (NULL, c = 1, a used entry not finite), ENOMEM, ECUDA.
 */
int blowchoc_set_cost_table(blowchoc_filter *f, const double *costs);

/*
 * blowchoc_cost_ranks -- the integer ranks the choose kernels compare in
 * place of the costs of Eq. 4-6 (Section 3.2, Appendix A): for block load
 * L = 0..512 and new bits a = 0..k with L + a <= 512, ranks[L * (k + 1) + a]
 * is the position of cost(j = L + a, a) among the distinct values of all
 * reachable costs, evaluated in IEEE double (equal costs share a rank), so
 * that comparing ranks is comparing the doubles. Unreachable entries
 * (L + a > 512) hold 0xFFFF. Host-only: needs no device. `ranks` is a host
 * array of `capacity` >= 513 (k + 1) entries owned by the caller.
 * Errors: EINVAL (NULL, k outside 1..32, unknown cost kind, a parameter that
 * is not finite, negative, or zero for cost^EXP, capacity too small).
 */
int blowchoc_cost_ranks(int cost, double cost_param, uint32_t k, uint16_t *ranks, uint64_t capacity);

/*
 * blowchoc_fpr_estimate -- the estimate blowchoc_stats reports, from a load
 * histogram: hist[L] blocks of load L (513 host entries, caller-owned).
 * A negative finds its bits in a block of load L with probability
 * p_L = (L / 512)^k for independent bit addresses (Section 2.1 per block) or
 * C(L, k) / C(512, k) for k distinct ones (Appendix B); q = the mean of p_L
 * over the blocks, and the estimate is 1 - (1 - q)^c, treating the c
 * candidate blocks as independent (exact in expectation for c = 1).
 * Host-only: needs no device.
 * Errors: EINVAL (NULL, k outside 1..32, c outside 1..3, bitsel > 1, a
 * histogram that counts no block).
 */
int blowchoc_fpr_estimate(const uint64_t *hist, uint32_t k, uint32_t choices, uint32_t bitsel, double *out);

/*
 * blowchoc_l2_residency -- keep part of the filter's words resident in L2
 * for the kernels later queued on `stream` (a created stream, not NULL):
 * sets aside fraction x the device's maximum persisting L2 for this process
 * (a limit of the CUDA context, which ends with it) and gives `stream` an
 * access-policy window over the words with persisting hits. fraction = 0
 * removes the window and releases persisting lines. Never changes results.
 * Errors: EINVAL (fraction outside [0, 1], NULL stream), ECUDA.
 */
int blowchoc_l2_residency(blowchoc_filter *f, double fraction, void *stream);

/*
 * blowchoc_read_words / blowchoc_write_words -- copy filter words
 * [first, first + count) to or from HOST memory (checkpoint and restore: a
 * filter is fully determined by its parameters and its words). Both run on
 * the home stream and synchronise it before returning. write_words leaves
 * the insert/skip counters unchanged.
 * Errors: EINVAL (NULL pointers, range past 8 M words), ECUDA.
 */
int blowchoc_read_words(blowchoc_filter *f, uint64_t first, uint64_t count, uint64_t *h_dst);
int blowchoc_write_words(blowchoc_filter *f, uint64_t first, uint64_t count, const uint64_t *h_src);

/*
 * blowchoc_clear -- reset the filter to empty (all words and counters
 * zero), queued on `stream`. Errors: EINVAL, ECUDA.
 */
int blowchoc_clear(blowchoc_filter *f, void *stream);

/*
 * blowchoc_query_count -- the query of blowchoc_query, counted instead of
 * written out: adds to *d_count the number of keys of d_keys[0..n) that are
 * reported present. For false-positive rates over large negative sets.
 *   d_count   device, in/out, one uint64 (the caller zeroes it).
 * Errors: EINVAL (NULL filter, NULL pointers with n > 0), ECUDA.
 */
int blowchoc_query_count(blowchoc_filter *f, const uint64_t *d_keys, uint64_t n, unsigned long long *d_count,
                         void *stream);

/*
 * blowchoc_generate_keys -- input generation, not part of the filter:
 * d_out[i] = output (start + i) of splitmix64 seeded with `seed`
 * (z = seed + (start + i + 1) * 0x9E3779B97F4A7C15, then the generator's two
 * xor-shift-multiply steps and a final xor-shift), i.e. the stream the
 * Python input generators give on the host.
 *   d_out     device, out, n uint64.
 * Errors: EINVAL (NULL d_out with n > 0), ECUDA.
 */
int blowchoc_generate_keys(uint64_t *d_out, uint64_t n, uint64_t seed, uint64_t start, void *stream);

/*
 * blowchoc_cluster_ctas -- CTAs per cluster that an insert of n keys into f
 * would run cluster-resident with (see blowchoc_tuning.cluster_max), or 0
 * when it would take the global-memory kernels. Needs the device (queries
 * its cluster limits once). Errors: EINVAL (NULL pointers).
 */
int blowchoc_cluster_ctas(blowchoc_filter *f, uint64_t n, uint32_t *ctas);

/*
 * blowchoc_launch_count -- number of kernels this library has launched in
 * this process so far (all filters, all threads). Diagnostic counter for
 * measuring how many launches a piece of work takes.
 */
uint64_t blowchoc_launch_count(void);

/*
 * ---- Many filters in one launch -------------------------------------------
 * A batch object runs the inserts (or queries) of many independent filters
 * in one launch over a device work list, instead of one launch per filter.
 * Each filter keeps its own parameters (M, k, hash multipliers, cost, B); the
 * results are exactly those of blowchoc_insert / blowchoc_query called on
 * each filter in turn. Not in the paper: a library service for workloads of
 * many uneven filters.
 */
typedef struct blowchoc_batch blowchoc_batch;

/* One filter's share of a many-filter call. d_bitmap is used by query only
 * (ceil(n/64) words, same layout as blowchoc_query). */
typedef struct {
    blowchoc_filter *filter;
    const uint64_t *d_keys;
    uint64_t n;
    uint64_t *d_bitmap;
} blowchoc_work;

/* Create / destroy a batch object on the current device. It owns the device
 * work list, the per-filter choice scratch and a recorded graph (if any).
 * Errors: EINVAL, ENOMEM, ECUDA. destroy accepts NULL. */
int blowchoc_batch_create(blowchoc_batch **out);
int blowchoc_batch_destroy(blowchoc_batch *b);

/*
 * blowchoc_insert_many -- insert items[i].d_keys into items[i].filter for
 * every i, with each filter's own batch rule (B of that filter): round r
 * runs the r-th batch of every filter that has one; a grid barrier separates
 * the choose and set phases and the rounds. One cooperative launch per
 * distinct choice count c among the items. Filters with B = 1, or whose
 * insert needs more than max(64, 4 x the median) batches of the call, run
 * through the single-filter kernels on the same stream instead, so that they
 * do not hold the launch's other filters behind their batches. A filter may
 * appear at most once
 * per call. Stream-ordered; the batch object must not be reused for another
 * call until this one's host-side setup has returned (it does not wait for
 * the GPU). Errors: EINVAL (NULL pointers, count 0, repeated filter,
 * filters on another device), ENOMEM, ECUDA.
 */
int blowchoc_insert_many(blowchoc_batch *b, const blowchoc_work *items, uint32_t count, void *stream);

/* blowchoc_query_many -- blowchoc_query for every item, one launch per
 * distinct c. Errors as insert_many. */
int blowchoc_query_many(blowchoc_batch *b, const blowchoc_work *items, uint32_t count, void *stream);

/*
 * blowchoc_batch_record -- record insert_many(ins) followed by
 * query_many(qry) (either list may be empty) as a CUDA graph held by the
 * batch object; blowchoc_batch_replay launches it on `stream`. The recorded
 * pointers and sizes are fixed at record time: replay repeats exactly that
 * work (on the filters' current contents). Recording again replaces the
 * graph. Errors: EINVAL, ENOMEM, ECUDA.
 */
int blowchoc_batch_record(blowchoc_batch *b, const blowchoc_work *ins, uint32_t n_ins,
                          const blowchoc_work *qry, uint32_t n_qry);
int blowchoc_batch_replay(blowchoc_batch *b, void *stream);

/*
 * ---- Serving --------------------------------------------------------------
 * A request-serving loop for device-resident filters: insert and query
 * requests arrive over time (host key buffers, arrival times); a scheduler
 * thread admits filters under an HBM budget, keeps one FIFO per filter, and
 * launches "waves": at most one request per filter (so two inserts of one
 * filter are never merged into one batch), coalesced across filters into one
 * insert_many and one query_many launch, on several streams, ordered per
 * filter by events. Each request's result is exactly what it gives when the
 * requests of its filter run alone, one after another, in arrival order.
 * Host buffers may be pinned (copied directly, asynchronously) or pageable
 * (staged through pinned arenas the server owns: staging_bytes for keys,
 * staging_bytes / 32 for bitmaps), so that no copy blocks the scheduler.
 * A request whose insert needs many batches (more than 64, from a small B)
 * runs in a wave of its own, so it never delays the light requests.
 * Not in the paper: a library service.
 */
typedef struct blowchoc_server blowchoc_server;

typedef struct {
    uint64_t hbm_budget_bytes;   /* device memory for admitted filters */
    uint64_t staging_bytes;      /* device memory for in-flight request keys/bitmaps */
    uint32_t streams;            /* concurrent waves, 1..16 */
    uint32_t max_wave_requests;  /* requests per wave, >= 1 */
} blowchoc_server_config;

#define BLOWCHOC_REQ_INSERT 0u
#define BLOWCHOC_REQ_QUERY 1u

typedef struct {
    uint64_t completed;          /* requests finished */
    uint64_t keys;               /* keys of finished requests */
    uint64_t waves;              /* launch waves */
    double first_arrival_s, last_done_s;
    double p50_latency_s, p99_latency_s, max_latency_s;  /* arrival -> completion */
    double mean_wave_requests;
    uint64_t max_filter_bytes_used;  /* high-water mark of admitted filter memory */
    uint32_t filters_admitted, filters_pending;
    double mean_wave_gpu_ms;     /* stream time from a wave's first copy to its completion */
    double launch_host_s;        /* scheduler time spent building and queueing waves */
} blowchoc_server_summary;

/* Create a server on the current device (its thread starts at
 * blowchoc_server_start). Errors: EINVAL, ENOMEM, ECUDA. */
int blowchoc_server_create(const blowchoc_server_config *cfg, blowchoc_server **out);

/* Register a filter. It is created (admitted) as soon as its memory fits the
 * budget, in registration order; until then its requests wait. *id receives
 * its index. Errors: EINVAL, EBUDGET (larger than the whole budget). */
int blowchoc_server_add_filter(blowchoc_server *s, const blowchoc_params *p, uint32_t *id);

/* Destroy a filter after all its submitted requests have completed, freeing
 * its budget for pending filters. Errors: EINVAL. */
int blowchoc_server_remove_filter(blowchoc_server *s, uint32_t id);

/* Submit a request (thread-safe). h_keys: n host keys (pinned memory copies
 * asynchronously); h_bitmap: query result, ceil(n/64) host words. Both stay
 * owned by the caller and must stay valid until the request completes. The
 * request counts as arriving at arrival_s seconds after start (or at submit
 * time if later). *req_id may be NULL. Errors: EINVAL, EBUDGET (request
 * larger than the staging memory). */
int blowchoc_server_submit(blowchoc_server *s, uint32_t filter_id, uint32_t kind, const uint64_t *h_keys,
                           uint64_t n, uint64_t *h_bitmap, double arrival_s, uint64_t *req_id);

/* Start the clock and the scheduler thread. Errors: EINVAL (started). */
int blowchoc_server_start(blowchoc_server *s);

/* Block until every submitted request has completed (or timeout_s passed:
 * ETIMEOUT). Errors: EINVAL, ECUDA (a launch failed), ETIMEOUT. */
int blowchoc_server_wait(blowchoc_server *s, double timeout_s);

/* Times of one request in seconds since start: arrival, launch, completion
 * (negative while not reached). Errors: EINVAL. */
int blowchoc_server_request_times(blowchoc_server *s, uint64_t req_id, double *arrival, double *launch,
                                  double *done);

/* Aggregate statistics of the completed requests. Errors: EINVAL. */
int blowchoc_server_stats(blowchoc_server *s, blowchoc_server_summary *out);

/* The filter behind an admitted id (NULL while pending); owned by the server.
 * Use only while no request of it is in flight. Errors: EINVAL. */
int blowchoc_server_filter(blowchoc_server *s, uint32_t id, blowchoc_filter **f);

/* Stop the thread, wait for the GPU, free everything. NULL is accepted.
 * Always returns OK. */
int blowchoc_server_destroy(blowchoc_server *s);

/*
 * ---- Learned cost (not in the paper) ----------------------------------------
 * A network g(x), x = ((L + a) / 512, a / k) -- the load after insertion and
 * the new bits relative to k, the arguments of the paper's costs -- with two
 * tanh hidden layers of 32 units and a linear output, fp32. Its values on the
 * whole (L, a) grid form a cost table for blowchoc_set_cost_table. Training
 * (score-function estimator) runs on the GPU: blowchoc_insert_sampled draws
 * each choice from softmax(-g / tau) and accumulates d log pi / d g per grid
 * point; blowchoc_mlp_backward turns those weights into parameter gradients
 * (fp64 accumulation); blowchoc_mlp_adam_step updates the parameters.
 * Parameter layout: W1[32][2], b1[32], W2[32][32] (row = output unit), b2[32],
 * w3[32], b3 (1185 floats).
 */
typedef struct blowchoc_mlp blowchoc_mlp;

/* Network for filters with k bit hashes; weights uniform in +-1/sqrt(fan in)
 * from splitmix64(seed), biases 0. Errors: EINVAL, ENOMEM, ECUDA. */
int blowchoc_mlp_create(uint32_t k, uint64_t seed, blowchoc_mlp **out);
/* Wait for the device, then free the network (NULL is accepted). Always
 * returns OK. */
int blowchoc_mlp_destroy(blowchoc_mlp *m);
uint32_t blowchoc_mlp_param_count(void);

/* Host copies of the parameters (1185 floats) and of the accumulated
 * gradient (1185 doubles); either pointer may be NULL. Synchronous.
 * set_params uploads 1185 floats. Errors: EINVAL (NULL network, NULL
 * h_params for set_params), ECUDA. */
int blowchoc_mlp_get_params(blowchoc_mlp *m, float *h_params, double *h_grad);
int blowchoc_mlp_set_params(blowchoc_mlp *m, const float *h_params);

/* d_table[L (k+1) + a] = g(((L + a) / 512, a / k)) for L = 0..512, a = 0..k
 * (a device array of 513 (k + 1) floats, caller-owned; stream-ordered).
 * Errors: EINVAL (NULL argument), ECUDA. */
int blowchoc_mlp_forward(blowchoc_mlp *m, float *d_table, void *stream);

/* gradient += sum_r d_scales[r] * sum_p d_w[r * P + p] * d g(x_p) / d params,
 * P = 513 (k + 1): `rows` rows of per-point weights (device), one device
 * scale per row (e.g. one training filter's advantage each). Stream-ordered.
 * Errors: EINVAL (NULL argument, rows = 0), ECUDA. */
int blowchoc_mlp_backward(blowchoc_mlp *m, const float *d_w, uint32_t rows, const double *d_scales,
                          void *stream);

/* One Adam step (lr; beta1 0.9, beta2 0.999, eps 1e-8) down the accumulated
 * gradient, which is then cleared. Stream-ordered.
 * Errors: EINVAL (NULL network, lr not > 0, NaN included), ECUDA. */
int blowchoc_mlp_adam_step(blowchoc_mlp *m, float lr, void *stream);

/*
 * blowchoc_insert_sampled -- training-mode insertion with the filter's batch
 * rule: a key already held by a candidate is skipped as usual; otherwise its
 * choice is drawn from softmax(-d_table[p_i] / tau) over its candidates
 * (p_i = L_i (k+1) + a_i), with the uniform taken from the splitmix64 stream
 * of `seed` at the key's index in this call, and
 * d_w[p_i] += (pi_i - 1{i chosen}) / tau  (= d log pi(chosen) / d g(p_i)).
 * d_choice (optional, n bytes) receives the choices (255 = skipped).
 * Errors: EINVAL (c = 1, tau <= 0, NULL pointers), ENOMEM, ECUDA.
 */
int blowchoc_insert_sampled(blowchoc_filter *f, const uint64_t *d_keys, uint64_t n, const float *d_table,
                            float tau, uint64_t seed, float *d_w, uint8_t *d_choice, void *stream);

/*
 * Launch configuration of a filter's kernels. It never changes any result
 * (words, bitmaps, counters are identical for every valid setting); it only
 * changes speed. Defaults are set at create.
 *   lanes_choose, lanes_set, lanes_query: lanes of a warp that share one key
 *       (1, 2, 4 or 8); each lane owns 8/lanes words of every 512-bit block.
 *       Defaults follow the filter's size against the device's L2:
 *       lanes_choose 4 up to L2/2, 2 up to 1.5 x L2, 4 beyond; lanes_query
 *       1 up to L2, 2 beyond.
 *   query_early: 1 = load candidate i+1 only if the key was not found in
 *       candidates 1..i (fewer block reads for members); 0 = load all first;
 *       2 = load the first two up front, later ones only while not found
 *       (three choices; two choices treat 2 as 1).
 *   ctas_per_sm: grid size of the grid-wide kernels, in CTAs per SM (1..16;
 *       the persistent insert caps it at what is co-resident).
 *   persistent: 1 = an insert of batches above 2048 keys runs as one
 *       cooperative launch with grid barriers between phases (each barrier
 *       wait is bounded; on expiry the filter's error word is set and
 *       blowchoc_stats returns ETIMEOUT); 0 = two launches per batch.
 *       lanes_choose then applies to both phases. Batches of 2 to 2048 keys
 *       run in one CTA with CTA barriers, B = 1 in one warp.
 *   keys_per_cta: grid of the persistent insert, as keys of one batch per
 *       CTA (grid = ceil(min(B, n) / keys_per_cta), at most ctas_per_sm CTAs
 *       per SM, at most what is co-resident). The default, 128, spreads a
 *       batch of up to about 39,000 keys over one CTA per 128 keys and gives
 *       larger batches the whole co-resident grid (two 512-thread CTAs per
 *       SM with 2 to 8 lanes per key, two of 256 threads with one); larger
 *       values trade parallelism for fewer CTAs at each grid barrier.
 *   set_mode: how the persistent insert ORs a batch in: 0 = 64-bit atomic OR
 *       reductions (no value returned) of each key's words at L2; 1 = sort by
 *       block: bucket the batch's keys by ranges of 256 blocks, stage each
 *       touched range in shared memory, OR there, write the range back
 *       (offered while ceil(M / 256) <= 65536; larger filters use 0); 2 =
 *       bulk: stage each key's 64-byte mask in shared memory and OR it into
 *       its block with one asynchronous bulk reduction of the copy engine.
 *       Default 2 for filters larger than the L2 size with c <= 2 and for
 *       filters larger than 1.5 times the L2 size with c = 3, else 0.
 *   seq_window: B = 1 (one key at a time) runs in parallel while staying
 *       exactly sequential: windows of seq_window keys (32..8192) go through
 *       rounds in which every pending key reserves its candidate blocks (the
 *       earliest key wins each block) and the keys that won all of theirs
 *       decide and set their bits; such keys share no candidate block with
 *       any earlier pending key. 0 = one warp inserting key after key.
 *       Batches of 2..16 keys (of a filter that does not run
 *       cluster-resident) use the same rounds with whole batches in place
 *       of keys, over windows of seq_window keys rounded to whole batches
 *       (at least four); 0 = one CTA running the batches one after another.
 *       Default 512, or 256 for batches of B = 2..16 keys when
 *       64 (B c)^2 >= M (their candidate blocks meet often); the window
 *       never changes the result.
 *   cluster_max: an insert of at least 4 batches (B >= 2; B <= 2048 while
 *       persistent is 1) into a filter that fits in the shared memory of one
 *       thread-block cluster runs cluster-resident: the cluster's CTAs hold the filter's words (a
 *       contiguous slice each), every batch reads and ORs them there over
 *       distributed shared memory with a cluster barrier between phases,
 *       and the words are written back at the end. cluster_max caps the
 *       CTAs per cluster (1..16, further capped by the device); 0 = never.
 *   lanes_cluster: lanes per key of the cluster-resident insert (4 or 8).
 *   cluster_keys: keys of a batch per CTA that the cluster-resident insert
 *       aims for: a cluster takes more CTAs than the filter needs (up to
 *       cluster_max) while a batch has more keys per CTA (16..2^20).
 *   host_ring_keys: device staging of blowchoc_insert_host / _query_host,
 *       in keys at most (0 = 2^27 keys, 1 GiB; else 2^16..2^31 - 1, rounded
 *       down to a multiple of 64). The ring is sized to the calls (never
 *       more than they need, never shrinking) and holds at least two chunks,
 *       so a batch size B above a quarter of it raises it to two batches.
 */
typedef struct {
    uint32_t lanes_choose;
    uint32_t lanes_set;
    uint32_t lanes_query;
    uint32_t query_early;
    uint32_t ctas_per_sm;
    uint32_t persistent;
    uint32_t keys_per_cta;
    uint32_t set_mode;
    uint32_t seq_window;
    uint32_t cluster_max;
    uint32_t lanes_cluster;
    uint32_t cluster_keys;
    uint32_t host_ring_keys;
} blowchoc_tuning;

/* Read / replace a filter's launch configuration. set_tuning checks every
 * field and changes nothing on error. Errors: EINVAL. */
int blowchoc_get_tuning(blowchoc_filter *f, blowchoc_tuning *out);
int blowchoc_set_tuning(blowchoc_filter *f, const blowchoc_tuning *t);

/* The same for a batch object's many-filter kernels (lanes_choose applies to
 * both insert phases; lanes_query, query_early, ctas_per_sm, cluster_max,
 * lanes_cluster, cluster_keys as above; cluster_max > 0 gives each eligible
 * filter of a call a cluster of its own, default 0). */
int blowchoc_batch_get_tuning(blowchoc_batch *b, blowchoc_tuning *out);
/* Errors (both): EINVAL (NULL argument, a field outside its range; nothing
 * changes then). */
int blowchoc_batch_set_tuning(blowchoc_batch *b, const blowchoc_tuning *t);

/* Launch configuration of a server's filters (applied as each is admitted,
 * like blowchoc_set_tuning) and of its many-filter calls (like
 * blowchoc_batch_set_tuning). Before blowchoc_server_start only; results
 * never change. Without it, a server's filters keep their defaults except
 * cluster_max = 16, lanes_cluster = 4, cluster_keys = 512, and its
 * many-filter calls use the same cluster fields.
 * Errors: EINVAL (bad fields, NULL, already started). */
int blowchoc_server_set_tuning(blowchoc_server *s, const blowchoc_tuning *t);

/*
 * ---- Per-size-class launch configuration of a batch object ----------------
 * A many-filter call treats each filter according to its size class, from
 * its bytes (64 M) against the device's L2 size:
 *   BLOWCHOC_CLASS_CACHE  64 M <= L2 / 16  (a few of them fit L2 at once)
 *   BLOWCHOC_CLASS_L2     64 M <= L2 / 2
 *   BLOWCHOC_CLASS_SPILL  64 M <= 2 L2     (partly L2-resident)
 *   BLOWCHOC_CLASS_HBM    larger           (HBM-resident)
 * and keeps one configuration per (class, k, c): the class tuning below. A
 * filter whose (class, k, c) has none uses the batch object's tuning (route
 * 0, its lanes, 128 keys per tile). Results never depend on the choice.
 */
enum {
    BLOWCHOC_CLASS_CACHE = 0,
    BLOWCHOC_CLASS_L2 = 1,
    BLOWCHOC_CLASS_SPILL = 2,
    BLOWCHOC_CLASS_HBM = 3,
    BLOWCHOC_NUM_CLASSES = 4
};
enum {
    BLOWCHOC_ROUTE_WORKLIST = 0,  /* inserted over the many-filter work list */
    BLOWCHOC_ROUTE_DIRECT = 1,    /* blowchoc_insert with the direct (atomic OR) set */
    BLOWCHOC_ROUTE_SORTED = 2     /* blowchoc_insert with the sort-by-block set */
};
typedef struct {
    uint32_t route;         /* BLOWCHOC_ROUTE_*: how the class's inserts run */
    uint32_t lanes_choose;  /* work-list insert: lanes per key, 1, 2, 4 or 8 */
    uint32_t tile;          /* work-list insert: keys per tile, 32 .. 1024, a power of two */
    uint32_t lanes_query;   /* work-list query: lanes per key, 1, 2, 4 or 8 */
    uint32_t query_early;   /* work-list query: 1 = stop at the first candidate holding the key */
} blowchoc_class_tuning;

/* Size class (BLOWCHOC_CLASS_*) of a filter of `nblocks` blocks on the batch
 * object's device. Errors: EINVAL (NULL). */
int blowchoc_batch_size_class(blowchoc_batch *b, uint64_t nblocks, uint32_t *cls);

/* The configuration of (cls, k, c): *is_set = 1 if one was set or tuned,
 * else 0 and *out holds the defaults that apply. Errors: EINVAL. */
int blowchoc_batch_get_class_tuning(blowchoc_batch *b, uint32_t cls, uint32_t k, uint32_t c,
                                    blowchoc_class_tuning *out, uint32_t *is_set);

/* Set the configuration of (cls, k, c); every field is checked and nothing
 * changes on error. A recorded graph keeps the configuration it was recorded
 * with. Errors: EINVAL. */
int blowchoc_batch_set_class_tuning(blowchoc_batch *b, uint32_t cls, uint32_t k, uint32_t c,
                                    const blowchoc_class_tuning *t);

/* Forget every class configuration. Errors: EINVAL (NULL). */
int blowchoc_batch_clear_class_tuning(blowchoc_batch *b);

/*
 * blowchoc_batch_autotune -- time insert_many + query_many of `ins` / `qry`
 * on scratch copies of the filters (same parameters, empty; the callers'
 * filters are not touched). First the batch object's tuning: lanes per key
 * for insert and query and CTAs per SM over the whole call. Then, for every
 * (size class, k, c) present, one dimension at a time on that class's
 * filters alone: lanes per key and keys per tile of the work-list insert,
 * the route (work list, direct or sort-by-block single-filter insert), and
 * lanes per key and early exit of the query. The fastest of each is kept on
 * the batch object (class tunings cached per (class, k, c) for later calls)
 * and the batch tuning is returned in *best (may be NULL). Results never
 * depend on the choices. Synchronises `stream`. Errors: EINVAL, ENOMEM,
 * ECUDA.
 */
int blowchoc_batch_autotune(blowchoc_batch *b, const blowchoc_work *ins, uint32_t n_ins,
                            const blowchoc_work *qry, uint32_t n_qry, void *stream,
                            blowchoc_tuning *best);

/*
 * blowchoc_gather_probe -- measurement aid, not part of the filter: reads
 * nreads pseudo-random whole 64-byte blocks of d_words[0 .. 8 nblocks) (the
 * access pattern of insert and query) with `lanes` lanes per block (1, 2, 4
 * or 8) on SMs x ctas_per_sm CTAs, each lane group keeping `inflight` (1, 2,
 * 4 or 8) independent block loads in flight before folding them, and writes
 * one folded word per warp to d_sink (at least SMs x ctas_per_sm x 8 words).
 * Timed by the caller, it gives the random-sector ceiling of the device.
 * Errors: EINVAL, ECUDA.
 */
int blowchoc_gather_probe(const uint64_t *d_words, uint64_t nblocks, uint64_t nreads, uint64_t seed,
                          uint32_t lanes, uint32_t ctas_per_sm, uint32_t inflight, uint64_t *d_sink,
                          void *stream);

/*
 * blowchoc_barrier_selftest -- diagnostic of the bounded device waits, not
 * part of the filter: a cooperative launch of `ctas` CTAs in which the last
 * CTA never arrives at a grid barrier; the others wait at most `seconds`
 * (0 < seconds <= 10) of SM clock and give up. Returns BLOWCHOC_ETIMEOUT when
 * the bound worked (the expected outcome), BLOWCHOC_OK never, and leaves the
 * context usable. Synchronises `stream`. Errors: EINVAL, ENOMEM, ECUDA.
 */
int blowchoc_barrier_selftest(uint32_t ctas, double seconds, void *stream);

/* Text of the calling thread's last error ("" if none). Never NULL. */
const char *blowchoc_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* BLOWCHOC_H */
