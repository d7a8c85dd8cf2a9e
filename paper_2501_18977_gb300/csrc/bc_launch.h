// Host-side launchers of the BlowChoc kernels (internal to the library).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "bc_device.cuh"

namespace bc {

// Largest batch the single-CTA batch kernel holds in shared memory.
constexpr uint64_t kSmallBatchMax = 16384;
// Batches up to this size use the single-CTA kernel in blowchoc_insert.
constexpr uint64_t kSingleCtaBatch = 2048;

struct Launch {
    int grid;          // CTAs
    int lanes;         // lanes per key (2, 4, 8)
    cudaStream_t stream;
    int early = 0;     // query: load later candidates only while not yet found
};

// Insertion, batch-synchronous (Section 3.2 with the batch rule of the
// library): phase 1 writes each key's choice (or kSkip) to sel[0..n),
// phase 2 OR-s the keys' bits into the chosen blocks.
cudaError_t launch_choose(int C, const Launch &L, const DevFilter &f, const uint64_t *keys,
                          uint64_t n, const uint16_t *rank, uint8_t *sel,
                          unsigned long long *counters);
cudaError_t launch_set(const Launch &L, const DevFilter &f, const uint64_t *keys, uint64_t n,
                       const uint8_t *sel);

// All batches of one insert in a single cooperative launch (grid barriers
// between phases; every CTA co-resident). L.grid is the wanted grid, capped
// at what fits on `sms` SMs. sel holds min(B, n) choices; bar is a zeroed
// arrival counter; a barrier wait that times out sets counters[2]. With
// `bulk` the set phase ORs each key's 64-byte mask in with one bulk
// reduction (set_mode 2) instead of a 64-bit red per word.
cudaError_t launch_persistent_insert(int C, const Launch &L, const DevFilter &f, const uint64_t *keys,
                                     uint64_t n, uint64_t B, const uint16_t *rank, uint8_t *sel,
                                     unsigned long long *counters, unsigned int *bar, int sms, bool bulk);

// Sort-by-block variant of the persistent insert: blocks per range, and the
// number of ranges up to which it is offered.
constexpr uint32_t kRangeBlocks = 256;
constexpr uint64_t kSortedMaxRanges = 1u << 16;

// scratch: 3 R + 1 + min(B, n) u32 (counts, cursors, offsets, key order).
cudaError_t launch_sorted_insert(int C, const Launch &L, const DevFilter &f, const uint64_t *keys, uint64_t n,
                                 uint64_t B, const uint16_t *rank, uint8_t *sel, unsigned long long *counters,
                                 unsigned int *bar, uint32_t *scratch, uint32_t R, int sms);

// B = 1 exactly, in parallel (reservation rounds over windows of keys, one
// CTA). resv: M zeroed u64 (zeroed by the launcher). window in 32..kSeqMaxWindow.
constexpr uint32_t kSeqMaxWindow = 8192;
cudaError_t launch_exact_sequential(int C, cudaStream_t s, const DevFilter &f, const uint64_t *keys, uint64_t n,
                                    uint32_t window, const uint16_t *rank, unsigned long long *counters,
                                    unsigned long long *resv);

// 2 <= B <= kSeqMaxBatch, exactly, by the same reservation rounds with a
// batch in place of a key; window is a multiple of B in B..kSeqMaxWindow.
constexpr uint64_t kSeqMaxBatch = 16;  // measured: beyond, the one-CTA batch loop is faster
cudaError_t launch_exact_batched(int C, cudaStream_t s, const DevFilter &f, const uint64_t *keys, uint64_t n,
                                 uint64_t B, uint32_t window, const uint16_t *rank, unsigned long long *counters,
                                 unsigned long long *resv);

// B = 1: one warp inserts the keys strictly one after another.
cudaError_t launch_sequential(int C, cudaStream_t s, const DevFilter &f, const uint64_t *keys,
                              uint64_t n, const uint16_t *rank, unsigned long long *counters);

// 1 < B <= kSmallBatchMax: one CTA runs all batches with CTA barriers.
cudaError_t launch_small_batch(int C, const Launch &L, const DevFilter &f, const uint64_t *keys,
                               uint64_t n, uint64_t B, const uint16_t *rank,
                               unsigned long long *counters);

// Membership query into an LSB-first bitmap of ceil(n/64) words (bitmap may
// be null); with count, the number of present keys is added to *count.
cudaError_t launch_query(int C, const Launch &L, const DevFilter &f, const uint64_t *keys,
                         uint64_t n, uint64_t *bitmap, unsigned long long *count = nullptr);

// d_out[i] = output start + i of splitmix64 seeded with `seed`.
cudaError_t launch_generate_keys(cudaStream_t s, int sms, uint64_t *d_out, uint64_t n, uint64_t seed,
                                 uint64_t start);

// Device work-list entry of one filter (many-filter and cluster launches).
struct ManyItem {
    DevFilter f;
    const uint16_t *rank;
    const uint64_t *keys;
    uint64_t n;
    uint64_t B;
    uint8_t *sel;                  // min(B, n) choice bytes (insert)
    unsigned long long *counters;  // the filter's counters (inserted, skipped)
    uint64_t *bitmap;              // query output
};

// Many-filter execution (bc_many.cu): one cooperative insert launch over the
// rounds of a work list, and one query launch over its bitmap words.
uint64_t many_tile();
// bitsel: some item uses distinct bit selection; pow2: every item's block
// count is a power of two (each picks a kernel instance, never a result).
cudaError_t launch_insert_many(int C, int lanes, bool bitsel, bool pow2, int grid, cudaStream_t s,
                               const ManyItem *items, uint32_t nitems, const uint32_t *prefix, uint32_t nrounds,
                               uint32_t tile, unsigned int *bar, unsigned long long *err, int sms);
cudaError_t launch_query_many(int C, int lanes, bool early, bool bitsel, bool pow2, int grid, cudaStream_t s,
                              const ManyItem *items, uint32_t nitems, const uint32_t *prefix);

// Cluster-resident insert (bc_cluster.cu): one thread-block cluster holds a
// whole filter in the distributed shared memory of its CTAs and runs every
// batch of the insert there (choose, cluster barrier, set, cluster barrier).
// Cluster i of the launch takes items[i]; with items == nullptr the launch
// has one cluster and takes `one`.
constexpr uint64_t kClusterMinRounds = 4;  // fewer batches take the global-memory kernels
constexpr uint64_t kClusterMaxPasses = 4;  // so do batches of more than 4 keys per lane group of a cluster
struct ClusterShape {
    int S = 0;              // CTAs per cluster (0: the filters do not fit)
    uint32_t slice = 0;     // blocks per CTA (the largest filter's)
    uint32_t rank_u16 = 0;  // rank-table entries per CTA (the largest k's)
    uint32_t kpc = 0;       // keys of one batch per CTA (key buffers and choice bytes)
    size_t smem = 0;        // dynamic shared memory per CTA
};
// Shape for filters of at most M blocks, k bit hashes and batches of at most
// Beff keys: the fewest CTAs per cluster (at most max_S, capped by the device)
// that hold the filter; with keys_per_cta > 0, more CTAs while a batch has
// more than keys_per_cta keys per CTA (fewer passes per batch).
// cluster_shape_at: the shape at exactly S CTAs (S = 0: no fit).
ClusterShape cluster_shape(int C, int lanes, uint64_t M, uint32_t k, uint64_t Beff, int max_S,
                           uint64_t keys_per_cta);
ClusterShape cluster_shape_at(int C, int lanes, int S, uint64_t M, uint32_t k, uint64_t Beff);
cudaError_t launch_cluster_insert(int C, int lanes, const ClusterShape &sh, int nclusters, cudaStream_t s,
                                  const ManyItem *items, const ManyItem &one);

// Load histogram: hist[L] += blocks with L set bits (hist has 513 entries).
cudaError_t launch_stats(const Launch &L, const uint64_t *words, uint64_t M,
                         unsigned long long *hist);

}  // namespace bc
