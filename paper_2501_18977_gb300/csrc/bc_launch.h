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
// arrival counter; a barrier wait that times out sets counters[2].
cudaError_t launch_persistent_insert(int C, const Launch &L, const DevFilter &f, const uint64_t *keys,
                                     uint64_t n, uint64_t B, const uint16_t *rank, uint8_t *sel,
                                     unsigned long long *counters, unsigned int *bar, int sms);

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

// B = 1: one warp inserts the keys strictly one after another.
cudaError_t launch_sequential(int C, cudaStream_t s, const DevFilter &f, const uint64_t *keys,
                              uint64_t n, const uint16_t *rank, unsigned long long *counters);

// 1 < B <= kSmallBatchMax: one CTA runs all batches with CTA barriers.
cudaError_t launch_small_batch(int C, const Launch &L, const DevFilter &f, const uint64_t *keys,
                               uint64_t n, uint64_t B, const uint16_t *rank,
                               unsigned long long *counters);

// Membership query into an LSB-first bitmap of ceil(n/64) words.
cudaError_t launch_query(int C, const Launch &L, const DevFilter &f, const uint64_t *keys,
                         uint64_t n, uint64_t *bitmap);

// Many-filter execution (bc_many.cu): one cooperative insert launch over the
// rounds of a work list, and one query launch over its bitmap words.
struct ManyItem;
uint64_t many_tile();
cudaError_t launch_insert_many(int C, int lanes, int grid, cudaStream_t s, const ManyItem *items,
                               uint32_t nitems, const uint32_t *prefix, uint32_t nrounds, unsigned int *bar,
                               unsigned long long *err, int sms);
cudaError_t launch_query_many(int C, int lanes, bool early, int grid, cudaStream_t s, const ManyItem *items,
                              uint32_t nitems, const uint32_t *prefix);

// Load histogram: hist[L] += blocks with L set bits (hist has 513 entries).
cudaError_t launch_stats(const Launch &L, const uint64_t *words, uint64_t M,
                         unsigned long long *hist);

}  // namespace bc
