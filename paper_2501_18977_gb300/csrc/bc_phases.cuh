// Phase helpers shared by the single-filter and many-filter kernels: the
// per-key decision, the OR into the chosen block, counter flushes, the
// bounded grid barrier and the query bitmap helpers.
#pragma once

#include "bc_device.cuh"

namespace bc {

constexpr unsigned kFull = 0xffffffffu;

// Copies the rank table into shared memory (only needed with choices).
template <int C>
__device__ __forceinline__ const uint16_t *stage_rank(const uint16_t *rank_g, uint16_t *s_rank,
                                                      uint32_t k1) {
    if constexpr (C == 1) {
        return rank_g;
    } else {
        for (uint32_t t = threadIdx.x; t < 513u * k1; t += blockDim.x) s_rank[t] = rank_g[t];
        __syncthreads();
        return s_rank;
    }
}

// Decision of one key by its group, given the group's share m of the key's
// mask: loads the C candidate blocks (the lane's W-word slice of each),
// computes L and a for each and returns the choice.
template <int C, int LANES, int PATH>
__device__ __forceinline__ uint32_t choose_one(const DevFilter &f, uint64_t x, bool valid, int q,
                                               const uint16_t *rank,
                                               const uint64_t (&m)[kBlockWords / LANES]) {
    constexpr int W = kBlockWords / LANES;
    uint64_t blk[C][W];
#pragma unroll
    for (int i = 0; i < C; ++i) {
        const uint64_t b = block_addr(f, f.a_block[i], x);
        if (valid) {
            load_words<W, PATH>(f.words + b * kBlockWords + (uint64_t)q * W, blk[i]);
        } else {
#pragma unroll
            for (int j = 0; j < W; ++j) blk[i][j] = ~0ull;
        }
    }
    uint32_t la[C];
#pragma unroll
    for (int i = 0; i < C; ++i) la[i] = group_sum<LANES>(load_and_new<W>(blk[i], m));
    return choose_from_terms<C>(la, rank, f.k + 1);
}

// The same decision, built for latency: the candidate blocks' loads are
// issued first, the key's mask is built (key_mask_shared, warp-collective)
// while they are in flight, then the terms are formed. m receives the mask.
template <int C, int LANES, int PATH>
__device__ __forceinline__ uint32_t choose_key(const DevFilter &f, uint64_t x, bool valid, int q,
                                               const uint16_t *rank, const uint64_t *s_amul, uint32_t *region,
                                               uint64_t (&m)[kBlockWords / LANES]) {
    constexpr int W = kBlockWords / LANES;
    uint64_t blk[C][W];
#pragma unroll
    for (int i = 0; i < C; ++i) {
        const uint64_t b = block_addr(f, f.a_block[i], x);
        if (valid) {
            load_words<W, PATH>(f.words + b * kBlockWords + (uint64_t)q * W, blk[i]);
        } else {
#pragma unroll
            for (int j = 0; j < W; ++j) blk[i][j] = ~0ull;
        }
    }
    key_mask_shared<LANES>(s_amul, f.k, x, q, region, m, f.bitsel);
    uint32_t la[C];
#pragma unroll
    for (int i = 0; i < C; ++i) la[i] = group_sum<LANES>(load_and_new<W>(blk[i], m));
    return choose_from_terms<C>(la, rank, f.k + 1);
}

// choose_key that also reports which of the chosen block's eight words get
// new bits (bit w of *words: word w of the key's mask has bits the block
// lacked at the batch start). Bits set then stay set, so a word without new
// bits needs no OR in the set phase.
template <int C, int LANES, int PATH>
__device__ __forceinline__ uint32_t choose_key_words(const DevFilter &f, uint64_t x, bool valid, int q,
                                                     const uint16_t *rank, const uint64_t *s_amul, uint32_t *region,
                                                     uint64_t (&m)[kBlockWords / LANES], uint32_t &words) {
    constexpr int W = kBlockWords / LANES;
    uint64_t blk[C][W];
#pragma unroll
    for (int i = 0; i < C; ++i) {
        const uint64_t b = block_addr(f, f.a_block[i], x);
        if (valid) {
            load_words<W, PATH>(f.words + b * kBlockWords + (uint64_t)q * W, blk[i]);
        } else {
#pragma unroll
            for (int j = 0; j < W; ++j) blk[i][j] = ~0ull;
        }
    }
    key_mask_shared<LANES>(s_amul, f.k, x, q, region, m, f.bitsel);
    uint32_t la[C];
#pragma unroll
    for (int i = 0; i < C; ++i) la[i] = group_sum<LANES>(load_and_new<W>(blk[i], m));
    const uint32_t s = choose_from_terms<C>(la, rank, f.k + 1);
    uint32_t v = 0;
#pragma unroll
    for (int i = 0; i < C; ++i) {
        if ((uint32_t)i == s) {
#pragma unroll
            for (int j = 0; j < W; ++j) v |= (m[j] & ~blk[i][j]) ? (1u << (q * W + j)) : 0u;
        }
    }
#pragma unroll
    for (int sh = LANES / 2; sh > 0; sh >>= 1) v |= __shfl_xor_sync(kFull, v, sh, LANES);
    words = v;
    return s;
}

// set_one restricted to the words flagged in `words` (bit w = word w).
template <int LANES>
__device__ __forceinline__ void set_words(const DevFilter &f, uint64_t b, int q, const uint64_t (&m)[kBlockWords / LANES],
                                          uint32_t words) {
    constexpr int W = kBlockWords / LANES;
    unsigned long long *dst =
        reinterpret_cast<unsigned long long *>(f.words + b * kBlockWords + (uint64_t)q * W);
#pragma unroll
    for (int j = 0; j < W; ++j)
        if ((words >> (q * W + j)) & 1u) red_or(dst + j, (unsigned long long)m[j]);
}

// OR of the key's bits into block b: lane q of the group owns W words.
template <int LANES>
__device__ __forceinline__ void set_one(const DevFilter &f, uint64_t b, int q,
                                        const uint64_t (&m)[kBlockWords / LANES]) {
    constexpr int W = kBlockWords / LANES;
    unsigned long long *dst =
        reinterpret_cast<unsigned long long *>(f.words + b * kBlockWords + (uint64_t)q * W);
#pragma unroll
    for (int j = 0; j < W; ++j)
        if (m[j]) red_or(dst + j, (unsigned long long)m[j]);
}

// Sums two per-thread counters over the CTA and adds them to counters[0..1].
__device__ __forceinline__ void flush_counts(uint32_t ins, uint32_t skp, unsigned long long *counters) {
    __shared__ unsigned long long s_cnt[2];
    if (threadIdx.x == 0) { s_cnt[0] = 0; s_cnt[1] = 0; }
    __syncthreads();
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
        ins += __shfl_xor_sync(kFull, ins, s);
        skp += __shfl_xor_sync(kFull, skp, s);
    }
    if ((threadIdx.x & 31) == 0 && (ins | skp)) {
        atomicAdd(&s_cnt[0], (unsigned long long)ins);
        atomicAdd(&s_cnt[1], (unsigned long long)skp);
    }
    __syncthreads();
    if (threadIdx.x == 0 && (s_cnt[0] | s_cnt[1])) {
        atomicAdd(&counters[0], s_cnt[0]);
        atomicAdd(&counters[1], s_cnt[1]);
    }
}

// Clock cycles a CTA waits at a grid barrier before it gives up (about 2 s).
constexpr long long kBarrierCycles = 4000000000ll;

__device__ __forceinline__ unsigned int ld_acquire(const unsigned int *p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid-wide barrier of a co-resident grid. *bar counts arrivals over the
// whole launch (zeroed before it); the barrier completes when it reaches
// `target`. A wait past kBarrierCycles, or an error word already set by
// another CTA, sets *err and returns false; the caller then leaves.
//
// Each CTA's first thread arrives with one release reduction (no value
// returned, so it starts polling at once) after a CTA barrier, which makes
// every write of the CTA part of that release; the acquiring load that sees
// the count complete then synchronises with every CTA's arrival, and the
// closing CTA barrier passes that on to the CTA's other threads. On the DNA
// insert (96 barriers) this took 3.679 ms against 3.716 ms for a full fence
// before a returning atomic add and after the wait; a last-arriver flag on a
// line of its own (3.772 ms) and a two-level arrival tree (3.831 ms) were
// slower, each adding a hop to the release.
__device__ __forceinline__ bool grid_barrier(unsigned int *bar, unsigned int target,
                                             unsigned long long *err, long long limit = kBarrierCycles) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(bar) : "memory");
        const long long t0 = clock64();
        while (ld_acquire(bar) < target) {
            if (*reinterpret_cast<volatile unsigned long long *>(err) != 0ull ||
                clock64() - t0 > limit) {
                atomicExch(err, 1ull);
                ok = 0;
                break;
            }
            __nanosleep(100);
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// ANDs each group's LANES ballot bits down onto the group's first bit.
template <int LANES>
__device__ __forceinline__ uint32_t fold_groups(uint32_t b) {
#pragma unroll
    for (int s = 1; s < LANES; s <<= 1) b &= b >> s;
    return b;
}

// Gathers bit g*LANES of v for g = 0..G-1 into bits 0..G-1 (mask-and-shift
// compaction in log2(G) steps).
template <int LANES>
__device__ __forceinline__ uint32_t compress_groups(uint32_t v) {
    if constexpr (LANES == 1) {
        return v;
    } else if constexpr (LANES == 2) {
        v &= 0x55555555u;
        v = (v | (v >> 1)) & 0x33333333u;
        v = (v | (v >> 2)) & 0x0F0F0F0Fu;
        v = (v | (v >> 4)) & 0x00FF00FFu;
        return (v | (v >> 8)) & 0x0000FFFFu;
    } else if constexpr (LANES == 4) {
        v &= 0x11111111u;
        v = (v | (v >> 3)) & 0x03030303u;
        v = (v | (v >> 6)) & 0x000F000Fu;
        return (v | (v >> 12)) & 0x000000FFu;
    } else {
        static_assert(LANES == 8, "LANES must be 1, 2, 4 or 8");
        v &= 0x01010101u;
        v = (v | (v >> 7)) & 0x00030003u;
        return (v | (v >> 14)) & 0x0000000Fu;
    }
}

// Answers keys [64 wd, 64 wd + 64) of `keys` (fewer at the tail) and
// returns their bitmap word. Per key, a group of LANES lanes builds the key's
// mask once (key_mask_shared), then tests the candidate blocks: each lane
// checks its W words for F(x) & ~block == 0, a ballot per candidate ANDs the
// lanes of each group, and the candidates OR. MODE 0 issues all C block
// loads before any test; MODE 1 loads candidate i+1 only for groups whose key
// was not found in candidates 1..i; MODE 2 loads the first two candidates up
// front and the others only while not found. The first loads are issued
// before the mask is built. Warp-collective.
template <int C, int LANES, int MODE>
__device__ __forceinline__ uint64_t query_word(const DevFilter &f, const uint64_t *__restrict__ keys,
                                               uint64_t n, uint64_t wd, const uint64_t *s_amul,
                                               uint32_t *region, int q, int g) {
    constexpr int W = kBlockWords / LANES;
    constexpr int G = 32 / LANES;
    constexpr int U = MODE == 0 ? C : (MODE == 2 && C >= 2 ? 2 : 1);  // candidates loaded up front
    uint64_t word = 0;
    uint64_t xn = wd * 64 + g < n ? load_key(keys + wd * 64 + g) : 0ull;  // one step ahead
    for (int it = 0; it < 64 / G; ++it) {
        const uint64_t i = wd * 64 + (uint64_t)it * G + g;
        const bool valid = i < n;
        const uint64_t x = xn;
        if (it + 1 < 64 / G) xn = i + G < n ? load_key(keys + i + G) : 0ull;
        uint64_t up[U][W];
#pragma unroll
        for (int c = 0; c < U; ++c) {
            if (valid) {
                load_words<W, kLoadNC>(f.words + block_addr(f, f.a_block[c], x) * kBlockWords + (uint64_t)q * W,
                                       up[c]);
            } else {
#pragma unroll
                for (int j = 0; j < W; ++j) up[c][j] = 0ull;
            }
        }
        uint64_t m[W];
        key_mask_shared<LANES>(s_amul, f.k, x, q, region, m, f.bitsel);
        uint32_t hits = 0;
        bool need = valid;
#pragma unroll
        for (int c = 0; c < C; ++c) {
            uint64_t blk[W];
            if (c < U) {
#pragma unroll
                for (int j = 0; j < W; ++j) blk[j] = up[c < U ? c : 0][j];
            } else if (need) {
                load_words<W, kLoadNC>(f.words + block_addr(f, f.a_block[c], x) * kBlockWords + (uint64_t)q * W,
                                       blk);
            } else {
#pragma unroll
                for (int j = 0; j < W; ++j) blk[j] = 0ull;
            }
            uint64_t miss = 0;
#pragma unroll
            for (int j = 0; j < W; ++j) miss |= m[j] & ~blk[j];
            const uint32_t got = fold_groups<LANES>(__ballot_sync(kFull, need && miss == 0));
            hits |= got;
            if (MODE != 0) need = need && !((got >> (g * LANES)) & 1u);
        }
        word |= (uint64_t)compress_groups<LANES>(hits) << (it * G);
    }
    return word;
}

}  // namespace bc
