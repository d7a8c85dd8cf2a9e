// Device-side building blocks of the BlowChoc filter kernels (sm_103a).
//
// A key is handled by a group of LANES consecutive lanes of a warp; lane q of
// the group owns W = 8 / LANES consecutive 64-bit words of every 512-bit block
// (words q*W .. q*W+W-1). One group therefore moves a whole 64-byte block with
// one W*8-byte vector access per lane, and a warp instruction touches
// 32 / LANES blocks, each as one contiguous 64-byte segment.
#pragma once

#include <cstdint>

namespace bc {

constexpr int kBlockWords = 8;  // 512 bits
constexpr uint32_t kSkip = 0xFFu;

// Hash range kinds of the linear hash (Section 3.4).
enum : uint32_t { kRangePow2 = 0, kRangeEven = 1, kRangeOdd = 2 };

// Everything a kernel needs to address one filter. Passed by value as a
// kernel parameter, so per-thread indexing of the multipliers reads the
// constant bank with a uniform address.
struct DevFilter {
    uint64_t *words;       // 8 * M words
    uint64_t M;            // blocks
    uint32_t k;            // bit hashes
    uint32_t range_kind;   // kRange* for M
    uint32_t shift;        // pow2 M: 64 - log2(M); 64 when M == 1
    uint32_t c;            // choices (for dispatch checks)
    uint32_t bitsel;       // 0 = random bit selection, 1 = distinct (Appendix B)
    uint32_t pad;
    uint64_t mod_mul;      // floor(2^64 / M) for M not a power of two (mod_fast)
    uint64_t a_block[3];   // h_1..h_c multipliers
    uint64_t a_bit[32];    // f_1..f_k multipliers
};

// y mod d for d >= 2 with mul = floor(2^64 / d): q = floor(y mul / 2^64) is
// floor(y / d) or one less (mul > 2^64 / d - 1 and y < 2^64), so y - q d
// lies in [0, 2d) and one conditional subtraction finishes it. Exact for
// every 64-bit y; replaces the library's 64-bit division.
__host__ __device__ constexpr uint64_t mod_mul_for(uint64_t d) {
    return ~0ull / d + (~0ull % d == d - 1 ? 1ull : 0ull);
}
__device__ __forceinline__ uint64_t mod_fast(uint64_t y, uint64_t d, uint64_t mul) {
    const uint64_t q = __umul64hi(y, mul);
    const uint64_t r = y - q * d;
    return r >= d ? r - d : r;
}

// h_i(x): linear hash into [M] (Section 3.4) with u = 64.
__device__ __forceinline__ uint64_t block_addr(const DevFilter &f, uint64_t a, uint64_t x) {
    uint64_t y = a * x;
    if (f.range_kind == kRangePow2) return f.shift >= 64 ? 0ull : (y >> f.shift);
    if (f.range_kind == kRangeEven) y ^= (y >> 32);
    return mod_fast(y, f.M, f.mod_mul);
}

// mod_mul_for(512 - i) for the ranges of distinct bit selection (i >= 1).
__constant__ const uint64_t kBitRangeMul[32] = {
    0, mod_mul_for(511), mod_mul_for(510), mod_mul_for(509), mod_mul_for(508), mod_mul_for(507),
    mod_mul_for(506), mod_mul_for(505), mod_mul_for(504), mod_mul_for(503), mod_mul_for(502),
    mod_mul_for(501), mod_mul_for(500), mod_mul_for(499), mod_mul_for(498), mod_mul_for(497),
    mod_mul_for(496), mod_mul_for(495), mod_mul_for(494), mod_mul_for(493), mod_mul_for(492),
    mod_mul_for(491), mod_mul_for(490), mod_mul_for(489), mod_mul_for(488), mod_mul_for(487),
    mod_mul_for(486), mod_mul_for(485), mod_mul_for(484), mod_mul_for(483), mod_mul_for(482),
    mod_mul_for(481)};

__device__ __forceinline__ uint64_t block_mult(const DevFilter &f, uint32_t i) {
    return i == 0 ? f.a_block[0] : (i == 1 ? f.a_block[1] : f.a_block[2]);
}

// f_i(x) for distinct selection: the linear hash of Section 3.4 into
// [range] (range = 512 - i + 1 <= 512): top bits for 512, xor-fold for even
// ranges, plain modulo for odd ones.
__device__ __forceinline__ uint32_t bit_hash_range(uint64_t a, uint64_t x, uint32_t range) {
    uint64_t y = a * x;
    if (range == 512u) return (uint32_t)(y >> 55);
    if ((range & 1u) == 0) y ^= (y >> 32);
    return (uint32_t)mod_fast(y, range, kBitRangeMul[512u - range]);
}

// Index of the r-th (0-based) zero bit of a 64-bit word that has more than
// r zero bits: binary search with popcounts of the low halves.
__device__ __forceinline__ uint32_t select_zero64(uint64_t word, uint32_t r) {
    uint64_t v = ~word;
    uint32_t p = 0;
#pragma unroll
    for (int s = 32; s >= 1; s >>= 1) {
        const uint32_t c = __popcll(v & ((1ull << s) - 1ull));
        if (r >= c) {
            r -= c;
            v >>= s;
            p += s;
        }
    }
    return p;
}

// Full 512-bit mask of F(x) under distinct selection (Appendix B): f_i maps
// into [512 - i + 1] and becomes the f_i-th position (in ascending order)
// not taken by f_1..f_{i-1} -- the paper's increment rule, computed by
// counting free positions per word.
__device__ __forceinline__ void distinct_mask(const uint64_t *amul, uint32_t k, uint64_t x, uint64_t (&w)[8]) {
#pragma unroll
    for (int j = 0; j < 8; ++j) w[j] = 0;
    for (uint32_t i = 0; i < k; ++i) {
        uint32_t r = bit_hash_range(amul[i], x, 512u - i);
        // word holding the r-th free position, and r's rank inside it: a
        // branch-free scan of the words' free counts, then one select
        uint32_t jw = 7;
        uint64_t word = w[7];
        bool found = false;
#pragma unroll
        for (int j = 0; j < 7; ++j) {
            const uint32_t z = 64u - (uint32_t)__popcll(w[j]);
            const bool here = !found && r < z;
            jw = here ? (uint32_t)j : jw;
            word = here ? w[j] : word;
            r -= (!found && !here) ? z : 0u;
            found = found || here;
        }
        const uint32_t p = 64u * jw + select_zero64(word, r);
#pragma unroll
        for (int j = 0; j < 8; ++j) w[j] |= ((p >> 6) == (uint32_t)j) ? (1ull << (p & 63)) : 0ull;
    }
}

// The group's share of the key's 512-bit mask: m[j] = word q*W + j of the
// bit set F(x), with f_i(x) = top 9 bits of a'_i x (range 512, Section 3.4).
template <int W>
__device__ __forceinline__ void key_mask(const DevFilter &f, uint64_t x, int q, uint64_t (&m)[W]) {
    if (f.bitsel) {
        uint64_t w[8];
        distinct_mask(f.a_bit, f.k, x, w);
#pragma unroll
        for (int j = 0; j < W; ++j) {
            uint64_t v = 0;
#pragma unroll
            for (int t = 0; t < 8; ++t) v = (t == q * W + j) ? w[t] : v;
            m[j] = v;
        }
        return;
    }
#pragma unroll
    for (int j = 0; j < W; ++j) m[j] = 0;
    const uint32_t first = (uint32_t)q * W;
    for (uint32_t i = 0; i < f.k; ++i) {
        uint32_t p = (uint32_t)((f.a_bit[i] * x) >> 55);
        uint32_t w = p >> 6;
        uint64_t bit = 1ull << (p & 63);
#pragma unroll
        for (int j = 0; j < W; ++j) m[j] |= (w == first + (uint32_t)j) ? bit : 0ull;
    }
}

// Bit multipliers staged in shared memory once per CTA, so that lanes can
// read a'_i with a lane-dependent i.
__device__ __forceinline__ void stage_bit_mults(const DevFilter &f, uint64_t *s_amul) {
    for (uint32_t t = threadIdx.x; t < f.k; t += blockDim.x) s_amul[t] = f.a_bit[t];
}

// u32 stride between the shared-memory mask regions of consecutive groups:
// 64 bytes, padded to 72 for one lane per key so that the lanes' 64-bit
// accesses spread over all banks.
template <int LANES>
constexpr int region_u32() { return LANES == 1 ? 18 : 16; }

// The group's share of the key's 512-bit mask, built once per group: lane q
// hashes only the bit addresses i = q, q + LANES, ... (each f_i(x) is the top
// 9 bits of a'_i x, Section 3.4) and ORs them into the group's 64-byte
// shared-memory region with 32-bit atomics; after a warp barrier each lane
// reads its W words. `region` is this group's 16 x u32 (8-byte aligned).
// Every lane of the warp must call this (it contains warp barriers).
template <int LANES>
__device__ __forceinline__ void key_mask_shared(const uint64_t *s_amul, uint32_t k, uint64_t x, int q,
                                                uint32_t *region, uint64_t (&m)[kBlockWords / LANES],
                                                uint32_t bitsel = 0) {
    constexpr int W = kBlockWords / LANES;
    uint64_t *r64 = reinterpret_cast<uint64_t *>(region);
    if (bitsel) {
        // distinct selection is sequential in i: the group's first lane builds
        // the whole mask, the others read their words
        if (q == 0) {
            uint64_t w[8];
            distinct_mask(s_amul, k, x, w);
#pragma unroll
            for (int j = 0; j < 8; ++j) r64[j] = w[j];
        }
        __syncwarp();
#pragma unroll
        for (int j = 0; j < W; ++j) m[j] = r64[q * W + j];
        __syncwarp();
        return;
    }
#pragma unroll
    for (int j = 0; j < W; ++j) r64[q * W + j] = 0;
    __syncwarp();
    for (uint32_t i = (uint32_t)q; i < k; i += LANES) {
        const uint32_t p = (uint32_t)((s_amul[i] * x) >> 55);
        atomicOr(region + (p >> 5), 1u << (p & 31));
    }
    __syncwarp();
#pragma unroll
    for (int j = 0; j < W; ++j) m[j] = r64[q * W + j];
}

// Vector loads of W words. NC: read-only path (filter not written during the
// kernel), not allocated in L1: random blocks are not reused, and keeping
// them out of L1 made the DNA query 11% faster. CG: L2-coherent path for
// kernels that read words other lanes or CTAs may have OR-ed in earlier in
// the same launch.
enum LoadPath { kLoadNC = 0, kLoadCG = 1 };

template <int W, int PATH>
__device__ __forceinline__ void load_words(const uint64_t *p, uint64_t (&v)[W]) {
    if constexpr (W == 1) {
        if constexpr (PATH == kLoadNC)
            asm volatile("ld.global.nc.L1::no_allocate.u64 %0, [%1];" : "=l"(v[0]) : "l"(p));
        else v[0] = __ldcg(reinterpret_cast<const unsigned long long *>(p));
    } else if constexpr (W == 2) {
        ulonglong2 t;
        if constexpr (PATH == kLoadNC)
            asm volatile("ld.global.nc.L1::no_allocate.v2.u64 {%0,%1}, [%2];" : "=l"(t.x), "=l"(t.y) : "l"(p));
        else t = __ldcg(reinterpret_cast<const ulonglong2 *>(p));
        v[0] = t.x; v[1] = t.y;
    } else if constexpr (W == 4) {
        if constexpr (PATH == kLoadNC)
            asm volatile("ld.global.nc.L1::no_allocate.v4.u64 {%0,%1,%2,%3}, [%4];"
                         : "=l"(v[0]), "=l"(v[1]), "=l"(v[2]), "=l"(v[3]) : "l"(p));
        else
            asm volatile("ld.global.cg.v4.u64 {%0,%1,%2,%3}, [%4];"
                         : "=l"(v[0]), "=l"(v[1]), "=l"(v[2]), "=l"(v[3]) : "l"(p));
    } else {
        static_assert(W == 8, "W must be 1, 2, 4 or 8");
        if constexpr (PATH == kLoadNC) {
            asm volatile("ld.global.nc.L1::no_allocate.v4.u64 {%0,%1,%2,%3}, [%4];"
                         : "=l"(v[0]), "=l"(v[1]), "=l"(v[2]), "=l"(v[3]) : "l"(p));
            asm volatile("ld.global.nc.L1::no_allocate.v4.u64 {%0,%1,%2,%3}, [%4];"
                         : "=l"(v[4]), "=l"(v[5]), "=l"(v[6]), "=l"(v[7]) : "l"(p + 4));
        } else {
            asm volatile("ld.global.cg.v4.u64 {%0,%1,%2,%3}, [%4];"
                         : "=l"(v[0]), "=l"(v[1]), "=l"(v[2]), "=l"(v[3]) : "l"(p));
            asm volatile("ld.global.cg.v4.u64 {%0,%1,%2,%3}, [%4];"
                         : "=l"(v[4]), "=l"(v[5]), "=l"(v[6]), "=l"(v[7]) : "l"(p + 4));
        }
    }
}

// Streaming read of a key (read once: evict-first in L2, no L1 allocation).
__device__ __forceinline__ uint64_t load_key(const uint64_t *p) {
    return __ldcs(reinterpret_cast<const unsigned long long *>(p));
}

// 64-bit OR at L2 as a reduction that returns nothing: the set phases never
// read the old value. Through atomicOr, ncu counted these as returning
// atomics (no reductions) and the DNA insert took 4.33 ms against 3.74.
__device__ __forceinline__ void red_or(unsigned long long *p, unsigned long long v) {
    asm volatile("red.relaxed.gpu.global.or.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Sum of v over the LANES lanes of this lane's group (butterfly).
template <int LANES>
__device__ __forceinline__ uint32_t group_sum(uint32_t v) {
#pragma unroll
    for (int s = LANES / 2; s > 0; s >>= 1) v += __shfl_xor_sync(0xffffffffu, v, s, LANES);
    return v;
}

// Per-candidate terms of the cost: L = popcount(block) and
// a = popcount(F(x) & ~block), packed as L | a << 16 and summed over the group.
template <int W>
__device__ __forceinline__ uint32_t load_and_new(const uint64_t (&blk)[W], const uint64_t (&m)[W]) {
    uint32_t L = 0, a = 0;
#pragma unroll
    for (int j = 0; j < W; ++j) {
        L += __popcll(blk[j]);
        a += __popcll(m[j] & ~blk[j]);
    }
    return L | (a << 16);
}

// Choice among C candidates from their (L, a) terms: kSkip if one of them
// already holds F(x) (a == 0); otherwise the index of least rank[L][a],
// lowest index on ties (Section 3.2). rank has (k+1) entries per load L.
template <int C>
__device__ __forceinline__ uint32_t choose_from_terms(const uint32_t (&la)[C], const uint16_t *rank,
                                                      uint32_t k1) {
    bool skip = false;
#pragma unroll
    for (int i = 0; i < C; ++i) skip |= ((la[i] >> 16) == 0);
    if (skip) return kSkip;
    if constexpr (C == 1) {
        return 0;
    } else {
        uint32_t best = 0xFFFFFFFFu;
#pragma unroll
        for (int i = 0; i < C; ++i) {
            uint32_t L = la[i] & 0xFFFFu, a = la[i] >> 16;
            uint32_t key = ((uint32_t)rank[L * k1 + a] << 2) | (uint32_t)i;
            best = key < best ? key : best;
        }
        return best & 3u;
    }
}

}  // namespace bc
