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

// Shared-memory area in which a warp builds its keys' masks: 512 / LANES
// u32 per warp, 64 bytes per lane group. Two layouts, by group width:
//  - one lane per key (W = 8): word-major interleaved, mask word j of lane l
//    at 64-bit index j * 32 + l. A bit OR of lane l lands in bank 2 l or
//    2 l + 1 (two lanes per bank pair), and each readback instruction reads
//    256 contiguous bytes;
//  - wider groups: group g's mask is u32 16 g .. 16 g + 15 in block word
//    order (64 contiguous bytes, which the bulk set of the persistent insert
//    sends to global memory as one piece), with the cheapest bit address
//    (one shift). Measured on the DNA insert, this beat both an interleaved
//    and a swizzled layout with conflict-free readback (3.73 ms against 3.90
//    and 3.82): the extra index arithmetic cost more than the conflicts.
template <int LANES>
constexpr int mask_u32_per_warp() { return 512 / LANES; }

// The warp's mask area inside s_mask (mask_u32_per_warp u32 per warp of the
// CTA), zeroed. Warp-collective; called once per warp before the first mask.
template <int LANES>
__device__ __forceinline__ uint32_t *warp_mask_area(uint32_t *s_mask, int warp_in_block) {
    uint32_t *area = s_mask + warp_in_block * mask_u32_per_warp<LANES>();
    uint64_t *r64 = reinterpret_cast<uint64_t *>(area);
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int j = 0; j < kBlockWords / LANES; ++j) r64[j * 32 + lane] = 0ull;
    __syncwarp();
    return area;
}

__device__ __forceinline__ void red_or_shared(uint32_t *p, uint32_t v) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("red.shared.or.b32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}

// Reads a shared 64-bit word and leaves 0 in its place (one exchange).
__device__ __forceinline__ uint64_t take_shared(uint64_t *p) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    uint64_t v;
    asm volatile("atom.shared.exch.b64 %0, [%1], %2;" : "=l"(v) : "r"(a), "l"(0ull) : "memory");
    return v;
}

// Builds the key's 512-bit mask F(x) into a group's 64 contiguous bytes
// `slot` (block word order), which the caller has zeroed: lane q hashes the
// bit addresses i = q, q + LANES, ... (each f_i(x) is the top 9 bits of
// a'_i x, Section 3.4) and ORs each bit into its 32-bit word. With distinct
// selection the group's first lane stores the whole mask. No barrier inside.
template <int LANES>
__device__ __forceinline__ void mask_into_slot(const uint64_t *s_amul, uint32_t k, uint64_t x, int q,
                                               uint32_t *slot, uint32_t bitsel) {
    if (bitsel) {
        if (q == 0) {
            uint64_t w[8];
            distinct_mask(s_amul, k, x, w);
            uint64_t *s64 = reinterpret_cast<uint64_t *>(slot);
#pragma unroll
            for (int t = 0; t < 8; ++t) s64[t] = w[t];
        }
        return;
    }
    for (uint32_t i = (uint32_t)q; i < k; i += LANES) {
        const uint32_t p = (uint32_t)((s_amul[i] * x) >> 55);
        red_or_shared(slot + (p >> 5), 1u << (p & 31));
    }
}

// The group's share of the key's 512-bit mask, built once per group: m[j] is
// mask word q W + j. `area` is the warp's mask area (warp_mask_area). Every
// lane of the warp must call this (it contains warp barriers).
template <int LANES>
__device__ __forceinline__ void key_mask_shared(const uint64_t *s_amul, uint32_t k, uint64_t x, int q,
                                                uint32_t *area, uint64_t (&m)[kBlockWords / LANES],
                                                uint32_t bitsel = 0) {
    constexpr int W = kBlockWords / LANES;
    uint64_t *r64 = reinterpret_cast<uint64_t *>(area);
    const int lane = threadIdx.x & 31;
    if constexpr (LANES == 1) {
        // interleaved; the area is zero between calls (the readback takes
        // the words and leaves zeros)
        __syncwarp();  // every lane has taken the previous key's words
        if (bitsel) {
            uint64_t w[8];
            distinct_mask(s_amul, k, x, w);
#pragma unroll
            for (int j = 0; j < 8; ++j) m[j] = w[j];
            return;
        }
        for (uint32_t i = 0; i < k; ++i) {
            const uint32_t p = (uint32_t)((s_amul[i] * x) >> 55);
            red_or_shared(area + 2u * ((p >> 6) * 32u + (uint32_t)lane) + ((p >> 5) & 1u), 1u << (p & 31));
        }
        __syncwarp();
#pragma unroll
        for (int j = 0; j < W; ++j) m[j] = take_shared(r64 + j * 32 + lane);
    } else {
        const int g = lane / LANES;
        uint32_t *slot = area + 16 * g;
        uint64_t *s64 = reinterpret_cast<uint64_t *>(slot);
#pragma unroll
        for (int j = 0; j < W; ++j) s64[q * W + j] = 0;
        __syncwarp();
        mask_into_slot<LANES>(s_amul, k, x, q, slot, bitsel);
        __syncwarp();
#pragma unroll
        for (int j = 0; j < W; ++j) m[j] = s64[q * W + j];
        // the next key's ORs wait at its first warp barrier, which this lane
        // reaches only after reading its words
    }
}

// ---- Bulk (TMA) OR of a whole 64-byte block ---------------------------------
// The set phase can send a key's mask, staged in shared memory in block word
// order, to its block as one asynchronous bulk reduction
// (cp.reduce.async.bulk ... .or.b64), instead of one 64-bit red per word.

// Makes this thread's (and, after a warp barrier, the warp's) generic-proxy
// shared-memory writes visible to the bulk copy engine.
__device__ __forceinline__ void fence_proxy_async_shared() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// Orders completed bulk writes to global memory before this thread's later
// generic accesses.
__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}
// *gdst |= slot[0 .. 64 bytes), as 64-bit ORs at L2. gdst and slot 16-byte aligned.
__device__ __forceinline__ void bulk_or_block(uint64_t *gdst, const uint32_t *slot) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(slot);
    asm volatile("cp.reduce.async.bulk.global.shared::cta.bulk_group.or.b64 [%0], [%1], 64;"
                 ::"l"(gdst), "r"(a) : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// Waits until at most N of this thread's bulk groups still read their source.
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
    asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}
// Waits until all of this thread's bulk groups have completed.
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// ---- Bulk copies of whole ranges between global and shared memory ---------
// A CTA-local mbarrier counts the bytes of a global-to-shared bulk copy.
__device__ __forceinline__ void mbar_init(uint64_t *mbar, uint32_t arrivals) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(mbar);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(arrivals) : "memory");
}
// Arrives on mbar and expects `bytes` more transaction bytes in this phase.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *mbar, uint32_t bytes) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(mbar);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *mbar, uint32_t parity) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(mbar);
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok) : "r"(a), "r"(parity) : "memory");
    return ok != 0;
}
// Waits for phase `parity` of mbar to complete, at most `limit` SM clock
// cycles; false if the wait gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t *mbar, uint32_t parity, long long limit) {
    const long long t0 = clock64();
    while (!mbar_try_wait(mbar, parity))
        if (clock64() - t0 > limit) return false;
    return true;
}
// sdst[0 .. bytes) = gsrc[0 .. bytes), completing `bytes` transactions on mbar.
// Both 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_load(void *sdst, const void *gsrc, uint32_t bytes, uint64_t *mbar) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(sdst);
    const unsigned m = (unsigned)__cvta_generic_to_shared(mbar);
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(d), "l"(gsrc), "r"(bytes), "r"(m) : "memory");
}
// gdst[0 .. bytes) = ssrc[0 .. bytes) as one bulk group entry.
__device__ __forceinline__ void bulk_store(void *gdst, const void *ssrc, uint32_t bytes) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(ssrc);
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(gdst), "r"(a), "r"(bytes)
                 : "memory");
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
