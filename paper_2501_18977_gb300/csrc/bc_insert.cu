// Insertion kernels of the BlowChoc filter (Section 3.2, Fig. 2B).
//
// Batch rule: the keys of one batch all decide against the filter as it is
// when the batch starts, and the batch's bits are OR-ed in afterwards. The
// result is therefore independent of the order of keys inside a batch and of
// the launch configuration; B = 1 is the paper's one-key-at-a-time insertion.
#include "bc_launch.h"
#include "bc_phases.cuh"

namespace bc {
namespace {

constexpr int kThreads = 256;  // CTA size of the grid-wide insert kernels

// Phase 1 of a batch: every key's choice against the unchanged filter.
template <int C, int LANES>
__global__ void __launch_bounds__(kThreads) choose_kernel(DevFilter f, const uint64_t *__restrict__ keys,
                                                          uint64_t n, const uint16_t *__restrict__ rank_g,
                                                          uint8_t *__restrict__ sel,
                                                          unsigned long long *counters) {
    constexpr int G = 32 / LANES;
    constexpr int W = kBlockWords / LANES;
    extern __shared__ uint16_t s_rank[];
    __shared__ uint64_t s_amul[32];
    __shared__ __align__(16) uint32_t s_mask[(kThreads / 32) * mask_u32_per_warp<LANES>()];
    stage_bit_mults(f, s_amul);
    const uint16_t *rank = stage_rank<C>(rank_g, s_rank, f.k + 1);
    if constexpr (C == 1) __syncthreads();
    const int lane = threadIdx.x & 31, q = lane % LANES, g = lane / LANES;
    uint32_t *region = warp_mask_area<LANES>(s_mask, threadIdx.x >> 5);
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    uint32_t ins = 0, skp = 0;
    for (uint64_t base = warp * G; base < n; base += nwarps * G) {
        const uint64_t i = base + g;
        const bool valid = i < n;
        const uint64_t x = valid ? load_key(keys + i) : 0ull;
        uint64_t m[W];
        const uint32_t s = choose_key<C, LANES, kLoadNC>(f, x, valid, q, rank, s_amul, region, m);
        if (valid && q == 0) {
            sel[i] = (uint8_t)s;
            if (s == kSkip) ++skp; else ++ins;
        }
    }
    flush_counts(ins, skp, counters);
}

// Phase 2 of a batch: OR every non-skipped key into its chosen block.
template <int LANES>
__global__ void __launch_bounds__(kThreads) set_kernel(DevFilter f, const uint64_t *__restrict__ keys,
                                                       uint64_t n, const uint8_t *__restrict__ sel) {
    constexpr int G = 32 / LANES;
    constexpr int W = kBlockWords / LANES;
    __shared__ uint64_t s_amul[32];
    __shared__ __align__(16) uint32_t s_mask[(kThreads / 32) * mask_u32_per_warp<LANES>()];
    stage_bit_mults(f, s_amul);
    __syncthreads();
    const int lane = threadIdx.x & 31, q = lane % LANES, g = lane / LANES;
    uint32_t *region = warp_mask_area<LANES>(s_mask, threadIdx.x >> 5);
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t base = warp * G; base < n; base += nwarps * G) {
        const uint64_t i = base + g;
        // the key is loaded beside the choice, not after it
        const uint32_t s = i < n ? (uint32_t)sel[i] : kSkip;
        const uint64_t x = i < n ? load_key(keys + i) : 0ull;
        uint64_t m[W];
        key_mask_shared<LANES>(s_amul, f.k, x, q, region, m, f.bitsel);
        if (s != kSkip) set_one<LANES>(f, block_addr(f, block_mult(f, s), x), q, m);
    }
}

// B = 1 in one warp. Lane 8i + j handles word j of candidate i (i < C); keys
// are prefetched 32 at a time and broadcast. A key's update is visible to the
// next key's loads through __syncwarp (the warp is the only writer).
template <int C>
__global__ void __launch_bounds__(32) sequential_kernel(DevFilter f, const uint64_t *__restrict__ keys,
                                                        uint64_t n, const uint16_t *__restrict__ rank_g,
                                                        unsigned long long *counters) {
    extern __shared__ uint16_t s_rank[];
    const uint16_t *rank = stage_rank<C>(rank_g, s_rank, f.k + 1);
    const int lane = threadIdx.x;
    const int i = lane >> 3, j = lane & 7;
    const bool active = i < C;
    uint64_t ins = 0, skp = 0;
    for (uint64_t base = 0; base < n; base += 32) {
        const uint64_t mine = base + lane < n ? load_key(keys + base + lane) : 0ull;
        const int cnt = (int)((n - base) < 32 ? (n - base) : 32);
        for (int t = 0; t < cnt; ++t) {
            const uint64_t x = __shfl_sync(kFull, mine, t);
            uint64_t m[1];
            key_mask<1>(f, x, j, m);
            const uint64_t b = active ? block_addr(f, block_mult(f, (uint32_t)i), x) : 0ull;
            unsigned long long *wp = reinterpret_cast<unsigned long long *>(f.words + b * kBlockWords + j);
            const uint64_t w = active ? __ldcg(wp) : ~0ull;
            const uint32_t v = group_sum<8>((uint32_t)__popcll(w) | ((uint32_t)__popcll(m[0] & ~w) << 16));
            uint32_t la[C];
#pragma unroll
            for (int ii = 0; ii < C; ++ii) la[ii] = __shfl_sync(kFull, v, 8 * ii);
            const uint32_t s = choose_from_terms<C>(la, rank, f.k + 1);
            if (s == kSkip) {
                ++skp;
            } else {
                ++ins;
                if (active && (uint32_t)i == s && (m[0] & ~w)) *wp = w | m[0];
            }
            __syncwarp();
        }
    }
    if (lane == 0) {
        atomicAdd(&counters[0], (unsigned long long)ins);
        atomicAdd(&counters[1], (unsigned long long)skp);
    }
}

// 1 < B <= kSmallBatchMax: one CTA of kSmallThreads, CTA barriers between the
// two phases of every batch; choices live in shared memory. Block loads take
// the L2 path because earlier batches of this launch have written the filter.
constexpr int kSmallThreads = 1024;

template <int LANES>
constexpr size_t small_mask_bytes() { return (kSmallThreads / 32) * mask_u32_per_warp<LANES>() * 4; }

// BITSEL and POW2 as in the persistent kernel.
template <int C, int LANES, bool BITSEL, bool POW2>
__global__ void __launch_bounds__(kSmallThreads) small_batch_kernel(const DevFilter fp,
                                                                    const uint64_t *__restrict__ keys,
                                                                    uint64_t n, uint64_t B,
                                                                    const uint16_t *__restrict__ rank_g,
                                                                    unsigned long long *counters) {
    DevFilter f = fp;
    if constexpr (!BITSEL) f.bitsel = 0;
    if constexpr (POW2) f.range_kind = kRangePow2;
    constexpr int G = 32 / LANES;
    constexpr int W = kBlockWords / LANES;
    extern __shared__ __align__(16) uint8_t s_dyn[];
    __shared__ uint64_t s_amul[32];
    uint32_t *s_mask = reinterpret_cast<uint32_t *>(s_dyn);
    uint8_t *sel = s_dyn + small_mask_bytes<LANES>();
    uint16_t *s_rank = reinterpret_cast<uint16_t *>(sel + kSmallBatchMax);
    stage_bit_mults(fp, s_amul);
    const uint16_t *rank = stage_rank<C>(rank_g, s_rank, f.k + 1);
    if constexpr (C == 1) __syncthreads();
    const int lane = threadIdx.x & 31, q = lane % LANES, g = lane / LANES;
    uint32_t *region = warp_mask_area<LANES>(s_mask, threadIdx.x >> 5);
    const uint32_t warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    uint32_t ins = 0, skp = 0;
    for (uint64_t s0 = 0; s0 < n; s0 += B) {
        const uint32_t cnt = (uint32_t)((n - s0) < B ? (n - s0) : B);
        for (uint32_t base = warp * G; base < cnt; base += nwarps * G) {
            const uint32_t i = base + g;
            const bool valid = i < cnt;
            const uint64_t x = valid ? load_key(keys + s0 + i) : 0ull;
            uint64_t m[W];
            const uint32_t s = choose_key<C, LANES, kLoadCG>(f, x, valid, q, rank, s_amul, region, m);
            if (valid && q == 0) {
                sel[i] = (uint8_t)s;
                if (s == kSkip) ++skp; else ++ins;
            }
        }
        __syncthreads();
        for (uint32_t base = warp * G; base < cnt; base += nwarps * G) {
            const uint32_t i = base + g;
            const uint32_t s = i < cnt ? (uint32_t)sel[i] : kSkip;
            const uint64_t x = i < cnt ? load_key(keys + s0 + i) : 0ull;
            uint64_t m[W];
            key_mask_shared<LANES>(s_amul, f.k, x, q, region, m, f.bitsel);
            if (s != kSkip) set_one<LANES>(f, block_addr(f, block_mult(f, s), x), q, m);
        }
        __syncthreads();
    }
    flush_counts(ins, skp, counters);
}

// ---------------------------------------------------------------------------
// Persistent insertion: one cooperative launch runs every batch. Between the
// choose phase and the set phase of a batch, and between batches, the whole
// grid meets at a barrier, which gives exactly the batch rule above.

// Registers per thread: one lane per key keeps three whole candidate blocks
// in registers (128; two 256-thread CTAs per SM). Wider groups are held to 64
// registers so that 32 warps fit per SM, which measured 13% faster on an
// L2-sized filter than letting them take 95 registers. They run as two
// 512-thread CTAs per SM: against four of 256 threads, half as many CTAs
// meet at each grid barrier, and the DNA insert measured 1-3% faster and a
// 2 MiB filter's 8% (1024-thread CTAs: 4% faster with four lanes, 3% slower
// with two).
template <int LANES>
constexpr int persistent_threads() { return LANES == 1 ? 256 : 512; }
template <int LANES>
constexpr int persistent_min_ctas() { return LANES == 1 ? 2 : 1024 / persistent_threads<LANES>(); }

// Bulk set (set_mode 2): the set phase stages each key's mask in a 64-byte
// slot and ORs it into the chosen block with one bulk reduction (the copy
// engine's cp.reduce.async.bulk) instead of a 64-bit red per word. A lane
// group cycles through kBulkRing slots, so a slot is rewritten only after
// the reduction issued kBulkRing keys earlier has read it. It pays from about
// the L2 size on (the default rule and its measurements are in
// blowchoc_create); smaller filters keep the 64-bit reds.
constexpr int kBulkRing = 4;
template <int LANES>
constexpr size_t bulk_ring_bytes() {
    return (size_t)(persistent_threads<LANES>() / LANES) * kBulkRing * 64;
}
// Offset of the slot ring in the dynamic shared memory, after the rank table.
__host__ __device__ inline size_t bulk_ring_offset(int C, uint32_t k) {
    return ((C > 1 ? 513u * (k + 1) * 2u : 0u) + 127u) & ~(size_t)127;
}

// BITSEL: the filter uses distinct bit selection; POW2: its block count is a
// power of two (block addresses are the top bits of a x). Each false instance
// compiles the other paths out: inlined as runtime branches they cost
// registers (the DNA insert spilled 72 bytes with the distinct path, none
// without) and time (DNA insert 3.70 -> 3.67 ms without the distinct path,
// -> 3.63 ms with the power-of-two addressing alone).
template <int C, int LANES, bool BULK, bool BITSEL, bool POW2>
__global__ void __launch_bounds__(persistent_threads<LANES>(), persistent_min_ctas<LANES>()) persistent_insert_kernel(
    const DevFilter fp, const uint64_t *__restrict__ keys, uint64_t n, uint64_t B,
    const uint16_t *__restrict__ rank_g, uint8_t *sel, unsigned long long *counters,
    unsigned int *bar) {
    // constants from here on: the paths this instance does not take fold away.
    // The bit multipliers are staged from the parameter itself: read with a
    // thread-dependent index through the modified copy, they made the compiler
    // keep the whole copy (328 bytes) in local memory and read every field there.
    DevFilter f = fp;
    if constexpr (!BITSEL) f.bitsel = 0;
    if constexpr (POW2) f.range_kind = kRangePow2;
    constexpr int G = 32 / LANES;
    constexpr int W = kBlockWords / LANES;
    extern __shared__ __align__(16) uint8_t s_dyn[];  // rank table | bulk slot ring (16-byte aligned slots)
    uint16_t *s_rank = reinterpret_cast<uint16_t *>(s_dyn);
    __shared__ uint64_t s_amul[32];
    __shared__ __align__(16) uint32_t s_mask[(persistent_threads<LANES>() / 32) * mask_u32_per_warp<LANES>()];
    stage_bit_mults(fp, s_amul);
    const uint16_t *rank = stage_rank<C>(rank_g, s_rank, f.k + 1);
    if constexpr (C == 1) __syncthreads();
    const int lane = threadIdx.x & 31, q = lane % LANES, g = lane / LANES;
    uint32_t *region = warp_mask_area<LANES>(s_mask, threadIdx.x >> 5);
    uint32_t *ring = reinterpret_cast<uint32_t *>(s_dyn + bulk_ring_offset(C, f.k)) +
                     (size_t)(threadIdx.x / LANES) * (kBulkRing * 16);  // used with BULK only
    uint32_t slot_i = 0;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    uint16_t *sel16 = reinterpret_cast<uint16_t *>(sel);  // choice | words with new bits << 8
    unsigned long long *err = counters + 2;
    unsigned int target = 0;
    uint32_t ins = 0, skp = 0;
    // Each lane group handles the same keys of a batch in both phases, so the
    // loads that start a phase (the batch's first key; the set phase's first
    // key and the choice this warp stored) need nothing from other CTAs: they
    // are issued before the grid barrier and arrive during its wait (measured
    // 0.4% faster on the DNA insert).
    uint64_t xfirst = warp * G + g < (n < B ? n : B) ? load_key(keys + warp * G + g) : 0ull;
    for (uint64_t s0 = 0; s0 < n; s0 += B) {
        const uint64_t cnt = (n - s0) < B ? (n - s0) : B;
        const uint64_t stride = nwarps * G;
        // the next step's key is loaded one step ahead
        uint64_t xn = xfirst;
        for (uint64_t base = warp * G; base < cnt; base += stride) {
            const uint64_t i = base + g;
            const bool valid = i < cnt;
            const uint64_t x = xn;
            xn = i + stride < cnt ? load_key(keys + s0 + i + stride) : 0ull;
            uint64_t m[W];
            // with 1 or 2 lanes per key, only words with new bits are OR-ed in
            // later (measured 1.4-4% faster); wider groups OR every word, which
            // measured faster for them (the flags cost registers)
            uint32_t words = 0xFFu;
            uint32_t s;
            if constexpr (LANES <= 2 && !BULK)
                s = choose_key_words<C, LANES, kLoadCG>(f, x, valid, q, rank, s_amul, region, m, words);
            else
                s = choose_key<C, LANES, kLoadCG>(f, x, valid, q, rank, s_amul, region, m);
            if (valid && q == 0) {
                sel16[i] = (uint16_t)(s | (words << 8));
                if (s == kSkip) ++skp; else ++ins;
            }
        }
        // the choice (stored by lane q = 0 of this group; read through L2 after
        // a warp barrier) and the key are loaded one step ahead
        __syncwarp();
        uint32_t swn = warp * G + g < cnt ? (uint32_t)__ldcg(sel16 + warp * G + g) : kSkip;
        uint64_t xs = warp * G + g < cnt ? load_key(keys + s0 + warp * G + g) : 0ull;
        target += gridDim.x;
        if (!grid_barrier(bar, target, err)) return;
        for (uint64_t base = warp * G; base < cnt; base += stride) {
            const uint64_t i = base + g;
            const uint32_t sw = swn;
            const uint64_t x = xs;
            swn = i + stride < cnt ? (uint32_t)__ldcg(sel16 + i + stride) : kSkip;
            xs = i + stride < cnt ? load_key(keys + s0 + i + stride) : 0ull;
            const uint32_t s = sw & 0xFFu;
            if constexpr (BULK) {
                // the group's next slot, free once the reduction that last
                // read it has (the group's first lane issued and waits for those)
                uint32_t *slot = ring + (slot_i % kBulkRing) * 16;
                ++slot_i;
                if (q == 0) bulk_wait_read<kBulkRing - 1>();
                __syncwarp();
                uint64_t *s64 = reinterpret_cast<uint64_t *>(slot);
#pragma unroll
                for (int j = 0; j < W; ++j) s64[q * W + j] = 0ull;
                __syncwarp();
                mask_into_slot<LANES>(s_amul, f.k, x, q, slot, f.bitsel);
                fence_proxy_async_shared();
                __syncwarp();
                if (q == 0) {
                    if (s != kSkip) bulk_or_block(f.words + block_addr(f, block_mult(f, s), x) * kBlockWords, slot);
                    bulk_commit();
                }
            } else {
                uint64_t m[W];
                key_mask_shared<LANES>(s_amul, f.k, x, q, region, m, f.bitsel);
                if (s != kSkip) set_words<LANES>(f, block_addr(f, block_mult(f, s), x), q, m, sw >> 8);
            }
        }
        if constexpr (BULK) {
            // every reduction of this batch has reached global memory before
            // the barrier that lets the next batch choose
            if (q == 0) bulk_wait_all();
            fence_proxy_async_global();
        }
        if (s0 + B < n) {
            const uint64_t cn = (n - s0 - B) < B ? (n - s0 - B) : B;
            xfirst = warp * G + g < cn ? load_key(keys + s0 + B + warp * G + g) : 0ull;
            target += gridDim.x;
            if (!grid_barrier(bar, target, err)) return;
        }
    }
    flush_counts(ins, skp, counters);
}

// ---------------------------------------------------------------------------
// Sort-by-block set variant. After the choose phase of a batch, the chosen
// blocks are bucketed by range of kRangeBlocks blocks (count, scan, scatter);
// then each CTA takes whole ranges, stages the range's words in shared memory
// with one bulk copy (cp.async.bulk, completion counted on an mbarrier), ORs
// the masks of the range's keys in with shared atomics and writes the range
// back with one bulk copy: no global atomics on the filter, one read and one
// write per touched range. Measured on one GB300 over filters of 1 to 512 MiB
// and 1/16 to 32 keys per block and batch, it never beat the direct or bulk
// set (1.4 to 10 times slower); the bulk copies made it up to 28% faster than
// staging with plain loads and stores.

template <int C, int LANES>
__global__ void __launch_bounds__(kThreads) sorted_insert_kernel(
    DevFilter f, const uint64_t *__restrict__ keys, uint64_t n, uint64_t B,
    const uint16_t *__restrict__ rank_g, uint8_t *sel, unsigned long long *counters, unsigned int *bar,
    uint32_t *cnt, uint32_t *cur, uint32_t *off, uint32_t *perm, uint32_t R) {
    constexpr int G = 32 / LANES;
    constexpr int W = kBlockWords / LANES;
    extern __shared__ __align__(16) uint8_t s_dyn[];
    uint64_t *s_range = reinterpret_cast<uint64_t *>(s_dyn);            // kRangeBlocks x 8 words
    uint32_t *s_range32 = reinterpret_cast<uint32_t *>(s_dyn);
    uint16_t *s_rank = reinterpret_cast<uint16_t *>(s_dyn + kRangeBlocks * 64);
    __shared__ uint64_t s_amul[32];
    __shared__ __align__(16) uint32_t s_mask[(kThreads / 32) * mask_u32_per_warp<LANES>()];
    __shared__ uint32_t s_part[kThreads];
    __shared__ uint64_t s_mbar;
    uint32_t phase = 0;
    if (threadIdx.x == 0) {
        mbar_init(&s_mbar, 1);
        fence_proxy_async_shared();
    }
    __syncthreads();
    stage_bit_mults(f, s_amul);
    const uint16_t *rank = stage_rank<C>(rank_g, s_rank, f.k + 1);
    if constexpr (C == 1) __syncthreads();
    const int lane = threadIdx.x & 31, q = lane % LANES, g = lane / LANES;
    const int wib = threadIdx.x >> 5, wpc = blockDim.x >> 5;
    uint32_t *region = warp_mask_area<LANES>(s_mask, wib);
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t nthreads = (uint64_t)gridDim.x * blockDim.x;
    unsigned long long *err = counters + 2;
    unsigned int target = 0;
    uint32_t ins = 0, skp = 0;
    for (uint64_t s0 = 0; s0 < n; s0 += B) {
        const uint64_t cnt_b = (n - s0) < B ? (n - s0) : B;
        const uint64_t *bk = keys + s0;
        // choose against the filter as the batch starts
        for (uint64_t base = warp * G; base < cnt_b; base += nwarps * G) {
            const uint64_t i = base + g;
            const bool valid = i < cnt_b;
            const uint64_t x = valid ? load_key(bk + i) : 0ull;
            uint64_t m[W];
            const uint32_t s = choose_key<C, LANES, kLoadCG>(f, x, valid, q, rank, s_amul, region, m);
            if (valid && q == 0) {
                sel[i] = (uint8_t)s;
                if (s == kSkip) ++skp; else ++ins;
            }
        }
        target += gridDim.x;
        if (!grid_barrier(bar, target, err)) return;
        // count keys per range
        for (uint64_t i = tid; i < cnt_b; i += nthreads) {
            const uint32_t s = __ldcg(sel + i);
            const uint64_t x = load_key(bk + i);
            if (s == kSkip) continue;
            atomicAdd(cnt + (uint32_t)(block_addr(f, block_mult(f, s), x) / kRangeBlocks), 1u);
        }
        target += gridDim.x;
        if (!grid_barrier(bar, target, err)) return;
        // exclusive scan of the counts (one CTA: each thread sums a run of
        // ranges, a shuffle scan over the threads' sums), cursors to zero
        if (blockIdx.x == 0) {
            const uint32_t per = (R + blockDim.x - 1) / blockDim.x;
            const uint32_t lo = threadIdx.x * per, hi = lo + per < R ? lo + per : R;
            uint32_t sum = 0;
            for (uint32_t r = lo; r < hi; ++r) sum += __ldcg(cnt + r);
            uint32_t v = sum;  // inclusive scan within the warp
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t u = __shfl_up_sync(kFull, v, d);
                if (lane >= d) v += u;
            }
            if (lane == 31) s_part[wib] = v;
            __syncthreads();
            if (wib == 0) {
                uint32_t t = lane < wpc ? s_part[lane] : 0u;
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const uint32_t u = __shfl_up_sync(kFull, t, d);
                    if (lane >= d) t += u;
                }
                if (lane < wpc) s_part[lane] = t;  // inclusive over warps
                if (lane == wpc - 1) off[R] = t;
            }
            __syncthreads();
            uint32_t acc = v - sum + (wib ? s_part[wib - 1] : 0u);
            for (uint32_t r = lo; r < hi; ++r) {
                off[r] = acc;
                acc += __ldcg(cnt + r);
                cur[r] = 0;
            }
        }
        target += gridDim.x;
        if (!grid_barrier(bar, target, err)) return;
        // scatter key indices into their ranges
        for (uint64_t i = tid; i < cnt_b; i += nthreads) {
            const uint32_t s = __ldcg(sel + i);
            const uint64_t x = load_key(bk + i);
            if (s == kSkip) continue;
            const uint32_t r = (uint32_t)(block_addr(f, block_mult(f, s), x) / kRangeBlocks);
            perm[__ldcg(off + r) + atomicAdd(cur + r, 1u)] = (uint32_t)i;
        }
        target += gridDim.x;
        if (!grid_barrier(bar, target, err)) return;
        // apply: one range at a time per CTA, staged in shared memory
        for (uint32_t r = blockIdx.x; r < R; r += gridDim.x) {
            const uint32_t c0 = __ldcg(off + r), c1 = __ldcg(off + r + 1);
            if (threadIdx.x == 0) cnt[r] = 0;  // ready for the next batch
            if (c0 == c1) continue;
            const uint64_t first = (uint64_t)r * kRangeBlocks;
            const uint64_t nb = f.M - first < kRangeBlocks ? f.M - first : kRangeBlocks;
            const uint64_t *src = f.words + first * kBlockWords;
            // one bulk copy of the range (after the previous range's write-back
            // has read the staging area), counted on the CTA's mbarrier
            if (threadIdx.x == 0) {
                bulk_wait_read<0>();
                mbar_arrive_expect_tx(&s_mbar, (uint32_t)(nb * 64));
                bulk_load(s_range, src, (uint32_t)(nb * 64), &s_mbar);
            }
            if (!mbar_wait(&s_mbar, phase, kBarrierCycles)) {
                atomicExch(err, 1ull);
                mbar_wait(&s_mbar, phase, kBarrierCycles);  // the copy in flight, bounded again
                return;
            }
            phase ^= 1u;
            __syncthreads();
            for (uint32_t base = c0 + wib * G; base < c1; base += wpc * G) {
                const uint32_t idx = base + g;
                const bool valid = idx < c1;
                const uint32_t i = valid ? __ldcg(perm + idx) : 0u;
                const uint32_t s = valid ? (uint32_t)__ldcg(sel + i) : kSkip;
                const uint64_t x = valid ? load_key(bk + i) : 0ull;
                uint64_t m[W];
                key_mask_shared<LANES>(s_amul, f.k, x, q, region, m, f.bitsel);
                if (valid) {
                    const uint64_t local = block_addr(f, block_mult(f, s), x) - first;
                    uint32_t *dst = s_range32 + (local * kBlockWords + (uint64_t)q * W) * 2;
#pragma unroll
                    for (int j = 0; j < W; ++j) {
                        if ((uint32_t)m[j]) atomicOr(dst + 2 * j, (uint32_t)m[j]);
                        if ((uint32_t)(m[j] >> 32)) atomicOr(dst + 2 * j + 1, (uint32_t)(m[j] >> 32));
                    }
                }
            }
            __syncthreads();
            uint64_t *dst = f.words + first * kBlockWords;
            fence_proxy_async_shared();  // every thread's ORs, visible to the bulk copy
            __syncthreads();
            if (threadIdx.x == 0) {
                bulk_store(dst, s_range, (uint32_t)(nb * 64));
                bulk_commit();
            }
        }
        if (threadIdx.x == 0) bulk_wait_all();  // the batch's ranges are written
        fence_proxy_async_global();
        if (s0 + B < n) {
            target += gridDim.x;
            if (!grid_barrier(bar, target, err)) return;
        }
    }
    flush_counts(ins, skp, counters);
}

// ---------------------------------------------------------------------------
// One-key-at-a-time insertion (B = 1, the paper's order) in parallel, exactly.
// Keys are taken in windows; in each round every pending key of the window
// reserves its candidate blocks with a 64-bit atomic max of
// (round << 32 | ~index), so the earliest pending key wins each block. A key
// that holds all of its own reservations has no earlier pending key sharing a
// candidate block with it: it decides against the current filter and sets its
// bits. Keys that commit in the same round touch disjoint blocks, so the
// outcome is that of inserting the keys one after another.

constexpr int kSeqThreads = 1024;

// BITSEL and POW2 as in the persistent kernel: the instance for a filter
// without distinct selection, or with a power-of-two block count, has the
// other paths compiled out.
template <int C, int LANES, bool BITSEL, bool POW2>
__global__ void __launch_bounds__(kSeqThreads) exact_sequential_kernel(
    const DevFilter fp, const uint64_t *__restrict__ keys, uint64_t n, uint32_t window,
    const uint16_t *__restrict__ rank_g, unsigned long long *counters, unsigned long long *resv) {
    DevFilter f = fp;
    if constexpr (!BITSEL) f.bitsel = 0;
    if constexpr (POW2) f.range_kind = kRangePow2;
    constexpr int G = 32 / LANES;
    constexpr int W = kBlockWords / LANES;
    extern __shared__ __align__(16) uint8_t s_dyn[];
    uint64_t *s_key = reinterpret_cast<uint64_t *>(s_dyn);                  // window keys
    uint8_t *s_state = s_dyn + (size_t)window * 8;                           // 1 = pending
    uint16_t *s_rank = reinterpret_cast<uint16_t *>(s_state + ((window + 15) & ~15u));
    __shared__ uint64_t s_amul[32];
    __shared__ __align__(16) uint32_t s_mask[(kSeqThreads / 32) * mask_u32_per_warp<LANES>()];
    __shared__ int s_left;
    stage_bit_mults(fp, s_amul);
    const uint16_t *rank = stage_rank<C>(rank_g, s_rank, f.k + 1);
    if constexpr (C == 1) __syncthreads();
    const int lane = threadIdx.x & 31, q = lane % LANES, g = lane / LANES;
    const int wib = threadIdx.x >> 5, wpc = blockDim.x >> 5;
    uint32_t *region = warp_mask_area<LANES>(s_mask, wib);
    uint32_t ins = 0, skp = 0;
    uint64_t round = 0;
    for (uint64_t s0 = 0; s0 < n; s0 += window) {
        const uint32_t cnt = (uint32_t)((n - s0) < window ? (n - s0) : window);
        for (uint32_t t = threadIdx.x; t < cnt; t += blockDim.x) {
            s_key[t] = load_key(keys + s0 + t);
            s_state[t] = 1;
        }
        __syncthreads();
        for (;;) {
            ++round;
            // reserve: the earliest pending key wins each candidate block
            for (uint32_t t = threadIdx.x; t < cnt; t += blockDim.x) {
                if (!s_state[t]) continue;
                const unsigned long long tag = ((unsigned long long)round << 32) | (unsigned long long)(~t);
#pragma unroll
                for (int c = 0; c < C; ++c)
                    atomicMax(resv + block_addr(f, f.a_block[c], s_key[t]), tag);
            }
            __syncthreads();
            // every thread has read the previous round's s_left before this barrier
            if (threadIdx.x == 0) s_left = 0;
            // commit the keys that hold every reservation of theirs
            for (uint32_t base = wib * G; base < cnt; base += wpc * G) {
                const uint32_t t = base + g;
                bool ready = t < cnt && s_state[t];
                const uint64_t x = ready ? s_key[t] : 0ull;
                if (ready) {
                    const unsigned long long tag = ((unsigned long long)round << 32) | (unsigned long long)(~t);
#pragma unroll
                    for (int c = 0; c < C; ++c)
                        ready = ready && __ldcg(resv + block_addr(f, f.a_block[c], x)) == tag;
                }
                uint64_t m[W];
                const uint32_t s = choose_key<C, LANES, kLoadCG>(f, x, ready, q, rank, s_amul, region, m);
                if (ready && s != kSkip) set_one<LANES>(f, block_addr(f, block_mult(f, s), x), q, m);
                if (ready && q == 0) {
                    s_state[t] = 0;
                    if (s == kSkip) ++skp; else ++ins;
                }
            }
            __syncthreads();
            for (uint32_t t = threadIdx.x; t < cnt; t += blockDim.x)
                if (s_state[t]) s_left = 1;
            __syncthreads();
            if (!s_left) break;
        }
    }
    flush_counts(ins, skp, counters);
}

// Batches of B > 1 keys (batch-synchronous: a batch decides against the
// state at its start, then sets) with the same reservation rounds, a batch
// taking the place of a key: every key of a pending batch reserves its
// candidate blocks with (round << 32 | ~batch), and a batch commits when all
// its keys hold all of their reservations. Then no earlier pending batch
// shares a candidate block with it, its keys decide against the current
// filter, and only after all of them decided do they set their bits. Batches
// that commit in the same round touch disjoint blocks. The outcome is that of
// inserting the batches one after another. The window holds whole batches.
template <int C, int LANES, bool BITSEL, bool POW2>
__global__ void __launch_bounds__(kSeqThreads) exact_batched_kernel(
    const DevFilter fp, const uint64_t *__restrict__ keys, uint64_t n, uint32_t B, uint32_t window,
    const uint16_t *__restrict__ rank_g, unsigned long long *counters, unsigned long long *resv) {
    DevFilter f = fp;
    if constexpr (!BITSEL) f.bitsel = 0;
    if constexpr (POW2) f.range_kind = kRangePow2;
    constexpr int G = 32 / LANES;
    constexpr int W = kBlockWords / LANES;
    extern __shared__ __align__(16) uint8_t s_dyn[];
    const uint32_t wpad = (window + 15) & ~15u;
    uint64_t *s_key = reinterpret_cast<uint64_t *>(s_dyn);  // window keys
    uint8_t *s_state = s_dyn + (size_t)window * 8;           // 1 = pending (per key)
    uint8_t *s_sel = s_state + wpad;                         // choices of a committing batch
    uint8_t *s_ok = s_sel + wpad;                            // per batch: every key holds its reservations
    uint16_t *s_rank = reinterpret_cast<uint16_t *>(s_ok + wpad);
    __shared__ uint64_t s_amul[32];
    __shared__ __align__(16) uint32_t s_mask[(kSeqThreads / 32) * mask_u32_per_warp<LANES>()];
    __shared__ int s_left;
    stage_bit_mults(fp, s_amul);
    const uint16_t *rank = stage_rank<C>(rank_g, s_rank, f.k + 1);
    if constexpr (C == 1) __syncthreads();
    const int lane = threadIdx.x & 31, q = lane % LANES, g = lane / LANES;
    const int wib = threadIdx.x >> 5, wpc = blockDim.x >> 5;
    uint32_t *region = warp_mask_area<LANES>(s_mask, wib);
    uint32_t ins = 0, skp = 0;
    uint64_t round = 0;
    for (uint64_t s0 = 0; s0 < n; s0 += window) {
        const uint32_t cnt = (uint32_t)((n - s0) < window ? (n - s0) : window);
        const uint32_t nb = (cnt + B - 1) / B;
        for (uint32_t t = threadIdx.x; t < cnt; t += blockDim.x) {
            s_key[t] = load_key(keys + s0 + t);
            s_state[t] = 1;
        }
        __syncthreads();
        for (;;) {
            ++round;
            for (uint32_t b = threadIdx.x; b < nb; b += blockDim.x) s_ok[b] = 1;
            // reserve: the earliest pending batch wins each candidate block
            for (uint32_t t = threadIdx.x; t < cnt; t += blockDim.x) {
                if (!s_state[t]) continue;
                const unsigned long long tag = ((unsigned long long)round << 32) | (unsigned long long)(~(t / B));
#pragma unroll
                for (int c = 0; c < C; ++c)
                    atomicMax(resv + block_addr(f, f.a_block[c], s_key[t]), tag);
            }
            __syncthreads();
            // every thread has read the previous round's s_left before this barrier
            if (threadIdx.x == 0) s_left = 0;
            // a batch with a key that lost one of its blocks waits for a later round
            for (uint32_t t = threadIdx.x; t < cnt; t += blockDim.x) {
                if (!s_state[t]) continue;
                const unsigned long long tag = ((unsigned long long)round << 32) | (unsigned long long)(~(t / B));
                bool won = true;
#pragma unroll
                for (int c = 0; c < C; ++c) won = won && __ldcg(resv + block_addr(f, f.a_block[c], s_key[t])) == tag;
                if (!won) s_ok[t / B] = 0;
            }
            __syncthreads();
            // the committing batches decide against the current filter ...
            for (uint32_t base = wib * G; base < cnt; base += wpc * G) {
                const uint32_t t = base + g;
                const bool ready = t < cnt && s_state[t] && s_ok[t / B];
                const uint64_t x = ready ? s_key[t] : 0ull;
                uint64_t m[W];
                const uint32_t s = choose_key<C, LANES, kLoadCG>(f, x, ready, q, rank, s_amul, region, m);
                if (ready && q == 0) s_sel[t] = (uint8_t)s;
            }
            __syncthreads();
            // ... and set their bits only after all of them decided
            for (uint32_t base = wib * G; base < cnt; base += wpc * G) {
                const uint32_t t = base + g;
                const bool ready = t < cnt && s_state[t] && s_ok[t / B];
                const uint32_t s = ready ? (uint32_t)s_sel[t] : kSkip;
                const uint64_t x = ready ? s_key[t] : 0ull;
                uint64_t m[W];
                key_mask_shared<LANES>(s_amul, f.k, x, q, region, m, f.bitsel);
                if (s != kSkip) set_one<LANES>(f, block_addr(f, block_mult(f, s), x), q, m);
                if (ready && q == 0) {
                    if (s == kSkip) ++skp; else ++ins;
                }
            }
            __syncthreads();
            for (uint32_t t = threadIdx.x; t < cnt; t += blockDim.x) {
                if (s_state[t] && s_ok[t / B]) s_state[t] = 0;
                else if (s_state[t]) s_left = 1;
            }
            __syncthreads();
            if (!s_left) break;
        }
    }
    flush_counts(ins, skp, counters);
}

inline size_t rank_bytes(int C, uint32_t k) { return C > 1 ? 513u * (k + 1) * sizeof(uint16_t) : 0; }

// Lets `fn` take `sm` bytes of dynamic shared memory (the default cap is
// 48 KB including static: the rank table of k = 32 next to a large static
// mask region exceeds it).
template <typename F>
cudaError_t allow_smem(F fn, size_t sm) {
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
}

template <int C, int LANES>
cudaError_t choose_launch(const Launch &L, const DevFilter &f, const uint64_t *keys, uint64_t n,
                          const uint16_t *rank, uint8_t *sel, unsigned long long *counters) {
    const size_t sm = rank_bytes(C, f.k);
    const cudaError_t e = allow_smem(choose_kernel<C, LANES>, sm);
    if (e != cudaSuccess) return e;
    choose_kernel<C, LANES><<<L.grid, kThreads, sm, L.stream>>>(f, keys, n, rank, sel, counters);
    return cudaGetLastError();
}

template <int C>
cudaError_t choose_dispatch(const Launch &L, const DevFilter &f, const uint64_t *keys, uint64_t n,
                            const uint16_t *rank, uint8_t *sel, unsigned long long *counters) {
    switch (L.lanes) {
        case 1: return choose_launch<C, 1>(L, f, keys, n, rank, sel, counters);
        case 2: return choose_launch<C, 2>(L, f, keys, n, rank, sel, counters);
        case 4: return choose_launch<C, 4>(L, f, keys, n, rank, sel, counters);
        case 8: return choose_launch<C, 8>(L, f, keys, n, rank, sel, counters);
        default: return cudaErrorInvalidValue;
    }
}

template <int C, int LANES, bool BITSEL, bool POW2>
cudaError_t small_launch(const Launch &L, const DevFilter &f, const uint64_t *keys, uint64_t n, uint64_t B,
                         const uint16_t *rank, unsigned long long *counters) {
    const size_t sm = small_mask_bytes<LANES>() + kSmallBatchMax + rank_bytes(C, f.k);
    cudaError_t e = cudaFuncSetAttribute(small_batch_kernel<C, LANES, BITSEL, POW2>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    small_batch_kernel<C, LANES, BITSEL, POW2><<<1, kSmallThreads, sm, L.stream>>>(f, keys, n, B, rank, counters);
    return cudaGetLastError();
}

// The instance for the filter's bit selection and block range (distinct
// selection always takes the general addressing).
template <int C, int LANES>
cudaError_t small_variant(const Launch &L, const DevFilter &f, const uint64_t *keys, uint64_t n, uint64_t B,
                          const uint16_t *rank, unsigned long long *counters) {
    if (f.bitsel) return small_launch<C, LANES, true, false>(L, f, keys, n, B, rank, counters);
    if (f.range_kind == kRangePow2) return small_launch<C, LANES, false, true>(L, f, keys, n, B, rank, counters);
    return small_launch<C, LANES, false, false>(L, f, keys, n, B, rank, counters);
}

template <int C>
cudaError_t small_dispatch(const Launch &L, const DevFilter &f, const uint64_t *keys, uint64_t n,
                           uint64_t B, const uint16_t *rank, unsigned long long *counters) {
    switch (L.lanes) {
        case 1:  // one lane per key needs more registers than a 1024-thread CTA allows
        case 2: return small_variant<C, 2>(L, f, keys, n, B, rank, counters);
        case 4: return small_variant<C, 4>(L, f, keys, n, B, rank, counters);
        case 8: return small_variant<C, 8>(L, f, keys, n, B, rank, counters);
        default: return cudaErrorInvalidValue;
    }
}

template <int C, int LANES, bool BULK, bool BITSEL, bool POW2>
cudaError_t persistent_launch(const Launch &L, const DevFilter &f, const uint64_t *keys, uint64_t n,
                              uint64_t B, const uint16_t *rank, uint8_t *sel,
                              unsigned long long *counters, unsigned int *bar, int sms) {
    const size_t sm = BULK ? bulk_ring_offset(C, f.k) + bulk_ring_bytes<LANES>() : rank_bytes(C, f.k);
    cudaError_t e = allow_smem(persistent_insert_kernel<C, LANES, BULK, BITSEL, POW2>, sm);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, persistent_insert_kernel<C, LANES, BULK, BITSEL, POW2>,
                                                      persistent_threads<LANES>(), sm);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int want = L.grid > 0 ? L.grid : 1;
    const int grid = want < per_sm * sms ? want : per_sm * sms;
    e = cudaMemsetAsync(bar, 0, sizeof(unsigned int), L.stream);
    if (e != cudaSuccess) return e;
    void *args[] = {(void *)&f, (void *)&keys, (void *)&n, (void *)&B, (void *)&rank,
                    (void *)&sel, (void *)&counters, (void *)&bar};
    return cudaLaunchCooperativeKernel((const void *)persistent_insert_kernel<C, LANES, BULK, BITSEL, POW2>, dim3(grid),
                                       dim3(persistent_threads<LANES>()), args, sm, L.stream);
}

// The instance for the filter's bit selection and block range (distinct
// selection always takes the general addressing).
template <int C, int LANES, bool BULK>
cudaError_t persistent_variant(const Launch &L, const DevFilter &f, const uint64_t *keys, uint64_t n,
                               uint64_t B, const uint16_t *rank, uint8_t *sel,
                               unsigned long long *counters, unsigned int *bar, int sms) {
    if (f.bitsel) return persistent_launch<C, LANES, BULK, true, false>(L, f, keys, n, B, rank, sel, counters, bar, sms);
    if (f.range_kind == kRangePow2)
        return persistent_launch<C, LANES, BULK, false, true>(L, f, keys, n, B, rank, sel, counters, bar, sms);
    return persistent_launch<C, LANES, BULK, false, false>(L, f, keys, n, B, rank, sel, counters, bar, sms);
}

template <int C, bool BULK>
cudaError_t persistent_dispatch(const Launch &L, const DevFilter &f, const uint64_t *keys, uint64_t n,
                                uint64_t B, const uint16_t *rank, uint8_t *sel,
                                unsigned long long *counters, unsigned int *bar, int sms) {
    switch (L.lanes) {
        case 1: return persistent_variant<C, 1, BULK>(L, f, keys, n, B, rank, sel, counters, bar, sms);
        case 2: return persistent_variant<C, 2, BULK>(L, f, keys, n, B, rank, sel, counters, bar, sms);
        case 4: return persistent_variant<C, 4, BULK>(L, f, keys, n, B, rank, sel, counters, bar, sms);
        case 8: return persistent_variant<C, 8, BULK>(L, f, keys, n, B, rank, sel, counters, bar, sms);
        default: return cudaErrorInvalidValue;
    }
}

template <int C, int LANES>
cudaError_t sorted_launch(const Launch &L, const DevFilter &f, const uint64_t *keys, uint64_t n, uint64_t B,
                          const uint16_t *rank, uint8_t *sel, unsigned long long *counters, unsigned int *bar,
                          uint32_t *scratch, uint32_t R, int sms) {
    const size_t sm = kRangeBlocks * 64 + rank_bytes(C, f.k);
    cudaError_t e = cudaFuncSetAttribute(sorted_insert_kernel<C, LANES>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sorted_insert_kernel<C, LANES>, kThreads, sm);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int want = L.grid > 0 ? L.grid : 1;
    const int grid = want < per_sm * sms ? want : per_sm * sms;
    e = cudaMemsetAsync(bar, 0, sizeof(unsigned int), L.stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(scratch, 0, (size_t)R * sizeof(uint32_t), L.stream);
    if (e != cudaSuccess) return e;
    uint32_t *cnt = scratch, *cur = scratch + R, *off = scratch + 2 * (size_t)R, *perm = scratch + 3 * (size_t)R + 1;
    void *args[] = {(void *)&f, (void *)&keys, (void *)&n, (void *)&B, (void *)&rank, (void *)&sel,
                    (void *)&counters, (void *)&bar, (void *)&cnt, (void *)&cur, (void *)&off, (void *)&perm,
                    (void *)&R};
    return cudaLaunchCooperativeKernel((const void *)sorted_insert_kernel<C, LANES>, dim3(grid), dim3(kThreads),
                                       args, sm, L.stream);
}

template <int C>
cudaError_t sorted_dispatch(const Launch &L, const DevFilter &f, const uint64_t *keys, uint64_t n, uint64_t B,
                            const uint16_t *rank, uint8_t *sel, unsigned long long *counters, unsigned int *bar,
                            uint32_t *scratch, uint32_t R, int sms) {
    switch (L.lanes) {
        case 1:  // one lane per key: register-hungry next to the staged range
        case 2: return sorted_launch<C, 2>(L, f, keys, n, B, rank, sel, counters, bar, scratch, R, sms);
        case 4: return sorted_launch<C, 4>(L, f, keys, n, B, rank, sel, counters, bar, scratch, R, sms);
        case 8: return sorted_launch<C, 8>(L, f, keys, n, B, rank, sel, counters, bar, scratch, R, sms);
        default: return cudaErrorInvalidValue;
    }
}

template <int C, int LANES, bool BITSEL, bool POW2>
cudaError_t exact_seq_launch(cudaStream_t s, const DevFilter &f, const uint64_t *keys, uint64_t n, uint32_t window,
                             const uint16_t *rank, unsigned long long *counters, unsigned long long *resv) {
    const size_t sm = (size_t)window * 8 + ((window + 15) & ~15u) + rank_bytes(C, f.k);
    cudaError_t e = cudaFuncSetAttribute(exact_sequential_kernel<C, LANES, BITSEL, POW2>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(resv, 0, f.M * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    exact_sequential_kernel<C, LANES, BITSEL, POW2><<<1, kSeqThreads, sm, s>>>(f, keys, n, window, rank, counters,
                                                                               resv);
    return cudaGetLastError();
}

// The instance for the filter's bit selection and block range (distinct
// selection always takes the general addressing).
template <int C, int LANES>
cudaError_t exact_seq_variant(cudaStream_t s, const DevFilter &f, const uint64_t *keys, uint64_t n, uint32_t window,
                              const uint16_t *rank, unsigned long long *counters, unsigned long long *resv) {
    if (f.bitsel) return exact_seq_launch<C, LANES, true, false>(s, f, keys, n, window, rank, counters, resv);
    if (f.range_kind == kRangePow2)
        return exact_seq_launch<C, LANES, false, true>(s, f, keys, n, window, rank, counters, resv);
    return exact_seq_launch<C, LANES, false, false>(s, f, keys, n, window, rank, counters, resv);
}

template <int C, int LANES, bool BITSEL, bool POW2>
cudaError_t exact_batched_launch(cudaStream_t s, const DevFilter &f, const uint64_t *keys, uint64_t n, uint32_t B,
                                 uint32_t window, const uint16_t *rank, unsigned long long *counters,
                                 unsigned long long *resv) {
    const size_t wpad = (window + 15) & ~15u;
    const size_t sm = (size_t)window * 8 + 3 * wpad + rank_bytes(C, f.k);
    cudaError_t e = allow_smem(exact_batched_kernel<C, LANES, BITSEL, POW2>, sm);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(resv, 0, f.M * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    exact_batched_kernel<C, LANES, BITSEL, POW2><<<1, kSeqThreads, sm, s>>>(f, keys, n, B, window, rank, counters,
                                                                            resv);
    return cudaGetLastError();
}

template <int C, int LANES>
cudaError_t exact_batched_variant(cudaStream_t s, const DevFilter &f, const uint64_t *keys, uint64_t n, uint32_t B,
                                  uint32_t window, const uint16_t *rank, unsigned long long *counters,
                                  unsigned long long *resv) {
    if (f.bitsel) return exact_batched_launch<C, LANES, true, false>(s, f, keys, n, B, window, rank, counters, resv);
    if (f.range_kind == kRangePow2)
        return exact_batched_launch<C, LANES, false, true>(s, f, keys, n, B, window, rank, counters, resv);
    return exact_batched_launch<C, LANES, false, false>(s, f, keys, n, B, window, rank, counters, resv);
}

}  // namespace

cudaError_t launch_exact_batched(int C, cudaStream_t s, const DevFilter &f, const uint64_t *keys, uint64_t n,
                                 uint64_t B, uint32_t window, const uint16_t *rank, unsigned long long *counters,
                                 unsigned long long *resv) {
    if (B < 2 || B > kSeqMaxBatch || window < B || window > kSeqMaxWindow || window % B) return cudaErrorInvalidValue;
    switch (C) {
        case 1: return exact_batched_variant<1, 2>(s, f, keys, n, (uint32_t)B, window, rank, counters, resv);
        case 2: return exact_batched_variant<2, 2>(s, f, keys, n, (uint32_t)B, window, rank, counters, resv);
        case 3: return exact_batched_variant<3, 2>(s, f, keys, n, (uint32_t)B, window, rank, counters, resv);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_exact_sequential(int C, cudaStream_t s, const DevFilter &f, const uint64_t *keys, uint64_t n,
                                    uint32_t window, const uint16_t *rank, unsigned long long *counters,
                                    unsigned long long *resv) {
    if (window < 32 || window > kSeqMaxWindow) return cudaErrorInvalidValue;
    switch (C) {
        case 1: return exact_seq_variant<1, 2>(s, f, keys, n, window, rank, counters, resv);
        case 2: return exact_seq_variant<2, 2>(s, f, keys, n, window, rank, counters, resv);
        case 3: return exact_seq_variant<3, 2>(s, f, keys, n, window, rank, counters, resv);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_sorted_insert(int C, const Launch &L, const DevFilter &f, const uint64_t *keys, uint64_t n,
                                 uint64_t B, const uint16_t *rank, uint8_t *sel, unsigned long long *counters,
                                 unsigned int *bar, uint32_t *scratch, uint32_t R, int sms) {
    switch (C) {
        case 1: return sorted_dispatch<1>(L, f, keys, n, B, rank, sel, counters, bar, scratch, R, sms);
        case 2: return sorted_dispatch<2>(L, f, keys, n, B, rank, sel, counters, bar, scratch, R, sms);
        case 3: return sorted_dispatch<3>(L, f, keys, n, B, rank, sel, counters, bar, scratch, R, sms);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_persistent_insert(int C, const Launch &L, const DevFilter &f, const uint64_t *keys,
                                     uint64_t n, uint64_t B, const uint16_t *rank, uint8_t *sel,
                                     unsigned long long *counters, unsigned int *bar, int sms, bool bulk) {
    switch (C) {
        case 1: return bulk ? persistent_dispatch<1, true>(L, f, keys, n, B, rank, sel, counters, bar, sms)
                            : persistent_dispatch<1, false>(L, f, keys, n, B, rank, sel, counters, bar, sms);
        case 2: return bulk ? persistent_dispatch<2, true>(L, f, keys, n, B, rank, sel, counters, bar, sms)
                            : persistent_dispatch<2, false>(L, f, keys, n, B, rank, sel, counters, bar, sms);
        case 3: return bulk ? persistent_dispatch<3, true>(L, f, keys, n, B, rank, sel, counters, bar, sms)
                            : persistent_dispatch<3, false>(L, f, keys, n, B, rank, sel, counters, bar, sms);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_choose(int C, const Launch &L, const DevFilter &f, const uint64_t *keys,
                          uint64_t n, const uint16_t *rank, uint8_t *sel,
                          unsigned long long *counters) {
    switch (C) {
        case 1: return choose_dispatch<1>(L, f, keys, n, rank, sel, counters);
        case 2: return choose_dispatch<2>(L, f, keys, n, rank, sel, counters);
        case 3: return choose_dispatch<3>(L, f, keys, n, rank, sel, counters);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_set(const Launch &L, const DevFilter &f, const uint64_t *keys, uint64_t n,
                       const uint8_t *sel) {
    switch (L.lanes) {
        case 1: set_kernel<1><<<L.grid, kThreads, 0, L.stream>>>(f, keys, n, sel); break;
        case 2: set_kernel<2><<<L.grid, kThreads, 0, L.stream>>>(f, keys, n, sel); break;
        case 4: set_kernel<4><<<L.grid, kThreads, 0, L.stream>>>(f, keys, n, sel); break;
        case 8: set_kernel<8><<<L.grid, kThreads, 0, L.stream>>>(f, keys, n, sel); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_sequential(int C, cudaStream_t s, const DevFilter &f, const uint64_t *keys,
                              uint64_t n, const uint16_t *rank, unsigned long long *counters) {
    const size_t sm = rank_bytes(C, f.k);
    switch (C) {
        case 1: sequential_kernel<1><<<1, 32, sm, s>>>(f, keys, n, rank, counters); break;
        case 2: sequential_kernel<2><<<1, 32, sm, s>>>(f, keys, n, rank, counters); break;
        case 3: sequential_kernel<3><<<1, 32, sm, s>>>(f, keys, n, rank, counters); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_small_batch(int C, const Launch &L, const DevFilter &f, const uint64_t *keys,
                               uint64_t n, uint64_t B, const uint16_t *rank,
                               unsigned long long *counters) {
    if (B > kSmallBatchMax) return cudaErrorInvalidValue;
    switch (C) {
        case 1: return small_dispatch<1>(L, f, keys, n, B, rank, counters);
        case 2: return small_dispatch<2>(L, f, keys, n, B, rank, counters);
        case 3: return small_dispatch<3>(L, f, keys, n, B, rank, counters);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace bc
