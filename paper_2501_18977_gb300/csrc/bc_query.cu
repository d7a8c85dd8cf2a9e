// Membership query (Section 3.1) and load statistics (Appendix C, Fig. 8).
#include "bc_launch.h"

namespace bc {
namespace {

constexpr unsigned kFull = 0xffffffffu;

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

constexpr int kThreads = 256;

// One warp answers 64 consecutive keys and writes one bitmap word. Per key, a
// group of LANES lanes builds the key's mask once (key_mask_shared), then
// tests the candidate blocks: each lane checks its W words for
// F(x) & ~block == 0, a ballot per candidate ANDs the lanes of each group,
// and the candidates OR. EARLY = false issues all C block loads before any
// test. EARLY = true loads candidate i+1 only for groups whose key was not
// found in candidates 1..i, so members cost fewer block reads.
template <int C, int LANES, bool EARLY>
__global__ void __launch_bounds__(kThreads) query_kernel(DevFilter f, const uint64_t *__restrict__ keys,
                                                         uint64_t n, uint64_t *__restrict__ bitmap) {
    constexpr int W = kBlockWords / LANES;
    constexpr int G = 32 / LANES;
    __shared__ uint64_t s_amul[32];
    __shared__ __align__(16) uint32_t s_mask[(kThreads / 32) * G * region_u32<LANES>()];
    stage_bit_mults(f, s_amul);
    __syncthreads();
    const int lane = threadIdx.x & 31, q = lane % LANES, g = lane / LANES;
    uint32_t *region = s_mask + ((threadIdx.x >> 5) * G + g) * region_u32<LANES>();
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint64_t nwords = (n + 63) / 64;
    for (uint64_t wd = warp; wd < nwords; wd += nwarps) {
        uint64_t word = 0;
        for (int it = 0; it < 64 / G; ++it) {
            const uint64_t i = wd * 64 + (uint64_t)it * G + g;
            const bool valid = i < n;
            const uint64_t x = valid ? load_key(keys + i) : 0ull;
            uint64_t m[W];
            key_mask_shared<LANES>(s_amul, f.k, x, q, region, m);
            uint32_t hits = 0;
            if constexpr (!EARLY) {
                uint64_t blk[C][W];
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    const uint64_t b = block_addr(f, f.a_block[c], x);
                    if (valid) {
                        load_words<W, kLoadNC>(f.words + b * kBlockWords + (uint64_t)q * W, blk[c]);
                    } else {
#pragma unroll
                        for (int j = 0; j < W; ++j) blk[c][j] = 0ull;
                    }
                }
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    uint64_t miss = 0;
#pragma unroll
                    for (int j = 0; j < W; ++j) miss |= m[j] & ~blk[c][j];
                    hits |= fold_groups<LANES>(__ballot_sync(kFull, valid && miss == 0));
                }
            } else {
                bool need = valid;
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    uint64_t blk[W];
                    if (need) {
                        const uint64_t b = block_addr(f, f.a_block[c], x);
                        load_words<W, kLoadNC>(f.words + b * kBlockWords + (uint64_t)q * W, blk);
                    } else {
#pragma unroll
                        for (int j = 0; j < W; ++j) blk[j] = 0ull;
                    }
                    uint64_t miss = 0;
#pragma unroll
                    for (int j = 0; j < W; ++j) miss |= m[j] & ~blk[j];
                    const uint32_t got = fold_groups<LANES>(__ballot_sync(kFull, need && miss == 0));
                    hits |= got;
                    need = need && !((got >> (g * LANES)) & 1u);
                }
            }
            word |= (uint64_t)compress_groups<LANES>(hits) << (it * G);
        }
        if (lane == 0) bitmap[wd] = word;
    }
}

// Histogram of set bits per block. Four lanes read one 64-byte block as
// consecutive 16-byte pieces (fully coalesced stream over the words).
__global__ void __launch_bounds__(256) stats_kernel(const uint64_t *__restrict__ words, uint64_t M,
                                                    unsigned long long *__restrict__ hist) {
    __shared__ unsigned int s_hist[513];
    for (int t = threadIdx.x; t < 513; t += blockDim.x) s_hist[t] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    // a warp covers 8 blocks per step
    for (uint64_t base = warp * 8; base < M; base += nwarps * 8) {
        const uint64_t b = base + (lane >> 2);
        uint32_t L = 0;
        if (b < M) {
            const ulonglong2 v = __ldcs(reinterpret_cast<const ulonglong2 *>(words + b * kBlockWords) + (lane & 3));
            L = __popcll(v.x) + __popcll(v.y);
        }
        L += __shfl_xor_sync(kFull, L, 1);
        L += __shfl_xor_sync(kFull, L, 2);
        if (b < M && (lane & 3) == 0) atomicAdd(&s_hist[L], 1u);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < 513; t += blockDim.x)
        if (s_hist[t]) atomicAdd(&hist[t], (unsigned long long)s_hist[t]);
}

template <int C, bool EARLY>
cudaError_t query_dispatch(const Launch &L, const DevFilter &f, const uint64_t *keys, uint64_t n,
                           uint64_t *bitmap) {
    switch (L.lanes) {
        case 1: query_kernel<C, 1, EARLY><<<L.grid, kThreads, 0, L.stream>>>(f, keys, n, bitmap); break;
        case 2: query_kernel<C, 2, EARLY><<<L.grid, kThreads, 0, L.stream>>>(f, keys, n, bitmap); break;
        case 4: query_kernel<C, 4, EARLY><<<L.grid, kThreads, 0, L.stream>>>(f, keys, n, bitmap); break;
        case 8: query_kernel<C, 8, EARLY><<<L.grid, kThreads, 0, L.stream>>>(f, keys, n, bitmap); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_query(int C, const Launch &L, const DevFilter &f, const uint64_t *keys,
                         uint64_t n, uint64_t *bitmap) {
    const bool early = L.early != 0;
    switch (C) {
        case 1: return query_dispatch<1, false>(L, f, keys, n, bitmap);
        case 2: return early ? query_dispatch<2, true>(L, f, keys, n, bitmap)
                             : query_dispatch<2, false>(L, f, keys, n, bitmap);
        case 3: return early ? query_dispatch<3, true>(L, f, keys, n, bitmap)
                             : query_dispatch<3, false>(L, f, keys, n, bitmap);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_stats(const Launch &L, const uint64_t *words, uint64_t M,
                         unsigned long long *hist) {
    stats_kernel<<<L.grid, 256, 0, L.stream>>>(words, M, hist);
    return cudaGetLastError();
}

}  // namespace bc
