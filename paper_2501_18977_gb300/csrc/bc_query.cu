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

// Gathers bit g*LANES of v for g = 0..G-1 into bits 0..G-1.
template <int LANES>
__device__ __forceinline__ uint32_t compress_groups(uint32_t v) {
    constexpr int G = 32 / LANES;
    uint32_t r = 0;
#pragma unroll
    for (int g = 0; g < G; ++g) r |= ((v >> (g * LANES)) & 1u) << g;
    return r;
}

// One warp answers 64 consecutive keys and writes one bitmap word. Per key,
// a group of LANES lanes loads the C candidate blocks (all loads issued
// before any test) and each lane checks its W words for F(x) & ~block == 0;
// a ballot per candidate ANDs the lanes of a group, and the candidates OR.
template <int C, int LANES>
__global__ void __launch_bounds__(256) query_kernel(DevFilter f, const uint64_t *__restrict__ keys,
                                                    uint64_t n, uint64_t *__restrict__ bitmap) {
    constexpr int W = kBlockWords / LANES;
    constexpr int G = 32 / LANES;
    const int lane = threadIdx.x & 31, q = lane % LANES, g = lane / LANES;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint64_t nwords = (n + 63) / 64;
    for (uint64_t wd = warp; wd < nwords; wd += nwarps) {
        uint64_t word = 0;
#pragma unroll 2
        for (int it = 0; it < 64 / G; ++it) {
            const uint64_t i = wd * 64 + (uint64_t)it * G + g;
            const bool valid = i < n;
            const uint64_t x = valid ? load_key(keys + i) : 0ull;
            uint64_t m[W];
            key_mask<W>(f, x, q, m);
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
            uint32_t hits = 0;
#pragma unroll
            for (int c = 0; c < C; ++c) {
                uint64_t miss = 0;
#pragma unroll
                for (int j = 0; j < W; ++j) miss |= m[j] & ~blk[c][j];
                hits |= fold_groups<LANES>(__ballot_sync(kFull, valid && miss == 0));
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

template <int C>
cudaError_t query_dispatch(const Launch &L, const DevFilter &f, const uint64_t *keys, uint64_t n,
                           uint64_t *bitmap) {
    switch (L.lanes) {
        case 2: query_kernel<C, 2><<<L.grid, 256, 0, L.stream>>>(f, keys, n, bitmap); break;
        case 4: query_kernel<C, 4><<<L.grid, 256, 0, L.stream>>>(f, keys, n, bitmap); break;
        case 8: query_kernel<C, 8><<<L.grid, 256, 0, L.stream>>>(f, keys, n, bitmap); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_query(int C, const Launch &L, const DevFilter &f, const uint64_t *keys,
                         uint64_t n, uint64_t *bitmap) {
    switch (C) {
        case 1: return query_dispatch<1>(L, f, keys, n, bitmap);
        case 2: return query_dispatch<2>(L, f, keys, n, bitmap);
        case 3: return query_dispatch<3>(L, f, keys, n, bitmap);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_stats(const Launch &L, const uint64_t *words, uint64_t M,
                         unsigned long long *hist) {
    stats_kernel<<<L.grid, 256, 0, L.stream>>>(words, M, hist);
    return cudaGetLastError();
}

}  // namespace bc
