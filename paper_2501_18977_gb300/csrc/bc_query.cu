// Membership query (Section 3.1) and load statistics (Appendix C, Fig. 8).
#include "bc_launch.h"
#include "bc_phases.cuh"

namespace bc {
namespace {

constexpr int kThreads = 256;

// One warp answers 64 consecutive keys per step (query_word) and writes one
// bitmap word; warps stride over the words of the bitmap. With `count`, the
// warp also adds its number of present keys to *count (bitmap may be null).
// BITSEL: distinct bit selection; POW2: a power-of-two block count. The
// false instances compile those paths out (inlined as runtime branches they
// cost registers; DNA query 2.80 -> 2.78 ms without the distinct path, ->
// 2.74 ms with the power-of-two addressing alone).
template <int C, int LANES, int MODE, bool BITSEL, bool POW2>
__global__ void __launch_bounds__(kThreads) query_kernel(DevFilter f, const uint64_t *__restrict__ keys,
                                                         uint64_t n, uint64_t *__restrict__ bitmap,
                                                         unsigned long long *__restrict__ count) {
    // constants from here on: the paths this instance does not take fold away
    if constexpr (!BITSEL) f.bitsel = 0;
    if constexpr (POW2) f.range_kind = kRangePow2;
    constexpr int G = 32 / LANES;
    __shared__ uint64_t s_amul[32];
    __shared__ __align__(16) uint32_t s_mask[(kThreads / 32) * mask_u32_per_warp<LANES>()];
    stage_bit_mults(f, s_amul);
    __syncthreads();
    const int lane = threadIdx.x & 31, q = lane % LANES, g = lane / LANES;
    uint32_t *region = warp_mask_area<LANES>(s_mask, threadIdx.x >> 5);
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint64_t nwords = (n + 63) / 64;
    uint32_t present = 0;
    for (uint64_t wd = warp; wd < nwords; wd += nwarps) {
        const uint64_t word = query_word<C, LANES, MODE>(f, keys, n, wd, s_amul, region, q, g);
        if (lane == 0) {
            if (bitmap) bitmap[wd] = word;
            present += (uint32_t)__popcll(word);
        }
    }
    if (count && lane == 0 && present) atomicAdd(count, (unsigned long long)present);
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

template <int C, int MODE, bool BITSEL, bool POW2>
cudaError_t query_lanes(const Launch &L, const DevFilter &f, const uint64_t *keys, uint64_t n,
                        uint64_t *bitmap, unsigned long long *count) {
    switch (L.lanes) {
        case 1: query_kernel<C, 1, MODE, BITSEL, POW2><<<L.grid, kThreads, 0, L.stream>>>(f, keys, n, bitmap, count); break;
        case 2: query_kernel<C, 2, MODE, BITSEL, POW2><<<L.grid, kThreads, 0, L.stream>>>(f, keys, n, bitmap, count); break;
        case 4: query_kernel<C, 4, MODE, BITSEL, POW2><<<L.grid, kThreads, 0, L.stream>>>(f, keys, n, bitmap, count); break;
        case 8: query_kernel<C, 8, MODE, BITSEL, POW2><<<L.grid, kThreads, 0, L.stream>>>(f, keys, n, bitmap, count); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int C, int MODE>
cudaError_t query_dispatch(const Launch &L, const DevFilter &f, const uint64_t *keys, uint64_t n,
                           uint64_t *bitmap, unsigned long long *count) {
    if (f.bitsel) return query_lanes<C, MODE, true, false>(L, f, keys, n, bitmap, count);
    return f.range_kind == kRangePow2 ? query_lanes<C, MODE, false, true>(L, f, keys, n, bitmap, count)
                                      : query_lanes<C, MODE, false, false>(L, f, keys, n, bitmap, count);
}

}  // namespace

cudaError_t launch_query(int C, const Launch &L, const DevFilter &f, const uint64_t *keys,
                         uint64_t n, uint64_t *bitmap, unsigned long long *count) {
    switch (C) {
        case 1: return query_dispatch<1, 0>(L, f, keys, n, bitmap, count);
        case 2: return L.early == 0 ? query_dispatch<2, 0>(L, f, keys, n, bitmap, count)
                                    : query_dispatch<2, 1>(L, f, keys, n, bitmap, count);
        case 3: return L.early == 0 ? query_dispatch<3, 0>(L, f, keys, n, bitmap, count)
                     : L.early == 1 ? query_dispatch<3, 1>(L, f, keys, n, bitmap, count)
                                    : query_dispatch<3, 2>(L, f, keys, n, bitmap, count);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_stats(const Launch &L, const uint64_t *words, uint64_t M,
                         unsigned long long *hist) {
    stats_kernel<<<L.grid, 256, 0, L.stream>>>(words, M, hist);
    return cudaGetLastError();
}

}  // namespace bc
