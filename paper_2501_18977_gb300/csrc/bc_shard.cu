// Sub-arrays (Section 3.4, parallelization): a filter of M blocks split into
// T sub-arrays of ceil(M / T) blocks, a key routed to sub-array h_0(x) by an
// additional linear hash with its own multiplier a_0. A sub-array is an
// ordinary filter whose hash seed is the generator state after a_0 was drawn,
// so every insert and query kernel applies unchanged; what is new here is the
// routing: a stable partition of a key array by h_0 (counting sort: per-warp
// counts, one exclusive scan, a scatter that ranks equal shards within a warp
// with __match_any_sync), and the scatter of per-sub-array query bitmaps back
// into the caller's key order.
#include <cstdio>

#include "bc_filter.h"
#include "bc_launch.h"

namespace {

constexpr int kThreads = 256;
constexpr uint32_t kMaxShards = 1024;
constexpr uint64_t kKeysPerWarp = 4096;   // partition work per warp (at least)
constexpr uint64_t kMaxWarps = 8192;
// Up to this many sub-arrays, each warp keeps its per-sub-array counts and
// output cursors in shared memory (8 bytes each); beyond it, in the global
// histogram. A cursor read from global memory put one dependent round trip
// in every 32-key step of the scatter.
constexpr uint32_t kSmemShards = 256;
// 32-key groups whose keys a warp loads together before ranking them in
// order (more key bytes in flight). On the DNA insert keys (5*10^7) the
// partition took 0.59 / 0.77 / 0.97 / 1.47 ms at T = 1 / 2 / 4 / 8 with
// global cursors and one group per step, 0.48 / 0.54 / 0.64 / 0.88 ms with
// shared cursors, and 0.33 / 0.40 / 0.50 / 0.77 ms with four groups.
constexpr int kGroups = 4;

// h_0 with the range rules of Section 3.4 (as bc::block_addr for the blocks).
struct ShardHash {
    uint64_t a0;
    uint64_t mod_mul;
    uint32_t T, kind, shift, pad;
};

__device__ __forceinline__ uint32_t shard_of(const ShardHash &h, uint64_t x) {
    uint64_t y = h.a0 * x;
    if (h.kind == bc::kRangePow2) return h.shift >= 64 ? 0u : (uint32_t)(y >> h.shift);
    if (h.kind == bc::kRangeEven) y ^= (y >> 32);
    return (uint32_t)bc::mod_fast(y, h.T, h.mod_mul);
}

ShardHash make_hash(uint64_t a0, uint32_t T) {
    ShardHash h{a0, 0, T, 0, 0, 0};
    if ((T & (T - 1)) == 0) {
        uint32_t lg = 0;
        while ((1u << lg) < T) ++lg;
        h.kind = bc::kRangePow2;
        h.shift = 64 - lg;
    } else {
        h.kind = (T & 1) ? bc::kRangeOdd : bc::kRangeEven;
        h.mod_mul = bc::mod_mul_for(T);
    }
    return h;
}

uint32_t warps_for(uint64_t n) {
    uint64_t w = (n + kKeysPerWarp - 1) / kKeysPerWarp;
    if (w < 1) w = 1;
    if (w > kMaxWarps) w = kMaxWarps;
    return (uint32_t)w;
}

// hist[s * nw + w] = keys of warp w's chunk that go to sub-array s (with
// T <= kSmemShards counted in the warp's shared counters and stored once;
// otherwise added to the zeroed hist directly).
__global__ void __launch_bounds__(kThreads) shard_count_kernel(const uint64_t *__restrict__ keys, uint64_t n,
                                                               ShardHash h, uint64_t chunk, uint32_t nw,
                                                               unsigned long long *__restrict__ hist) {
    __shared__ unsigned long long s_cnt[(kThreads / 32) * kSmemShards];
    const uint32_t w = (uint32_t)(((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (w >= nw) return;  // whole warps
    const bool local = h.T <= kSmemShards;
    unsigned long long *cnt = s_cnt + (threadIdx.x >> 5) * kSmemShards;
    if (local) {
        for (uint32_t t = lane; t < h.T; t += 32) cnt[t] = 0ull;
        __syncwarp();
    }
    const uint64_t b0 = (uint64_t)w * chunk;
    const uint64_t b1 = b0 + chunk < n ? b0 + chunk : n;
    for (uint64_t base = b0; base < b1; base += 32 * kGroups) {
        uint64_t x[kGroups];  // kGroups loads in flight per lane
#pragma unroll
        for (int j = 0; j < kGroups; ++j) {
            const uint64_t i = base + 32 * j + lane;
            x[j] = i < b1 ? bc::load_key(keys + i) : 0ull;
        }
#pragma unroll
        for (int j = 0; j < kGroups; ++j) {
            const bool valid = base + 32 * j + lane < b1;
            const uint32_t s = valid ? shard_of(h, x[j]) : 0xFFFFFFFFu;
            const uint32_t same = __match_any_sync(0xFFFFFFFFu, s);
            if (valid && lane == __ffs(same) - 1) {
                if (local) cnt[s] += (unsigned long long)__popc(same);  // one leader per sub-array per group
                else atomicAdd(&hist[(uint64_t)s * nw + w], (unsigned long long)__popc(same));
            }
            __syncwarp();
        }
    }
    if (local)
        for (uint32_t t = lane; t < h.T; t += 32) hist[(uint64_t)t * nw + w] = cnt[t];
}

// Exclusive scan of hist[0 .. L) in place (one CTA of 1024 threads; shard-
// major order makes the result each warp's first output position per
// sub-array), then offsets[s] = first position of sub-array s, offsets[T] = n.
__global__ void __launch_bounds__(1024) shard_scan_kernel(unsigned long long *hist, uint64_t L, uint32_t T,
                                                          uint32_t nw, uint64_t n, uint64_t *offsets) {
    __shared__ unsigned long long s_warp[32];
    const uint32_t tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const uint64_t per = (L + blockDim.x - 1) / blockDim.x;
    const uint64_t lo = (uint64_t)tid * per;
    const uint64_t hi = lo + per < L ? lo + per : L;
    unsigned long long sum = 0;
    for (uint64_t r = lo; r < hi; ++r) sum += hist[r];
    // inclusive scan of the per-thread sums: within warps, then over warps
    unsigned long long v = sum;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const unsigned long long u = __shfl_up_sync(0xFFFFFFFFu, v, d);
        if ((int)lane >= d) v += u;
    }
    if (lane == 31) s_warp[wid] = v;
    __syncthreads();
    if (wid == 0) {
        unsigned long long t = lane < (blockDim.x >> 5) ? s_warp[lane] : 0ull;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned long long u = __shfl_up_sync(0xFFFFFFFFu, t, d);
            if ((int)lane >= d) t += u;
        }
        s_warp[lane] = t;  // inclusive over warps
    }
    __syncthreads();
    unsigned long long acc = v - sum + (wid ? s_warp[wid - 1] : 0ull);  // exclusive start of this thread
    for (uint64_t r = lo; r < hi; ++r) {
        const unsigned long long c = hist[r];
        hist[r] = acc;
        acc += c;
    }
    __syncthreads();
    for (uint32_t s = tid; s < T; s += blockDim.x) offsets[s] = hist[(uint64_t)s * nw];
    if (tid == 0) offsets[T] = n;
}

// Writes each key of warp w's chunk to its sub-array's next position, in
// input order within the sub-array: lanes with equal h_0 rank themselves by
// lane index, the group's first lane advances the warp's cursor.
__global__ void __launch_bounds__(kThreads) shard_scatter_kernel(const uint64_t *__restrict__ keys, uint64_t n,
                                                                 ShardHash h, uint64_t chunk, uint32_t nw,
                                                                 unsigned long long *pos,
                                                                 uint64_t *__restrict__ out_keys,
                                                                 uint64_t *__restrict__ out_index) {
    __shared__ unsigned long long s_cur[(kThreads / 32) * kSmemShards];
    const uint32_t w = (uint32_t)(((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (w >= nw) return;
    // the warp's cursors: in shared memory for T <= kSmemShards, else in pos
    const bool local = h.T <= kSmemShards;
    unsigned long long *cur = local ? s_cur + (threadIdx.x >> 5) * kSmemShards : nullptr;
    if (local) {
        for (uint32_t t = lane; t < h.T; t += 32) cur[t] = pos[(uint64_t)t * nw + w];
        __syncwarp();
    }
    const uint64_t b0 = (uint64_t)w * chunk;
    const uint64_t b1 = b0 + chunk < n ? b0 + chunk : n;
    const uint32_t below = (1u << lane) - 1u;
    for (uint64_t base = b0; base < b1; base += 32 * kGroups) {
        uint64_t xs[kGroups];  // kGroups loads in flight per lane; groups then go out in order
#pragma unroll
        for (int j = 0; j < kGroups; ++j) {
            const uint64_t i = base + 32 * j + lane;
            xs[j] = i < b1 ? bc::load_key(keys + i) : 0ull;
        }
#pragma unroll
        for (int j = 0; j < kGroups; ++j) {
            const uint64_t i = base + 32 * j + lane;
            const bool valid = i < b1;
            const uint64_t x = xs[j];
            const uint32_t s = valid ? shard_of(h, x) : 0xFFFFFFFFu;
            const uint32_t same = __match_any_sync(0xFFFFFFFFu, s);
            const int leader = __ffs(same) - 1;
            unsigned long long b = 0;
            if (valid && lane == leader) b = local ? cur[s] : pos[(uint64_t)s * nw + w];
            b = __shfl_sync(0xFFFFFFFFu, b, leader);
            if (valid) {
                const uint64_t dst = b + (uint64_t)__popc(same & below);
                out_keys[dst] = x;
                out_index[dst] = i;
                if (lane == leader) {
                    if (local) cur[s] = b + (unsigned long long)__popc(same);
                    else pos[(uint64_t)s * nw + w] = b + (unsigned long long)__popc(same);
                }
            }
            __syncwarp();  // the cursor written above is read by any lane next group
        }
    }
}

// bitmap bit index[j] = bit (j - offsets[t]) of sub-array t's segment, for
// the t with offsets[t] <= j < offsets[t + 1]; segment t starts at word
// sum over t' < t of ceil(count_t' / 64). The bitmap is zeroed beforehand.
__global__ void __launch_bounds__(kThreads) shard_unpermute_kernel(const uint64_t *__restrict__ seg_bits,
                                                                   const uint64_t *__restrict__ offsets,
                                                                   const uint64_t *__restrict__ index, uint64_t n,
                                                                   uint32_t T, unsigned long long *bitmap) {
    __shared__ uint64_t s_off[kMaxShards + 1];
    __shared__ uint64_t s_woff[kMaxShards];
    for (uint32_t t = threadIdx.x; t <= T; t += blockDim.x) s_off[t] = offsets[t];
    __syncthreads();
    if (threadIdx.x == 0) {
        uint64_t wsum = 0;
        for (uint32_t t = 0; t < T; ++t) {
            s_woff[t] = wsum;
            wsum += (s_off[t + 1] - s_off[t] + 63) / 64;
        }
    }
    __syncthreads();
    for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
         j += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t lo = 0, hi = T;  // the last t with s_off[t] <= j
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (s_off[mid] <= j) lo = mid; else hi = mid;
        }
        const uint64_t bit = s_woff[lo] * 64 + (j - s_off[lo]);
        if ((__ldg(seg_bits + (bit >> 6)) >> (bit & 63)) & 1ull) {
            const uint64_t dst = __ldg(index + j);
            atomicOr(bitmap + (dst >> 6), 1ull << (dst & 63));
        }
    }
}

}  // namespace

extern "C" int blowchoc_shard_partition_scratch(uint64_t n, uint32_t T, uint64_t *words) {
    if (!words || T < 1 || T > kMaxShards) return bc_set_error(BLOWCHOC_EINVAL, "T in 1..1024, words not NULL");
    *words = (uint64_t)T * warps_for(n);
    return BLOWCHOC_OK;
}

extern "C" int blowchoc_shard_partition(const uint64_t *d_keys, uint64_t n, uint32_t T, uint64_t a0,
                                        uint64_t *d_out_keys, uint64_t *d_out_index, uint64_t *d_offsets,
                                        uint64_t *d_scratch, uint64_t scratch_words, void *stream) {
    if (T < 1 || T > kMaxShards) return bc_set_error(BLOWCHOC_EINVAL, "T must be in 1..1024");
    if (T > 1 && (a0 & 1) == 0) return bc_set_error(BLOWCHOC_EINVAL, "a0 must be odd");
    if (!d_offsets || (n && (!d_keys || !d_out_keys || !d_out_index || !d_scratch)))
        return bc_set_error(BLOWCHOC_EINVAL, "NULL buffer");
    const uint32_t nw = warps_for(n);
    if (scratch_words < (uint64_t)T * nw)
        return bc_set_error(BLOWCHOC_EINVAL, "scratch smaller than blowchoc_shard_partition_scratch");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e;
    if (n == 0) {
        e = cudaMemsetAsync(d_offsets, 0, (T + 1) * sizeof(uint64_t), s);
        if (e != cudaSuccess) return bc_set_error(BLOWCHOC_ECUDA, cudaGetErrorString(e));
        return BLOWCHOC_OK;
    }
    const ShardHash h = make_hash(T > 1 ? a0 : 0, T);
    const uint64_t chunk = ((n + nw - 1) / nw + 31) / 32 * 32;
    const int grid = (int)((nw + kThreads / 32 - 1) / (kThreads / 32));
    unsigned long long *hist = reinterpret_cast<unsigned long long *>(d_scratch);
    e = cudaMemsetAsync(hist, 0, (size_t)T * nw * sizeof(uint64_t), s);
    if (e == cudaSuccess) {
        shard_count_kernel<<<grid, kThreads, 0, s>>>(d_keys, n, h, chunk, nw, hist);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        shard_scan_kernel<<<1, 1024, 0, s>>>(hist, (uint64_t)T * nw, T, nw, n, d_offsets);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        shard_scatter_kernel<<<grid, kThreads, 0, s>>>(d_keys, n, h, chunk, nw, hist, d_out_keys, d_out_index);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return bc_set_error(BLOWCHOC_ECUDA, cudaGetErrorString(e));
    bc_note_launch();
    bc_note_launch();
    bc_note_launch();
    return BLOWCHOC_OK;
}

extern "C" int blowchoc_shard_unpermute(const uint64_t *d_seg_bits, const uint64_t *d_offsets,
                                        const uint64_t *d_index, uint64_t n, uint32_t T, uint64_t *d_bitmap,
                                        void *stream) {
    if (T < 1 || T > kMaxShards) return bc_set_error(BLOWCHOC_EINVAL, "T must be in 1..1024");
    if (n && (!d_seg_bits || !d_offsets || !d_index || !d_bitmap)) return bc_set_error(BLOWCHOC_EINVAL, "NULL buffer");
    if (n == 0) return BLOWCHOC_OK;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(d_bitmap, 0, (n + 63) / 64 * sizeof(uint64_t), s);
    if (e == cudaSuccess) {
        int sms = 0, dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const uint64_t want = (n + kThreads - 1) / kThreads;
        const uint64_t cap = (uint64_t)(sms > 0 ? sms : 1) * 8;
        shard_unpermute_kernel<<<(int)(want < cap ? want : cap), kThreads, 0, s>>>(
            d_seg_bits, d_offsets, d_index, n, T, reinterpret_cast<unsigned long long *>(d_bitmap));
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return bc_set_error(BLOWCHOC_ECUDA, cudaGetErrorString(e));
    bc_note_launch();
    return BLOWCHOC_OK;
}
