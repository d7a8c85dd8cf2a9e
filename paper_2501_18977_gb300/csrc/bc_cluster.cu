// Cluster-resident insertion: a filter small enough for the distributed
// shared memory of one thread-block cluster is loaded into it once, every
// batch of the insert runs there, and the words are written back at the end.
//
// CTA r of a cluster of S CTAs holds blocks [r * slice, (r + 1) * slice) of
// the filter (slice = ceil(M / S)). A batch (Section 3.2, with the batch rule
// of the library: all keys of a batch decide against the state at its start)
// is one choose pass over the batch's keys, a cluster barrier, one set pass,
// and a second cluster barrier. Candidate blocks are read with
// ld.shared::cluster from the CTA that owns them, and bits are OR-ed in with
// red.shared::cluster; the barriers' release/acquire order makes a batch's
// ORs visible to the next batch's reads. Per round this replaces the round
// trips to L2 of the global-memory kernels by shared-memory round trips
// inside one GPC, and the grid barrier by the cluster barrier.
#include <cooperative_groups.h>

#include <algorithm>
#include <mutex>

#include "bc_launch.h"
#include "bc_phases.cuh"

namespace cg = cooperative_groups;

namespace bc {
namespace {

constexpr int kClThreads = 1024;

// 32-bit shared::cluster address of `local` (a shared-memory address of this
// CTA) in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t cluster_addr(const void *local, uint32_t rank) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(local);
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}

// The lane's W words of a block in distributed shared memory.
template <int W>
__device__ __forceinline__ void dsmem_load(uint32_t addr, uint64_t (&v)[W]) {
    if constexpr (W == 1) {
        asm volatile("ld.shared::cluster.u64 %0, [%1];" : "=l"(v[0]) : "r"(addr) : "memory");
    } else {
#pragma unroll
        for (int j = 0; j < W; j += 2)
            asm volatile("ld.shared::cluster.v2.u64 {%0,%1}, [%2];"
                         : "=l"(v[j]), "=l"(v[j + 1]) : "r"(addr + 8u * j) : "memory");
    }
}

// OR of v into the 64-bit word at addr, as two 32-bit ORs of the non-zero
// halves (little-endian: the low half at addr). Measured on GB300 with
// driver 580 and CUDA 13.0: a 64-bit red/atom OR into another CTA's shared
// memory loses bits, while 32-bit OR, 64-bit add and 64-bit CAS do not.
__device__ __forceinline__ void dsmem_or(uint32_t addr, uint64_t v) {
    const uint32_t lo = (uint32_t)v, hi = (uint32_t)(v >> 32);
    if (lo) asm volatile("red.relaxed.cluster.shared::cluster.or.b32 [%0], %1;" :: "r"(addr), "r"(lo) : "memory");
    if (hi) asm volatile("red.relaxed.cluster.shared::cluster.or.b32 [%0], %1;" :: "r"(addr + 4u), "r"(hi) : "memory");
}

// Cluster-wide barrier (release on arrival, acquire on wait): every thread's
// earlier shared-memory accesses, local and remote, are ordered before every
// thread's later ones.
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// 8-byte asynchronous copy global -> shared (completes at cp_async_wait).
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" :: "r"(d), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Field-wise read of the cluster's work item: from the global work list, or
// from the by-value parameter of a single-filter launch.
#define CL_FIELD(field) (items ? items[ci].field : one.field)

template <int C, int LANES>
__global__ void __launch_bounds__(kClThreads, 1)
    cluster_insert_kernel(const ManyItem *__restrict__ items, const ManyItem one, uint32_t slice_max,
                          uint32_t rank_u16, uint32_t kpc) {
    constexpr int W = kBlockWords / LANES;    // words per lane
    constexpr int TC = kClThreads / LANES;    // groups per CTA
    __shared__ uint64_t s_amul[32];
    __shared__ __align__(16) uint32_t s_mask[(kClThreads / 32) * mask_u32_per_warp<LANES>()];
    // dynamic: the slice's words | two key buffers of kpc keys (one batch's
    // keys of this CTA, the next batch's arriving) | rank table | kpc choices
    extern __shared__ __align__(16) uint8_t s_dyn[];
    uint64_t *s_words = reinterpret_cast<uint64_t *>(s_dyn);
    uint64_t *s_keys = reinterpret_cast<uint64_t *>(s_dyn + (size_t)slice_max * 64);
    uint16_t *s_rank = reinterpret_cast<uint16_t *>(s_dyn + (size_t)slice_max * 64 + (size_t)kpc * 16);
    uint8_t *s_sel = reinterpret_cast<uint8_t *>(s_rank) + ((rank_u16 * 2u + 15u) & ~15u);

    cg::cluster_group cl = cg::this_cluster();
    const uint32_t S = cl.num_blocks();
    const uint32_t me = cl.block_rank();
    const uint32_t ci = blockIdx.x / S;

    DevFilter f;
    f.words = CL_FIELD(f.words);
    f.M = CL_FIELD(f.M);
    f.k = CL_FIELD(f.k);
    f.range_kind = CL_FIELD(f.range_kind);
    f.shift = CL_FIELD(f.shift);
    f.c = CL_FIELD(f.c);
    f.bitsel = CL_FIELD(f.bitsel);
    f.mod_mul = CL_FIELD(f.mod_mul);
    f.a_block[0] = CL_FIELD(f.a_block[0]);
    f.a_block[1] = CL_FIELD(f.a_block[1]);
    f.a_block[2] = CL_FIELD(f.a_block[2]);
    const uint64_t *keys = CL_FIELD(keys);
    const uint64_t n = CL_FIELD(n);
    const uint64_t B = CL_FIELD(B);
    const uint16_t *rank_g = CL_FIELD(rank);
    unsigned long long *counters = CL_FIELD(counters);
    if (threadIdx.x < f.k) s_amul[threadIdx.x] = CL_FIELD(f.a_bit[threadIdx.x]);

    // this CTA's slice of the filter
    const uint32_t slice = (uint32_t)((f.M + S - 1) / S);
    // owner CTA and offset of block b: q = floor(b mul / 2^32) with
    // mul = floor(2^32 / slice) is b / slice or one less; one correction step
    const uint32_t slice_mul = slice > 1 ? (uint32_t)(0x100000000ull / slice) : 0u;
    auto locate = [slice, slice_mul](uint32_t b, uint32_t &owner, uint32_t &off) {
        uint32_t q = slice > 1 ? __umulhi(b, slice_mul) : b;
        uint32_t r = b - q * slice;
        if (r >= slice) {
            ++q;
            r -= slice;
        }
        owner = q;
        off = r;
    };
    const uint64_t b0 = (uint64_t)me * slice;
    const uint64_t nb = b0 < f.M ? (f.M - b0 < slice ? f.M - b0 : slice) : 0;
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(f.words + b0 * kBlockWords);
        uint4 *dst = reinterpret_cast<uint4 *>(s_words);
        for (uint64_t t = threadIdx.x; t < nb * 4; t += kClThreads) dst[t] = __ldcg(src + t);
    }
    const uint32_t k1 = f.k + 1;
    const uint16_t *rank = rank_g;
    if constexpr (C > 1) {
        for (uint32_t t = threadIdx.x; t < 513u * k1; t += kClThreads) s_rank[t] = rank_g[t];
        rank = s_rank;
    }
    cluster_sync();  // every slice loaded before any CTA reads another's

    const int lane = threadIdx.x & 31, q = lane % LANES;
    uint32_t *region = warp_mask_area<LANES>(s_mask, threadIdx.x >> 5);
    const uint32_t gl = threadIdx.x / LANES;  // group within the CTA
    const int lead = lane & ~(LANES - 1);     // the group's first lane
    static_assert(LANES >= C, "a group locates its candidates one per lane");
    const uint32_t T = S * TC;                // groups in the cluster
    const uint32_t gid = me * TC + gl;
    uint32_t ins = 0, skp = 0;
    const uint64_t rounds = (n + B - 1) / B;
    // key j of a batch is taken by group j mod T of the cluster in pass j / T;
    // this CTA's keys of pass p sit at [p * TC, (p + 1) * TC) of its buffer
    auto stage = [&](uint64_t r, uint64_t *buf) {
        const uint64_t base = r * B;
        const uint32_t cnt = (uint32_t)(n - base < B ? n - base : B);
        const uint32_t slots = (cnt + T - 1) / T * TC;
        for (uint32_t u = threadIdx.x; u < slots; u += kClThreads) {
            const uint32_t j = (u / TC) * T + me * TC + (u % TC);
            if (j < cnt) cp_async8(buf + u, keys + base + j);
        }
        cp_async_commit();
    };
    stage(0, s_keys);
    for (uint64_t r = 0; r < rounds; ++r) {
        const uint32_t cnt = (uint32_t)(n - r * B < B ? n - r * B : B);
        const uint32_t passes = (cnt + T - 1) / T;
        const uint64_t *kb = s_keys + (r & 1) * kpc;
        cp_async_wait();
        __syncthreads();  // this batch's keys are in shared memory
        if (r + 1 < rounds) stage(r + 1, s_keys + ((r + 1) & 1) * kpc);  // the next batch's keys, meanwhile
        // choose
        for (uint32_t p = 0; p < passes; ++p) {
            const uint32_t j = p * T + gid;
            const bool valid = j < cnt;
            const uint64_t x = valid ? kb[p * TC + gl] : 0ull;
            // lane i of the group locates candidate i once; the group shares it
            uint32_t mine = 0;
            if (valid && q < C) {
                uint32_t owner, off;
                locate((uint32_t)block_addr(f, block_mult(f, (uint32_t)q), x), owner, off);
                mine = cluster_addr(s_words + (size_t)off * kBlockWords, owner);
            }
            uint64_t blk[C][W];
#pragma unroll
            for (int i = 0; i < C; ++i) {
                const uint32_t base = __shfl_sync(kFull, mine, lead + i);
                if (valid) {
                    dsmem_load<W>(base + 8u * W * q, blk[i]);
                } else {
#pragma unroll
                    for (int w = 0; w < W; ++w) blk[i][w] = ~0ull;
                }
            }
            uint64_t m[W];
            key_mask_shared<LANES>(s_amul, f.k, x, q, region, m, f.bitsel);
            uint32_t la[C];
#pragma unroll
            for (int i = 0; i < C; ++i) la[i] = group_sum<LANES>(load_and_new<W>(blk[i], m));
            const uint32_t s = choose_from_terms<C>(la, rank, k1);
            if (valid && q == 0) {
                s_sel[p * TC + gl] = (uint8_t)s;
                if (s == kSkip) ++skp; else ++ins;
            }
        }
        cluster_sync();  // all reads of the batch-start state done
        // set: the same groups OR their keys' bits into the chosen blocks
        for (uint32_t p = 0; p < passes; ++p) {
            const uint32_t j = p * T + gid;
            const uint32_t s = j < cnt ? s_sel[p * TC + gl] : kSkip;
            const uint64_t x = s != kSkip ? kb[p * TC + gl] : 0ull;
            uint64_t m[W];
            key_mask_shared<LANES>(s_amul, f.k, x, q, region, m, f.bitsel);
            uint32_t mine = 0;
            if (s != kSkip && q == 0) {
                uint32_t owner, off;
                locate((uint32_t)block_addr(f, block_mult(f, s), x), owner, off);
                mine = cluster_addr(s_words + (size_t)off * kBlockWords, owner);
            }
            const uint32_t a = __shfl_sync(kFull, mine, lead) + 8u * W * q;
            if (s != kSkip) {
#pragma unroll
                for (int w = 0; w < W; ++w)
                    if (m[w]) dsmem_or(a + 8u * w, m[w]);
            }
        }
        cluster_sync();  // the batch's ORs land before the next batch reads
    }
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(s_words);
        uint4 *dst = reinterpret_cast<uint4 *>(f.words + b0 * kBlockWords);
        for (uint64_t t = threadIdx.x; t < nb * 4; t += kClThreads) dst[t] = src[t];
    }
    flush_counts(ins, skp, counters);
}

#undef CL_FIELD

template <int C, int LANES>
struct ClusterKernel {
    static constexpr auto fn = cluster_insert_kernel<C, LANES>;
};

// Per instantiation: static shared memory and the largest cluster the
// device can co-schedule with a full shared-memory budget per CTA.
struct ClusterInfo {
    bool ok = false;
    size_t static_smem = 0;
    size_t optin = 0;
    int max_S = 0;
};

template <int C, int LANES>
const ClusterInfo &cluster_info() {
    static ClusterInfo info;
    static std::once_flag once;
    std::call_once(once, [] {
        auto fn = cluster_insert_kernel<C, LANES>;
        int dev = 0, optin = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return;
        if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return;
        cudaFuncAttributes fa;
        if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess) return;
        const int dyn = optin - (int)fa.sharedSizeBytes;
        if (dyn <= 0) return;
        if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn) != cudaSuccess) return;
        if (cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
            cudaGetLastError();
        }
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(16, 1, 1);
        cfg.blockDim = dim3(kClThreads, 1, 1);
        cfg.dynamicSmemBytes = (size_t)dyn;
        int cs = 0;
        if (cudaOccupancyMaxPotentialClusterSize(&cs, fn, &cfg) != cudaSuccess || cs < 1) {
            cudaGetLastError();
            return;
        }
        info.static_smem = fa.sharedSizeBytes;
        info.optin = (size_t)optin;
        info.max_S = std::min(cs, 16);
        info.ok = true;
    });
    return info;
}

const ClusterInfo &info_for(int C, int lanes) {
    static const ClusterInfo none;
    if (lanes == 4) {
        if (C == 1) return cluster_info<1, 4>();
        if (C == 2) return cluster_info<2, 4>();
        if (C == 3) return cluster_info<3, 4>();
    } else if (lanes == 8) {
        if (C == 1) return cluster_info<1, 8>();
        if (C == 2) return cluster_info<2, 8>();
        if (C == 3) return cluster_info<3, 8>();
    }
    return none;
}

}  // namespace

ClusterShape cluster_shape_at(int C, int lanes, int S, uint64_t M, uint32_t k, uint64_t Beff) {
    ClusterShape sh;
    const ClusterInfo &info = info_for(C, lanes);
    if (!info.ok || S < 1 || S > info.max_S || M == 0 || Beff == 0 || k == 0 || k > 32) return sh;
    const uint32_t TC = kClThreads / lanes;
    const uint32_t rank_u16 = C > 1 ? 513u * (k + 1) : 0u;
    const size_t rank_b = ((size_t)rank_u16 * 2 + 15) & ~size_t(15);
    const uint64_t slice = (M + S - 1) / S;
    const uint64_t passes = (Beff + (uint64_t)S * TC - 1) / ((uint64_t)S * TC);
    const uint64_t kpc = passes * TC;  // keys of one batch per CTA (TC is a multiple of 16)
    const size_t smem = (size_t)slice * 64 + (size_t)kpc * 16 + rank_b + (size_t)kpc;
    if (smem + info.static_smem > info.optin) return sh;
    sh.S = S;
    sh.slice = (uint32_t)slice;
    sh.rank_u16 = rank_u16;
    sh.kpc = (uint32_t)kpc;
    sh.smem = smem;
    return sh;
}

ClusterShape cluster_shape(int C, int lanes, uint64_t M, uint32_t k, uint64_t Beff, int max_S,
                           uint64_t keys_per_cta) {
    const ClusterInfo &info = info_for(C, lanes);
    if (!info.ok) return ClusterShape();
    const int cap = std::min(max_S, info.max_S);
    ClusterShape sh;
    int S = 1;
    for (; S <= cap; ++S) {
        sh = cluster_shape_at(C, lanes, S, M, k, Beff);
        if (sh.S) break;
    }
    if (S > cap) return ClusterShape();
    if (keys_per_cta) {
        const uint64_t want = (Beff + keys_per_cta - 1) / keys_per_cta;
        const int S2 = (int)std::min<uint64_t>((uint64_t)cap, want);
        if (S2 > S) {
            const ClusterShape wider = cluster_shape_at(C, lanes, S2, M, k, Beff);
            if (wider.S) sh = wider;
        }
    }
    // a batch takes passes one after another on each CTA; beyond a few the
    // grid-wide kernels, which spread a batch over every SM, are faster
    const uint64_t TC = (uint64_t)(kClThreads / lanes);
    if ((Beff + (uint64_t)sh.S * TC - 1) / ((uint64_t)sh.S * TC) > kClusterMaxPasses) return ClusterShape();
    return sh;
}

cudaError_t launch_cluster_insert(int C, int lanes, const ClusterShape &sh, int nclusters, cudaStream_t s,
                                  const ManyItem *items, const ManyItem &one) {
    if (sh.S < 1 || nclusters < 1) return cudaErrorInvalidValue;
    void (*fn)(const ManyItem *, const ManyItem, uint32_t, uint32_t, uint32_t) = nullptr;
    if (lanes == 4) {
        fn = C == 1 ? cluster_insert_kernel<1, 4> : C == 2 ? cluster_insert_kernel<2, 4> : cluster_insert_kernel<3, 4>;
    } else if (lanes == 8) {
        fn = C == 1 ? cluster_insert_kernel<1, 8> : C == 2 ? cluster_insert_kernel<2, 8> : cluster_insert_kernel<3, 8>;
    }
    if (!fn || C < 1 || C > 3 || !info_for(C, lanes).ok) return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(sh.S * nclusters), 1, 1);
    cfg.blockDim = dim3(kClThreads, 1, 1);
    cfg.dynamicSmemBytes = sh.smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)sh.S;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, fn, items, one, sh.slice, sh.rank_u16, sh.kpc);
}

}  // namespace bc
