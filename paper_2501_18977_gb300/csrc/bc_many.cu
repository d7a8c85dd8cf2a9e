// Many independent filters in one launch per phase (work-list execution).
//
// The work list holds one entry per filter (its addressing, hash multipliers,
// rank table, keys, batch size, choice scratch, counters, bitmap). Insertion
// proceeds in rounds: round r runs the r-th batch of every filter that has
// one, as a choose phase, a grid barrier, a set phase and another barrier, so
// each filter sees exactly its own batch rule. Work inside a phase is cut
// into tiles of kTile keys of one filter; warps take tiles in turn and find a
// tile's filter by binary search over the round's tile prefix sums.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <utility>
#include <vector>

#include "bc_filter.h"
#include "bc_launch.h"
#include "bc_phases.cuh"

namespace bc {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
// Default keys per insert tile (a class tuning may choose another): one tile
// per warp at the grid's 1024 keys of a round per CTA. Tiles of 512 keys left
// three warps in four idle and measured 13.8 ms for the 256-filter workload
// against 11.7 with 128 (64: 11.8).
constexpr uint64_t kTile = 128;

// Index of the tile's item: the last f with prefix[f] <= t (prefix has
// nitems + 1 ascending entries, prefix[0] = 0).
__device__ __forceinline__ uint32_t find_item(const uint32_t *prefix, uint32_t nitems, uint32_t t) {
    uint32_t lo = 0, hi = nitems;  // answer in [lo, hi)
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (__ldg(prefix + mid) <= t) lo = mid; else hi = mid;
    }
    return lo;
}

// Copies the item's addressing (not its bit multipliers) into registers and
// its bit multipliers into the warp's shared slot.
__device__ __forceinline__ void load_item(const ManyItem *it, DevFilter &f, uint64_t *s_amul, int lane) {
    f.words = it->f.words;
    f.M = it->f.M;
    f.k = it->f.k;
    f.range_kind = it->f.range_kind;
    f.shift = it->f.shift;
    f.c = it->f.c;
    f.bitsel = it->f.bitsel;
    f.mod_mul = it->f.mod_mul;
    f.a_block[0] = it->f.a_block[0];
    f.a_block[1] = it->f.a_block[1];
    f.a_block[2] = it->f.a_block[2];
    __syncwarp();
    if ((uint32_t)lane < f.k) s_amul[lane] = it->f.a_bit[lane];
    __syncwarp();
}

// BITSEL: some item of the launch uses distinct bit selection; POW2: every
// item's block count is a power of two. The instances without a path compile
// it out (as in the single-filter kernels: inlined runtime branches cost the
// hot path registers).
template <int C, int LANES, bool BITSEL, bool POW2>
__global__ void __launch_bounds__(kThreads) insert_many_kernel(const ManyItem *__restrict__ items, uint32_t nitems,
                                                               const uint32_t *__restrict__ prefix,
                                                               uint32_t nrounds, uint32_t tile,
                                                               unsigned int *bar, unsigned long long *err) {
    constexpr int G = 32 / LANES;
    constexpr int W = kBlockWords / LANES;
    __shared__ uint64_t s_amul[kWarps][32];
    __shared__ __align__(16) uint32_t s_mask[kWarps * mask_u32_per_warp<LANES>()];
    const int lane = threadIdx.x & 31, q = lane % LANES, g = lane / LANES;
    const int wib = threadIdx.x >> 5;
    uint32_t *region = warp_mask_area<LANES>(s_mask, wib);
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    unsigned int target = 0;
    for (uint32_t r = 0; r < nrounds; ++r) {
        const uint32_t *pre = prefix + (uint64_t)r * (nitems + 1);
        const uint32_t ntiles = __ldg(pre + nitems);
        for (int phase = 0; phase < 2; ++phase) {
            for (uint32_t t = warp; t < ntiles; t += nwarps) {
                const uint32_t fi = find_item(pre, nitems, t);
                const ManyItem *it = items + fi;
                DevFilter f;
                load_item(it, f, s_amul[wib], lane);
                if constexpr (!BITSEL) f.bitsel = 0;
                if constexpr (POW2) f.range_kind = kRangePow2;
                const uint64_t B = it->B, n = it->n;
                const uint64_t bstart = (uint64_t)r * B;
                const uint64_t bend = bstart + B < n ? bstart + B : n;
                const uint64_t start = bstart + (uint64_t)(t - __ldg(pre + fi)) * tile;
                const uint64_t cnt = bend - start < tile ? bend - start : (uint64_t)tile;
                uint32_t ins = 0, skp = 0;
                for (uint64_t base = 0; base < cnt; base += G) {
                    const uint64_t i = start + base + g;  // key index within the filter
                    if (phase == 0) {
                        const bool valid = base + g < cnt;
                        const uint64_t x = valid ? load_key(it->keys + i) : 0ull;
                        uint64_t m[W];
                        const uint32_t s = choose_key<C, LANES, kLoadCG>(f, x, valid, q, it->rank, s_amul[wib], region, m);
                        if (valid && q == 0) {
                            it->sel[i - bstart] = (uint8_t)s;
                            if (s == kSkip) ++skp; else ++ins;
                        }
                    } else {
                        const uint32_t s = base + g < cnt ? (uint32_t)__ldcg(it->sel + (i - bstart)) : kSkip;
                        const uint64_t x = base + g < cnt ? load_key(it->keys + i) : 0ull;
                        uint64_t m[W];
                        key_mask_shared<LANES>(s_amul[wib], f.k, x, q, region, m, f.bitsel);
                        if (s != kSkip) set_one<LANES>(f, block_addr(f, block_mult(f, s), x), q, m);
                    }
                }
                if (phase == 0) {
#pragma unroll
                    for (int sh = 16; sh > 0; sh >>= 1) {
                        ins += __shfl_xor_sync(kFull, ins, sh);
                        skp += __shfl_xor_sync(kFull, skp, sh);
                    }
                    if (lane == 0) {
                        if (ins) atomicAdd(&it->counters[0], (unsigned long long)ins);
                        if (skp) atomicAdd(&it->counters[1], (unsigned long long)skp);
                    }
                }
            }
            if (phase == 1 && r + 1 == nrounds) break;
            target += gridDim.x;
            if (!grid_barrier(bar, target, err)) return;
        }
    }
}

template <int C, int LANES, int MODE, bool BITSEL, bool POW2>
__global__ void __launch_bounds__(kThreads) query_many_kernel(const ManyItem *__restrict__ items, uint32_t nitems,
                                                              const uint32_t *__restrict__ prefix) {
    __shared__ uint64_t s_amul[kWarps][32];
    __shared__ __align__(16) uint32_t s_mask[kWarps * mask_u32_per_warp<LANES>()];
    const int lane = threadIdx.x & 31, q = lane % LANES, g = lane / LANES;
    const int wib = threadIdx.x >> 5;
    uint32_t *region = warp_mask_area<LANES>(s_mask, wib);
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    const uint32_t ntiles = __ldg(prefix + nitems);
    uint32_t cur = 0xFFFFFFFFu;
    DevFilter f;
    const ManyItem *it = items;
    for (uint32_t t = warp; t < ntiles; t += nwarps) {
        const uint32_t fi = find_item(prefix, nitems, t);
        if (fi != cur) {
            it = items + fi;
            load_item(it, f, s_amul[wib], lane);
            if constexpr (!BITSEL) f.bitsel = 0;
            if constexpr (POW2) f.range_kind = kRangePow2;
            cur = fi;
        }
        const uint64_t wd = t - __ldg(prefix + fi);
        const uint64_t word = query_word<C, LANES, MODE>(f, it->keys, it->n, wd, s_amul[wib], region, q, g);
        if (lane == 0) it->bitmap[wd] = word;
    }
}

template <int C, int LANES, bool BITSEL, bool POW2>
cudaError_t insert_many_launch(int grid, cudaStream_t s, const ManyItem *items, uint32_t nitems,
                               const uint32_t *prefix, uint32_t nrounds, uint32_t tile, unsigned int *bar,
                               unsigned long long *err, int sms) {
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, insert_many_kernel<C, LANES, BITSEL, POW2>,
                                                                  kThreads, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int g = std::min(std::max(grid, 1), per_sm * sms);
    e = cudaMemsetAsync(bar, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    void *args[] = {(void *)&items, (void *)&nitems, (void *)&prefix, (void *)&nrounds, (void *)&tile,
                    (void *)&bar, (void *)&err};
    return cudaLaunchCooperativeKernel((const void *)insert_many_kernel<C, LANES, BITSEL, POW2>, dim3(g), dim3(kThreads),
                                       args, 0, s);
}

template <int C, bool BITSEL, bool POW2>
cudaError_t insert_many_lanes(int lanes, int grid, cudaStream_t s, const ManyItem *items, uint32_t nitems,
                              const uint32_t *prefix, uint32_t nrounds, uint32_t tile, unsigned int *bar,
                              unsigned long long *err, int sms) {
    switch (lanes) {
        case 1: return insert_many_launch<C, 1, BITSEL, POW2>(grid, s, items, nitems, prefix, nrounds, tile, bar, err, sms);
        case 2: return insert_many_launch<C, 2, BITSEL, POW2>(grid, s, items, nitems, prefix, nrounds, tile, bar, err, sms);
        case 4: return insert_many_launch<C, 4, BITSEL, POW2>(grid, s, items, nitems, prefix, nrounds, tile, bar, err, sms);
        case 8: return insert_many_launch<C, 8, BITSEL, POW2>(grid, s, items, nitems, prefix, nrounds, tile, bar, err, sms);
        default: return cudaErrorInvalidValue;
    }
}

// The instance for the launch's items (distinct selection always takes the
// general addressing).
template <int C>
cudaError_t insert_many_dispatch(int lanes, bool bitsel, bool pow2, int grid, cudaStream_t s, const ManyItem *items,
                                 uint32_t nitems, const uint32_t *prefix, uint32_t nrounds, uint32_t tile,
                                 unsigned int *bar, unsigned long long *err, int sms) {
    if (bitsel) return insert_many_lanes<C, true, false>(lanes, grid, s, items, nitems, prefix, nrounds, tile, bar, err, sms);
    if (pow2) return insert_many_lanes<C, false, true>(lanes, grid, s, items, nitems, prefix, nrounds, tile, bar, err, sms);
    return insert_many_lanes<C, false, false>(lanes, grid, s, items, nitems, prefix, nrounds, tile, bar, err, sms);
}

template <int C, int MODE, bool BITSEL, bool POW2>
cudaError_t query_many_lanes(int lanes, int grid, cudaStream_t s, const ManyItem *items, uint32_t nitems,
                             const uint32_t *prefix) {
    switch (lanes) {
        case 1: query_many_kernel<C, 1, MODE, BITSEL, POW2><<<grid, kThreads, 0, s>>>(items, nitems, prefix); break;
        case 2: query_many_kernel<C, 2, MODE, BITSEL, POW2><<<grid, kThreads, 0, s>>>(items, nitems, prefix); break;
        case 4: query_many_kernel<C, 4, MODE, BITSEL, POW2><<<grid, kThreads, 0, s>>>(items, nitems, prefix); break;
        case 8: query_many_kernel<C, 8, MODE, BITSEL, POW2><<<grid, kThreads, 0, s>>>(items, nitems, prefix); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int C, int MODE>
cudaError_t query_many_dispatch(int lanes, bool bitsel, bool pow2, int grid, cudaStream_t s, const ManyItem *items,
                                uint32_t nitems, const uint32_t *prefix) {
    if (bitsel) return query_many_lanes<C, MODE, true, false>(lanes, grid, s, items, nitems, prefix);
    if (pow2) return query_many_lanes<C, MODE, false, true>(lanes, grid, s, items, nitems, prefix);
    return query_many_lanes<C, MODE, false, false>(lanes, grid, s, items, nitems, prefix);
}

}  // namespace

cudaError_t launch_insert_many(int C, int lanes, bool bitsel, bool pow2, int grid, cudaStream_t s,
                               const ManyItem *items, uint32_t nitems, const uint32_t *prefix, uint32_t nrounds,
                               uint32_t tile, unsigned int *bar, unsigned long long *err, int sms) {
    switch (C) {
        case 1: return insert_many_dispatch<1>(lanes, bitsel, pow2, grid, s, items, nitems, prefix, nrounds, tile, bar, err, sms);
        case 2: return insert_many_dispatch<2>(lanes, bitsel, pow2, grid, s, items, nitems, prefix, nrounds, tile, bar, err, sms);
        case 3: return insert_many_dispatch<3>(lanes, bitsel, pow2, grid, s, items, nitems, prefix, nrounds, tile, bar, err, sms);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_query_many(int C, int lanes, bool early, bool bitsel, bool pow2, int grid, cudaStream_t s,
                              const ManyItem *items, uint32_t nitems, const uint32_t *prefix) {
    switch (C) {
        case 1: return query_many_dispatch<1, 0>(lanes, bitsel, pow2, grid, s, items, nitems, prefix);
        case 2: return early ? query_many_dispatch<2, 1>(lanes, bitsel, pow2, grid, s, items, nitems, prefix)
                             : query_many_dispatch<2, 0>(lanes, bitsel, pow2, grid, s, items, nitems, prefix);
        case 3: return early ? query_many_dispatch<3, 1>(lanes, bitsel, pow2, grid, s, items, nitems, prefix)
                             : query_many_dispatch<3, 0>(lanes, bitsel, pow2, grid, s, items, nitems, prefix);
        default: return cudaErrorInvalidValue;
    }
}

uint64_t many_tile() { return kTile; }

}  // namespace bc

// ---------------------------------------------------------------------------
// Host side: the batch object.

namespace {

using bc::ManyItem;

// One call's device work list, uploaded through a ring of pinned staging
// slots: a call reuses a slot only once the upload and launch that last used
// it have completed, so the host can prepare several calls ahead of the GPU.
constexpr int kStageSlots = 4;

struct ManyPlan {
    struct Group {
        int C;
        uint32_t item0, nitems;   // range in the item array
        size_t prefix0;           // offset in the prefix array
        uint32_t nrounds;         // insert only
        uint64_t keys;            // keys of the group's items
        int lanes;                // lanes per key of the group's launch
        uint32_t tile;            // insert: keys per tile
        int early;                // query: stop at the first candidate holding the key
        bool bitsel = false;      // some item uses distinct bit selection
        bool pow2 = true;         // every item's block count is a power of two
    };
    struct Slot {
        ManyItem *d_items = nullptr, *h_items = nullptr;
        size_t d_items_cap = 0, h_items_cap = 0;
        uint32_t *d_prefix = nullptr, *h_prefix = nullptr;
        size_t d_prefix_cap = 0, h_prefix_cap = 0;
        cudaEvent_t done = nullptr;  // the slot's last upload and launches completed
        cudaStream_t last = nullptr;  // stream of the slot's last use
    };
    Slot slots[kStageSlots];
    int cur = 0;                     // slot of the prepared call
    uint8_t *d_sel = nullptr;
    size_t sel_cap = 0;
    cudaStream_t sel_last = nullptr;
    std::vector<Group> groups;
    struct ClusterGroup {         // items inserted cluster-resident, one cluster each
        int C;
        bc::ClusterShape sh;
        uint32_t item0, nitems;   // range in the item array
    };
    std::vector<ClusterGroup> cgroups;
    std::vector<blowchoc_work> side;  // items run by the single-filter kernels
    std::vector<int> side_mode;       // per side item: -1 the filter's own tuning, else its set_mode
};

void free_plan(ManyPlan &p) {
    for (ManyPlan::Slot &sl : p.slots) {
        cudaFree(sl.d_items);
        cudaFree(sl.d_prefix);
        cudaFreeHost(sl.h_items);
        cudaFreeHost(sl.h_prefix);
        if (sl.done) cudaEventDestroy(sl.done);
    }
    cudaFree(p.d_sel);
    p = ManyPlan();
}

}  // namespace

struct blowchoc_batch {
    int device = 0;
    int sms = 0;
    unsigned long long *d_state = nullptr;  // [0] error word, [1] barrier arrivals (u32)
    ManyPlan live_ins, live_qry, rec_ins, rec_qry;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int lanes_choose = 1, lanes_query = 1, query_early = 1, ctas_per_sm = 8;  // one lane per key: 14.3 ms against 18.7 (256 filters)
    // cluster-resident items are off by default here: a work list of many
    // filters spreads every round over all SMs, which measured faster than one
    // cluster per filter (256 lognormal filters: 18.3 ms against 20.8-33 ms)
    int cluster_max = 0, lanes_cluster = 8, cluster_keys = 128;
    uint64_t l2_bytes = 0;  // the device's L2, for the size classes
    std::map<uint64_t, blowchoc_class_tuning> ctune;  // per (size class, k, c)
};

namespace {

// A launch runs as many rounds as its item with the most batches. An item
// that inserts one key at a time (B = 1), or needs more than
// max(kManyMinRounds, 4 x the median round count of the call) rounds, runs
// through the single-filter kernels on the same stream instead, so that it
// does not hold every other item of the launch behind its rounds.
constexpr uint64_t kManyMinRounds = 64;
constexpr uint64_t kManyWarpsPerCta = 8;  // the work-list kernels' 256-thread CTAs

uint32_t size_class_of(const blowchoc_batch *b, uint64_t M) {
    const uint64_t bytes = 64 * M;
    const uint64_t l2 = b->l2_bytes ? b->l2_bytes : (126ull << 20);
    if (bytes <= l2 / 16) return BLOWCHOC_CLASS_CACHE;
    if (bytes <= l2 / 2) return BLOWCHOC_CLASS_L2;
    if (bytes <= 2 * l2) return BLOWCHOC_CLASS_SPILL;
    return BLOWCHOC_CLASS_HBM;
}

uint64_t class_key(uint32_t cls, uint32_t k, uint32_t c) {
    return ((uint64_t)cls << 40) | ((uint64_t)k << 8) | (uint64_t)c;
}

blowchoc_class_tuning default_class(const blowchoc_batch *b) {
    blowchoc_class_tuning t;
    t.route = BLOWCHOC_ROUTE_WORKLIST;
    t.lanes_choose = (uint32_t)b->lanes_choose;
    t.tile = (uint32_t)bc::many_tile();
    t.lanes_query = (uint32_t)b->lanes_query;
    t.query_early = (uint32_t)b->query_early;
    return t;
}

// The configuration a filter runs with in a many-filter call.
blowchoc_class_tuning class_tuning(const blowchoc_batch *b, const blowchoc_filter *f) {
    const auto it = b->ctune.find(class_key(size_class_of(b, f->dev.M), f->dev.k, f->p.choices));
    return it == b->ctune.end() ? default_class(b) : it->second;
}

uint64_t rounds_of(const blowchoc_work &w) {
    const uint64_t B = w.filter->p.batch;
    return (w.n + B - 1) / B;
}

uint64_t round_cap(const blowchoc_work *items, uint32_t count) {
    std::vector<uint64_t> r;
    for (uint32_t i = 0; i < count; ++i)
        if (items[i].n) r.push_back(rounds_of(items[i]));
    if (r.empty()) return kManyMinRounds;
    std::nth_element(r.begin(), r.begin() + r.size() / 2, r.end());
    return std::max<uint64_t>(kManyMinRounds, 4 * r[r.size() / 2]);
}

bool side_path(const blowchoc_work &w, uint64_t cap) {
    return w.filter->p.batch == 1 || rounds_of(w) > cap;
}

int set_err(int code, const char *msg) { return bc_set_error(code, msg); }

int cuda_err(cudaError_t e, const char *what) {
    char msg[256];
    std::snprintf(msg, sizeof msg, "%s: %s", what, cudaGetErrorString(e));
    return bc_set_error(e == cudaErrorMemoryAllocation ? BLOWCHOC_ENOMEM : BLOWCHOC_ECUDA, msg);
}

#define MANY_CUDA(call, what)                                \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return cuda_err(e_, what);    \
    } while (0)

// Grows a device buffer with stream-ordered allocation: the old buffer is
// released after the work already queued on `last` (its last user), the new
// one is allocated on `s`. No device-wide synchronisation.
template <typename T>
int grow_device(T *&ptr, size_t &cap, size_t need, cudaStream_t s, cudaStream_t &last, const char *what) {
    if (need <= cap) {
        last = s;
        return BLOWCHOC_OK;
    }
    if (ptr) {
        if (last != s) {
            // order the release after the last user's work, seen from `s`
            cudaEvent_t ev;
            MANY_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), what);
            MANY_CUDA(cudaEventRecord(ev, last), what);
            MANY_CUDA(cudaStreamWaitEvent(s, ev, 0), what);
            cudaEventDestroy(ev);
        }
        MANY_CUDA(cudaFreeAsync(ptr, s), what);
    }
    ptr = nullptr;
    const size_t n = std::max(need, cap * 2);
    cap = 0;
    MANY_CUDA(cudaMallocAsync((void **)&ptr, n * sizeof(T), s), what);
    cap = n;
    last = s;
    return BLOWCHOC_OK;
}

template <typename T>
int grow_host(T *&ptr, size_t &cap, size_t need, const char *what) {
    if (need <= cap) return BLOWCHOC_OK;
    cudaFreeHost(ptr);
    ptr = nullptr;
    const size_t n = std::max(need, cap * 2);
    cap = 0;
    MANY_CUDA(cudaHostAlloc((void **)&ptr, n * sizeof(T), cudaHostAllocDefault), what);
    cap = n;
    return BLOWCHOC_OK;
}

int check_items(const blowchoc_batch *b, const blowchoc_work *items, uint32_t count, bool query) {
    if (!b) return set_err(BLOWCHOC_EINVAL, "batch is NULL");
    if (count && !items) return set_err(BLOWCHOC_EINVAL, "items is NULL");
    std::vector<const blowchoc_filter *> seen;
    seen.reserve(count);
    for (uint32_t i = 0; i < count; ++i) {
        const blowchoc_work &w = items[i];
        if (!w.filter) return set_err(BLOWCHOC_EINVAL, "item without a filter");
        if (w.n && !w.d_keys) return set_err(BLOWCHOC_EINVAL, "item keys are NULL");
        if (query && w.n && !w.d_bitmap) return set_err(BLOWCHOC_EINVAL, "item bitmap is NULL");
        if (w.filter->device != b->device) return set_err(BLOWCHOC_EINVAL, "item filter is on another device");
        seen.push_back(w.filter);
    }
    std::sort(seen.begin(), seen.end());
    if (std::adjacent_find(seen.begin(), seen.end()) != seen.end())
        return set_err(BLOWCHOC_EINVAL, "a filter appears twice in one many-filter call");
    return BLOWCHOC_OK;
}

ManyItem make_item(const blowchoc_work &w) {
    ManyItem it;
    std::memset(&it, 0, sizeof it);
    it.f = w.filter->dev;
    it.rank = w.filter->d_rank;
    it.keys = w.d_keys;
    it.n = w.n;
    it.B = w.filter->p.batch;
    it.counters = w.filter->d_counters;
    it.bitmap = w.d_bitmap;
    return it;
}

// Builds one call's work list into `p` and uploads it on stream `s`: from
// pinned staging, asynchronously; or with a synchronous copy if `sync`.
int prepare(const blowchoc_batch *b, ManyPlan &p, const blowchoc_work *items, uint32_t count, bool query,
            cudaStream_t s, bool sync) {
    p.cur = (p.cur + 1) % kStageSlots;
    ManyPlan::Slot &sl = p.slots[p.cur];
    if (sl.done) MANY_CUDA(cudaEventSynchronize(sl.done), "batch staging");
    else MANY_CUDA(cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming), "batch event");
    p.groups.clear();
    p.cgroups.clear();
    p.side.clear();
    p.side_mode.clear();
    std::vector<ManyItem> list;
    std::vector<uint32_t> prefix;
    const uint64_t cap = query ? 0 : round_cap(items, count);
    for (int C = 1; C <= 3; ++C) {
        // work-list items by launch configuration: (lanes, tile) for inserts,
        // (lanes, early exit) for queries, from each filter's class tuning
        std::map<std::pair<int, uint32_t>, std::vector<ManyItem>> buckets;
        std::vector<std::pair<int, ManyItem>> clustered;  // (CTAs per cluster, item)
        for (uint32_t i = 0; i < count; ++i) {
            const blowchoc_work &w = items[i];
            if ((int)w.filter->p.choices != C || w.n == 0) continue;
            if (!query && b->cluster_max > 0 && w.filter->p.batch >= 2 &&
                rounds_of(w) >= bc::kClusterMinRounds) {
                const bc::ClusterShape sh =
                    bc::cluster_shape(C, b->lanes_cluster, w.filter->dev.M, w.filter->dev.k,
                                      std::min<uint64_t>(w.filter->p.batch, w.n), b->cluster_max,
                                      (uint64_t)b->cluster_keys);
                if (sh.S) {
                    clustered.emplace_back(sh.S, make_item(w));
                    continue;
                }
            }
            if (!query && side_path(w, cap)) {
                p.side.push_back(w);
                p.side_mode.push_back(-1);
                continue;
            }
            const blowchoc_class_tuning ct = class_tuning(b, w.filter);
            if (!query && ct.route != BLOWCHOC_ROUTE_WORKLIST) {
                p.side.push_back(w);
                p.side_mode.push_back(ct.route == BLOWCHOC_ROUTE_SORTED ? 1 : 0);
                continue;
            }
            const std::pair<int, uint32_t> key =
                query ? std::make_pair((int)ct.lanes_query, ct.query_early) : std::make_pair((int)ct.lanes_choose, ct.tile);
            buckets[key].push_back(make_item(w));
        }
        // clustered items: launches of equal cluster size, packed while one
        // shared-memory layout (largest slice, rank table, choice bytes) fits
        std::stable_sort(clustered.begin(), clustered.end(),
                         [](const std::pair<int, ManyItem> &a, const std::pair<int, ManyItem> &c) {
                             return a.first < c.first;
                         });
        for (size_t i = 0; i < clustered.size();) {
            const int S = clustered[i].first;
            uint64_t Mx = 0, Bx = 0;
            uint32_t kx = 0;
            ManyPlan::ClusterGroup cg{C, bc::ClusterShape(), (uint32_t)list.size(), 0};
            while (i < clustered.size() && clustered[i].first == S) {
                const ManyItem &it = clustered[i].second;
                const uint64_t M2 = std::max(Mx, it.f.M), B2 = std::max(Bx, std::min(it.B, it.n));
                const uint32_t k2 = std::max(kx, it.f.k);
                const bc::ClusterShape sh = bc::cluster_shape_at(C, b->lanes_cluster, S, M2, k2, B2);
                if (!sh.S) break;  // does not fit with the group: it starts the next one
                Mx = M2;
                Bx = B2;
                kx = k2;
                cg.sh = sh;
                list.push_back(it);
                ++cg.nitems;
                ++i;
            }
            p.cgroups.push_back(cg);
        }
        for (auto &kv : buckets) {
            std::vector<ManyItem> &mine = kv.second;
            ManyPlan::Group g{C, (uint32_t)list.size(), (uint32_t)mine.size(), prefix.size(), 0, 0,
                              kv.first.first, query ? 0u : kv.first.second, query ? (int)kv.first.second : 0};
            for (const ManyItem &it : mine) {
                g.keys += it.n;
                g.bitsel = g.bitsel || it.f.bitsel != 0;
                g.pow2 = g.pow2 && it.f.range_kind == bc::kRangePow2;
            }
            if (query) {
                prefix.push_back(0);
                for (const ManyItem &it : mine) {
                    const uint64_t next = prefix.back() + (it.n + 63) / 64;
                    if (next > 0xFFFFFFFFull) return set_err(BLOWCHOC_EINVAL, "work list too large");
                    prefix.push_back((uint32_t)next);
                }
            } else {
                uint64_t rounds = 0;
                for (const ManyItem &it : mine) rounds = std::max<uint64_t>(rounds, (it.n + it.B - 1) / it.B);
                if (rounds > (1u << 24)) return set_err(BLOWCHOC_EINVAL, "too many batches in one call");
                g.nrounds = (uint32_t)rounds;
                const uint64_t T = g.tile;
                for (uint64_t r = 0; r < rounds; ++r) {
                    prefix.push_back(0);
                    for (const ManyItem &it : mine) {
                        const uint64_t s0 = r * it.B;
                        const uint64_t cnt = s0 < it.n ? std::min(it.B, it.n - s0) : 0;
                        const uint64_t next = prefix.back() + (cnt + T - 1) / T;
                        if (next > 0xFFFFFFFFull) return set_err(BLOWCHOC_EINVAL, "work list too large");
                        prefix.push_back((uint32_t)next);
                    }
                }
            }
            list.insert(list.end(), mine.begin(), mine.end());
            p.groups.push_back(g);
        }
    }
    int rc = BLOWCHOC_OK;
    if (!query) {
        // choice bytes of one batch per work-list item, 16-byte aligned slices
        size_t sel_total = 0;
        for (const ManyPlan::Group &g : p.groups)
            for (uint32_t i = 0; i < g.nitems; ++i) {
                const ManyItem &it = list[g.item0 + i];
                sel_total += (std::min(it.B, it.n) + 15) & ~uint64_t(15);
            }
        if (sel_total) {
            rc = grow_device(p.d_sel, p.sel_cap, sel_total, s, p.sel_last, "batch choice scratch");
            if (rc) return rc;
            size_t off = 0;
            for (const ManyPlan::Group &g : p.groups)
                for (uint32_t i = 0; i < g.nitems; ++i) {
                    ManyItem &it = list[g.item0 + i];
                    it.sel = p.d_sel + off;
                    off += (std::min(it.B, it.n) + 15) & ~uint64_t(15);
                }
        }
    }
    if (list.empty()) return BLOWCHOC_OK;
    cudaStream_t last_items = sl.last, last_prefix = sl.last;
    rc = grow_device(sl.d_items, sl.d_items_cap, list.size(), s, last_items, "batch work list");
    if (!rc) rc = grow_device(sl.d_prefix, sl.d_prefix_cap, prefix.size(), s, last_prefix, "batch tile table");
    sl.last = s;
    if (rc) return rc;
    if (sync) {
        MANY_CUDA(cudaStreamSynchronize(s), "batch work list");
        MANY_CUDA(cudaMemcpy(sl.d_items, list.data(), list.size() * sizeof(ManyItem), cudaMemcpyHostToDevice),
                  "upload work list");
        MANY_CUDA(cudaMemcpy(sl.d_prefix, prefix.data(), prefix.size() * sizeof(uint32_t), cudaMemcpyHostToDevice),
                  "upload tile table");
        return BLOWCHOC_OK;
    }
    rc = grow_host(sl.h_items, sl.h_items_cap, list.size(), "batch staging");
    if (!rc) rc = grow_host(sl.h_prefix, sl.h_prefix_cap, prefix.size(), "batch staging");
    if (rc) return rc;
    std::memcpy(sl.h_items, list.data(), list.size() * sizeof(ManyItem));
    std::memcpy(sl.h_prefix, prefix.data(), prefix.size() * sizeof(uint32_t));
    MANY_CUDA(cudaMemcpyAsync(sl.d_items, sl.h_items, list.size() * sizeof(ManyItem), cudaMemcpyHostToDevice, s),
              "upload work list");
    MANY_CUDA(cudaMemcpyAsync(sl.d_prefix, sl.h_prefix, prefix.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, s),
              "upload tile table");
    return BLOWCHOC_OK;
}

// Queues the prepared work on stream `s` and marks its staging slot.
int launch(blowchoc_batch *b, const ManyPlan &p, bool query, cudaStream_t s, bool mark = true) {
    unsigned long long *err = b->d_state;
    unsigned int *bar = reinterpret_cast<unsigned int *>(b->d_state + 1);
    const ManyPlan::Slot &sl = p.slots[p.cur];
    if (!query) {
        ManyItem none;
        std::memset(&none, 0, sizeof none);
        for (const ManyPlan::ClusterGroup &g : p.cgroups) {
            const cudaError_t e =
                bc::launch_cluster_insert(g.C, b->lanes_cluster, g.sh, (int)g.nitems, s, sl.d_items + g.item0, none);
            if (e != cudaSuccess) return cuda_err(e, "cluster insert launch");
            bc_note_launch();
        }
    }
    for (const ManyPlan::Group &g : p.groups) {
        const ManyItem *items = sl.d_items + g.item0;
        const uint32_t *prefix = sl.d_prefix + g.prefix0;
        // insert: about one tile of a round per warp, so that rounds with
        // little work meet at cheap barriers
        int grid = b->sms * b->ctas_per_sm;
        if (!query && g.nrounds) {
            const uint64_t per_round = (g.keys + g.nrounds - 1) / g.nrounds;
            const uint64_t per_cta = (uint64_t)g.tile * kManyWarpsPerCta;
            grid = (int)std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)grid, (per_round + per_cta - 1) / per_cta));
        }
        cudaError_t e;
        if (query)
            e = bc::launch_query_many(g.C, g.lanes, g.early != 0, g.bitsel, g.pow2, grid, s, items, g.nitems, prefix);
        else
            e = bc::launch_insert_many(g.C, g.lanes, g.bitsel, g.pow2, grid, s, items, g.nitems, prefix, g.nrounds, g.tile,
                                       bar, err,
                                       b->sms);
        if (e != cudaSuccess) return cuda_err(e, query ? "query_many launch" : "insert_many launch");
        bc_note_launch();
    }
    for (size_t i = 0; i < p.side.size(); ++i) {
        const blowchoc_work &w = p.side[i];
        blowchoc_filter *f = w.filter;
        int rc;
        if (p.side_mode[i] < 0) {
            rc = blowchoc_insert(f, w.d_keys, w.n, s);
        } else {
            // a routed class: the single-filter insert with the class's set
            // (host-side launch fields, restored once the launch is queued)
            const int set_mode = f->set_mode, persistent = f->persistent;
            f->set_mode = p.side_mode[i];
            f->persistent = 1;
            rc = blowchoc_insert(f, w.d_keys, w.n, s);
            f->set_mode = set_mode;
            f->persistent = persistent;
        }
        if (rc) return rc;
    }
    if (mark) MANY_CUDA(cudaEventRecord(sl.done, s), "batch event");
    return BLOWCHOC_OK;
}

int run_many(blowchoc_batch *b, ManyPlan &p, const blowchoc_work *items, uint32_t count, bool query,
             cudaStream_t s) {
    int rc = check_items(b, items, count, query);
    if (rc) return rc;
    if (count == 0) return BLOWCHOC_OK;
    rc = prepare(b, p, items, count, query, s, false);
    if (rc) return rc;
    return launch(b, p, query, s);
}

bool lanes_ok(uint32_t l) { return l == 1 || l == 2 || l == 4 || l == 8; }

int check_class_tuning(const blowchoc_class_tuning *t) {
    if (t->route > BLOWCHOC_ROUTE_SORTED) return set_err(BLOWCHOC_EINVAL, "route must be 0, 1 or 2");
    if (!lanes_ok(t->lanes_choose) || !lanes_ok(t->lanes_query))
        return set_err(BLOWCHOC_EINVAL, "lanes must be 1, 2, 4 or 8");
    if (t->tile < 32 || t->tile > 1024 || (t->tile & (t->tile - 1)))
        return set_err(BLOWCHOC_EINVAL, "tile must be a power of two in 32..1024");
    if (t->query_early > 1) return set_err(BLOWCHOC_EINVAL, "query_early must be 0 or 1");
    return BLOWCHOC_OK;
}

bool class_args_ok(uint32_t cls, uint32_t k, uint32_t c) {
    return cls < BLOWCHOC_NUM_CLASSES && k >= 1 && k <= 32 && c >= 1 && c <= 3;
}

}  // namespace

extern "C" {

int blowchoc_batch_create(blowchoc_batch **out) {
    if (!out) return set_err(BLOWCHOC_EINVAL, "out is NULL");
    *out = nullptr;
    blowchoc_batch *b = new blowchoc_batch();
    cudaError_t e = cudaGetDevice(&b->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device);
    int l2 = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, b->device);
    b->l2_bytes = (uint64_t)(l2 > 0 ? l2 : 0);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_state, 4 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(b->d_state, 0, 4 * sizeof(unsigned long long));
    if (e != cudaSuccess) {
        cudaFree(b->d_state);
        delete b;
        return cuda_err(e, "blowchoc_batch_create");
    }
    *out = b;
    return BLOWCHOC_OK;
}

int blowchoc_batch_destroy(blowchoc_batch *b) {
    if (!b) return BLOWCHOC_OK;
    cudaError_t e = cudaDeviceSynchronize();
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    free_plan(b->live_ins);
    free_plan(b->live_qry);
    free_plan(b->rec_ins);
    free_plan(b->rec_qry);
    cudaFree(b->d_state);
    delete b;
    if (e != cudaSuccess) return cuda_err(e, "blowchoc_batch_destroy");
    return BLOWCHOC_OK;
}

int blowchoc_insert_many(blowchoc_batch *b, const blowchoc_work *items, uint32_t count, void *stream) {
    if (!b) return set_err(BLOWCHOC_EINVAL, "batch is NULL");
    return run_many(b, b->live_ins, items, count, false, (cudaStream_t)stream);
}

int blowchoc_query_many(blowchoc_batch *b, const blowchoc_work *items, uint32_t count, void *stream) {
    if (!b) return set_err(BLOWCHOC_EINVAL, "batch is NULL");
    return run_many(b, b->live_qry, items, count, true, (cudaStream_t)stream);
}

int blowchoc_batch_record(blowchoc_batch *b, const blowchoc_work *ins, uint32_t n_ins,
                          const blowchoc_work *qry, uint32_t n_qry) {
    if (!b) return set_err(BLOWCHOC_EINVAL, "batch is NULL");
    int rc = check_items(b, ins, n_ins, false);
    if (!rc) rc = check_items(b, qry, n_qry, true);
    if (rc) return rc;
    if (n_ins) rc = prepare(b, b->rec_ins, ins, n_ins, false, nullptr, true);
    if (!rc && n_qry) rc = prepare(b, b->rec_qry, qry, n_qry, true, nullptr, true);
    // the single-filter inserts of side items allocate their scratch on first
    // use, which a capture does not allow: allocate it now, with the launch
    // fields each will run with
    for (size_t i = 0; !rc && i < b->rec_ins.side.size(); ++i) {
        const blowchoc_work &w = b->rec_ins.side[i];
        blowchoc_filter *f = w.filter;
        const int set_mode = f->set_mode, persistent = f->persistent;
        if (b->rec_ins.side_mode[i] >= 0) {
            f->set_mode = b->rec_ins.side_mode[i];
            f->persistent = 1;
        }
        rc = bc_reserve_insert_scratch(f, w.n);
        f->set_mode = set_mode;
        f->persistent = persistent;
    }
    if (rc) return rc;
    if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
    if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
    cudaStream_t cs;
    MANY_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "record stream");
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        cudaStreamDestroy(cs);
        return cuda_err(e, "begin capture");
    }
    if (n_ins) rc = launch(b, b->rec_ins, false, cs, false);
    if (!rc && n_qry) rc = launch(b, b->rec_qry, true, cs, false);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(cs, &g);
    cudaStreamDestroy(cs);
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return cuda_err(e, "end capture");
    e = cudaGraphInstantiate(&b->exec, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return cuda_err(e, "graph instantiate");
    }
    b->graph = g;
    return BLOWCHOC_OK;
}

int blowchoc_batch_replay(blowchoc_batch *b, void *stream) {
    if (!b || !b->exec) return set_err(BLOWCHOC_EINVAL, "no recorded graph");
    MANY_CUDA(cudaGraphLaunch(b->exec, (cudaStream_t)stream), "graph launch");
    return BLOWCHOC_OK;
}

int blowchoc_batch_get_tuning(blowchoc_batch *b, blowchoc_tuning *out) {
    if (!b || !out) return set_err(BLOWCHOC_EINVAL, "NULL argument");
    out->lanes_choose = (uint32_t)b->lanes_choose;
    out->lanes_set = (uint32_t)b->lanes_choose;
    out->lanes_query = (uint32_t)b->lanes_query;
    out->query_early = (uint32_t)b->query_early;
    out->ctas_per_sm = (uint32_t)b->ctas_per_sm;
    out->persistent = 1;
    out->keys_per_cta = 0;
    out->set_mode = 0;
    out->seq_window = 0;
    out->cluster_max = (uint32_t)b->cluster_max;
    out->lanes_cluster = (uint32_t)b->lanes_cluster;
    out->cluster_keys = (uint32_t)b->cluster_keys;
    out->host_ring_keys = 0;
    return BLOWCHOC_OK;
}

int blowchoc_batch_set_tuning(blowchoc_batch *b, const blowchoc_tuning *t) {
    if (!b || !t) return set_err(BLOWCHOC_EINVAL, "NULL argument");
    if (!lanes_ok(t->lanes_choose) || !lanes_ok(t->lanes_query))
        return set_err(BLOWCHOC_EINVAL, "lanes must be 1, 2, 4 or 8");
    if (t->query_early > 1) return set_err(BLOWCHOC_EINVAL, "query_early must be 0 or 1");
    if (t->ctas_per_sm < 1 || t->ctas_per_sm > 16) return set_err(BLOWCHOC_EINVAL, "ctas_per_sm must be in 1..16");
    if (t->cluster_max > 16) return set_err(BLOWCHOC_EINVAL, "cluster_max must be in 0..16");
    if (t->lanes_cluster != 4 && t->lanes_cluster != 8) return set_err(BLOWCHOC_EINVAL, "lanes_cluster must be 4 or 8");
    if (t->cluster_keys < 16 || t->cluster_keys > (1u << 20))
        return set_err(BLOWCHOC_EINVAL, "cluster_keys must be in 16..2^20");
    b->lanes_choose = (int)t->lanes_choose;
    b->cluster_max = (int)t->cluster_max;
    b->lanes_cluster = (int)t->lanes_cluster;
    b->cluster_keys = (int)t->cluster_keys;
    b->lanes_query = (int)t->lanes_query;
    b->query_early = (int)t->query_early;
    b->ctas_per_sm = (int)t->ctas_per_sm;
    return BLOWCHOC_OK;
}

int blowchoc_batch_size_class(blowchoc_batch *b, uint64_t nblocks, uint32_t *cls) {
    if (!b || !cls) return set_err(BLOWCHOC_EINVAL, "NULL argument");
    *cls = size_class_of(b, nblocks);
    return BLOWCHOC_OK;
}

int blowchoc_batch_get_class_tuning(blowchoc_batch *b, uint32_t cls, uint32_t k, uint32_t c,
                                    blowchoc_class_tuning *out, uint32_t *is_set) {
    if (!b || !out) return set_err(BLOWCHOC_EINVAL, "NULL argument");
    if (!class_args_ok(cls, k, c)) return set_err(BLOWCHOC_EINVAL, "class 0..3, k 1..32, c 1..3");
    const auto it = b->ctune.find(class_key(cls, k, c));
    *out = it == b->ctune.end() ? default_class(b) : it->second;
    if (is_set) *is_set = it == b->ctune.end() ? 0u : 1u;
    return BLOWCHOC_OK;
}

int blowchoc_batch_set_class_tuning(blowchoc_batch *b, uint32_t cls, uint32_t k, uint32_t c,
                                    const blowchoc_class_tuning *t) {
    if (!b || !t) return set_err(BLOWCHOC_EINVAL, "NULL argument");
    if (!class_args_ok(cls, k, c)) return set_err(BLOWCHOC_EINVAL, "class 0..3, k 1..32, c 1..3");
    const int rc = check_class_tuning(t);
    if (rc) return rc;
    b->ctune[class_key(cls, k, c)] = *t;
    return BLOWCHOC_OK;
}

int blowchoc_batch_clear_class_tuning(blowchoc_batch *b) {
    if (!b) return set_err(BLOWCHOC_EINVAL, "batch is NULL");
    b->ctune.clear();
    return BLOWCHOC_OK;
}

int blowchoc_batch_autotune(blowchoc_batch *b, const blowchoc_work *ins, uint32_t n_ins,
                            const blowchoc_work *qry, uint32_t n_qry, void *stream, blowchoc_tuning *best) {
    if (!b) return set_err(BLOWCHOC_EINVAL, "batch is NULL");
    int rc = check_items(b, ins, n_ins, false);
    if (!rc) rc = check_items(b, qry, n_qry, true);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    // scratch copies of every filter, so that the callers' filters stay untouched
    std::vector<blowchoc_filter *> scratch;
    std::vector<blowchoc_work> sins(ins, ins + n_ins), sqry(qry, qry + n_qry);
    auto clone = [&](blowchoc_filter *orig) -> blowchoc_filter * {
        for (size_t i = 0; i < scratch.size(); i += 2)
            if ((blowchoc_filter *)scratch[i + 1] == orig) return scratch[i];
        blowchoc_filter *c = nullptr;
        if (blowchoc_create(&orig->p, stream, &c)) return nullptr;
        scratch.push_back(c);
        scratch.push_back(orig);
        return c;
    };
    uint64_t bitmap_words = 0;
    for (auto &w : sqry) bitmap_words += (w.n + 63) / 64;
    uint64_t *d_bm = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (bitmap_words && cudaMalloc(&d_bm, bitmap_words * sizeof(uint64_t)) != cudaSuccess) {
        return set_err(BLOWCHOC_ENOMEM, "autotune bitmap");
    }
    rc = BLOWCHOC_OK;
    for (auto &w : sins) if (!rc && !(w.filter = clone(w.filter))) rc = BLOWCHOC_ENOMEM;
    uint64_t off = 0;
    for (auto &w : sqry) {
        if (!rc && !(w.filter = clone(w.filter))) rc = BLOWCHOC_ENOMEM;
        w.d_bitmap = d_bm + off;
        off += (w.n + 63) / 64;
    }
    if (!rc && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
        rc = set_err(BLOWCHOC_ECUDA, "autotune events");
    const int saved[4] = {b->lanes_choose, b->lanes_query, b->query_early, b->ctas_per_sm};
    const std::map<uint64_t, blowchoc_class_tuning> saved_classes = b->ctune;

    // Time of `wi` inserted then `wq` queried on cleared scratch filters, summed
    // over two repetitions after a warm-up; with query_only the inserts run
    // untimed before the timed queries.
    auto timed = [&](const std::vector<blowchoc_work> &wi, const std::vector<blowchoc_work> &wq,
                     bool query_only, float *out_ms) -> int {
        float total = 0.0f;
        for (int rep = 0; rep < 3; ++rep) {
            for (size_t i = 0; i < scratch.size(); i += 2) {
                const int r = blowchoc_clear(scratch[i], stream);
                if (r) return r;
            }
            int r = BLOWCHOC_OK;
            if (query_only && !wi.empty()) r = blowchoc_insert_many(b, wi.data(), (uint32_t)wi.size(), stream);
            if (r) return r;
            if (cudaEventRecord(e0, s) != cudaSuccess) return set_err(BLOWCHOC_ECUDA, "autotune event");
            if (!query_only && !wi.empty()) r = blowchoc_insert_many(b, wi.data(), (uint32_t)wi.size(), stream);
            if (!r && !wq.empty()) r = blowchoc_query_many(b, wq.data(), (uint32_t)wq.size(), stream);
            if (r) return r;
            if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess)
                return set_err(BLOWCHOC_ECUDA, "autotune sync");
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep) total += ms;
        }
        *out_ms = total;
        return BLOWCHOC_OK;
    };

    // 1. the batch object's tuning over the whole call, class tunings aside
    b->ctune.clear();
    float best_ms = -1.0f;
    int best_cfg[4] = {saved[0], saved[1], saved[2], saved[3]};
    const int lanes_c[] = {1, 2, 4}, lanes_q[] = {1, 2}, ctas[] = {4, 8};
    for (int lc : lanes_c)
        for (int lq : lanes_q)
            for (int cp : ctas) {
                if (rc) break;
                b->lanes_choose = lc;
                b->lanes_query = lq;
                b->query_early = 1;
                b->ctas_per_sm = cp;
                float ms = 0.0f;
                rc = timed(sins, sqry, false, &ms);
                if (!rc && (best_ms < 0.0f || ms < best_ms)) {
                    best_ms = ms;
                    best_cfg[0] = lc; best_cfg[1] = lq; best_cfg[2] = 1; best_cfg[3] = cp;
                }
            }
    if (!rc) {
        b->lanes_choose = best_cfg[0];
        b->lanes_query = best_cfg[1];
        b->query_early = best_cfg[2];
        b->ctas_per_sm = best_cfg[3];
    }

    // 2. per (size class, k, c): one dimension at a time on that class's filters
    std::map<uint64_t, std::pair<std::vector<blowchoc_work>, std::vector<blowchoc_work>>> by_class;
    for (const auto &w : sins)
        by_class[class_key(size_class_of(b, w.filter->dev.M), w.filter->dev.k, w.filter->p.choices)].first.push_back(w);
    for (const auto &w : sqry)
        by_class[class_key(size_class_of(b, w.filter->dev.M), w.filter->dev.k, w.filter->p.choices)].second.push_back(w);
    const std::vector<blowchoc_work> none;
    for (auto &kv : by_class) {
        if (rc) break;
        const uint64_t key = kv.first;
        const std::vector<blowchoc_work> &wi = kv.second.first, &wq = kv.second.second;
        blowchoc_class_tuning cur = default_class(b);
        float cur_ms = -1.0f;
        // keeps t (and its time) if it beats the best so far
        auto consider = [&](const blowchoc_class_tuning &t, bool query_only) -> int {
            b->ctune[key] = t;
            float ms = 0.0f;
            const int r = query_only ? timed(wi, wq, true, &ms) : timed(wi, none, false, &ms);
            if (r) return r;
            if (cur_ms < 0.0f || ms < cur_ms) {
                cur_ms = ms;
                cur = t;
            }
            return BLOWCHOC_OK;
        };
        if (!wi.empty()) {
            for (uint32_t lanes : {1u, 2u, 4u, 8u}) {
                blowchoc_class_tuning t = cur;
                t.lanes_choose = lanes;
                if (!rc) rc = consider(t, false);
            }
            const blowchoc_class_tuning base = cur;
            for (uint32_t tile : {64u, 128u, 256u, 512u}) {
                blowchoc_class_tuning t = base;
                t.tile = tile;
                if (!rc) rc = consider(t, false);
            }
            const blowchoc_class_tuning listed = cur;
            for (uint32_t route : {(uint32_t)BLOWCHOC_ROUTE_DIRECT, (uint32_t)BLOWCHOC_ROUTE_SORTED}) {
                blowchoc_class_tuning t = listed;
                t.route = route;
                if (!rc) rc = consider(t, false);
            }
        }
        if (!wq.empty()) {
            cur_ms = -1.0f;
            const blowchoc_class_tuning base = cur;
            for (uint32_t lanes : {1u, 2u, 4u, 8u})
                for (uint32_t early : {0u, 1u}) {
                    blowchoc_class_tuning t = base;
                    t.lanes_query = lanes;
                    t.query_early = early;
                    if (!rc) rc = consider(t, true);
                }
        }
        b->ctune[key] = cur;
    }

    for (size_t i = 0; i < scratch.size(); i += 2) blowchoc_destroy(scratch[i]);
    cudaFree(d_bm);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (rc) {
        b->lanes_choose = saved[0];
        b->lanes_query = saved[1];
        b->query_early = saved[2];
        b->ctas_per_sm = saved[3];
        b->ctune = saved_classes;
        return rc;
    }
    if (best) blowchoc_batch_get_tuning(b, best);
    return BLOWCHOC_OK;
}

}  // extern "C"
