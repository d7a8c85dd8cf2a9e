// C ABI of the BlowChoc filter library (declared in include/blowchoc.h).
//
// Host side: parameter checks, hash-multiplier derivation, the cost rank
// table, device memory, batch scheduling and kernel dispatch. Every step of
// the filter's arithmetic on keys runs in the CUDA kernels.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/blowchoc.h"
#include "bc_filter.h"
#include "bc_launch.h"


namespace {

thread_local std::string g_err;
constexpr size_t kCounterWords = 520;  // see blowchoc_filter::d_counters
std::atomic<uint64_t> g_launches{0};

// Every bc::launch_* call launches exactly one kernel.
inline cudaError_t counted(cudaError_t e) {
    if (e == cudaSuccess) g_launches.fetch_add(1, std::memory_order_relaxed);
    return e;
}

int fail(int code, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char *what) {
    return fail(e == cudaErrorMemoryAllocation ? BLOWCHOC_ENOMEM : BLOWCHOC_ECUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

#define BC_CUDA(call, what)                                  \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return cuda_fail(e_, what);   \
    } while (0)

// splitmix64 (Steele, Lea and Flood, OOPSLA 2014): golden-ratio increment
// followed by the published finaliser.
uint64_t splitmix64(uint64_t &state) {
    uint64_t z = (state += 0x9e3779b97f4a7c15ull);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

uint64_t gcd64(uint64_t a, uint64_t b) {
    while (b) {
        uint64_t t = a % b;
        a = b;
        b = t;
    }
    return a;
}

// Section 3.4: multipliers are random, odd and coprime to the hash range:
// M for the block hashes; 512 for random bit selection, 512 - i for the
// (i+1)-th hash of distinct bit selection (Appendix B).
void derive_multipliers(uint64_t seed, uint64_t M, uint32_t k, uint32_t c, uint32_t bitsel, uint64_t *a_block,
                        uint64_t *a_bit) {
    uint64_t st = seed;
    for (uint32_t i = 0; i < c; ++i) {
        uint64_t a;
        do a = splitmix64(st) | 1ull;
        while (gcd64(a, M) != 1);
        a_block[i] = a;
    }
    for (uint32_t i = 0; i < k; ++i) {
        const uint64_t range = bitsel ? 512u - i : 512u;
        uint64_t a;
        do a = splitmix64(st) | 1ull;
        while (gcd64(a, range) != 1);
        a_bit[i] = a;
    }
}

// Cost of Eq. 4-6 in double; j = L + a.
double cost_value(int kind, double par, uint32_t k, uint32_t j, uint32_t a) {
    const double dk = (double)k;
    if (kind == BLOWCHOC_COST_MIX) return (par * dk) * std::pow((double)j / 256.0, dk) + (double)a;
    if (kind == BLOWCHOC_COST_LA) return dk * std::pow(((double)j + par * dk) / 256.0, dk) + (double)a;
    return std::pow(par, (double)j / 128.0) + (double)a / dk;
}

// FPR estimate from the load histogram: a negative finds all its bits set in
// a block of load L with probability (L / 512)^k for independent bit
// addresses, C(L, k) / C(512, k) for k distinct ones (Appendix B); q is the
// mean over blocks, and c candidates are treated as independent.
double fpr_from_hist(const uint64_t *hist, uint32_t k, uint32_t choices, uint32_t bitsel) {
    double q = 0.0, blocks = 0.0;
    for (int L = 0; L <= 512; ++L) {
        double pL = 1.0;
        if (bitsel) {
            for (uint32_t i = 0; i < k; ++i) pL *= (double)((int)L - (int)i) / (double)(512 - i);
            if (pL < 0.0) pL = 0.0;
        } else {
            pL = std::pow((double)L / 512.0, (double)k);
        }
        q += (double)hist[L] * pL;
        blocks += (double)hist[L];
    }
    q /= blocks;
    return 1.0 - std::pow(1.0 - q, (double)choices);
}

// Integer rank of every reachable (L, a) cost: equal doubles share a rank,
// so comparing ranks on the device is comparing the doubles exactly. With
// `given` the costs come from a table instead of Eq. 4-6.
std::vector<uint16_t> rank_table(int kind, double par, uint32_t k, const double *given = nullptr) {
    const uint32_t k1 = k + 1;
    std::vector<double> cost(513 * k1, INFINITY);
    std::vector<double> vals;
    vals.reserve(513 * k1);
    for (uint32_t L = 0; L <= 512; ++L)
        for (uint32_t a = 0; a <= k && L + a <= 512; ++a) {
            cost[L * k1 + a] = given ? given[L * k1 + a] : cost_value(kind, par, k, L + a, a);
            vals.push_back(cost[L * k1 + a]);
        }
    std::sort(vals.begin(), vals.end());
    vals.erase(std::unique(vals.begin(), vals.end()), vals.end());
    std::vector<uint16_t> rank(513 * k1, 0xFFFF);
    for (uint32_t t = 0; t < 513 * k1; ++t)
        if (std::isfinite(cost[t]))
            rank[t] = (uint16_t)(std::lower_bound(vals.begin(), vals.end(), cost[t]) - vals.begin());
    return rank;
}

int check_params(const blowchoc_params *p) {
    if (!p) return fail(BLOWCHOC_EINVAL, "params is NULL");
    if (p->nblocks == 0 || p->nblocks > (1ull << 32))
        return fail(BLOWCHOC_EINVAL, "nblocks must be in 1..2^32 (got %llu)", (unsigned long long)p->nblocks);
    if (p->k < 1 || p->k > BLOWCHOC_MAX_K) return fail(BLOWCHOC_EINVAL, "k must be in 1..32 (got %u)", p->k);
    if (p->choices < 1 || p->choices > BLOWCHOC_MAX_CHOICES)
        return fail(BLOWCHOC_EINVAL, "choices must be in 1..3 (got %u)", p->choices);
    if (p->cost < BLOWCHOC_COST_MIX || p->cost > BLOWCHOC_COST_EXP)
        return fail(BLOWCHOC_EINVAL, "unknown cost kind %d", p->cost);
    if (!std::isfinite(p->cost_param) || p->cost_param < 0.0 ||
        (p->cost == BLOWCHOC_COST_EXP && p->cost_param <= 0.0))
        return fail(BLOWCHOC_EINVAL, "bad cost parameter %g", p->cost_param);
    if (p->bitsel > 1) return fail(BLOWCHOC_EINVAL, "bitsel must be 0 (random) or 1 (distinct)");
    if (p->batch == 0) return fail(BLOWCHOC_EINVAL, "batch must be >= 1");
    return BLOWCHOC_OK;
}

int grid_for(const blowchoc_filter *f, uint64_t work_groups, int threads_per_cta, int ctas_per_sm) {
    const uint64_t per_cta = (uint64_t)threads_per_cta;
    uint64_t need = (work_groups + per_cta - 1) / per_cta;
    const uint64_t cap = (uint64_t)f->sms * (uint64_t)ctas_per_sm;
    if (need > cap) need = cap;
    if (need < 1) need = 1;
    return (int)need;
}

int ensure_sel(blowchoc_filter *f, uint64_t need) {
    if (need <= f->sel_cap) return BLOWCHOC_OK;
    if (f->d_sel) {
        cudaError_t e = cudaFree(f->d_sel);
        f->d_sel = nullptr;
        f->sel_cap = 0;
        if (e != cudaSuccess) return cuda_fail(e, "cudaFree(sel)");
    }
    BC_CUDA(cudaMalloc(&f->d_sel, need), "cudaMalloc(sel)");
    f->sel_cap = need;
    return BLOWCHOC_OK;
}

int ensure_sorted(blowchoc_filter *f, uint64_t need) {
    if (need <= f->sorted_cap) return BLOWCHOC_OK;
    cudaFree(f->d_sorted);
    f->d_sorted = nullptr;
    f->sorted_cap = 0;
    BC_CUDA(cudaMalloc(&f->d_sorted, need * sizeof(uint32_t)), "cudaMalloc(sorted scratch)");
    f->sorted_cap = need;
    return BLOWCHOC_OK;
}

}  // namespace

extern "C" {

const char *blowchoc_last_error(void) { return g_err.c_str(); }

uint64_t blowchoc_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

}  // extern "C"

void bc_note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

int bc_set_error(int code, const char *msg) {
    g_err = msg;
    return code;
}

extern "C" {

int blowchoc_create(const blowchoc_params *params, void *stream, blowchoc_filter **out) {
    if (!out) return fail(BLOWCHOC_EINVAL, "out is NULL");
    *out = nullptr;
    int rc = check_params(params);
    if (rc) return rc;
    blowchoc_filter *f = new blowchoc_filter();
    f->p = *params;
    f->home = (cudaStream_t)stream;
    cudaError_t e = cudaGetDevice(&f->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&f->sms, cudaDevAttrMultiProcessorCount, f->device);
    int l2 = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, f->device);
    if (e != cudaSuccess) {
        delete f;
        return cuda_fail(e, "no usable CUDA device");
    }
    // measured defaults (one GB300 with 129 MiB of L2, one process, persistent
    // insert over a full grid, B = 2^20, 12 bits per key): inserts decide
    // fastest with four lanes per key up to half the L2 size (2 MiB: 0.112 ms
    // against 0.131 with one lane; 64 MiB, three choices: 3.07 ms against 3.21
    // with two), with two lanes up to 1.5 times the L2 size (128 MiB: 6.36 ms
    // against 6.50 with four; 192 MiB: 11.46 against 11.75) and, with three
    // choices, four beyond (256 MiB: 16.42 ms against 17.41 with two);
    // queries with one lane while the filter fits in L2 and two beyond
    const uint64_t bytes = params->nblocks * 64ull;
    // Beyond 1.5 L2 with two choices (and the bulk set) two lanes won too:
    // 256 MiB 12.77 against 14.02 ms, 512 MiB 30.58 against 30.79.
    f->lanes_choose = bytes <= (uint64_t)l2 / 2 ? 4
                      : bytes <= 3ull * (uint64_t)l2 / 2 ? 2
                      : params->choices <= 2 ? 2 : 4;
    f->lanes_query = bytes <= (uint64_t)l2 ? 1 : 2;
    // the bulk set paid at the L2 size and beyond, except with three choices
    // at about the L2 size (one GB300, c = 2, k = 12: 128 MiB 3.26 against
    // 4.18 ms at 32 keys per block and batch, 3.91 against 4.23 at 1/2;
    // 512 MiB 21.0-21.8 against 23.2-23.4; 16 MiB and below 3-18% slower;
    // the 128 MiB DNA shape, c = 3, k = 16: 2.83 against 2.59)
    f->set_mode = (bytes > (uint64_t)l2 && (params->choices <= 2 || bytes > 3ull * (uint64_t)l2 / 2)) ? 2 : 0;
    // reservation window of the exact inserts of B <= 16 (one GB300, 2^15 to
    // 2^21 blocks, 2.8 M keys or 12 bits per key): 512 keys, one commit pass
    // of the 1024-thread CTA at two lanes per key, was the fastest window or
    // within 5% of it for B = 1 (2^16 blocks, c = 2: 47.5 ms against 54.2
    // with 2048 and 72.2 with 128). Windows of batches whose candidate blocks
    // often meet, 64 (B c)^2 >= M, did best at 256 (2^16 blocks, B = 16,
    // c = 3: 145.8 ms against 164.9 with 512 and 326.6 with 2048); larger
    // filters at 512 (2^21 blocks, B = 16, c = 2: 53.7 against 61.7 with 256).
    {
        const uint64_t bcw = params->batch * params->choices;
        f->seq_window = (params->batch > 1 && params->batch <= bc::kSeqMaxBatch && 64 * bcw * bcw >= params->nblocks)
                            ? 256
                            : 512;
    }
    bc::DevFilter &d = f->dev;
    std::memset(&d, 0, sizeof d);
    d.M = params->nblocks;
    d.k = params->k;
    d.c = params->choices;
    if ((d.M & (d.M - 1)) == 0) {
        uint32_t lg = 0;
        while ((1ull << lg) < d.M) ++lg;
        d.range_kind = bc::kRangePow2;
        d.shift = 64 - lg;
    } else {
        d.range_kind = (d.M & 1) ? bc::kRangeOdd : bc::kRangeEven;
        d.shift = 0;
        d.mod_mul = bc::mod_mul_for(d.M);
    }
    d.bitsel = params->bitsel;
    derive_multipliers(params->hash_seed, d.M, d.k, d.c, d.bitsel, d.a_block, d.a_bit);

    const size_t wbytes = (size_t)d.M * bc::kBlockWords * sizeof(uint64_t);
    e = cudaMalloc(&d.words, wbytes);
    if (e == cudaSuccess) e = cudaMalloc(&f->d_counters, kCounterWords * sizeof(unsigned long long));
    if (e == cudaSuccess && d.c > 1) {
        std::vector<uint16_t> rank = rank_table(params->cost, params->cost_param, d.k);
        e = cudaMalloc(&f->d_rank, rank.size() * sizeof(uint16_t));
        if (e == cudaSuccess)
            e = cudaMemcpy(f->d_rank, rank.data(), rank.size() * sizeof(uint16_t), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(d.words, 0, wbytes, f->home);
    if (e == cudaSuccess) e = cudaMemsetAsync(f->d_counters, 0, kCounterWords * sizeof(unsigned long long), f->home);
    if (e != cudaSuccess) {
        rc = cuda_fail(e, "blowchoc_create");
        cudaFree(d.words);
        cudaFree(f->d_counters);
        cudaFree(f->d_rank);
        delete f;
        return rc;
    }
    *out = f;
    return BLOWCHOC_OK;
}

namespace {

// Shape of the cluster-resident insert for n keys, S = 0 if not taken.
// The cluster-resident insert replaces the global-memory kernels where those
// run a batch in one CTA (B <= 2048) or in two launches (persistent off).
// Against the persistent insert over the whole grid it lost from B = 4096
// on (one GB300, ~10^6 keys, 8,192 to 45,000 blocks: 1.72 ms against 1.41
// at B = 4096, 1.45 against 0.74 at B = 8192), and won 1.6 to 5 times at
// B = 512 to 2048.
bc::ClusterShape cluster_plan(const blowchoc_filter *f, uint64_t n) {
    const uint64_t B = f->p.batch;
    if (f->cluster_max == 0 || B < 2 || n == 0 || (n + B - 1) / B < bc::kClusterMinRounds) return bc::ClusterShape();
    if (f->persistent && B > bc::kSingleCtaBatch) return bc::ClusterShape();
    return bc::cluster_shape((int)f->p.choices, f->lanes_cluster, f->dev.M, f->dev.k, std::min(B, n),
                             f->cluster_max, (uint64_t)f->cluster_keys);
}

}  // namespace

// Allocates what blowchoc_insert of n keys would allocate on first use
// (reservation words, choice bytes, sort-by-block scratch) without launching
// anything, so that the insert can then be captured in a CUDA graph.
int bc_reserve_insert_scratch(blowchoc_filter *f, uint64_t n) {
    if (!f) return fail(BLOWCHOC_EINVAL, "filter is NULL");
    if (n == 0) return BLOWCHOC_OK;
    const uint64_t B = f->p.batch;
    const bool resv = (B == 1 && f->seq_window > 0) ||
                      (B > 1 && B <= bc::kSeqMaxBatch && f->seq_window > 0 && n > B && !cluster_plan(f, n).S);
    if (resv && !f->d_resv)
        BC_CUDA(cudaMalloc(&f->d_resv, f->dev.M * sizeof(unsigned long long)), "cudaMalloc(reservations)");
    if (B == 1 || cluster_plan(f, n).S || (B <= bc::kSeqMaxBatch && f->seq_window > 0 && n > B) ||
        B <= bc::kSingleCtaBatch || (!f->persistent && B <= bc::kSmallBatchMax))
        return BLOWCHOC_OK;
    const uint64_t per = std::min(B, n);
    int rc = ensure_sel(f, 2 * per);
    if (rc) return rc;
    const uint64_t R = (f->dev.M + bc::kRangeBlocks - 1) / bc::kRangeBlocks;
    if (f->persistent && f->set_mode == 1 && R <= bc::kSortedMaxRanges) return ensure_sorted(f, 3 * R + 1 + per);
    return BLOWCHOC_OK;
}

int blowchoc_cluster_ctas(blowchoc_filter *f, uint64_t n, uint32_t *ctas) {
    if (!f || !ctas) return fail(BLOWCHOC_EINVAL, "NULL argument");
    *ctas = (uint32_t)cluster_plan(f, n).S;
    return BLOWCHOC_OK;
}

int blowchoc_insert(blowchoc_filter *f, const uint64_t *d_keys, uint64_t n, void *stream) {
    if (!f) return fail(BLOWCHOC_EINVAL, "filter is NULL");
    if (n == 0) return BLOWCHOC_OK;
    if (!d_keys) return fail(BLOWCHOC_EINVAL, "keys is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    const int C = (int)f->p.choices;
    const uint64_t B = f->p.batch;
    if (B == 1) {
        if (f->seq_window > 0) {
            if (!f->d_resv)
                BC_CUDA(cudaMalloc(&f->d_resv, f->dev.M * sizeof(unsigned long long)), "cudaMalloc(reservations)");
            BC_CUDA(counted(bc::launch_exact_sequential(C, s, f->dev, d_keys, n, (uint32_t)f->seq_window, f->d_rank,
                                                        f->d_counters, f->d_resv)),
                    "sequential insert launch");
            return BLOWCHOC_OK;
        }
        BC_CUDA(counted(bc::launch_sequential(C, s, f->dev, d_keys, n, f->d_rank, f->d_counters)),
                "sequential insert launch");
        return BLOWCHOC_OK;
    }
    {
        const bc::ClusterShape sh = cluster_plan(f, n);
        if (sh.S) {
            bc::ManyItem one;
            std::memset(&one, 0, sizeof one);
            one.f = f->dev;
            one.rank = f->d_rank;
            one.keys = d_keys;
            one.n = n;
            one.B = B;
            one.counters = f->d_counters;
            BC_CUDA(counted(bc::launch_cluster_insert(C, f->lanes_cluster, sh, 1, s, nullptr, one)),
                    "cluster insert launch");
            return BLOWCHOC_OK;
        }
    }
    if (B <= bc::kSeqMaxBatch && f->seq_window > 0 && n > B) {
        // small batches of a filter beyond one cluster: reservation rounds
        // over windows of whole batches
        uint64_t window = (uint64_t)f->seq_window / B * B;
        if (window < 4 * B) window = 4 * B;
        if (window > bc::kSeqMaxWindow) window = bc::kSeqMaxWindow / B * B;
        if (!f->d_resv)
            BC_CUDA(cudaMalloc(&f->d_resv, f->dev.M * sizeof(unsigned long long)), "cudaMalloc(reservations)");
        BC_CUDA(counted(bc::launch_exact_batched(C, s, f->dev, d_keys, n, B, (uint32_t)window, f->d_rank,
                                                 f->d_counters, f->d_resv)),
                "batched insert launch");
        return BLOWCHOC_OK;
    }
    if (B <= bc::kSingleCtaBatch || (!f->persistent && B <= bc::kSmallBatchMax)) {
        bc::Launch L{1, f->lanes_choose, s};
        BC_CUDA(counted(bc::launch_small_batch(C, L, f->dev, d_keys, n, B, f->d_rank, f->d_counters)),
                "small-batch insert launch");
        return BLOWCHOC_OK;
    }
    int rc = ensure_sel(f, 2 * std::min(B, n));  // the persistent insert keeps two bytes per key
    if (rc) return rc;
    if (f->persistent) {
        const uint64_t per = std::min(B, n);
        const uint64_t want = (per + (uint64_t)f->keys_per_cta - 1) / (uint64_t)f->keys_per_cta;
        const uint64_t cap = (uint64_t)f->sms * (uint64_t)f->ctas_per_sm;
        bc::Launch L{(int)std::max<uint64_t>(1, std::min(want, cap)), f->lanes_choose, s};
        const uint64_t R = (f->dev.M + bc::kRangeBlocks - 1) / bc::kRangeBlocks;
        if (f->set_mode == 1 && R <= bc::kSortedMaxRanges) {
            rc = ensure_sorted(f, 3 * R + 1 + per);
            if (rc) return rc;
            unsigned int *bar = reinterpret_cast<unsigned int *>(f->d_counters + 516);
            BC_CUDA(counted(bc::launch_sorted_insert(C, L, f->dev, d_keys, n, B, f->d_rank, f->d_sel,
                                                     f->d_counters, bar, f->d_sorted, (uint32_t)R, f->sms)),
                    "sorted insert launch");
            return BLOWCHOC_OK;
        }
        unsigned int *bar = reinterpret_cast<unsigned int *>(f->d_counters + 516);
        BC_CUDA(counted(bc::launch_persistent_insert(C, L, f->dev, d_keys, n, B, f->d_rank, f->d_sel,
                                                     f->d_counters, bar, f->sms, f->set_mode == 2)),
                "persistent insert launch");
        return BLOWCHOC_OK;
    }
    for (uint64_t s0 = 0; s0 < n; s0 += B) {
        const uint64_t cnt = std::min(B, n - s0);
        bc::Launch Lc{grid_for(f, cnt * f->lanes_choose, 256, f->ctas_per_sm), f->lanes_choose, s};
        BC_CUDA(counted(bc::launch_choose(C, Lc, f->dev, d_keys + s0, cnt, f->d_rank, f->d_sel, f->d_counters)),
                "choose launch");
        bc::Launch Ls{grid_for(f, cnt * f->lanes_set, 256, f->ctas_per_sm), f->lanes_set, s};
        BC_CUDA(counted(bc::launch_set(Ls, f->dev, d_keys + s0, cnt, f->d_sel)), "set launch");
    }
    return BLOWCHOC_OK;
}

int blowchoc_query(blowchoc_filter *f, const uint64_t *d_keys, uint64_t n, uint64_t *d_bitmap,
                   void *stream) {
    if (!f) return fail(BLOWCHOC_EINVAL, "filter is NULL");
    if (n == 0) return BLOWCHOC_OK;
    if (!d_keys || !d_bitmap) return fail(BLOWCHOC_EINVAL, "keys or bitmap is NULL");
    const uint64_t nwords = (n + 63) / 64;
    bc::Launch L{grid_for(f, nwords * 32, 256, f->ctas_per_sm), f->lanes_query, (cudaStream_t)stream, f->query_early};
    BC_CUDA(counted(bc::launch_query((int)f->p.choices, L, f->dev, d_keys, n, d_bitmap)), "query launch");
    return BLOWCHOC_OK;
}

int blowchoc_query_count(blowchoc_filter *f, const uint64_t *d_keys, uint64_t n, unsigned long long *d_count,
                         void *stream) {
    if (!f) return fail(BLOWCHOC_EINVAL, "filter is NULL");
    if (n == 0) return BLOWCHOC_OK;
    if (!d_keys || !d_count) return fail(BLOWCHOC_EINVAL, "keys or count is NULL");
    const uint64_t nwords = (n + 63) / 64;
    bc::Launch L{grid_for(f, nwords * 32, 256, f->ctas_per_sm), f->lanes_query, (cudaStream_t)stream, f->query_early};
    BC_CUDA(counted(bc::launch_query((int)f->p.choices, L, f->dev, d_keys, n, nullptr, d_count)),
            "query count launch");
    return BLOWCHOC_OK;
}

int blowchoc_generate_keys(uint64_t *d_out, uint64_t n, uint64_t seed, uint64_t start, void *stream) {
    if (n == 0) return BLOWCHOC_OK;
    if (!d_out) return fail(BLOWCHOC_EINVAL, "out is NULL");
    int dev = 0, sms = 0;
    BC_CUDA(cudaGetDevice(&dev), "device");
    BC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
    BC_CUDA(counted(bc::launch_generate_keys((cudaStream_t)stream, sms, d_out, n, seed, start)),
            "key generation launch");
    return BLOWCHOC_OK;
}

int blowchoc_stats_async(blowchoc_filter *f, uint64_t *h_raw, void *stream) {
    if (!f || !h_raw) return fail(BLOWCHOC_EINVAL, "filter or h_raw is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long *d_hist = f->d_counters + 3;
    BC_CUDA(cudaMemsetAsync(d_hist, 0, 513 * sizeof(unsigned long long), s), "memset hist");
    bc::Launch L{grid_for(f, (f->dev.M + 7) / 8 * 32, 256, 8), 4, s};
    BC_CUDA(counted(bc::launch_stats(L, f->dev.words, f->dev.M, d_hist)), "stats launch");
    BC_CUDA(cudaMemcpyAsync(h_raw, f->d_counters, BLOWCHOC_STATS_RAW_WORDS * sizeof(uint64_t),
                            cudaMemcpyDeviceToHost, s),
            "stats copy");
    return BLOWCHOC_OK;
}

int blowchoc_stats_decode(const blowchoc_filter *f, const uint64_t *h, blowchoc_filter_stats *out) {
    if (!f || !h || !out) return fail(BLOWCHOC_EINVAL, "NULL argument");
    std::memset(out, 0, sizeof *out);
    out->inserted = h[0];
    out->skipped = h[1];
    for (int L = 0; L <= 512; ++L) {
        out->hist[L] = h[3 + L];
        out->set_bits += (uint64_t)L * h[3 + L];
    }
    out->fpr_est = fpr_from_hist(out->hist, f->p.k, f->p.choices, f->p.bitsel);
    if (h[2]) return fail(BLOWCHOC_ETIMEOUT, "a bounded device wait of this filter gave up");
    return BLOWCHOC_OK;
}

int blowchoc_stats(blowchoc_filter *f, blowchoc_filter_stats *out) {
    if (!f || !out) return fail(BLOWCHOC_EINVAL, "filter or out is NULL");
    uint64_t h[BLOWCHOC_STATS_RAW_WORDS];
    const int rc = blowchoc_stats_async(f, h, f->home);
    if (rc) return rc;
    BC_CUDA(cudaStreamSynchronize(f->home), "stats sync");
    return blowchoc_stats_decode(f, h, out);
}

int blowchoc_destroy(blowchoc_filter *f) {
    if (!f) return BLOWCHOC_OK;
    cudaError_t e = cudaStreamSynchronize(f->home);
    cudaFree(f->dev.words);
    cudaFree(f->d_counters);
    cudaFree(f->d_rank);
    cudaFree(f->d_sel);
    cudaFree(f->d_sorted);
    cudaFree(f->d_resv);
    bc_free_host_stage(f);
    delete f;
    if (e != cudaSuccess) return cuda_fail(e, "blowchoc_destroy");
    return BLOWCHOC_OK;
}

int blowchoc_words(blowchoc_filter *f, uint64_t **d_words, uint64_t *nwords) {
    if (!f || !d_words || !nwords) return fail(BLOWCHOC_EINVAL, "NULL argument");
    *d_words = f->dev.words;
    *nwords = f->dev.M * bc::kBlockWords;
    return BLOWCHOC_OK;
}

int blowchoc_multipliers(blowchoc_filter *f, uint64_t *a_block, uint64_t *a_bit) {
    if (!f || !a_block || !a_bit) return fail(BLOWCHOC_EINVAL, "NULL argument");
    for (int i = 0; i < 3; ++i) a_block[i] = i < (int)f->dev.c ? f->dev.a_block[i] : 0;
    for (int i = 0; i < 32; ++i) a_bit[i] = i < (int)f->dev.k ? f->dev.a_bit[i] : 0;
    return BLOWCHOC_OK;
}

int blowchoc_read_words(blowchoc_filter *f, uint64_t first, uint64_t count, uint64_t *h_dst) {
    if (!f || (!h_dst && count)) return fail(BLOWCHOC_EINVAL, "NULL argument");
    const uint64_t nw = f->dev.M * bc::kBlockWords;
    if (first > nw || count > nw - first) return fail(BLOWCHOC_EINVAL, "word range past the filter");
    if (count == 0) return BLOWCHOC_OK;
    BC_CUDA(cudaMemcpyAsync(h_dst, f->dev.words + first, count * sizeof(uint64_t), cudaMemcpyDeviceToHost,
                            f->home), "read words");
    BC_CUDA(cudaStreamSynchronize(f->home), "read words sync");
    return BLOWCHOC_OK;
}

int blowchoc_write_words(blowchoc_filter *f, uint64_t first, uint64_t count, const uint64_t *h_src) {
    if (!f || (!h_src && count)) return fail(BLOWCHOC_EINVAL, "NULL argument");
    const uint64_t nw = f->dev.M * bc::kBlockWords;
    if (first > nw || count > nw - first) return fail(BLOWCHOC_EINVAL, "word range past the filter");
    if (count == 0) return BLOWCHOC_OK;
    BC_CUDA(cudaMemcpyAsync(f->dev.words + first, h_src, count * sizeof(uint64_t), cudaMemcpyHostToDevice,
                            f->home), "write words");
    BC_CUDA(cudaStreamSynchronize(f->home), "write words sync");
    return BLOWCHOC_OK;
}

int blowchoc_set_cost_table(blowchoc_filter *f, const double *costs) {
    if (!f || !costs) return fail(BLOWCHOC_EINVAL, "NULL argument");
    if (f->dev.c < 2 || !f->d_rank) return fail(BLOWCHOC_EINVAL, "one choice has no cost");
    const uint32_t k = f->dev.k, k1 = k + 1;
    for (uint32_t L = 0; L <= 512; ++L)
        for (uint32_t a = 0; a <= k && L + a <= 512; ++a)
            if (!std::isfinite(costs[L * k1 + a])) return fail(BLOWCHOC_EINVAL, "cost table value not finite");
    std::vector<uint16_t> rank = rank_table(0, 0.0, k, costs);
    // ordered after earlier work on the home stream, like an insert would be
    BC_CUDA(cudaMemcpyAsync(f->d_rank, rank.data(), rank.size() * sizeof(uint16_t), cudaMemcpyHostToDevice,
                            f->home), "cost table upload");
    BC_CUDA(cudaStreamSynchronize(f->home), "cost table upload");
    return BLOWCHOC_OK;
}

int blowchoc_derive_multipliers(const blowchoc_params *params, uint64_t *a_block, uint64_t *a_bit) {
    if (!a_block || !a_bit) return fail(BLOWCHOC_EINVAL, "NULL argument");
    const int rc = check_params(params);
    if (rc) return rc;
    derive_multipliers(params->hash_seed, params->nblocks, params->k, params->choices, params->bitsel, a_block,
                       a_bit);
    return BLOWCHOC_OK;
}

int blowchoc_shard_layout(uint64_t nblocks, uint32_t T, uint64_t hash_seed, uint64_t *a0, uint64_t *sub_nblocks,
                          uint64_t *sub_seed) {
    if (!a0 || !sub_nblocks || !sub_seed) return fail(BLOWCHOC_EINVAL, "NULL argument");
    if (nblocks == 0 || T < 1 || T > 1024) return fail(BLOWCHOC_EINVAL, "nblocks >= 1 and T in 1..1024");
    *sub_nblocks = (nblocks + T - 1) / T;
    if (T == 1) {
        *a0 = 0;
        *sub_seed = hash_seed;
        return BLOWCHOC_OK;
    }
    uint64_t st = hash_seed, a;
    do a = splitmix64(st) | 1ull;
    while (gcd64(a, T) != 1);
    *a0 = a;
    *sub_seed = st;
    return BLOWCHOC_OK;
}

int blowchoc_fpr_estimate(const uint64_t *hist, uint32_t k, uint32_t choices, uint32_t bitsel, double *out) {
    if (!hist || !out) return fail(BLOWCHOC_EINVAL, "NULL argument");
    if (k < 1 || k > BLOWCHOC_MAX_K) return fail(BLOWCHOC_EINVAL, "k must be in 1..32 (got %u)", k);
    if (choices < 1 || choices > BLOWCHOC_MAX_CHOICES) return fail(BLOWCHOC_EINVAL, "choices must be in 1..3");
    if (bitsel > 1) return fail(BLOWCHOC_EINVAL, "bitsel must be 0 (random) or 1 (distinct)");
    uint64_t blocks = 0;
    for (int L = 0; L <= 512; ++L) blocks += hist[L];
    if (blocks == 0) return fail(BLOWCHOC_EINVAL, "the histogram counts no block");
    *out = fpr_from_hist(hist, k, choices, bitsel);
    return BLOWCHOC_OK;
}

int blowchoc_cost_ranks(int cost, double cost_param, uint32_t k, uint16_t *ranks, uint64_t capacity) {
    if (!ranks) return fail(BLOWCHOC_EINVAL, "ranks is NULL");
    if (k < 1 || k > BLOWCHOC_MAX_K) return fail(BLOWCHOC_EINVAL, "k must be in 1..32 (got %u)", k);
    if (cost < BLOWCHOC_COST_MIX || cost > BLOWCHOC_COST_EXP) return fail(BLOWCHOC_EINVAL, "unknown cost kind %d", cost);
    if (!std::isfinite(cost_param) || cost_param < 0.0 || (cost == BLOWCHOC_COST_EXP && cost_param <= 0.0))
        return fail(BLOWCHOC_EINVAL, "bad cost parameter %g", cost_param);
    const uint64_t need = 513ull * (k + 1);
    if (capacity < need) return fail(BLOWCHOC_EINVAL, "ranks needs 513 (k + 1) = %llu entries", (unsigned long long)need);
    const std::vector<uint16_t> rank = rank_table(cost, cost_param, k);
    std::memcpy(ranks, rank.data(), rank.size() * sizeof(uint16_t));
    return BLOWCHOC_OK;
}

int blowchoc_l2_residency(blowchoc_filter *f, double fraction, void *stream) {
    if (!f || !(fraction >= 0.0) || fraction > 1.0) return fail(BLOWCHOC_EINVAL, "fraction must be in [0, 1]");
    cudaStream_t s = (cudaStream_t)stream;
    if (!s) return fail(BLOWCHOC_EINVAL, "a created stream is required (not the legacy default stream)");
    int max_persist = 0, max_window = 0;
    BC_CUDA(cudaDeviceGetAttribute(&max_persist, cudaDevAttrMaxPersistingL2CacheSize, f->device), "L2 attribute");
    BC_CUDA(cudaDeviceGetAttribute(&max_window, cudaDevAttrMaxAccessPolicyWindowSize, f->device), "L2 attribute");
    cudaStreamAttrValue attr;
    std::memset(&attr, 0, sizeof attr);
    const size_t bytes = (size_t)f->dev.M * bc::kBlockWords * sizeof(uint64_t);
    if (fraction > 0.0 && max_persist > 0 && max_window > 0) {
        const size_t set_aside = (size_t)(fraction * (double)max_persist);
        BC_CUDA(cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, set_aside), "persisting L2 limit");
        const size_t window = std::min(bytes, (size_t)max_window);
        attr.accessPolicyWindow.base_ptr = f->dev.words;
        attr.accessPolicyWindow.num_bytes = window;
        attr.accessPolicyWindow.hitRatio = (float)std::min(1.0, (double)set_aside / (double)window);
        attr.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
        attr.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
    } else {
        attr.accessPolicyWindow.base_ptr = f->dev.words;
        attr.accessPolicyWindow.num_bytes = 0;
        attr.accessPolicyWindow.hitRatio = 0.0f;
        attr.accessPolicyWindow.hitProp = cudaAccessPropertyNormal;
        attr.accessPolicyWindow.missProp = cudaAccessPropertyNormal;
    }
    BC_CUDA(cudaStreamSetAttribute(s, cudaStreamAttributeAccessPolicyWindow, &attr), "access policy window");
    if (fraction == 0.0) BC_CUDA(cudaCtxResetPersistingL2Cache(), "reset persisting L2");
    return BLOWCHOC_OK;
}

int blowchoc_get_tuning(blowchoc_filter *f, blowchoc_tuning *out) {
    if (!f || !out) return fail(BLOWCHOC_EINVAL, "NULL argument");
    out->lanes_choose = (uint32_t)f->lanes_choose;
    out->lanes_set = (uint32_t)f->lanes_set;
    out->lanes_query = (uint32_t)f->lanes_query;
    out->query_early = (uint32_t)f->query_early;
    out->ctas_per_sm = (uint32_t)f->ctas_per_sm;
    out->persistent = (uint32_t)f->persistent;
    out->keys_per_cta = (uint32_t)f->keys_per_cta;
    out->set_mode = (uint32_t)f->set_mode;
    out->seq_window = (uint32_t)f->seq_window;
    out->cluster_max = (uint32_t)f->cluster_max;
    out->lanes_cluster = (uint32_t)f->lanes_cluster;
    out->cluster_keys = (uint32_t)f->cluster_keys;
    out->host_ring_keys = f->host_ring_keys;
    return BLOWCHOC_OK;
}

// Field checks of a filter's launch configuration (blowchoc_set_tuning).
int bc_check_tuning(const blowchoc_tuning *t) {
    auto lanes_ok = [](uint32_t l) { return l == 1 || l == 2 || l == 4 || l == 8; };
    if (!lanes_ok(t->lanes_choose) || !lanes_ok(t->lanes_set) || !lanes_ok(t->lanes_query))
        return fail(BLOWCHOC_EINVAL, "lanes must be 1, 2, 4 or 8");
    if (t->query_early > 2) return fail(BLOWCHOC_EINVAL, "query_early must be 0, 1 or 2");
    if (t->ctas_per_sm < 1 || t->ctas_per_sm > 16) return fail(BLOWCHOC_EINVAL, "ctas_per_sm must be in 1..16");
    if (t->persistent > 1) return fail(BLOWCHOC_EINVAL, "persistent must be 0 or 1");
    if (t->keys_per_cta < 32 || t->keys_per_cta > (1u << 24))
        return fail(BLOWCHOC_EINVAL, "keys_per_cta must be in 32..2^24");
    if (t->set_mode > 2) return fail(BLOWCHOC_EINVAL, "set_mode must be 0, 1 or 2");
    if (t->seq_window != 0 && (t->seq_window < 32 || t->seq_window > bc::kSeqMaxWindow))
        return fail(BLOWCHOC_EINVAL, "seq_window must be 0 or in 32..8192");
    if (t->cluster_max > 16) return fail(BLOWCHOC_EINVAL, "cluster_max must be in 0..16");
    if (t->lanes_cluster != 4 && t->lanes_cluster != 8) return fail(BLOWCHOC_EINVAL, "lanes_cluster must be 4 or 8");
    if (t->cluster_keys < 16 || t->cluster_keys > (1u << 20))
        return fail(BLOWCHOC_EINVAL, "cluster_keys must be in 16..2^20");
    if (t->host_ring_keys != 0 && (t->host_ring_keys < (1u << 16) || t->host_ring_keys > 0x7FFFFFFFu))
        return fail(BLOWCHOC_EINVAL, "host_ring_keys must be 0 or in 2^16..2^31-1");
    return BLOWCHOC_OK;
}

int blowchoc_set_tuning(blowchoc_filter *f, const blowchoc_tuning *t) {
    if (!f || !t) return fail(BLOWCHOC_EINVAL, "NULL argument");
    const int rc = bc_check_tuning(t);
    if (rc) return rc;
    f->lanes_choose = (int)t->lanes_choose;
    f->lanes_set = (int)t->lanes_set;
    f->lanes_query = (int)t->lanes_query;
    f->query_early = (int)t->query_early;
    f->ctas_per_sm = (int)t->ctas_per_sm;
    f->persistent = (int)t->persistent;
    f->keys_per_cta = (int)t->keys_per_cta;
    f->set_mode = (int)t->set_mode;
    f->seq_window = (int)t->seq_window;
    f->cluster_max = (int)t->cluster_max;
    f->lanes_cluster = (int)t->lanes_cluster;
    f->cluster_keys = (int)t->cluster_keys;
    f->host_ring_keys = t->host_ring_keys;
    return BLOWCHOC_OK;
}

int blowchoc_clear(blowchoc_filter *f, void *stream) {
    if (!f) return fail(BLOWCHOC_EINVAL, "filter is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    BC_CUDA(cudaMemsetAsync(f->dev.words, 0, f->dev.M * bc::kBlockWords * sizeof(uint64_t), s), "clear words");
    BC_CUDA(cudaMemsetAsync(f->d_counters, 0, 3 * sizeof(unsigned long long), s), "clear counters");
    return BLOWCHOC_OK;
}

}  // extern "C"
