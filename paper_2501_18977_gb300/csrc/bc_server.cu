// Request-serving loop for device-resident filters (continuous batching).
//
// A scheduler thread owns all GPU work: it releases submitted requests at
// their arrival times into per-filter FIFOs, admits registered filters in
// order while their memory fits the HBM budget, and launches waves. A wave
// takes, for every ready filter, its head request if that is an insert (one
// insert per filter, so consecutive inserts stay separate calls with their
// own batches), or its run of consecutive queries (they see the same filter,
// so they share one launch item, each padded to whole bitmap words), up to
// the wave size and the free staging memory; it copies the keys in,
// runs one insert_many and one query_many over the whole wave, copies the
// bitmaps out and records an event. Waves rotate over several streams, so
// copies and kernels of different waves overlap; a filter's next request
// waits on the event of the wave that ran its previous one.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "bc_filter.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Req {
    uint64_t id;
    uint32_t filter;
    uint32_t kind;
    const uint64_t *h_keys;
    uint64_t n;
    uint64_t *h_bitmap;
    double arrival = 0.0;   // seconds since start
    double launched = -1.0;
    double done = -1.0;
    uint64_t staging = 0;   // device bytes while in flight
    bool keys_pinned = false, bitmap_pinned = false;
    bool clear_tail = false;  // a coalesced query followed by padding: bits n..63 of its last word
    size_t key_bounce = SIZE_MAX, bm_bounce = SIZE_MAX;  // offsets in the pinned arenas
};

// First-fit allocator over a fixed pinned host buffer (offsets, 256-byte
// granules): bounce space for requests whose host buffers are pageable,
// because copies to or from pageable memory would block the scheduler.
struct Arena {
    uint8_t *base = nullptr;
    size_t size = 0;
    std::map<size_t, size_t> free_;  // offset -> length
    void init(uint8_t *b, size_t n) {
        base = b;
        size = n;
        free_.clear();
        if (n) free_[0] = n;
    }
    size_t alloc(size_t n) {
        n = (n + 255) & ~size_t(255);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < n) continue;
            const size_t off = it->first, len = it->second;
            free_.erase(it);
            if (len > n) free_[off + n] = len - n;
            return off;
        }
        return SIZE_MAX;
    }
    void release(size_t off, size_t n) {
        n = (n + 255) & ~size_t(255);
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

bool is_pinned(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

struct Slot {               // one registered filter
    blowchoc_params params;
    uint64_t bytes = 0;
    blowchoc_filter *f = nullptr;
    bool admitted = false, remove = false, removed = false;
    std::deque<Req *> fifo; // arrived, not yet launched
    int last_wave = -1;     // wave that ran its latest launched request (while in flight)
    uint32_t inflight = 0;
    uint64_t unlaunched = 0; // submitted (arrived or not) and not yet launched
};

struct Wave {
    int stream = 0;
    cudaEvent_t ev = nullptr;
    cudaEvent_t start = nullptr;  // timing: recorded before the wave's first copy
    std::vector<Req *> reqs;
    uint64_t staging = 0;
    bool active = false;
};

uint64_t filter_bytes(const blowchoc_params &p) {
    return p.nblocks * 64ull + 513ull * (p.k + 1) * 2ull + 520ull * 8ull;
}

}  // namespace

struct blowchoc_server {
    blowchoc_server_config cfg;
    int device = 0;
    bool tuned = false;                        // apply `tuning` to admitted filters
    blowchoc_tuning tuning;
    std::vector<cudaStream_t> streams;
    std::vector<blowchoc_batch *> batches;     // one per stream
    std::vector<int> stream_inflight;
    cudaMemPool_t pool = nullptr;
    uint8_t *h_keys_arena = nullptr, *h_bm_arena = nullptr;  // pinned bounce buffers
    Arena keys_arena, bm_arena;
    std::vector<Wave> waves;                   // pool of wave records
    std::vector<Slot> slots;
    std::vector<std::unique_ptr<Req>> reqs;
    std::vector<Req *> incoming;               // submitted, not yet arrived
    uint64_t used_bytes = 0, max_used = 0, staging_used = 0;
    uint64_t outstanding = 0;                  // submitted, not completed
    uint64_t completed = 0, keys_done = 0, nwaves = 0, wave_reqs = 0;
    double wave_gpu_ms = 0.0, launch_host_s = 0.0;
    int error = BLOWCHOC_OK;
    char error_msg[256] = {0};
    std::mutex mu;
    std::condition_variable cv_done, cv_work;
    std::thread th;
    std::atomic<bool> stop{false};
    bool started = false;
    Clock::time_point t0;
    int rr = 0;                                // round-robin start of the filter scan
    int next_stream = 0;

    double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

namespace {

constexpr int kWavesPerStream = 2;
constexpr uint64_t kHeavyRounds = 64;  // inserts needing more batches run in a wave of their own
constexpr size_t kQueryRun = 64;        // queries of one filter sharing one launch item, at most

// Cluster-resident inserts in the server: moderate clusters (4 lanes per key,
// 512 keys of a batch per CTA) for its filters and many-filter calls. Under
// concurrent waves, smaller clusters schedule more easily than the largest
// ones, and cluster launches keep waves clear of cooperative grid-wide
// kernels (64 filters, 10^4 requests: 2.2 G keys/s against 0.6 with the
// work list).
blowchoc_tuning *server_cluster_defaults(blowchoc_tuning *t) {
    t->cluster_max = 16;
    t->lanes_cluster = 4;
    t->cluster_keys = 512;
    return t;
}

int fail_locked(blowchoc_server *s, int code, const char *what, cudaError_t e) {
    if (s->error == BLOWCHOC_OK) {
        s->error = code;
        std::snprintf(s->error_msg, sizeof s->error_msg, "%s: %s", what,
                      e == cudaSuccess ? "failed" : cudaGetErrorString(e));
    }
    return code;
}

// Admit pending filters in registration order while they fit.
void admit(blowchoc_server *s) {
    for (Slot &sl : s->slots) {
        if (sl.admitted || sl.removed) continue;
        if (s->used_bytes + sl.bytes > s->cfg.hbm_budget_bytes) break;
        blowchoc_filter *f = nullptr;
        int rc = blowchoc_create(&sl.params, nullptr, &f);
        if (!rc && s->tuned) {
            rc = blowchoc_set_tuning(f, &s->tuning);
        } else if (!rc) {
            blowchoc_tuning t;
            rc = blowchoc_get_tuning(f, &t);
            if (!rc) rc = blowchoc_set_tuning(f, server_cluster_defaults(&t));
        }
        if (rc) {
            if (f) blowchoc_destroy(f);
            fail_locked(s, rc, "admitting a filter", cudaSuccess);
            return;
        }
        const cudaError_t e = cudaStreamSynchronize(nullptr);  // its zeroing is done
        if (e != cudaSuccess) {
            fail_locked(s, BLOWCHOC_ECUDA, "admitting a filter", e);
            return;
        }
        sl.f = f;
        sl.admitted = true;
        s->used_bytes += sl.bytes;
        s->max_used = std::max(s->max_used, s->used_bytes);
    }
}

void retire(blowchoc_server *s) {
    for (Slot &sl : s->slots) {
        if (sl.remove && !sl.removed && sl.admitted && sl.unlaunched == 0 && sl.inflight == 0) {
            blowchoc_destroy(sl.f);
            sl.f = nullptr;
            sl.removed = true;
            s->used_bytes -= sl.bytes;
        }
    }
}

// Completed waves: requests done, staging and stream slot released.
void collect(blowchoc_server *s) {
    for (size_t w = 0; w < s->waves.size(); ++w) {
        Wave &wv = s->waves[w];
        if (!wv.active) continue;
        const cudaError_t q = cudaEventQuery(wv.ev);
        if (q == cudaErrorNotReady) continue;
        if (q != cudaSuccess) {
            fail_locked(s, BLOWCHOC_ECUDA, "a wave failed", q);
            continue;
        }
        for (Req *r : wv.reqs) {
            if (r->bm_bounce != SIZE_MAX) {
                std::memcpy(r->h_bitmap, s->h_bm_arena + r->bm_bounce, (r->n + 63) / 64 * 8);
                s->bm_arena.release(r->bm_bounce, (r->n + 63) / 64 * 8);
                r->bm_bounce = SIZE_MAX;
            }
            if (r->clear_tail && (r->n & 63)) {
                // the padding keys after this request answered too: their bits go
                r->h_bitmap[r->n / 64] &= (1ull << (r->n & 63)) - 1ull;
                r->clear_tail = false;
            }
            if (r->key_bounce != SIZE_MAX) {
                s->keys_arena.release(r->key_bounce, r->n * 8);
                r->key_bounce = SIZE_MAX;
            }
        }
        const double t = s->now();
        for (Req *r : wv.reqs) {
            r->done = t;
            Slot &sl = s->slots[r->filter];
            sl.inflight--;
            if (sl.last_wave == (int)w) sl.last_wave = -1;
            s->completed++;
            s->keys_done += r->n;
            s->outstanding--;
        }
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, wv.start, wv.ev) == cudaSuccess) s->wave_gpu_ms += ms;
        s->staging_used -= wv.staging;
        s->stream_inflight[wv.stream]--;
        wv.active = false;
        wv.reqs.clear();
    }
    s->cv_done.notify_all();
}

// Builds and launches one wave; returns false if nothing was ready.
bool launch_wave(blowchoc_server *s) {
    int st = -1;
    for (int i = 0; i < (int)s->streams.size(); ++i) {
        const int c = (s->next_stream + i) % (int)s->streams.size();
        if (s->stream_inflight[c] < kWavesPerStream) { st = c; break; }
    }
    if (st < 0) return false;
    int wi = -1;
    for (size_t w = 0; w < s->waves.size(); ++w)
        if (!s->waves[w].active) { wi = (int)w; break; }
    if (wi < 0) return false;
    Wave &wv = s->waves[wi];
    // a wave takes, per filter, its next insert, or its next run of queries
    // (queries with no insert between them see the same filter and share one
    // launch item: their keys are concatenated, each padded to a multiple of
    // 64 so that its bitmap starts on a word of the item's bitmap)
    std::vector<std::vector<Req *>> groups;
    std::vector<Req *> take;
    uint64_t staging = 0;
    const int nf = (int)s->slots.size();
    // a heavy insert (many batches) runs alone; light requests share waves
    auto heavy = [s](const Req *r) {
        const uint64_t B = s->slots[r->filter].params.batch;
        return r->kind == BLOWCHOC_REQ_INSERT && (r->n + B - 1) / B > kHeavyRounds;
    };
    // host bounce space for a request whose buffers are not pinned
    auto bounce = [s](Req *r) {
        if (!r->keys_pinned && r->key_bounce == SIZE_MAX) {
            r->key_bounce = s->keys_arena.alloc(r->n * 8);
            if (r->key_bounce == SIZE_MAX) return false;
        }
        if (r->kind == BLOWCHOC_REQ_QUERY && !r->bitmap_pinned && r->bm_bounce == SIZE_MAX) {
            r->bm_bounce = s->bm_arena.alloc((r->n + 63) / 64 * 8);
            if (r->bm_bounce == SIZE_MAX) return false;
        }
        return true;
    };
    bool alone = false;
    for (int i = 0; i < nf && take.size() < s->cfg.max_wave_requests && !alone; ++i) {
        Slot &sl = s->slots[(s->rr + i) % nf];
        if (!sl.admitted || sl.removed || sl.fifo.empty()) continue;
        // a filter with work in flight on another stream waits for it here,
        // on the host: a device-side wait would hold the whole wave behind it
        if (sl.last_wave >= 0 && s->waves[sl.last_wave].stream != st) continue;
        Req *r = sl.fifo.front();
        if (s->staging_used + staging + r->staging > s->cfg.staging_bytes) continue;
        if (!bounce(r)) continue;
        if (heavy(r)) {
            if (take.empty()) {
                groups.push_back({r});
                take.push_back(r);
                staging += r->staging;
                alone = true;
            }
            continue;
        }
        std::vector<Req *> g{r};
        take.push_back(r);
        staging += r->staging;
        if (r->kind == BLOWCHOC_REQ_QUERY) {
            for (size_t j = 1; j < sl.fifo.size() && take.size() < s->cfg.max_wave_requests &&
                               g.size() < kQueryRun; ++j) {
                Req *q = sl.fifo[j];
                if (q->kind != BLOWCHOC_REQ_QUERY) break;
                if (s->staging_used + staging + q->staging > s->cfg.staging_bytes) break;
                if (!bounce(q)) break;
                g.push_back(q);
                take.push_back(q);
                staging += q->staging;
            }
        }
        groups.push_back(g);
    }
    if (take.empty()) return false;
    s->rr = (s->rr + 1) % std::max(nf, 1);
    s->next_stream = (st + 1) % (int)s->streams.size();
    cudaStream_t stream = s->streams[st];
    std::vector<blowchoc_work> ins, qry;
    std::vector<std::vector<Req *>> qry_groups;  // the requests behind each query item
    std::vector<void *> bufs;
    const double t = s->now();
    const auto h0 = Clock::now();
    {
        const cudaError_t e0 = cudaEventRecord(wv.start, stream);
        if (e0 != cudaSuccess) { fail_locked(s, BLOWCHOC_ECUDA, "wave event", e0); return false; }
    }
    for (const std::vector<Req *> &g : groups) {
        Slot &sl = s->slots[g.front()->filter];
        // the filter's earlier work, if still in flight, is on this stream
        // (selection above): stream order keeps its requests in FIFO order
        uint64_t padded = 0;  // keys of the item, each request but the last padded to 64
        for (size_t j = 0; j < g.size(); ++j) {
            sl.fifo.pop_front();
            padded += j + 1 < g.size() ? (g[j]->n + 63) / 64 * 64 : g[j]->n;
        }
        void *dk = nullptr, *db = nullptr;
        cudaError_t e = cudaMallocFromPoolAsync(&dk, ((padded + 63) / 64 * 64) * 8, s->pool, stream);
        uint64_t off = 0;
        for (Req *r : g) {
            if (e != cudaSuccess) break;
            const void *src = r->h_keys;
            if (r->key_bounce != SIZE_MAX) {
                std::memcpy(s->h_keys_arena + r->key_bounce, r->h_keys, r->n * 8);
                src = s->h_keys_arena + r->key_bounce;
            }
            e = cudaMemcpyAsync((uint64_t *)dk + off, src, r->n * 8, cudaMemcpyHostToDevice, stream);
            off += (r->n + 63) / 64 * 64;
        }
        if (e == cudaSuccess && g.front()->kind == BLOWCHOC_REQ_QUERY)
            e = cudaMallocFromPoolAsync(&db, (padded + 63) / 64 * 8, s->pool, stream);
        if (e != cudaSuccess) { fail_locked(s, BLOWCHOC_ECUDA, "wave staging", e); return false; }
        bufs.push_back(dk);
        if (db) bufs.push_back(db);
        blowchoc_work w{sl.f, (const uint64_t *)dk, padded, (uint64_t *)db};
        if (g.front()->kind == BLOWCHOC_REQ_QUERY) {
            qry.push_back(w);
            qry_groups.push_back(g);
        } else {
            ins.push_back(w);
        }
        for (size_t j = 0; j < g.size(); ++j) {
            Req *r = g[j];
            r->launched = t;
            r->clear_tail = j + 1 < g.size();  // padded: not the item's last request
            sl.inflight++;
            sl.unlaunched--;
        }
        sl.last_wave = wi;
    }
    int rc = BLOWCHOC_OK;
    if (!ins.empty()) rc = blowchoc_insert_many(s->batches[st], ins.data(), (uint32_t)ins.size(), stream);
    if (!rc && !qry.empty()) rc = blowchoc_query_many(s->batches[st], qry.data(), (uint32_t)qry.size(), stream);
    if (rc) { fail_locked(s, rc, "wave launch", cudaSuccess); return false; }
    for (size_t qi = 0; qi < qry_groups.size(); ++qi) {
        uint64_t woff = 0;  // each request's bitmap starts on a word of the item's bitmap
        for (Req *r : qry_groups[qi]) {
            void *dst = r->bm_bounce != SIZE_MAX ? (void *)(s->h_bm_arena + r->bm_bounce) : (void *)r->h_bitmap;
            const cudaError_t e = cudaMemcpyAsync(dst, qry[qi].d_bitmap + woff, (r->n + 63) / 64 * 8,
                                                  cudaMemcpyDeviceToHost, stream);
            if (e != cudaSuccess) { fail_locked(s, BLOWCHOC_ECUDA, "bitmap copy", e); return false; }
            woff += (r->n + 63) / 64;
        }
    }
    for (void *p : bufs) cudaFreeAsync(p, stream);
    cudaError_t e = cudaEventRecord(wv.ev, stream);
    if (e != cudaSuccess) { fail_locked(s, BLOWCHOC_ECUDA, "wave event", e); return false; }
    wv.active = true;
    wv.stream = st;
    wv.reqs = take;
    wv.staging = staging;
    s->staging_used += staging;
    s->stream_inflight[st]++;
    s->nwaves++;
    s->wave_reqs += take.size();
    s->launch_host_s += std::chrono::duration<double>(Clock::now() - h0).count();
    return true;
}

void scheduler(blowchoc_server *s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (!s->stop.load()) {
        const double t = s->now();
        // release arrived requests into their filters' FIFOs (in arrival order)
        std::vector<Req *> keep;
        for (Req *r : s->incoming) {
            if (r->arrival <= t) s->slots[r->filter].fifo.push_back(r);
            else keep.push_back(r);
        }
        s->incoming.swap(keep);
        collect(s);
        retire(s);
        admit(s);
        bool launched = false;
        if (s->error == BLOWCHOC_OK)
            while (launch_wave(s)) launched = true;
        if (s->error != BLOWCHOC_OK) s->cv_done.notify_all();
        if (!launched) {
            // sleep until the next arrival, a submission, or a short poll interval
            double next = 1e30;
            for (Req *r : s->incoming) next = std::min(next, r->arrival);
            const double wait = std::max(0.0, std::min(next - s->now(), 2e-5));
            s->cv_work.wait_for(lk, std::chrono::duration<double>(wait));
        }
    }
}

}  // namespace

extern "C" {

int blowchoc_server_create(const blowchoc_server_config *cfg, blowchoc_server **out) {
    if (!cfg || !out) return bc_set_error(BLOWCHOC_EINVAL, "NULL argument");
    *out = nullptr;
    if (cfg->streams < 1 || cfg->streams > 16 || cfg->max_wave_requests < 1 || cfg->staging_bytes == 0)
        return bc_set_error(BLOWCHOC_EINVAL, "bad server configuration");
    blowchoc_server *s = new blowchoc_server();
    s->cfg = *cfg;
    cudaError_t e = cudaGetDevice(&s->device);
    for (uint32_t i = 0; e == cudaSuccess && i < cfg->streams; ++i) {
        cudaStream_t st;
        e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (e == cudaSuccess) s->streams.push_back(st);
        blowchoc_batch *b = nullptr;
        if (e == cudaSuccess && blowchoc_batch_create(&b)) e = cudaErrorMemoryAllocation;
        if (e == cudaSuccess) {
            s->batches.push_back(b);
            blowchoc_tuning t;
            if (blowchoc_batch_get_tuning(b, &t) || blowchoc_batch_set_tuning(b, server_cluster_defaults(&t)))
                e = cudaErrorInvalidValue;
        }
    }
    if (e == cudaSuccess) {
        cudaMemPoolProps props;
        std::memset(&props, 0, sizeof props);
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = s->device;
        e = cudaMemPoolCreate(&s->pool, &props);
        if (e == cudaSuccess) {
            uint64_t keep = cfg->staging_bytes;
            e = cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
    }
    if (e == cudaSuccess) {
        const size_t kb = (size_t)cfg->staging_bytes, bb = (size_t)(cfg->staging_bytes / 32 + (1 << 20));
        e = cudaHostAlloc((void **)&s->h_keys_arena, kb, cudaHostAllocDefault);
        if (e == cudaSuccess) e = cudaHostAlloc((void **)&s->h_bm_arena, bb, cudaHostAllocDefault);
        if (e == cudaSuccess) {
            s->keys_arena.init(s->h_keys_arena, kb);
            s->bm_arena.init(s->h_bm_arena, bb);
        }
    }
    s->stream_inflight.assign(s->streams.size(), 0);
    s->waves.resize(s->streams.size() * kWavesPerStream + 1);
    for (Wave &w : s->waves) {
        if (e == cudaSuccess) e = cudaEventCreate(&w.ev);
        if (e == cudaSuccess) e = cudaEventCreate(&w.start);
    }
    if (e != cudaSuccess) {
        blowchoc_server_destroy(s);
        return bc_set_error(BLOWCHOC_ECUDA, "blowchoc_server_create failed");
    }
    *out = s;
    return BLOWCHOC_OK;
}

int blowchoc_server_add_filter(blowchoc_server *s, const blowchoc_params *p, uint32_t *id) {
    if (!s || !p || !id) return bc_set_error(BLOWCHOC_EINVAL, "NULL argument");
    if (p->nblocks == 0 || p->k < 1 || p->k > 32 || p->choices < 1 || p->choices > 3 || p->batch == 0)
        return bc_set_error(BLOWCHOC_EINVAL, "bad filter parameters");
    Slot sl;
    sl.params = *p;
    sl.bytes = filter_bytes(*p);
    if (sl.bytes > s->cfg.hbm_budget_bytes)
        return bc_set_error(BLOWCHOC_EBUDGET, "filter larger than the whole HBM budget");
    std::lock_guard<std::mutex> lk(s->mu);
    *id = (uint32_t)s->slots.size();
    s->slots.push_back(std::move(sl));
    if (!s->started) admit(s);
    s->cv_work.notify_one();
    return BLOWCHOC_OK;
}

int blowchoc_server_remove_filter(blowchoc_server *s, uint32_t id) {
    if (!s) return bc_set_error(BLOWCHOC_EINVAL, "server is NULL");
    std::lock_guard<std::mutex> lk(s->mu);
    if (id >= s->slots.size()) return bc_set_error(BLOWCHOC_EINVAL, "unknown filter id");
    s->slots[id].remove = true;
    s->cv_work.notify_one();
    return BLOWCHOC_OK;
}

int blowchoc_server_submit(blowchoc_server *s, uint32_t filter_id, uint32_t kind, const uint64_t *h_keys,
                           uint64_t n, uint64_t *h_bitmap, double arrival_s, uint64_t *req_id) {
    if (!s) return bc_set_error(BLOWCHOC_EINVAL, "server is NULL");
    if (kind > 1 || n == 0 || !h_keys || (kind == BLOWCHOC_REQ_QUERY && !h_bitmap))
        return bc_set_error(BLOWCHOC_EINVAL, "bad request");
    std::unique_ptr<Req> r(new Req());
    r->filter = filter_id;
    r->kind = kind;
    r->h_keys = h_keys;
    r->n = n;
    r->h_bitmap = h_bitmap;
    r->staging = ((n * 8 + 511) & ~uint64_t(511)) + (kind ? ((n + 63) / 64 * 8 + 511) & ~uint64_t(511) : 0);
    r->keys_pinned = is_pinned(h_keys);
    r->bitmap_pinned = kind == BLOWCHOC_REQ_QUERY && is_pinned(h_bitmap);
    if (r->staging > s->cfg.staging_bytes) return bc_set_error(BLOWCHOC_EBUDGET, "request larger than staging");
    std::lock_guard<std::mutex> lk(s->mu);
    if (filter_id >= s->slots.size() || s->slots[filter_id].remove)
        return bc_set_error(BLOWCHOC_EINVAL, "unknown or removed filter");
    r->id = s->reqs.size();
    r->arrival = s->started ? std::max(arrival_s, s->now()) : arrival_s;
    if (req_id) *req_id = r->id;
    s->incoming.push_back(r.get());
    s->slots[filter_id].unlaunched++;
    s->reqs.push_back(std::move(r));
    s->outstanding++;
    s->cv_work.notify_one();
    return BLOWCHOC_OK;
}

int blowchoc_server_set_tuning(blowchoc_server *s, const blowchoc_tuning *t) {
    if (!s || !t) return bc_set_error(BLOWCHOC_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->started) return bc_set_error(BLOWCHOC_EINVAL, "server already started");
    int rc0 = bc_check_tuning(t);
    if (rc0) return rc0;
    for (blowchoc_batch *b : s->batches) {
        const int rc = blowchoc_batch_set_tuning(b, t);
        if (rc) return rc;
    }
    s->tuning = *t;
    s->tuned = true;
    return BLOWCHOC_OK;
}

int blowchoc_server_start(blowchoc_server *s) {
    if (!s) return bc_set_error(BLOWCHOC_EINVAL, "server is NULL");
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->started) return bc_set_error(BLOWCHOC_EINVAL, "server already started");
    std::sort(s->incoming.begin(), s->incoming.end(),
              [](const Req *a, const Req *b) { return a->arrival < b->arrival || (a->arrival == b->arrival && a->id < b->id); });
    s->t0 = Clock::now();
    s->started = true;
    s->th = std::thread(scheduler, s);
    return BLOWCHOC_OK;
}

int blowchoc_server_wait(blowchoc_server *s, double timeout_s) {
    if (!s || !s->started) return bc_set_error(BLOWCHOC_EINVAL, "server not started");
    std::unique_lock<std::mutex> lk(s->mu);
    const bool ok = s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s),
                                        [s] { return s->outstanding == 0 || s->error != BLOWCHOC_OK; });
    if (s->error != BLOWCHOC_OK) return bc_set_error(s->error, s->error_msg);
    if (!ok) return bc_set_error(BLOWCHOC_ETIMEOUT, "requests still outstanding");
    return BLOWCHOC_OK;
}

int blowchoc_server_request_times(blowchoc_server *s, uint64_t req_id, double *arrival, double *launch,
                                  double *done) {
    if (!s || !arrival || !launch || !done) return bc_set_error(BLOWCHOC_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    if (req_id >= s->reqs.size()) return bc_set_error(BLOWCHOC_EINVAL, "unknown request");
    const Req &r = *s->reqs[req_id];
    *arrival = r.arrival;
    *launch = r.launched;
    *done = r.done;
    return BLOWCHOC_OK;
}

int blowchoc_server_stats(blowchoc_server *s, blowchoc_server_summary *out) {
    if (!s || !out) return bc_set_error(BLOWCHOC_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    std::memset(out, 0, sizeof *out);
    std::vector<double> lat;
    double first = 1e30, last = 0.0;
    for (const auto &r : s->reqs) {
        if (r->done < 0.0) continue;
        lat.push_back(r->done - r->arrival);
        first = std::min(first, r->arrival);
        last = std::max(last, r->done);
    }
    out->completed = s->completed;
    out->keys = s->keys_done;
    out->waves = s->nwaves;
    out->mean_wave_requests = s->nwaves ? (double)s->wave_reqs / (double)s->nwaves : 0.0;
    out->max_filter_bytes_used = s->max_used;
    out->mean_wave_gpu_ms = s->nwaves ? s->wave_gpu_ms / (double)s->nwaves : 0.0;
    out->launch_host_s = s->launch_host_s;
    for (const Slot &sl : s->slots) {
        if (sl.admitted && !sl.removed) out->filters_admitted++;
        if (!sl.admitted && !sl.removed) out->filters_pending++;
    }
    if (!lat.empty()) {
        std::sort(lat.begin(), lat.end());
        auto pct = [&](double p) { return lat[std::min(lat.size() - 1, (size_t)(p * (double)lat.size()))]; };
        out->p50_latency_s = pct(0.50);
        out->p99_latency_s = pct(0.99);
        out->max_latency_s = lat.back();
        out->first_arrival_s = first;
        out->last_done_s = last;
    }
    return BLOWCHOC_OK;
}

int blowchoc_server_filter(blowchoc_server *s, uint32_t id, blowchoc_filter **f) {
    if (!s || !f) return bc_set_error(BLOWCHOC_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    if (id >= s->slots.size()) return bc_set_error(BLOWCHOC_EINVAL, "unknown filter id");
    *f = s->slots[id].admitted && !s->slots[id].removed ? s->slots[id].f : nullptr;
    return BLOWCHOC_OK;
}

int blowchoc_server_destroy(blowchoc_server *s) {
    if (!s) return BLOWCHOC_OK;
    s->stop.store(true);
    s->cv_work.notify_all();
    if (s->th.joinable()) s->th.join();
    for (cudaStream_t st : s->streams) cudaStreamSynchronize(st);
    for (Slot &sl : s->slots)
        if (sl.f) blowchoc_destroy(sl.f);
    for (blowchoc_batch *b : s->batches) blowchoc_batch_destroy(b);
    for (Wave &w : s->waves) {
        if (w.ev) cudaEventDestroy(w.ev);
        if (w.start) cudaEventDestroy(w.start);
    }
    for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
    if (s->pool) cudaMemPoolDestroy(s->pool);
    cudaFreeHost(s->h_keys_arena);
    cudaFreeHost(s->h_bm_arena);
    delete s;
    return BLOWCHOC_OK;
}

}  // extern "C"
