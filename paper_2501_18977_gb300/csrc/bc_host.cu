// Insert and query from host buffers: the keys move to the device in chunks
// through a staging ring on a copy stream, so that the copies of the next
// chunks overlap the kernels of chunk i on the caller's stream (and the
// copies of a query's first chunks overlap the previous insert's kernels);
// query bitmaps come back on a second stream, so that they never queue in
// front of keys. Insert chunks are whole multiples of the filter's batch size
// B, so that the batch sequence is exactly that of one blowchoc_insert over
// all keys (each call starts its batches at its first key, and every chunk
// edge is a batch edge). Query chunks are multiples of 64 keys, so that each
// chunk's bitmap is a run of whole words of the caller's bitmap.
#include <cstdio>
#include <cstring>
#include <deque>
#include <vector>

#include "bc_filter.h"

// Staging of the host-buffer calls: one contiguous device ring of keys (and
// a bitmap ring of one word per 64 keys at the same offsets), a stream for
// keys to the device, one for bitmaps back, and per chunk a set of events
// that order its piece of the ring between those streams and the caller's.
//
// Chunks grow within a call, from 2^20 keys up to 2^24 (or a quarter of the
// ring): the first copy is short, so the kernels start early, and the later
// ones are few, so the launches are few. A chunk takes the next free span of
// the ring (wrapping to its start when it does not fit before the end); the
// copy stream first waits until every earlier chunk that held any of that
// span has been consumed (and, for a query chunk, until its bitmap left). The
// ring position runs on across calls, so a query's first copies go to space
// that the previous insert's kernels release first, and overlap them.
//
// A query call on an idle device is bound by the copies (the query kernel
// consumes keys faster than they arrive), and its last chunk's kernel time is
// exposed after the last copy: its chunks stop at 2^22 keys. Whether the
// device is idle is read from the previous chunk's consumed event: while
// earlier work is queued, the copies run ahead of the kernels and chunks
// grow to 2^24. Inserts are bound by their kernels either way.
//
// The DNA benchmark step end to end (1.2 GB of keys from pinned memory,
// 50 M inserted, 100 M queried) ran 7.25 ms with eight fixed slots of 2^22
// keys, whose 36 launches per step cost 0.32 ms of kernel time over one
// launch per phase, and 6.95 ms with this ring. A model of the copy engine
// and the kernels gave 7.04 and 6.75 ms; for 10^8 queries alone it gave
// 3.97 ms with chunks of 2^22 and 4.35 ms with chunks growing to 2^24
// (4.36 ms measured).
struct HostStage {
    struct Chunk {
        uint64_t lo, hi;  // span of the ring, in keys (multiples of 64)
        int ev;           // its event set
        bool query;       // a bitmap leaves through the bitmap ring
    };
    uint64_t *d_keys = nullptr;    // ring keys
    uint64_t *d_bitmap = nullptr;  // ring / 64 words: a chunk's bitmap at its keys' offset / 64
    uint64_t ring = 0;             // keys in the ring (a multiple of 64)
    uint64_t pos = 0;              // where the next chunk goes (a multiple of 64)
    cudaStream_t copy = nullptr;   // keys to the device
    cudaStream_t back = nullptr;   // bitmaps to the host (its own queue, so that it never holds up keys)
    std::deque<Chunk> pending;     // chunks whose span was not handed out again, oldest first
    std::vector<cudaEvent_t> copied, used, drained;  // event sets: keys on the device, consumed, bitmap out
    std::vector<int> free_sets;
    cudaEvent_t done = nullptr;    // the bitmap stream's last work
};

namespace {

constexpr uint64_t kRingDefaultKeys = 1ull << 27;  // 1 GiB of keys
constexpr uint64_t kFirstChunkKeys = 1ull << 20;
constexpr uint64_t kMaxChunkKeys = 1ull << 24;
constexpr uint64_t kIdleQueryChunkKeys = 1ull << 22;  // query chunks on an idle device
constexpr int kEventSets = 64;  // chunks tracked at once; the oldest is retired when all are taken

uint64_t round64(uint64_t v) { return (v + 63) / 64 * 64; }

int cuda_fail(cudaError_t e, const char *what) {
    char msg[256];
    std::snprintf(msg, sizeof msg, "%s: %s", what, cudaGetErrorString(e));
    return bc_set_error(e == cudaErrorMemoryAllocation ? BLOWCHOC_ENOMEM : BLOWCHOC_ECUDA, msg);
}

#define HOST_CUDA(call, what)                              \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

// The ring limit of f, in keys (a multiple of 64).
uint64_t ring_limit(const blowchoc_filter *f) {
    return f->host_ring_keys ? (uint64_t)f->host_ring_keys / 64 * 64 : kRingDefaultKeys;
}

// Largest chunk of a call on f, before rounding to whole batches.
uint64_t chunk_cap(const blowchoc_filter *f) {
    const uint64_t q = ring_limit(f) / 4 / 64 * 64;
    return q < kMaxChunkKeys ? (q > 64 ? q : 64) : kMaxChunkKeys;
}

// Chunk sizes of one call: start at min(2^20, cap), double up to cap; with
// unit > 1 (inserts: the batch size) every chunk is a whole number of units.
struct ChunkSizes {
    uint64_t unit, cap, next;
    ChunkSizes(uint64_t unit_, uint64_t cap_) : unit(unit_), cap(cap_) {
        next = kFirstChunkKeys < cap ? kFirstChunkKeys : cap;
    }
    uint64_t whole(uint64_t c) const { return c < unit ? unit : c / unit * unit; }
    uint64_t largest() const { return whole(cap); }
    uint64_t take(uint64_t left) {
        uint64_t c = whole(next);
        next = next * 2 < cap ? next * 2 : cap;
        return c < left ? c : left;
    }
};

// Streams, events and a ring of at least `want` keys (a multiple of 64).
int ensure_stage(blowchoc_filter *f, uint64_t want) {
    if (!f->host) f->host = new HostStage();
    HostStage &h = *f->host;
    if (!h.copy) {
        HOST_CUDA(cudaStreamCreateWithFlags(&h.copy, cudaStreamNonBlocking), "copy stream");
        HOST_CUDA(cudaStreamCreateWithFlags(&h.back, cudaStreamNonBlocking), "copy stream");
        h.copied.assign(kEventSets, nullptr);
        h.used.assign(kEventSets, nullptr);
        h.drained.assign(kEventSets, nullptr);
        for (int i = 0; i < kEventSets; ++i) {
            HOST_CUDA(cudaEventCreateWithFlags(&h.copied[i], cudaEventDisableTiming), "staging events");
            HOST_CUDA(cudaEventCreateWithFlags(&h.used[i], cudaEventDisableTiming), "staging events");
            HOST_CUDA(cudaEventCreateWithFlags(&h.drained[i], cudaEventDisableTiming), "staging events");
            h.free_sets.push_back(i);
        }
        HOST_CUDA(cudaEventCreateWithFlags(&h.done, cudaEventDisableTiming), "staging events");
    }
    if (h.ring >= want) return BLOWCHOC_OK;
    HOST_CUDA(cudaStreamSynchronize(h.copy), "staging resize");
    HOST_CUDA(cudaStreamSynchronize(h.back), "staging resize");
    HOST_CUDA(cudaDeviceSynchronize(), "staging resize");  // earlier kernels may still read the old ring
    for (const HostStage::Chunk &c : h.pending) h.free_sets.push_back(c.ev);
    h.pending.clear();
    cudaFree(h.d_keys);
    cudaFree(h.d_bitmap);
    h.d_keys = nullptr;
    h.d_bitmap = nullptr;
    h.ring = 0;
    h.pos = 0;
    HOST_CUDA(cudaMalloc(&h.d_keys, want * sizeof(uint64_t)), "staging keys");
    HOST_CUDA(cudaMalloc(&h.d_bitmap, want / 64 * sizeof(uint64_t)), "staging bitmap");
    h.ring = want;
    return BLOWCHOC_OK;
}

// Ring for a call of n keys whose chunks are at most `largest`: no more than
// the call needs up to the limit, and room for two of its chunks at least.
int stage_for(blowchoc_filter *f, uint64_t n, uint64_t largest) {
    const uint64_t lim = ring_limit(f);
    const uint64_t big = round64(largest < n ? largest : n);
    uint64_t want = round64(n < lim ? n : lim);
    if (want < 2 * big) want = 2 * big;
    return ensure_stage(f, want);
}

// Hands chunk set `c` back once the copy stream waits for it: its keys were
// consumed and, for a query chunk, its bitmap reached the host.
int retire(HostStage &h, const HostStage::Chunk &c) {
    HOST_CUDA(cudaStreamWaitEvent(h.copy, h.used[c.ev], 0), "staging order");
    if (c.query) HOST_CUDA(cudaStreamWaitEvent(h.copy, h.drained[c.ev], 0), "staging order");
    h.free_sets.push_back(c.ev);
    return BLOWCHOC_OK;
}

// The span and event set of the next chunk of `cnt` keys. Before the copy
// stream writes the span, it waits for every earlier chunk that held part of
// it. Any kernel that later uses the span waits for the chunk's copy, which
// follows those waits on the copy stream.
int place(HostStage &h, uint64_t cnt, bool query, HostStage::Chunk *out) {
    const uint64_t span = round64(cnt);
    if (h.pos + span > h.ring) h.pos = 0;
    const uint64_t lo = h.pos, hi = lo + span;
    h.pos = hi;
    for (auto it = h.pending.begin(); it != h.pending.end();) {
        if (it->lo < hi && lo < it->hi) {
            int rc = retire(h, *it);
            if (rc) return rc;
            it = h.pending.erase(it);
        } else {
            ++it;
        }
    }
    if (h.free_sets.empty()) {  // every set is taken: retire the oldest chunk
        int rc = retire(h, h.pending.front());
        if (rc) return rc;
        h.pending.pop_front();
    }
    const int ev = h.free_sets.back();
    h.free_sets.pop_back();
    *out = HostStage::Chunk{lo, hi, ev, query};
    h.pending.push_back(*out);
    return BLOWCHOC_OK;
}

}  // namespace

void bc_free_host_stage(blowchoc_filter *f) {
    if (!f->host) return;
    HostStage &h = *f->host;
    if (h.copy) cudaStreamSynchronize(h.copy);
    if (h.back) cudaStreamSynchronize(h.back);
    cudaFree(h.d_keys);
    cudaFree(h.d_bitmap);
    for (size_t i = 0; i < h.copied.size(); ++i) {
        if (h.copied[i]) cudaEventDestroy(h.copied[i]);
        if (h.used[i]) cudaEventDestroy(h.used[i]);
        if (h.drained[i]) cudaEventDestroy(h.drained[i]);
    }
    if (h.done) cudaEventDestroy(h.done);
    if (h.copy) cudaStreamDestroy(h.copy);
    if (h.back) cudaStreamDestroy(h.back);
    delete f->host;
    f->host = nullptr;
}

extern "C" {

int blowchoc_insert_host(blowchoc_filter *f, const uint64_t *h_keys, uint64_t n, void *stream) {
    if (!f) return bc_set_error(BLOWCHOC_EINVAL, "filter is NULL");
    if (n == 0) return BLOWCHOC_OK;
    if (!h_keys) return bc_set_error(BLOWCHOC_EINVAL, "keys are NULL");
    cudaStream_t s = (cudaStream_t)stream;
    ChunkSizes sizes(f->p.batch, chunk_cap(f));  // whole batches; a batch above the cap is one chunk
    int rc = stage_for(f, n, sizes.largest());
    if (rc) return rc;
    HostStage &h = *f->host;
    for (uint64_t off = 0; off < n;) {
        const uint64_t cnt = sizes.take(n - off);
        HostStage::Chunk c;
        rc = place(h, cnt, false, &c);
        if (rc) return rc;
        uint64_t *dst = h.d_keys + c.lo;
        HOST_CUDA(cudaMemcpyAsync(dst, h_keys + off, cnt * sizeof(uint64_t), cudaMemcpyHostToDevice, h.copy),
                  "keys to the device");
        HOST_CUDA(cudaEventRecord(h.copied[c.ev], h.copy), "staging order");
        HOST_CUDA(cudaStreamWaitEvent(s, h.copied[c.ev], 0), "staging order");
        rc = blowchoc_insert(f, dst, cnt, s);
        if (rc) return rc;
        HOST_CUDA(cudaEventRecord(h.used[c.ev], s), "staging order");
        off += cnt;
    }
    return BLOWCHOC_OK;
}

int blowchoc_query_host(blowchoc_filter *f, const uint64_t *h_keys, uint64_t n, uint64_t *h_bitmap, void *stream) {
    if (!f) return bc_set_error(BLOWCHOC_EINVAL, "filter is NULL");
    if (n == 0) return BLOWCHOC_OK;
    if (!h_keys || !h_bitmap) return bc_set_error(BLOWCHOC_EINVAL, "keys or bitmap is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    uint64_t cap = chunk_cap(f);
    const bool busy = f->host && !f->host->pending.empty() &&
                      cudaEventQuery(f->host->used[f->host->pending.back().ev]) == cudaErrorNotReady;
    if (!busy && cap > kIdleQueryChunkKeys) cap = kIdleQueryChunkKeys;
    ChunkSizes sizes(64, cap);  // whole bitmap words
    int rc = stage_for(f, n, sizes.largest());
    if (rc) return rc;
    HostStage &h = *f->host;
    for (uint64_t off = 0; off < n;) {
        const uint64_t cnt = sizes.take(n - off);
        HostStage::Chunk c;
        rc = place(h, cnt, true, &c);
        if (rc) return rc;
        uint64_t *dk = h.d_keys + c.lo;
        uint64_t *db = h.d_bitmap + c.lo / 64;
        HOST_CUDA(cudaMemcpyAsync(dk, h_keys + off, cnt * sizeof(uint64_t), cudaMemcpyHostToDevice, h.copy),
                  "keys to the device");
        HOST_CUDA(cudaEventRecord(h.copied[c.ev], h.copy), "staging order");
        HOST_CUDA(cudaStreamWaitEvent(s, h.copied[c.ev], 0), "staging order");
        rc = blowchoc_query(f, dk, cnt, db, s);
        if (rc) return rc;
        HOST_CUDA(cudaEventRecord(h.used[c.ev], s), "staging order");
        HOST_CUDA(cudaStreamWaitEvent(h.back, h.used[c.ev], 0), "staging order");
        HOST_CUDA(cudaMemcpyAsync(h_bitmap + off / 64, db, (cnt + 63) / 64 * sizeof(uint64_t),
                                  cudaMemcpyDeviceToHost, h.back),
                  "bitmap to the host");
        HOST_CUDA(cudaEventRecord(h.drained[c.ev], h.back), "staging order");
        off += cnt;
    }
    // the caller's stream completes only after the last bitmap reached the host
    HOST_CUDA(cudaEventRecord(h.done, h.back), "staging order");
    HOST_CUDA(cudaStreamWaitEvent(s, h.done, 0), "staging order");
    return BLOWCHOC_OK;
}

}  // extern "C"
