// Insert and query from host buffers: the keys move to the device in chunks
// through a ring of staging slots on a copy stream, so that the copies of the
// next chunks overlap the kernels of chunk i on the caller's stream (and the
// copies of a query's first chunks overlap the previous insert's kernels); query bitmaps come
// back on a second stream, so that they never queue in front of keys. Insert chunks are
// whole multiples of the filter's batch size B, so that the batch sequence is
// exactly that of one blowchoc_insert over all keys (each call starts its
// batches at its first key, and every chunk edge is a batch edge). Query
// chunks are multiples of 64 keys, so that each chunk's bitmap is a run of
// whole words of the caller's bitmap.
#include <cstdio>
#include <cstring>

#include "bc_filter.h"

// Staging of the host-buffer calls: a ring of device slots, a stream for
// keys to the device, one for bitmaps back, and the events that order each
// slot between those streams and the caller's stream. The ring's cursor runs
// on across calls, so the copies of a call's first chunks go to slots that
// the previous call's kernels have already released, and overlap them.
// The DNA benchmark step end to end (1.2 GB of keys from pinned memory on a
// box copying 211 GB/s) took 7.95 ms with 2 slots, 7.63 with 4, 7.28 with 8,
// and 7.26 to 10.77 ms with 16 (deeper prefetch competed with the kernels).
constexpr int kHostSlots = 8;

struct HostStage {
    uint64_t *d_keys = nullptr;    // kHostSlots x chunk keys
    uint64_t *d_bitmap = nullptr;  // kHostSlots x chunk / 64 words
    uint64_t chunk = 0;            // keys per slot
    int nslots = 0;                // slots in the ring: kHostSlots, or 2 for chunks above 2^22 keys
    int next = 0;                  // the ring's next slot
    cudaStream_t copy = nullptr;   // keys to the device
    cudaStream_t back = nullptr;   // bitmaps to the host (its own queue, so that it never holds up keys)
    cudaEvent_t copied[kHostSlots] = {};   // keys of the slot are on the device
    cudaEvent_t used[kHostSlots] = {};     // the slot's keys were consumed
    cudaEvent_t drained[kHostSlots] = {};  // the slot's bitmap was copied out
    cudaEvent_t done = nullptr;            // the bitmap stream's last work
};

namespace {

constexpr uint64_t kHostChunkKeys = 1ull << 22;  // about 32 MB of keys per slot (256 MB in all)

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

// Staging of at least `chunk` keys per slot (and chunk / 64 bitmap words).
int ensure_stage(blowchoc_filter *f, uint64_t chunk) {
    if (!f->host) f->host = new HostStage();
    HostStage &h = *f->host;
    if (!h.copy) {
        HOST_CUDA(cudaStreamCreateWithFlags(&h.copy, cudaStreamNonBlocking), "copy stream");
        HOST_CUDA(cudaStreamCreateWithFlags(&h.back, cudaStreamNonBlocking), "copy stream");
        for (int i = 0; i < kHostSlots; ++i) {
            HOST_CUDA(cudaEventCreateWithFlags(&h.copied[i], cudaEventDisableTiming), "staging events");
            HOST_CUDA(cudaEventCreateWithFlags(&h.used[i], cudaEventDisableTiming), "staging events");
            HOST_CUDA(cudaEventCreateWithFlags(&h.drained[i], cudaEventDisableTiming), "staging events");
        }
        HOST_CUDA(cudaEventCreateWithFlags(&h.done, cudaEventDisableTiming), "staging events");
    }
    if (h.chunk >= chunk) return BLOWCHOC_OK;
    HOST_CUDA(cudaStreamSynchronize(h.copy), "staging resize");
    HOST_CUDA(cudaStreamSynchronize(h.back), "staging resize");
    HOST_CUDA(cudaDeviceSynchronize(), "staging resize");  // earlier kernels may still read the old slots
    cudaFree(h.d_keys);
    cudaFree(h.d_bitmap);
    h.d_keys = nullptr;
    h.d_bitmap = nullptr;
    h.chunk = 0;
    const int nslots = chunk <= kHostChunkKeys ? kHostSlots : 2;  // whole batches above 2^22 keys: two
    HOST_CUDA(cudaMalloc(&h.d_keys, nslots * chunk * sizeof(uint64_t)), "staging keys");
    HOST_CUDA(cudaMalloc(&h.d_bitmap, nslots * (chunk / 64) * sizeof(uint64_t)), "staging bitmap");
    h.chunk = chunk;
    h.nslots = nslots;
    h.next = 0;
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
    for (int i = 0; i < kHostSlots; ++i) {
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
    const uint64_t B = f->p.batch;
    // whole batches per chunk; a batch larger than the chunk is one chunk
    uint64_t chunk = B >= kHostChunkKeys ? B : (kHostChunkKeys / B) * B;
    if (chunk > n) chunk = n;
    int rc = ensure_stage(f, chunk);
    if (rc) return rc;
    HostStage &h = *f->host;
    for (uint64_t off = 0; off < n; off += chunk) {
        const int slot = h.next;
        h.next = (h.next + 1) % h.nslots;
        const uint64_t cnt = n - off < chunk ? n - off : chunk;
        uint64_t *dst = h.d_keys + (uint64_t)slot * h.chunk;
        HOST_CUDA(cudaStreamWaitEvent(h.copy, h.used[slot], 0), "staging order");
        HOST_CUDA(cudaMemcpyAsync(dst, h_keys + off, cnt * sizeof(uint64_t), cudaMemcpyHostToDevice, h.copy),
                  "keys to the device");
        HOST_CUDA(cudaEventRecord(h.copied[slot], h.copy), "staging order");
        HOST_CUDA(cudaStreamWaitEvent(s, h.copied[slot], 0), "staging order");
        rc = blowchoc_insert(f, dst, cnt, s);
        if (rc) return rc;
        HOST_CUDA(cudaEventRecord(h.used[slot], s), "staging order");
    }
    return BLOWCHOC_OK;
}

int blowchoc_query_host(blowchoc_filter *f, const uint64_t *h_keys, uint64_t n, uint64_t *h_bitmap, void *stream) {
    if (!f) return bc_set_error(BLOWCHOC_EINVAL, "filter is NULL");
    if (n == 0) return BLOWCHOC_OK;
    if (!h_keys || !h_bitmap) return bc_set_error(BLOWCHOC_EINVAL, "keys or bitmap is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    uint64_t chunk = kHostChunkKeys;  // a multiple of 64
    int rc = ensure_stage(f, chunk < n ? chunk : ((n + 63) / 64) * 64);
    if (rc) return rc;
    HostStage &h = *f->host;
    chunk = h.chunk / 64 * 64;  // a slot may be larger (an insert sized it to whole batches)
    for (uint64_t off = 0; off < n; off += chunk) {
        const int slot = h.next;
        h.next = (h.next + 1) % h.nslots;
        const uint64_t cnt = n - off < chunk ? n - off : chunk;
        uint64_t *dk = h.d_keys + (uint64_t)slot * h.chunk;
        uint64_t *db = h.d_bitmap + (uint64_t)slot * (h.chunk / 64);
        HOST_CUDA(cudaStreamWaitEvent(h.copy, h.used[slot], 0), "staging order");
        HOST_CUDA(cudaMemcpyAsync(dk, h_keys + off, cnt * sizeof(uint64_t), cudaMemcpyHostToDevice, h.copy),
                  "keys to the device");
        HOST_CUDA(cudaEventRecord(h.copied[slot], h.copy), "staging order");
        HOST_CUDA(cudaStreamWaitEvent(s, h.copied[slot], 0), "staging order");
        HOST_CUDA(cudaStreamWaitEvent(s, h.drained[slot], 0), "staging order");  // the slot's last bitmap is out
        rc = blowchoc_query(f, dk, cnt, db, s);
        if (rc) return rc;
        HOST_CUDA(cudaEventRecord(h.used[slot], s), "staging order");
        HOST_CUDA(cudaStreamWaitEvent(h.back, h.used[slot], 0), "staging order");
        HOST_CUDA(cudaMemcpyAsync(h_bitmap + off / 64, db, (cnt + 63) / 64 * sizeof(uint64_t),
                                  cudaMemcpyDeviceToHost, h.back),
                  "bitmap to the host");
        HOST_CUDA(cudaEventRecord(h.drained[slot], h.back), "staging order");
    }
    // the caller's stream completes only after the last bitmap reached the host
    HOST_CUDA(cudaEventRecord(h.done, h.back), "staging order");
    HOST_CUDA(cudaStreamWaitEvent(s, h.done, 0), "staging order");
    return BLOWCHOC_OK;
}

}  // extern "C"
