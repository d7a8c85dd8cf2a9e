// blowchoc_insert_noalloc: insertion that never allocates device memory.
//
// The regular blowchoc_insert keeps each batch's per-key choices in a device
// buffer that it allocates (and grows) on demand. Some callers cannot let a
// library call cudaMalloc at insert time: applications whose device memory is
// entirely handed out by their own allocator or fixed budget, and latency-
// critical loops (a serving loop, code between CUDA graph replays) where an
// allocation may synchronise the device. This entry point keeps the choices
// in a fixed array in the library's own device image instead.
#include <cstdio>
#include <mutex>

#include "bc_filter.h"
#include "bc_launch.h"

// Choice bytes of one batch: at most this many keys per batch on the path
// that needs them (batches that run over the whole grid).
static constexpr uint64_t kNoAllocMaxBatch = 1ull << 22;  // 4,194,304 keys, 4 MiB

// Every device that loads the library holds its own copy until the process
// exits. In host code this name is only a host-side stand-in: the device
// address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) uint8_t g_noalloc_choices[kNoAllocMaxBatch];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
uint8_t *g_choices_addr[kMaxDevices] = {};

// Device address of g_noalloc_choices on the current device `dev`, looked up
// once per device (with that device current) and kept for the life of the
// process: a device reset, which unloads the module, leaves it stale, so the
// library must not be used after one. Returns nullptr on failure.
uint8_t *choices_on(int dev, cudaError_t *err) {
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (g_choices_addr[dev] == nullptr) {
        void *ptr = nullptr;
        *err = cudaGetSymbolAddress(&ptr, g_noalloc_choices);
        if (*err != cudaSuccess) return nullptr;
        g_choices_addr[dev] = static_cast<uint8_t *>(ptr);
    }
    *err = cudaSuccess;
    return g_choices_addr[dev];
}

int noalloc_cuda_error(cudaError_t e) {
    char msg[200];
    std::snprintf(msg, sizeof msg, "blowchoc_insert_noalloc: %s", cudaGetErrorString(e));
    return bc_set_error(BLOWCHOC_ECUDA, msg);
}

}  // namespace

extern "C" int blowchoc_insert_noalloc(blowchoc_filter *f, const uint64_t *d_keys, uint64_t n,
                                       void *stream) {
    if (!f) return bc_set_error(BLOWCHOC_EINVAL, "filter is NULL");
    if (n == 0) return BLOWCHOC_OK;
    if (!d_keys) return bc_set_error(BLOWCHOC_EINVAL, "keys is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    const int C = (int)f->p.choices;
    const uint64_t B = f->p.batch;
    cudaError_t e = cudaSuccess;
    if (B == 1) {
        e = bc::launch_sequential(C, s, f->dev, d_keys, n, f->d_rank, f->d_counters);
        if (e != cudaSuccess) return noalloc_cuda_error(e);
        bc_note_launch();
        return BLOWCHOC_OK;
    }
    // the single-CTA kernel takes the batches that blowchoc_insert also runs in
    // one CTA; larger ones run over the whole grid (choose/set pairs below)
    if (B <= bc::kSingleCtaBatch || (!f->persistent && B <= bc::kSmallBatchMax)) {
        bc::Launch L{1, f->lanes_choose, s};
        e = bc::launch_small_batch(C, L, f->dev, d_keys, n, B, f->d_rank, f->d_counters);
        if (e != cudaSuccess) return noalloc_cuda_error(e);
        bc_note_launch();
        return BLOWCHOC_OK;
    }
    const uint64_t per_batch = B < n ? B : n;
    if (per_batch > kNoAllocMaxBatch) {
        char msg[160];
        std::snprintf(msg, sizeof msg,
                      "blowchoc_insert_noalloc: a batch of %llu keys exceeds the fixed scratch of %llu keys",
                      (unsigned long long)per_batch, (unsigned long long)kNoAllocMaxBatch);
        return bc_set_error(BLOWCHOC_EINVAL, msg);
    }
    int dev = -1;
    e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_cuda_error(e);
    if (dev != f->device || dev < 0 || dev >= kMaxDevices)
        return bc_set_error(BLOWCHOC_EINVAL, "blowchoc_insert_noalloc: make the filter's device current");
    uint8_t *sel = choices_on(dev, &e);
    if (!sel) return noalloc_cuda_error(e);
    for (uint64_t s0 = 0; s0 < n; s0 += B) {
        const uint64_t cnt = (n - s0) < B ? (n - s0) : B;
        // every choice byte of the batch is written before the set phase
        // reads it, so the array needs no clearing between calls
        const uint64_t gc = (cnt * (uint64_t)f->lanes_choose + 255) / 256;
        const uint64_t gs = (cnt * (uint64_t)f->lanes_set + 255) / 256;
        const uint64_t cap = (uint64_t)f->sms * 8;
        bc::Launch Lc{(int)(gc < cap ? (gc ? gc : 1) : cap), f->lanes_choose, s};
        e = bc::launch_choose(C, Lc, f->dev, d_keys + s0, cnt, f->d_rank, sel, f->d_counters);
        if (e != cudaSuccess) return noalloc_cuda_error(e);
        bc_note_launch();
        bc::Launch Ls{(int)(gs < cap ? (gs ? gs : 1) : cap), f->lanes_set, s};
        e = bc::launch_set(Ls, f->dev, d_keys + s0, cnt, sel);
        if (e != cudaSuccess) return noalloc_cuda_error(e);
        bc_note_launch();
    }
    return BLOWCHOC_OK;
}
