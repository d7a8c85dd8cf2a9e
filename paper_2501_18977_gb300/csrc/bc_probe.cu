// Random 64-byte gather probe: the ceiling that random block reads (the
// access pattern of insert and query) reach on this device, measured beside
// the streaming copy bandwidth.
#include "bc_filter.h"
#include "bc_launch.h"
#include "bc_phases.cuh"

namespace {

constexpr int kThreads = 256;

// Each group of LANES lanes reads `per_group` pseudo-random whole blocks
// (block index from a multiplicative hash of a counter, so addresses are
// spread uniformly) and folds them into one word per warp. A trip issues U
// independent block loads before folding any of them, so U loads per lane
// group are in flight at once (memory-level parallelism beyond one load per
// thread).
template <int LANES, int U>
__global__ void __launch_bounds__(kThreads) gather_probe_kernel(const uint64_t *__restrict__ words,
                                                                uint64_t mask_or_m, int pow2,
                                                                uint64_t nreads, uint64_t seed,
                                                                uint64_t *__restrict__ sink) {
    constexpr int W = bc::kBlockWords / LANES;
    const int lane = threadIdx.x & 31, q = lane % LANES;
    const uint64_t gid = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) / LANES;
    const uint64_t ngroups = ((uint64_t)gridDim.x * blockDim.x) / LANES;
    uint64_t acc = 0;
    const uint64_t per_trip = ngroups * U;
    const uint64_t trips = (nreads + per_trip - 1) / per_trip;
    for (uint64_t t = 0; t < trips; ++t) {
        uint64_t v[U][W];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint64_t r = t * per_trip + (uint64_t)u * ngroups + gid;
            const uint64_t h = (r + seed) * 0x9E3779B97F4A7C15ull;
            const uint64_t b = pow2 ? ((h >> 20) & mask_or_m) : ((h >> 20) % mask_or_m);
            if (r < nreads) {
                bc::load_words<W, bc::kLoadNC>(words + b * bc::kBlockWords + (uint64_t)q * W, v[u]);
            } else {
#pragma unroll
                for (int j = 0; j < W; ++j) v[u][j] = 0;
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int j = 0; j < W; ++j) acc ^= v[u][j];
    }
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) acc ^= __shfl_xor_sync(0xffffffffu, acc, s);
    if (lane == 0) sink[((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5] = acc;
}

template <int LANES>
cudaError_t launch_probe(int grid, cudaStream_t s, uint32_t inflight, const uint64_t *w, uint64_t mm,
                         int pow2, uint64_t nreads, uint64_t seed, uint64_t *sink) {
    switch (inflight) {
        case 1: gather_probe_kernel<LANES, 1><<<grid, kThreads, 0, s>>>(w, mm, pow2, nreads, seed, sink); break;
        case 2: gather_probe_kernel<LANES, 2><<<grid, kThreads, 0, s>>>(w, mm, pow2, nreads, seed, sink); break;
        case 4: gather_probe_kernel<LANES, 4><<<grid, kThreads, 0, s>>>(w, mm, pow2, nreads, seed, sink); break;
        case 8: gather_probe_kernel<LANES, 8><<<grid, kThreads, 0, s>>>(w, mm, pow2, nreads, seed, sink); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// Barrier self-test: every CTA but the last arrives at one grid barrier; the
// last never does, so the others must give up after `limit` clock cycles and
// set *err. Nothing spins without a bound.
__global__ void barrier_selftest_kernel(unsigned int *bar, unsigned long long *err, long long limit) {
    if (blockIdx.x + 1 == gridDim.x) return;  // the CTA that never arrives
    bc::grid_barrier(bar, gridDim.x, err, limit);
}

}  // namespace

extern "C" int blowchoc_barrier_selftest(uint32_t ctas, double seconds, void *stream) {
    if (ctas < 2 || ctas > 1024 || !(seconds > 0.0) || seconds > 10.0)
        return bc_set_error(BLOWCHOC_EINVAL, "ctas in 2..1024, seconds in (0, 10]");
    int dev = 0, rate_khz = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&rate_khz, cudaDevAttrClockRate, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return bc_set_error(BLOWCHOC_ECUDA, "no usable CUDA device");
    if ((int)ctas > sms) return bc_set_error(BLOWCHOC_EINVAL, "more CTAs than SMs");
    const long long limit = (long long)(seconds * 1e3 * (double)(rate_khz > 0 ? rate_khz : 2000000));
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long *d = nullptr;  // [0] error word, [1] arrivals
    if (cudaMalloc(&d, 2 * sizeof(unsigned long long)) != cudaSuccess)
        return bc_set_error(BLOWCHOC_ENOMEM, "self-test words");
    unsigned long long h[2] = {0, 0};
    cudaError_t e = cudaMemsetAsync(d, 0, 2 * sizeof(unsigned long long), s);
    unsigned int *bar = reinterpret_cast<unsigned int *>(d + 1);
    void *args[] = {(void *)&bar, (void *)&d, (void *)&limit};
    if (e == cudaSuccess)
        e = cudaLaunchCooperativeKernel((const void *)barrier_selftest_kernel, dim3(ctas), dim3(32), args, 0, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, d, sizeof h, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d);
    if (e != cudaSuccess) return bc_set_error(BLOWCHOC_ECUDA, cudaGetErrorString(e));
    bc_note_launch();
    if (h[0] != 0) return bc_set_error(BLOWCHOC_ETIMEOUT, "grid barrier wait gave up (as intended)");
    return BLOWCHOC_OK;
}

extern "C" int blowchoc_gather_probe(const uint64_t *d_words, uint64_t nblocks, uint64_t nreads,
                                     uint64_t seed, uint32_t lanes, uint32_t ctas_per_sm, uint32_t inflight,
                                     uint64_t *d_sink, void *stream) {
    if (!d_words || !d_sink || nblocks == 0) return bc_set_error(BLOWCHOC_EINVAL, "bad probe arguments");
    if (ctas_per_sm < 1 || ctas_per_sm > 16) return bc_set_error(BLOWCHOC_EINVAL, "ctas_per_sm must be in 1..16");
    if (inflight != 1 && inflight != 2 && inflight != 4 && inflight != 8)
        return bc_set_error(BLOWCHOC_EINVAL, "inflight must be 1, 2, 4 or 8");
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return bc_set_error(BLOWCHOC_ECUDA, "no usable CUDA device");
    const int grid = sms * (int)ctas_per_sm;
    const int pow2 = (nblocks & (nblocks - 1)) == 0;
    const uint64_t mm = pow2 ? nblocks - 1 : nblocks;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e;
    switch (lanes) {
        case 1: e = launch_probe<1>(grid, s, inflight, d_words, mm, pow2, nreads, seed, d_sink); break;
        case 2: e = launch_probe<2>(grid, s, inflight, d_words, mm, pow2, nreads, seed, d_sink); break;
        case 4: e = launch_probe<4>(grid, s, inflight, d_words, mm, pow2, nreads, seed, d_sink); break;
        case 8: e = launch_probe<8>(grid, s, inflight, d_words, mm, pow2, nreads, seed, d_sink); break;
        default: return bc_set_error(BLOWCHOC_EINVAL, "lanes must be 1, 2, 4 or 8");
    }
    if (e != cudaSuccess) return bc_set_error(BLOWCHOC_ECUDA, cudaGetErrorString(e));
    bc_note_launch();
    return BLOWCHOC_OK;
}
