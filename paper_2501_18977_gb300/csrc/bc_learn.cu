// Learned block-selection cost (not in the paper).
//
// A small network g(x) with x = (j / 512, a / k) -- the load after insertion
// and the new bits relative to k, the two arguments of the paper's costs --
// is evaluated on the whole (L, a) grid into a cost table, which a filter then
// uses through blowchoc_set_cost_table exactly like a built-in cost. Training
// is on the GPU by a score-function (REINFORCE) estimator: a sampling choose
// kernel picks among a key's candidates with probability softmax(-g / tau)
// and accumulates d log pi / d g at every grid point it touched; the backward
// kernel turns those per-point weights into parameter gradients; Adam steps.
//
// Network: 2 -> H -> H -> 1, tanh on the hidden layers, linear output, fp32.
// Parameter layout: W1[H][2], b1[H], W2[H][H] (row o, column i), b2[H],
// w3[H], b3 -- H*H + 5H + 1 floats.
#include <cmath>
#include <cstring>
#include <vector>

#include "bc_filter.h"
#include "bc_launch.h"
#include "bc_phases.cuh"

namespace {

constexpr int kH = 32;
constexpr int kParams = kH * kH + 5 * kH + 1;
constexpr int kW1 = 0, kB1 = 2 * kH, kW2 = 3 * kH, kB2 = 3 * kH + kH * kH, kW3 = 4 * kH + kH * kH,
              kB3 = 5 * kH + kH * kH;

__device__ __forceinline__ void mlp_hidden(const float *p, float x0, float x1, float (&h1)[kH], float (&h2)[kH]) {
#pragma unroll
    for (int h = 0; h < kH; ++h) h1[h] = tanhf(p[kW1 + 2 * h] * x0 + p[kW1 + 2 * h + 1] * x1 + p[kB1 + h]);
#pragma unroll 4
    for (int o = 0; o < kH; ++o) {
        float acc = p[kB2 + o];
#pragma unroll
        for (int i = 0; i < kH; ++i) acc += p[kW2 + o * kH + i] * h1[i];
        h2[o] = tanhf(acc);
    }
}

// table[L (k+1) + a] = g(((L + a) / 512, a / k)) for every grid point.
__global__ void __launch_bounds__(128) mlp_forward_kernel(const float *__restrict__ params, uint32_t k,
                                                          float *__restrict__ table) {
    __shared__ float p[kParams];
    for (int t = threadIdx.x; t < kParams; t += blockDim.x) p[t] = params[t];
    __syncthreads();
    const uint32_t k1 = k + 1;
    const uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 513u * k1) return;
    const uint32_t L = idx / k1, a = idx % k1;
    float h1[kH], h2[kH];
    mlp_hidden(p, (float)(L + a) / 512.0f, (float)a / (float)k, h1, h2);
    float g = p[kB3];
#pragma unroll
    for (int h = 0; h < kH; ++h) g += p[kW3 + h] * h2[h];
    table[idx] = g;
}

// Warp sum of v, added (in double) to *dst by lane 0.
__device__ __forceinline__ void warp_add(double *dst, float v, int lane) {
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) v += __shfl_xor_sync(0xffffffffu, v, s);
    if (lane == 0 && v != 0.0f) atomicAdd(dst, (double)v);
}

// grad += sum_r scales[r] * sum_p w[r][p] * d g(x_p) / d params: rows r of
// per-point weights (one per training filter) with one scale each; one
// thread per grid point.
__global__ void __launch_bounds__(128) mlp_backward_kernel(const float *__restrict__ params, uint32_t k,
                                                           const float *__restrict__ w, uint32_t rows,
                                                           const double *__restrict__ scales,
                                                           double *__restrict__ grad) {
    __shared__ float p[kParams];
    for (int t = threadIdx.x; t < kParams; t += blockDim.x) p[t] = params[t];
    __syncthreads();
    const uint32_t k1 = k + 1, npts = 513u * k1;
    const uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const bool valid = idx < npts;
    double acc = 0.0;
    if (valid)
        for (uint32_t r = 0; r < rows; ++r) acc += scales[r] * (double)w[(uint64_t)r * npts + idx];
    const float gw = (float)acc;
    if (__ballot_sync(0xffffffffu, gw != 0.0f) == 0u) return;  // whole warp idle
    const uint32_t L = valid ? idx / k1 : 0, a = valid ? idx % k1 : 0;
    const float x0 = (float)(L + a) / 512.0f, x1 = (float)a / (float)k;
    float h1[kH], h2[kH];
    mlp_hidden(p, x0, x1, h1, h2);
    warp_add(grad + kB3, gw, lane);
    float d2[kH];
#pragma unroll
    for (int o = 0; o < kH; ++o) {
        warp_add(grad + kW3 + o, gw * h2[o], lane);
        d2[o] = gw * p[kW3 + o] * (1.0f - h2[o] * h2[o]);
        warp_add(grad + kB2 + o, d2[o], lane);
    }
    for (int o = 0; o < kH; ++o)
#pragma unroll
        for (int i = 0; i < kH; ++i) warp_add(grad + kW2 + o * kH + i, d2[o] * h1[i], lane);
    for (int i = 0; i < kH; ++i) {
        float back = 0.0f;
#pragma unroll
        for (int o = 0; o < kH; ++o) back += p[kW2 + o * kH + i] * d2[o];
        const float d1 = back * (1.0f - h1[i] * h1[i]);
        warp_add(grad + kB1 + i, d1, lane);
        warp_add(grad + kW1 + 2 * i, d1 * x0, lane);
        warp_add(grad + kW1 + 2 * i + 1, d1 * x1, lane);
    }
}

// Adam on the parameters (minimises: the caller passes the gradient of the
// loss), then clears the gradient.
__global__ void adam_kernel(float *__restrict__ params, double *__restrict__ grad, float *__restrict__ m1,
                            float *__restrict__ m2, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= kParams) return;
    const float g = (float)grad[t];
    grad[t] = 0.0;
    m1[t] = b1 * m1[t] + (1.0f - b1) * g;
    m2[t] = b2 * m2[t] + (1.0f - b2) * g * g;
    params[t] -= lr * (m1[t] / c1) / (sqrtf(m2[t] / c2) + eps);
}

// Uniform in [0, 1) from the splitmix64 stream of `seed` at position idx.
__device__ __forceinline__ double rng_uniform(uint64_t seed, uint64_t idx) {
    uint64_t z = seed + (idx + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

// Sampling choose phase for training: per key, skip exactly as the greedy
// rule does; otherwise draw the choice from softmax(-g / tau) over the
// candidates' table values, and add d log pi(chosen) / d g = -(1{p = chosen} -
// pi_p) / tau to w at the candidates' grid points.
template <int C, int LANES>
__global__ void __launch_bounds__(256) sampled_choose_kernel(bc::DevFilter f, const uint64_t *__restrict__ keys,
                                                             uint64_t n, uint64_t idx0,
                                                             const float *__restrict__ table, float tau,
                                                             uint64_t seed, uint8_t *__restrict__ sel,
                                                             float *__restrict__ w, uint8_t *choice_out,
                                                             unsigned long long *counters) {
    constexpr int G = 32 / LANES;
    constexpr int W = bc::kBlockWords / LANES;
    extern __shared__ float s_w[];  // 513 (k+1) per-point weights of this CTA
    __shared__ uint64_t s_amul[32];
    __shared__ __align__(16) uint32_t s_mask[8 * bc::mask_u32_per_warp<LANES>()];
    const uint32_t k1 = f.k + 1, npts = 513u * k1;
    for (uint32_t t = threadIdx.x; t < npts; t += blockDim.x) s_w[t] = 0.0f;
    bc::stage_bit_mults(f, s_amul);
    __syncthreads();
    const int lane = threadIdx.x & 31, q = lane % LANES, g = lane / LANES;
    uint32_t *region = bc::warp_mask_area<LANES>(s_mask, threadIdx.x >> 5);
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    uint32_t ins = 0, skp = 0;
    for (uint64_t base = warp * G; base < n; base += nwarps * G) {
        const uint64_t i = base + g;
        const bool valid = i < n;
        const uint64_t x = valid ? bc::load_key(keys + i) : 0ull;
        uint64_t m[W];
        bc::key_mask_shared<LANES>(s_amul, f.k, x, q, region, m, f.bitsel);
        uint32_t la[C];
#pragma unroll
        for (int c = 0; c < C; ++c) {
            uint64_t blk[W];
            const uint64_t b = bc::block_addr(f, f.a_block[c], x);
            if (valid) {
                bc::load_words<W, bc::kLoadNC>(f.words + b * bc::kBlockWords + (uint64_t)q * W, blk);
            } else {
#pragma unroll
                for (int j = 0; j < W; ++j) blk[j] = ~0ull;
            }
            la[c] = bc::group_sum<LANES>(bc::load_and_new<W>(blk, m));
        }
        if (!valid || q != 0) continue;
        bool skip = false;
#pragma unroll
        for (int c = 0; c < C; ++c) skip |= ((la[c] >> 16) == 0);
        uint32_t s = bc::kSkip;
        if (!skip) {
            uint32_t pt[C];
            double gv[C], gmin = 1e300;
#pragma unroll
            for (int c = 0; c < C; ++c) {
                pt[c] = (la[c] & 0xFFFFu) * k1 + (la[c] >> 16);
                gv[c] = (double)table[pt[c]];
                gmin = gv[c] < gmin ? gv[c] : gmin;
            }
            double e[C], z = 0.0;
#pragma unroll
            for (int c = 0; c < C; ++c) {
                e[c] = exp(-(gv[c] - gmin) / (double)tau);
                z += e[c];
            }
            // the first candidate whose cumulative weight exceeds u z
            const double u = rng_uniform(seed, idx0 + i) * z;
            double cdf = 0.0;
            s = C - 1;
            bool found = false;
#pragma unroll
            for (int c = 0; c < C - 1; ++c) {
                cdf += e[c];
                if (!found && u < cdf) {
                    s = c;
                    found = true;
                }
            }
#pragma unroll
            for (int c = 0; c < C; ++c)
                atomicAdd(s_w + pt[c], (float)((e[c] / z - (c == (int)s ? 1.0 : 0.0)) / (double)tau));
        }
        sel[i] = (uint8_t)s;
        if (choice_out) choice_out[i] = (uint8_t)s;
        if (s == bc::kSkip) ++skp; else ++ins;
    }
    __syncthreads();
    for (uint32_t t = threadIdx.x; t < npts; t += blockDim.x)
        if (s_w[t] != 0.0f) atomicAdd(w + t, s_w[t]);
    bc::flush_counts(ins, skp, counters);
}

template <int C>
cudaError_t sampled_launch(int grid, cudaStream_t s, const bc::DevFilter &f, const uint64_t *keys, uint64_t n,
                           uint64_t idx0, const float *table, float tau, uint64_t seed, uint8_t *sel, float *w,
                           uint8_t *choice_out, unsigned long long *counters) {
    const size_t sm = 513u * (f.k + 1) * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(sampled_choose_kernel<C, 2>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    sampled_choose_kernel<C, 2><<<grid, 256, sm, s>>>(f, keys, n, idx0, table, tau, seed, sel, w, choice_out,
                                                      counters);
    return cudaGetLastError();
}

}  // namespace

struct blowchoc_mlp {
    uint32_t k = 0;
    float *d_params = nullptr, *d_m1 = nullptr, *d_m2 = nullptr;
    double *d_grad = nullptr;
    int step = 0;
};

extern "C" {

int blowchoc_mlp_create(uint32_t k, uint64_t seed, blowchoc_mlp **out) {
    if (!out || k < 1 || k > 32) return bc_set_error(BLOWCHOC_EINVAL, "bad network arguments");
    *out = nullptr;
    blowchoc_mlp *m = new blowchoc_mlp();
    m->k = k;
    // weights uniform in +-1/sqrt(fan_in) from splitmix64(seed); biases 0
    std::vector<float> p(kParams, 0.0f);
    uint64_t st = seed;
    auto next = [&st]() {
        uint64_t z = (st += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        return (double)(z >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
    };
    for (int t = 0; t < 2 * kH; ++t) p[kW1 + t] = (float)(next() / std::sqrt(2.0));
    for (int t = 0; t < kH * kH; ++t) p[kW2 + t] = (float)(next() / std::sqrt((double)kH));
    for (int t = 0; t < kH; ++t) p[kW3 + t] = (float)(next() / std::sqrt((double)kH));
    cudaError_t e = cudaMalloc(&m->d_params, kParams * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&m->d_m1, kParams * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&m->d_m2, kParams * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&m->d_grad, kParams * sizeof(double));
    if (e == cudaSuccess) e = cudaMemcpy(m->d_params, p.data(), kParams * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(m->d_m1, 0, kParams * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(m->d_m2, 0, kParams * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(m->d_grad, 0, kParams * sizeof(double));
    if (e != cudaSuccess) {
        cudaFree(m->d_params); cudaFree(m->d_m1); cudaFree(m->d_m2); cudaFree(m->d_grad);
        delete m;
        return bc_set_error(e == cudaErrorMemoryAllocation ? BLOWCHOC_ENOMEM : BLOWCHOC_ECUDA, cudaGetErrorString(e));
    }
    *out = m;
    return BLOWCHOC_OK;
}

int blowchoc_mlp_destroy(blowchoc_mlp *m) {
    if (!m) return BLOWCHOC_OK;
    cudaDeviceSynchronize();
    cudaFree(m->d_params); cudaFree(m->d_m1); cudaFree(m->d_m2); cudaFree(m->d_grad);
    delete m;
    return BLOWCHOC_OK;
}

uint32_t blowchoc_mlp_param_count(void) { return (uint32_t)kParams; }

int blowchoc_mlp_get_params(blowchoc_mlp *m, float *h_params, double *h_grad) {
    if (!m) return bc_set_error(BLOWCHOC_EINVAL, "network is NULL");
    if (h_params && cudaMemcpy(h_params, m->d_params, kParams * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
        return bc_set_error(BLOWCHOC_ECUDA, "copy parameters");
    if (h_grad && cudaMemcpy(h_grad, m->d_grad, kParams * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
        return bc_set_error(BLOWCHOC_ECUDA, "copy gradient");
    return BLOWCHOC_OK;
}

int blowchoc_mlp_set_params(blowchoc_mlp *m, const float *h_params) {
    if (!m || !h_params) return bc_set_error(BLOWCHOC_EINVAL, "NULL argument");
    if (cudaMemcpy(m->d_params, h_params, kParams * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
        return bc_set_error(BLOWCHOC_ECUDA, "copy parameters");
    return BLOWCHOC_OK;
}

int blowchoc_mlp_forward(blowchoc_mlp *m, float *d_table, void *stream) {
    if (!m || !d_table) return bc_set_error(BLOWCHOC_EINVAL, "NULL argument");
    const uint32_t npts = 513u * (m->k + 1);
    mlp_forward_kernel<<<(npts + 127) / 128, 128, 0, (cudaStream_t)stream>>>(m->d_params, m->k, d_table);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return bc_set_error(BLOWCHOC_ECUDA, cudaGetErrorString(e));
    bc_note_launch();
    return BLOWCHOC_OK;
}

int blowchoc_mlp_backward(blowchoc_mlp *m, const float *d_w, uint32_t rows, const double *d_scales,
                          void *stream) {
    if (!m || !d_w || !d_scales || rows == 0) return bc_set_error(BLOWCHOC_EINVAL, "bad backward arguments");
    const uint32_t npts = 513u * (m->k + 1);
    mlp_backward_kernel<<<(npts + 127) / 128, 128, 0, (cudaStream_t)stream>>>(m->d_params, m->k, d_w, rows,
                                                                              d_scales, m->d_grad);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return bc_set_error(BLOWCHOC_ECUDA, cudaGetErrorString(e));
    bc_note_launch();
    return BLOWCHOC_OK;
}

int blowchoc_mlp_adam_step(blowchoc_mlp *m, float lr, void *stream) {
    if (!m || !(lr > 0.0f)) return bc_set_error(BLOWCHOC_EINVAL, "bad Adam arguments");
    m->step++;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - std::pow(b1, (float)m->step), c2 = 1.0f - std::pow(b2, (float)m->step);
    adam_kernel<<<(kParams + 255) / 256, 256, 0, (cudaStream_t)stream>>>(m->d_params, m->d_grad, m->d_m1, m->d_m2,
                                                                       lr, b1, b2, 1e-8f, c1, c2);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return bc_set_error(BLOWCHOC_ECUDA, cudaGetErrorString(e));
    bc_note_launch();
    return BLOWCHOC_OK;
}

int blowchoc_insert_sampled(blowchoc_filter *f, const uint64_t *d_keys, uint64_t n, const float *d_table,
                            float tau, uint64_t seed, float *d_w, uint8_t *d_choice, void *stream) {
    if (!f || !d_table || !d_w || !(tau > 0.0f)) return bc_set_error(BLOWCHOC_EINVAL, "bad arguments");
    if (f->p.choices < 2) return bc_set_error(BLOWCHOC_EINVAL, "one choice has nothing to sample");
    if (n == 0) return BLOWCHOC_OK;
    if (!d_keys) return bc_set_error(BLOWCHOC_EINVAL, "keys is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    const uint64_t B = f->p.batch;
    const uint64_t per = B < n ? B : n;
    if (per > f->sel_cap) {
        cudaFree(f->d_sel);
        f->d_sel = nullptr;
        f->sel_cap = 0;
        if (cudaMalloc(&f->d_sel, per) != cudaSuccess) return bc_set_error(BLOWCHOC_ENOMEM, "choice scratch");
        f->sel_cap = per;
    }
    for (uint64_t s0 = 0; s0 < n; s0 += B) {
        const uint64_t cnt = (n - s0) < B ? (n - s0) : B;
        const uint64_t groups = (cnt * 2 + 255) / 256;
        const int grid = (int)(groups < (uint64_t)f->sms * 8 ? (groups ? groups : 1) : (uint64_t)f->sms * 8);
        cudaError_t e = f->p.choices == 2
            ? sampled_launch<2>(grid, s, f->dev, d_keys + s0, cnt, s0, d_table, tau, seed, f->d_sel, d_w,
                                d_choice ? d_choice + s0 : nullptr, f->d_counters)
            : sampled_launch<3>(grid, s, f->dev, d_keys + s0, cnt, s0, d_table, tau, seed, f->d_sel, d_w,
                                d_choice ? d_choice + s0 : nullptr, f->d_counters);
        if (e != cudaSuccess) return bc_set_error(BLOWCHOC_ECUDA, cudaGetErrorString(e));
        bc_note_launch();
        bc::Launch Ls{grid, f->lanes_set, s};
        e = bc::launch_set(Ls, f->dev, d_keys + s0, cnt, f->d_sel);
        if (e != cudaSuccess) return bc_set_error(BLOWCHOC_ECUDA, cudaGetErrorString(e));
        bc_note_launch();
    }
    return BLOWCHOC_OK;
}

}  // extern "C"
