// Device-side key generation for large synthetic workloads: successive
// outputs of splitmix64 (Steele, Lea and Flood, OOPSLA 2014) of a seed, the
// same stream the Python input generators produce on the host. Input
// generation only; no part of the filter's arithmetic.
#include "bc_launch.h"

namespace bc {
namespace {

__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t i) {
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void __launch_bounds__(256) generate_keys_kernel(uint64_t *__restrict__ out, uint64_t n, uint64_t seed,
                                                            uint64_t start) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        __stcs(reinterpret_cast<unsigned long long *>(out + i), splitmix64_at(seed, start + i));
}

}  // namespace

cudaError_t launch_generate_keys(cudaStream_t s, int sms, uint64_t *d_out, uint64_t n, uint64_t seed,
                                 uint64_t start) {
    if (n == 0) return cudaSuccess;
    const uint64_t want = (n + 255) / 256;
    const int grid = (int)(want < (uint64_t)sms * 8 ? want : (uint64_t)sms * 8);
    generate_keys_kernel<<<grid, 256, 0, s>>>(d_out, n, seed, start);
    return cudaGetLastError();
}

}  // namespace bc
