// k_debug_curand.cu -- test probe only: blocks of NVIDIA's device Philox4_32_10
// generator (cuRAND device API), used by the GPU tests to check the library's
// own counter-based Philox bit for bit against an independent implementation.
// Never on the propagation path.
#include <curand_kernel.h>

#include <cstdint>

#include "internal.h"

namespace cosmica {

namespace {
__global__ void k_debug_curand_philox(uint32_t n, uint64_t seed, const unsigned long long *subseq,
                                      const unsigned long long *offset, uint32_t *out)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    curandStatePhilox4_32_10_t st;
    curand_init(seed, subseq[i], offset[i], &st);
    const uint4 w = curand4(&st);
    out[4 * i] = w.x; out[4 * i + 1] = w.y; out[4 * i + 2] = w.z; out[4 * i + 3] = w.w;
}
}  // namespace

cudaError_t launch_debug_curand_philox(uint32_t n, uint64_t seed, const unsigned long long *subseq,
                                       const unsigned long long *offset, uint32_t *out, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    cudaGetLastError();
    k_debug_curand_philox<<<(n + 127) / 128, 128, 0, s>>>(n, seed, subseq, offset, out);
    note_launch();
    return cudaGetLastError();
}

}  // namespace cosmica
