// k_debug32.cu -- test probe only: the mixed path's FP32 normals.
//
// Built with the mixed kernels' floating-point flags (-ftz=true
// -prec-div=false -prec-sqrt=false -fmad=false), so m32::normals compiles to
// the same arithmetic that the propagation kernels draw each step.  Besides
// the three normals of step `step` of each particle it returns the Philox
// words they come from, so that a test can evaluate Box-Muller on exactly
// those words independently.  Never on the propagation path.
#include <cstdint>

#include "common.cuh"
#include "internal.h"
#include "model32.cuh"
#include "philox.cuh"

namespace cosmica {

namespace {
__global__ void k_debug_normals32(uint64_t seed, uint64_t pid0, uint32_t n, uint32_t step, float *__restrict__ z,
                                  uint32_t *__restrict__ words)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint64_t pid = pid0 + i;
    float z0, z1, z2;
    m32::normals(seed, pid, step, z0, z1, z2);
    z[3 * (size_t)i] = z0;
    z[3 * (size_t)i + 1] = z1;
    z[3 * (size_t)i + 2] = z2;
    if (words) {
        const uint4 w = philox_step_block(seed, pid, step);
        words[4 * (size_t)i] = w.x;
        words[4 * (size_t)i + 1] = w.y;
        words[4 * (size_t)i + 2] = w.z;
        words[4 * (size_t)i + 3] = w.w;
    }
}
}  // namespace

cudaError_t launch_debug_normals32(uint64_t seed, uint64_t pid0, uint32_t n, uint32_t step, float *z,
                                   uint32_t *words, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    cudaGetLastError();
    k_debug_normals32<<<(n + 255u) / 256u, 256, 0, s>>>(seed, pid0, n, step, z, words);
    note_launch();
    return cudaGetLastError();
}

}  // namespace cosmica
