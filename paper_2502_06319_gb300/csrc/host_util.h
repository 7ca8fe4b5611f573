// host_util.h -- host-side helpers shared by the C-ABI layer and the server:
// thread-local error reporting, grow-only device buffers, pinned staging
// buffers guarded by an event, and parameter conversion/validation.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <cstddef>
#include <cstdint>

#include "common.cuh"
#include "cosmica.h"

namespace cosmica {
namespace host {

cosmica_status fail(cosmica_status st, const char *fmt, ...);
cosmica_status cuda_fail(cudaError_t e, const char *what);

#define CK(call, what)                                   \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

// Grow-only device buffer.  cudaFree synchronises the device, so a buffer is
// never released while a kernel that uses it is in flight.
struct DevBuf {
    void *d = nullptr;
    size_t cap = 0;
    cosmica_status reserve(size_t n)
    {
        if (n <= cap) return COSMICA_OK;
        if (d) cudaFree(d);
        d = nullptr;
        cap = 0;
        size_t want = std::max<size_t>(n, 4096);
        cudaError_t e = cudaMalloc(&d, want);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(scratch)");
        cap = want;
        return COSMICA_OK;
    }
    void release()
    {
        if (d) cudaFree(d);
        d = nullptr;
        cap = 0;
    }
};

// Pinned staging buffer for the small per-call tables.  Before it is
// rewritten, the host waits for the previous upload from it to complete.
struct Staging {
    void *h = nullptr;
    size_t cap = 0;
    cudaEvent_t ev = nullptr;
    bool pending = false;
    cosmica_status reserve(size_t n)
    {
        if (pending) {
            cudaError_t e = cudaEventSynchronize(ev);
            if (e != cudaSuccess) return cuda_fail(e, "cudaEventSynchronize(staging)");
            pending = false;
        }
        if (!ev) {
            cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
            if (e != cudaSuccess) return cuda_fail(e, "cudaEventCreate");
        }
        if (n <= cap) return COSMICA_OK;
        if (h) cudaFreeHost(h);
        h = nullptr;
        cap = 0;
        size_t want = std::max<size_t>(n, 4096);
        cudaError_t e = cudaMallocHost(&h, want);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMallocHost(staging)");
        cap = want;
        return COSMICA_OK;
    }
    cosmica_status upload(void *dst, size_t n, cudaStream_t s)
    {
        CK(cudaMemcpyAsync(dst, h, n, cudaMemcpyHostToDevice, s), "cudaMemcpyAsync(tables)");
        CK(cudaEventRecord(ev, s), "cudaEventRecord(staging)");
        pending = true;
        return COSMICA_OK;
    }
    void release()
    {
        if (pending && ev) cudaEventSynchronize(ev);
        if (h) cudaFreeHost(h);
        if (ev) cudaEventDestroy(ev);
        h = nullptr;
        ev = nullptr;
        cap = 0;
        pending = false;
    }
};

size_t align_up(size_t x, size_t a);
bool is_device_ptr(const void *p);
cosmica_status check_params(const cosmica_params *p);
cosmica_status check_species(const cosmica_species *s);
DevParams to_dev(const cosmica_params &p);
DevSpecies to_dev(const cosmica_species &s);
// a start position inside the heliosphere of p: r_in <= r0 < R_out, th0 in (0, pi), finite ph0
bool valid_start(const cosmica_params &p, double r0, double th0, double ph0);

inline DevItem make_item(double T, uint64_t first_pid, uint64_t seed, uint32_t param_idx, uint32_t species_idx,
                         double r0, double th0, double ph0, uint32_t out_item)
{
    DevItem it;
    it.T = T;
    it.first_pid = first_pid;
    it.seed = seed;
    it.param_idx = param_idx;
    it.species_idx = species_idx;
    it.r0 = r0;
    it.th0 = th0;
    it.ph0 = ph0;
    it.out_item = out_item;
    it.pad = 0;
    return it;
}
int num_sms();

}  // namespace host
}  // namespace cosmica
